"""Host-side arithmetic of bench.py's JSON line: the roofline fraction is the
paper-form algorithmic bytes of one iteration (304 B per factor, 288 B per
keyframe, 108 B per point) over the measured time and the copy bandwidth;
per-belief errors are relative world-frame errors; the committed ncu traffic
is used only for the kernel source it was captured from."""
import json
import os

import numpy as np
import pytest

import bench
from paper_2003_03134_gb300 import synth


def test_roofline_fraction_follows_the_paper_form_bytes():
    p = synth.make_circle(0)
    iter_ms = 0.0125
    r = bench.roofline(p, iter_ms, 0.008, mode=2)
    bytes_iter = 304 * p.n_obs + 288 * p.n_kf + 108 * p.n_lm
    assert r["bytes_per_iteration"] == bytes_iter
    achieved = bytes_iter / (iter_ms * 1e-3) / 1e9
    assert r["achieved"] == pytest.approx(achieved, rel=1e-12)
    assert r["frac"] == pytest.approx(achieved / r["peak"], rel=1e-12)
    assert r["implementation_bytes_per_iteration"] == bytes_iter + 40 * p.n_obs
    assert r["unit"] == "GB/s" and r["bound"] == "hbm"
    assert r["ms_per_iteration"] == iter_ms


def test_per_belief_error_statistics():
    okf = np.zeros((4, 12))
    okf[:, 0] = 2.0             # |x_orc| = 2: errors are relative to it
    kf = okf.copy()
    kf[1, 3] = 2e-5             # 1e-5 relative
    kf[2, 3] = 6e-5             # 3e-5 relative
    olm = np.full((6, 3), 0.1)  # |x_orc| < 1: errors are absolute
    lm = olm.copy()
    lm[5, 0] += 4e-6
    e = bench.per_belief_error(kf, lm, okf, olm)
    assert e["beliefs"] == 10
    assert e["max"] == pytest.approx(3e-5)
    assert e["keyframes_max"] == pytest.approx(3e-5)
    assert e["over_1e-5"] == 1   # 1e-5 exactly is within the bar
    assert e["median"] == 0.0
    expect = np.percentile(np.array([0, 1e-5, 3e-5, 0, 0, 0, 0, 0, 0, 4e-6]), 99)
    assert e["p99"] == pytest.approx(expect)


def test_traffic_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    with open(tmp_path / "profiles" / "factor_kernel_traffic.json", "w") as f:
        json.dump({"kernel_source_hash": "abc", "l2_resident": {"dram_bytes_per_factor": 181.1},
                   "hbm": {"dram_bytes_per_factor": 157.5}}, f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.ncu_traffic(1000, "l2_resident") == pytest.approx(181100.0)
    assert bench.ncu_traffic(2000, "hbm") == pytest.approx(315000.0)
    assert bench.ncu_traffic(1000, "unknown") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.ncu_traffic(1000, "l2_resident") is None

