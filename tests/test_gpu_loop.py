"""The large single problem (2000 keyframes on two laps of a 30 m loop,
200k points, ~2M factors; FP32 messages with the FP64 fallback for
ill-conditioned keyframe marginals) against the FP64 oracle.

The oracle runs on a 10% subgraph (keyframes 0-199 and every point they see
twice, ~190k factors): per-belief FP32 error against it, with the
deterministic relinearisation schedule (every factor at t = 10, 20, ...)
so that threshold decisions cannot part the trajectories.  On the whole
graph the FP32 path is compared with the device's FP64 mode (itself pinned
to the oracle to 1e-9 on smaller graphs), per belief.

The error is stated as a distribution.  A few dozen weakly observed points
(seen two or three times, some through outlier pixels) still move after
hundreds of iterations, and there the iteration amplifies any difference
in rounding: the device's FP64 mode, whose arithmetic differs from the
oracle's only in summation order, departs from it by up to 6e-7 on those
points after 60 iterations (4e-5 after 300) while its 99th percentile stays
at 1e-9.  The bar is therefore: 99th percentile and every keyframe within
the 1e-5 tolerance, at most 0.1% of the beliefs beyond it, and the average
reprojection error within 1e-3 px."""
import os
import time

import numpy as np
import pytest

import oracle
from paper_2003_03134_gb300 import build, gbp, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL32 = 1e-5
DET = dict(relin_beta=0.0, relin_interval=10, huber_nsigma=2.0)


@pytest.fixture(scope="module")
def loop():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    return synth.make_loop(0)


def per_belief(kf, lm, okf, olm):
    ek = np.linalg.norm(kf - okf, axis=1) / np.maximum(np.linalg.norm(okf, axis=1), 1.0)
    el = np.linalg.norm(lm - olm, axis=1) / np.maximum(np.linalg.norm(olm, axis=1), 1.0)
    e = np.concatenate([ek, el])
    return e, dict(max=float(e.max()), p99=float(np.percentile(e, 99)), median=float(np.median(e)),
                   kf_max=float(ek.max()), lm_max=float(el.max()), frac_over=float((e > TOL32).mean()))


def check(s):
    assert s["p99"] <= TOL32, s
    assert s["kf_max"] <= TOL32, s
    assert s["frac_over"] <= 1e-3, s


def test_loop_subgraph_fp32_against_oracle(loop):
    q = synth.subgraph(loop, 200)
    assert 150_000 < q.n_obs < 250_000
    n = 60
    g = gbp.Graph(q, **DET)
    g.iterate(n)
    kf, lm = g.beliefs()
    st = g.stats()
    g.close()
    o = oracle.Oracle(q, **DET)
    t0 = time.perf_counter()
    o.iterate(n)
    dt = time.perf_counter() - t0
    okf, olm = o.world()
    e, s = per_belief(kf, lm, okf, olm)
    print("subgraph", q.n_kf, q.n_lm, q.n_obs, s, "ARE", st["are"], o.are()[0],
          "oracle factor-updates/s", q.n_obs * n / dt, "fp64 fallbacks", st["fp64_fallbacks"])
    check(s)
    assert abs(st["are"] - o.are()[0]) <= 1e-3


def test_loop_full_graph_fp32_against_fp64(loop):
    n = 60
    out = {}
    for mode in (0, 2):
        g = gbp.Graph(loop, precision_mode=mode, **DET)
        t0 = time.perf_counter()
        g.iterate(n)
        out[mode] = (g.beliefs(), g.stats())
        print("precision_mode", mode, "seconds", time.perf_counter() - t0, out[mode][1])
        g.close()
    (kf, lm), st32 = out[0]
    (dkf, dlm), st64 = out[2]
    e, s = per_belief(kf, lm, dkf, dlm)
    print("full graph", loop.n_kf, loop.n_lm, loop.n_obs, s)
    assert np.isfinite(kf).all() and np.isfinite(lm).all()
    check(s)
    assert abs(st32["are"] - st64["are"]) <= 1e-3
