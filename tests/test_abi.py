"""C-ABI checks that need no GPU: the library loads, exports every entry
point that include/gbp.h declares, reports the paper's defaults and rejects
invalid input before touching the device."""
import json
import os
import re

import numpy as np
import pytest

from paper_2003_03134_gb300 import build, gbp, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gbp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gbp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gbp.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(gbp.EXPORTS) == sorted(n for n in names if n in gbp.EXPORTS)
    assert set(names) <= set(gbp.EXPORTS) | {n for n in names if n.startswith("gbp_")}


def test_defaults_are_the_papers_constants(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = gbp.gbp_default_params()
    assert p.damping == pytest.approx(g["damping"]["value"])
    assert p.relin_beta == pytest.approx(g["relin_beta"]["value"])
    assert p.relin_interval == g["relin_interval"]["value"]
    assert p.undamped_iters == g["undamped_iters"]["value"]
    assert p.prior_anneal_iters == g["prior_anneal_iters"]["value"]
    assert p.prior_final_scale == pytest.approx(g["prior_final_scale"]["value"])
    # the trailing fields, as the library wrote them: the binding's layout matches the header's
    assert (p.factor_shape, p.persistent_shape, p.fp64_exact_cavity) == (-1, -1, 0)


def test_status_strings(lib):
    for s in range(7):
        assert lib.gbp_status_string(s)
    assert lib.gbp_status_string(99) == b"unknown status"


@pytest.mark.parametrize("mutate", ["kf_index", "lm_index", "nan_uv", "nan_pose", "anchor", "behind"])
def test_invalid_input_rejected_before_device_work(lib, mutate):
    p = synth.make_circle(0, n_kf=4, n_lm=10)
    kf, lm = p.kf_Rt_init.copy(), p.lm_init.copy()
    ok, ol, uv = p.obs_kf.copy(), p.obs_lm.copy(), p.obs_uv.copy()
    anc = p.anchor_kf.copy()
    if mutate == "kf_index":
        ok[3] = p.n_kf
    elif mutate == "lm_index":
        ol[0] = -1
    elif mutate == "nan_uv":
        uv[2, 1] = np.nan
    elif mutate == "nan_pose":
        kf[1, 10] = np.inf
    elif mutate == "anchor":
        anc = np.array([7], np.int32)
    elif mutate == "behind":
        # put the first observed point behind its camera
        R = kf[ok[0], :9].reshape(3, 3)
        c = -R.T @ kf[ok[0], 9:]
        lm[ol[0]] = c - 2.0 * R[2]
    with pytest.raises(gbp.GBPError) as e:
        gbp.gbp_create_graph(p.intrinsics(), kf, lm, ok, ol, uv, anc)
    assert e.value.status == gbp.GBP_EINVAL
