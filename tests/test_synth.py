"""The synthetic input generator's data selection helpers (no arithmetic of
the method)."""
import numpy as np

from paper_2003_03134_gb300 import synth


def test_subgraph_keeps_what_the_first_keyframes_see():
    p = synth.make_walk(0, n_kf=40, n_lm=400)
    q = synth.subgraph(p, 15)
    assert q.n_kf == 15
    assert (q.obs_kf < 15).all()
    assert np.bincount(q.obs_lm, minlength=q.n_lm).min() >= 2
    assert list(q.anchor_kf) == [0]
    # every kept observation is one of p's, with the same pixel and the same point
    kept = {(int(k), tuple(np.round(p.lm_true[l], 12)), tuple(uv)) for k, l, uv in
            zip(p.obs_kf, p.obs_lm, map(tuple, p.obs_uv)) if k < 15}
    for k, l, uv in zip(q.obs_kf, q.obs_lm, map(tuple, q.obs_uv)):
        assert (int(k), tuple(np.round(q.lm_true[l], 12)), uv) in kept
    # and every point of p seen twice by those keyframes is kept
    cnt = np.bincount(p.obs_lm[p.obs_kf < 15], minlength=p.n_lm)
    assert q.n_lm == int((cnt >= 2).sum())
    np.testing.assert_array_equal(q.kf_Rt_init, p.kf_Rt_init[:15])
