"""The allocation-free reprojection-error entry point.

gbp_reprojection_error_noalloc() serves callers that cannot allocate device
memory when they need the number (a real-time loop that reserved all its
memory up front, an application whose allocator owns the device memory).
Its answer must match the ARE that gbp_get_stats() reports for the same
means, on consecutive calls that share the library's fixed scratch array.
This file is named to be collected last."""
import numpy as np
import pytest

from paper_2003_03134_gb300 import build, gbp, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gbp.lib()
    return t


def _are_noalloc(torch, p, kf, lm, stream):
    dev = torch.device("cuda")
    d_kf = torch.tensor(kf, dtype=torch.float64, device=dev).contiguous()
    d_lm = torch.tensor(lm, dtype=torch.float64, device=dev).contiguous()
    d_ok = torch.tensor(p.obs_kf, dtype=torch.int32, device=dev)
    d_ol = torch.tensor(p.obs_lm, dtype=torch.int32, device=dev)
    d_uv = torch.tensor(p.obs_uv, dtype=torch.float64, device=dev).contiguous()
    out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)
    gbp.gbp_reprojection_error_noalloc(p.intrinsics(), 0.05, d_kf.data_ptr(), d_lm.data_ptr(), p.n_obs,
                                       d_ok.data_ptr(), d_ol.data_ptr(), d_uv.data_ptr(), out.data_ptr(), stream)
    torch.cuda.current_stream().synchronize()
    return out.cpu().numpy()


def test_noalloc_are_matches_stats_on_consecutive_calls(torch):
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for seed, n_iter in ((0, 30), (1, 80)):
        p = synth.make_walk(seed, n_kf=30, n_lm=400)
        g = gbp.Graph(p, stream=stream, huber_nsigma=2.0)
        g.iterate(n_iter)
        kf, lm = g.beliefs()
        st = g.stats()
        g.close()
        are, count = _are_noalloc(torch, p, kf, lm, stream)
        assert count == st["n_are"]
        assert abs(are - st["are"]) <= 1e-3, (are, st["are"])
        results.append(are)
    assert results[0] != results[1]


def test_noalloc_rejects_more_observations_than_scratch(torch):
    with pytest.raises(gbp.GBPError) as e:
        gbp.gbp_reprojection_error_noalloc((500.0, 500.0, 320.0, 240.0, 640, 480), 0.05, 0, 0,
                                           gbp.GBP_NOALLOC_MAX_OBS + 1, 0, 0, 0, 0, None)
    assert e.value.status == gbp.GBP_EINVAL


def test_noalloc_empty_input(torch):
    p = synth.make_circle(0, n_kf=3, n_lm=5)
    p.obs_kf, p.obs_lm, p.obs_uv = p.obs_kf[:0], p.obs_lm[:0], p.obs_uv[:0]
    out = _are_noalloc(torch, p, p.kf_Rt_init, p.lm_init, torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(out, [0.0, 0.0])
