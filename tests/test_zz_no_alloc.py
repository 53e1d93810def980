"""The allocation-free reprojection-error entry point.

gbp_reprojection_error_noalloc() serves callers that cannot allocate device
memory when they need the number (a real-time loop that reserved all its
memory up front, an application whose allocator owns the device memory).
Its answer must match the ARE that gbp_get_stats() reports for the same
means, on consecutive calls that share the library's fixed scratch array,
and repeated calls must leave the device's free memory unchanged.
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


class _DeviceInputs:
    """The caller-owned device arrays of one call, allocated up front."""

    def __init__(self, torch, p, kf, lm):
        dev = torch.device("cuda")
        self.p = p
        self.n_kf, self.n_lm = len(kf), len(lm)
        self.kf = torch.tensor(kf, dtype=torch.float64, device=dev).contiguous()
        self.lm = torch.tensor(lm, dtype=torch.float64, device=dev).contiguous()
        self.ok = torch.tensor(p.obs_kf, dtype=torch.int32, device=dev)
        self.ol = torch.tensor(p.obs_lm, dtype=torch.int32, device=dev)
        self.uv = torch.tensor(p.obs_uv, dtype=torch.float64, device=dev).contiguous()
        self.out = torch.full((2,), -1.0, dtype=torch.float64, device=dev)

    def call(self, torch, stream):
        gbp.gbp_reprojection_error_noalloc(self.p.intrinsics(), 0.05, self.n_kf, self.kf.data_ptr(), self.n_lm,
                                           self.lm.data_ptr(), self.p.n_obs, self.ok.data_ptr(), self.ol.data_ptr(),
                                           self.uv.data_ptr(), self.out.data_ptr(), stream)
        torch.cuda.current_stream().synchronize()
        return self.out.cpu().numpy()


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
        are, count = _DeviceInputs(torch, p, kf, lm).call(torch, stream)
        assert count == st["n_are"]
        assert abs(are - st["are"]) <= 1e-3, (are, st["are"])
        results.append(are)
    assert results[0] != results[1]


def test_noalloc_calls_leave_free_device_memory_unchanged(torch):
    """After a first call (module load, symbol lookup), further calls take no
    device memory: the free byte count is the same before and after."""
    stream = torch.cuda.current_stream().cuda_stream
    p = synth.make_walk(2, n_kf=20, n_lm=300)
    inp = _DeviceInputs(torch, p, p.kf_Rt_init, p.lm_init)
    first = inp.call(torch, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats().get("num_alloc_retries", 0), torch.cuda.memory_allocated()
    for _ in range(5):
        np.testing.assert_array_equal(inp.call(torch, stream), first)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert (torch.cuda.memory_stats().get("num_alloc_retries", 0), torch.cuda.memory_allocated()) == stats0


def test_noalloc_leaves_out_observations_with_bad_indices(torch):
    stream = torch.cuda.current_stream().cuda_stream
    p = synth.make_circle(0, n_kf=4, n_lm=20)
    good = _DeviceInputs(torch, p, p.kf_Rt_init, p.lm_init).call(torch, stream)
    q = synth.make_circle(0, n_kf=4, n_lm=20)
    q.obs_kf = np.concatenate([q.obs_kf, [4, -1, 0]]).astype(np.int32)
    q.obs_lm = np.concatenate([q.obs_lm, [0, 0, 20]]).astype(np.int32)
    q.obs_uv = np.concatenate([q.obs_uv, np.full((3, 2), 100.0)])
    bad = _DeviceInputs(torch, q, q.kf_Rt_init, q.lm_init).call(torch, stream)
    np.testing.assert_array_equal(bad, good)


def test_noalloc_rejects_more_observations_than_scratch(torch):
    with pytest.raises(gbp.GBPError) as e:
        gbp.gbp_reprojection_error_noalloc((500.0, 500.0, 320.0, 240.0, 640, 480), 0.05, 0, 0, 0, 0,
                                           gbp.GBP_NOALLOC_MAX_OBS + 1, 0, 0, 0, 0, None)
    assert e.value.status == gbp.GBP_EINVAL


def test_noalloc_empty_input(torch):
    p = synth.make_circle(0, n_kf=3, n_lm=5)
    p.obs_kf, p.obs_lm, p.obs_uv = p.obs_kf[:0], p.obs_lm[:0], p.obs_uv[:0]
    out = _DeviceInputs(torch, p, p.kf_Rt_init, p.lm_init).call(torch, torch.cuda.current_stream().cuda_stream)
    np.testing.assert_array_equal(out, [0.0, 0.0])
