"""GPU damping network (BF16 tensor-core forward, backward and Adam through
the C ABI) against the FP64 reference network.

Tolerances come from the arithmetic: the GPU rounds weights and
activations to BF16 (unit roundoff 2^-8 = 3.9e-3) and accumulates in FP32,
so each layer carries a relative error of a few 2^-8.  Outputs lie in
(0, 0.9): |y_gpu - y_ref| <= 0.02 everywhere and <= 0.002 on average.
Gradient blocks, in relative norm: a model of the rounding (FP64 products of
BF16-rounded operands) differs from the exact gradient by up to 4% for W1
(its operands X and dz1 are both rounded and its sums cancel), 1.6% b1,
1.4% W2, 0.9% b2, 0.4% W3, 0.3% b3; the bounds below are about twice that.
A transposed or shifted weight, a dropped ReLU mask or a wrong sign moves
the results by far more.

Device buffers are kept referenced for as long as a kernel may read them:
a temporary tensor's memory returns to the caching allocator at once."""
import numpy as np
import pytest

from oracle import mlp
from paper_2003_03134_gb300 import build, gbp

pytestmark = pytest.mark.gpu

BLOCKS = [("W1", 0, 1024, 0.08), ("b1", 1024, 1088, 0.04), ("W2", 1088, 5184, 0.03), ("b2", 5184, 5248, 0.02),
          ("W3", 5248, 5312, 0.01), ("b3", 5312, 5313, 0.01)]


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    gbp.lib()
    return t


def _params(seed):
    """Reference initialisation with a stronger output layer, so that the
    predictions spread over (0, 0.9) and every layer's gradient matters."""
    p = mlp.unpack(mlp.init_params(seed))
    rng = np.random.default_rng(seed + 100)
    p["W3"] = rng.normal(0.0, 0.5, 64)
    p["b1"] = rng.normal(0.0, 0.1, 64)
    p["b2"] = rng.normal(0.0, 0.1, 64)
    return mlp.pack(p).astype(np.float32).astype(np.float64)


def _data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    t = rng.uniform(0.0, 0.9, n).astype(np.float32)
    return X, t


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 31, 128, 1000, 4099])
def test_forward_matches_reference(torch, n):
    p = _params(0)
    X, _ = _data(n, n)
    net = gbp.DampingNet(p)
    Xd = _dev(torch, X)
    yd = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    net.forward(Xd.data_ptr(), n, yd.data_ptr())
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    ref, _ = mlp.forward(p, X.astype(np.float64))
    err = np.abs(y - ref)
    assert err.max() <= 0.02, err.max()
    if n >= 100:   # the average is only meaningful over many rows
        assert err.mean() <= 0.002, err.mean()
    assert ((y > 0) & (y < 0.9)).all()
    net.close()


@pytest.mark.parametrize("n,seed", [(128, 1), (777, 2), (5000, 3)])
def test_gradient_matches_reference(torch, n, seed):
    p = _params(seed)
    X, t = _data(seed + 50, n)
    net = gbp.DampingNet(p)
    Xd, td = _dev(torch, X), _dev(torch, t)
    loss, g = net.gradient(Xd.data_ptr(), td.data_ptr(), n)
    rloss, rg = mlp.loss_and_grad(p, X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= 0.01 * rloss
    for name, a, b, tol in BLOCKS:
        num = np.linalg.norm(g[a:b] - rg[a:b])
        den = np.linalg.norm(rg[a:b])
        assert num <= tol * den, (name, num, den)
    net.close()


def test_gradient_is_reproducible(torch):
    p = _params(4)
    X, t = _data(9, 3000)
    Xd, td = _dev(torch, X), _dev(torch, t)
    net = gbp.DampingNet(p)
    l1, g1 = net.gradient(Xd.data_ptr(), td.data_ptr(), 3000)
    l2, g2 = net.gradient(Xd.data_ptr(), td.data_ptr(), 3000)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)
    net.close()


def test_first_adam_step_matches_reference(torch):
    """Adam's first step moves each parameter by lr * g / (|g| + eps), i.e.
    by +-lr wherever the gradient is clearly non-zero."""
    p = _params(5)
    X, t = _data(11, 2048)
    lr = 1e-3
    net = gbp.DampingNet(p)
    Xd, td = _dev(torch, X), _dev(torch, t)
    net.train_step(Xd.data_ptr(), td.data_ptr(), 2048, lr)
    p1 = net.params.astype(np.float64)
    _, rg = mlp.loss_and_grad(p, X.astype(np.float64), t.astype(np.float64))
    rp1, _, _ = mlp.adam_step(p, rg, np.zeros_like(p), np.zeros_like(p), 1, lr)
    d, rd = p1 - p, rp1 - p
    assert np.abs(d - rd).max() <= 2.0 * lr * (1 + 1e-3)
    clear = np.abs(rg) > 1e-3 * np.abs(rg).max()
    agree = np.abs(d[clear] - rd[clear]) <= 1e-2 * lr
    assert agree.mean() >= 0.95, agree.mean()
    net.close()


def test_training_fits_a_teacher_network(torch):
    """Regression onto a teacher network's outputs: the loss falls by more
    than 10x in 600 Adam steps on minibatches given by index."""
    teacher = _params(6)
    X, _ = _data(13, 16384)
    t, _ = mlp.forward(teacher, X.astype(np.float64))
    t = t.astype(np.float32)
    Xd, td = _dev(torch, X), _dev(torch, t)
    net = gbp.DampingNet(mlp.init_params(7))
    loss0, _ = net.gradient(Xd.data_ptr(), td.data_ptr(), 16384)
    gen = torch.Generator(device="cpu").manual_seed(0)
    for _ in range(600):
        idx = torch.randint(0, 16384, (512,), generator=gen, dtype=torch.int32).cuda()
        net.train_step(Xd.data_ptr(), td.data_ptr(), 512, 3e-3, idx_ptr=idx.data_ptr())
    loss1, _ = net.gradient(Xd.data_ptr(), td.data_ptr(), 16384)
    assert loss1 < loss0 / 10, (loss0, loss1)
    net.close()


def test_indexed_minibatch_equals_gathered_rows(torch):
    p = _params(8)
    X, t = _data(15, 1000)
    idx = np.random.default_rng(3).permutation(1000)[:300].astype(np.int32)
    a = gbp.DampingNet(p)
    b = gbp.DampingNet(p)
    Xd, td, idxd = _dev(torch, X), _dev(torch, t), _dev(torch, idx)
    Xg, tg = _dev(torch, X[idx]), _dev(torch, t[idx])
    la = a.train_step(Xd.data_ptr(), td.data_ptr(), 300, 1e-3, idx_ptr=idxd.data_ptr(), want_loss=True)
    lb = b.train_step(Xg.data_ptr(), tg.data_ptr(), 300, 1e-3, want_loss=True)
    assert la == lb
    np.testing.assert_array_equal(a.params, b.params)
    a.close()
    b.close()


def test_invalid_arguments(torch):
    p = mlp.init_params(0).astype(np.float32)
    bad = p.copy()
    bad[17] = np.nan
    with pytest.raises(gbp.GBPError):
        gbp.DampingNet(bad)
    net = gbp.DampingNet(p)
    X, t = _data(0, 4)
    Xd, td = _dev(torch, X), _dev(torch, t)
    with pytest.raises(gbp.GBPError):
        net.gradient(Xd.data_ptr(), td.data_ptr(), 0)
    with pytest.raises(gbp.GBPError):
        net.train_step(Xd.data_ptr(), td.data_ptr(), 4, 0.0)
    with pytest.raises(gbp.GBPError):
        net.set_params(bad)
    net.forward(Xd.data_ptr(), 0, td.data_ptr())   # empty batch is a no-op
    np.testing.assert_array_equal(net.params, p)
    net.close()
