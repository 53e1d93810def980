"""Pins for the FP64 damping-network reference: gradients against central
finite differences, the output range, and Adam against its closed form on a
quadratic."""
import numpy as np
import pytest

from oracle import mlp


def _batch(seed, B=37):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, mlp.N_IN))
    t = rng.uniform(0.0, 0.9, B)
    return X, t


def test_parameter_count():
    assert mlp.N_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1
    p = mlp.init_params(0)
    assert p.size == mlp.N_PARAMS
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(p)), p)


def test_initial_output_is_the_papers_damping():
    p = mlp.unpack(mlp.init_params(3))
    p["W3"][:] = 0.0
    y, _ = mlp.forward(mlp.pack(p), np.random.default_rng(0).normal(size=(5, 16)))
    np.testing.assert_allclose(y, 0.4, rtol=1e-12)


def test_output_range():
    p = mlp.init_params(1) * 30.0
    y, _ = mlp.forward(p, np.random.default_rng(1).normal(size=(200, 16)) * 10)
    assert (y >= 0).all() and (y <= 0.9).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    p = mlp.init_params(seed)
    X, t = _batch(seed)
    loss, g = mlp.loss_and_grad(p, X, t)
    rng = np.random.default_rng(seed + 10)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp, _ = mlp.loss_and_grad(p + e, X, t)
        lm, _ = mlp.loss_and_grad(p - e, X, t)
        fd = (lp - lm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_adam_on_a_quadratic():
    """Adam's first step moves every coordinate by lr (bias-corrected m/sqrt(v)
    equals sign(g) on step 1)."""
    x = np.array([1.0, -2.0, 3.0])
    g = 2 * x
    x1, m, v = mlp.adam_step(x, g, np.zeros(3), np.zeros(3), 1, 0.1)
    np.testing.assert_allclose(x1, x - 0.1 * np.sign(g), rtol=1e-7)
