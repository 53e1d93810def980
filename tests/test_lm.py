"""The CPU Levenberg-Marquardt bundle adjuster (dense Schur complement), the
comparison baseline: pinned against the oracle's GBP on the objective both
minimise.  (CPU only.)"""
import numpy as np
import pytest

import oracle
from paper_2003_03134_gb300 import synth
from paper_2003_03134_gb300.lm import LM, reprojection_error


@pytest.mark.parametrize("make", [lambda: synth.make_circle(1, n_kf=5, n_lm=25),
                                  lambda: synth.make_circle(0)])
def test_lm_optimum_is_the_gbp_fixed_point(make):
    """With the quadratic loss, relinearised GBP's fixed point is the
    stationary point of the objective (Sec. 4, eq. residuals; the oracle's
    Gauss-Newton pin) -- the optimum LM reaches by a different route."""
    p = make()
    lm = LM(p)
    lm.solve(200)
    assert lm.converged
    kf, lx = lm.world()
    o = oracle.Oracle(p, relin_beta=0.0, relin_interval=10)
    _, d = o.run_to_convergence(1e-12, 20000, chunk=10)
    assert d < 1e-11
    okf, olm = o.world()
    np.testing.assert_allclose(kf, okf, atol=1e-7)
    np.testing.assert_allclose(lx, olm, atol=1e-7)
    assert reprojection_error(p, kf, lx) == pytest.approx(o.are()[0], abs=1e-9)


def test_lm_cost_decreases_every_iteration():
    p = synth.make_walk(2, n_kf=15, n_lm=150)
    lm = LM(p, huber_nsigma=2.0)
    costs = [lm.cost]
    while not lm.converged and lm.iterations < 50:
        lm.step(1)
        costs.append(lm.cost)
    assert np.all(np.diff(costs) <= 0)
    assert costs[-1] < 0.5 * costs[0]


def test_lm_with_huber_down_weights_outliers():
    """Sec. 6: with 5% uniform outlier pixels, the Huber loss keeps the inlier
    error near the noise level where the quadratic loss does not."""
    p = synth.make_walk(3, n_kf=20, n_lm=250, outlier_frac=0.05)
    res = {}
    for n in (0.0, 2.0):
        lm = LM(p, huber_nsigma=n)
        lm.solve(100)
        res[n] = reprojection_error(p, *lm.world(), mask=~p.obs_outlier)
    assert res[2.0] < 1.5 < res[0.0] or res[2.0] < 0.8 * res[0.0]
