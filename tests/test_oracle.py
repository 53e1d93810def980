"""Pins for the FP64 oracle, each against something other than the oracle:
library rotations, finite differences, covariance-form Gaussian marginals,
dense linear solves, ground truth on noise-free data and constants the paper
prints.  (CPU only.)"""
import copy
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2003_03134_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cam(p):
    return (p.fx, p.fy, p.cx, p.cy)


def _refs(p):
    R = p.kf_Rt_init[:, :9].reshape(-1, 3, 3)
    t = p.kf_Rt_init[:, 9:]
    C = -np.einsum("kji,kj->ki", R, t)
    return R, C, p.lm_init


# ---------------------------------------------------------------- rotations

@pytest.mark.parametrize("scale", [0.0, 1e-7, 1e-5, 1e-3, 0.3, 2.5])
def test_so3_exp_matches_library(scale):
    rng = np.random.default_rng(0)
    for _ in range(5):
        w = rng.normal(size=3) * scale
        np.testing.assert_allclose(oracle.so3_exp(w), Rotation.from_rotvec(w).as_matrix(), atol=1e-14)


@pytest.mark.parametrize("scale", [1e-6, 1e-3, 0.4, 2.0])
def test_left_jacobian_first_order(scale):
    rng = np.random.default_rng(1)
    w = rng.normal(size=3) * scale
    J = oracle.so3_left_jacobian(w)
    R = Rotation.from_rotvec(w).as_matrix()
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        # Exp(w + e) Exp(w)^T = Exp(Jl e) to first order
        D = Rotation.from_rotvec(w + e).as_matrix() @ R.T
        D2 = Rotation.from_rotvec(w - e).as_matrix() @ R.T
        v = (Rotation.from_matrix(D).as_rotvec() - Rotation.from_matrix(D2).as_rotvec()) / (2 * h)
        np.testing.assert_allclose(v, J[:, i], atol=1e-8)


# ------------------------------------------------------------ measurement

def test_projection_matches_pose_convention():
    p = synth.make_circle(0)
    R, C, L = _refs(p)
    rng = np.random.default_rng(2)
    for f in range(0, p.n_obs, 37):
        k, m = p.obs_kf[f], p.obs_lm[f]
        # at the reference: pi(R l + t) straight from the world pose
        Rt = p.kf_Rt_init[k]
        pc = Rt[:9].reshape(3, 3) @ p.lm_init[m] + Rt[9:]
        uv0 = np.array([p.fx * pc[0] / pc[2] + p.cx, p.fy * pc[1] / pc[2] + p.cy])
        uv, depth = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], np.zeros(6), np.zeros(3))
        np.testing.assert_allclose(uv, uv0, rtol=1e-12)
        assert depth == pytest.approx(pc[2])
        # perturbed chart: R = Exp(dw) Rref, c = cref + dc, l = lref + dl
        xk = rng.normal(0, 0.05, 6)
        xl = rng.normal(0, 0.05, 3)
        Rn = Rotation.from_rotvec(xk[3:]).as_matrix() @ R[k]
        pc = Rn @ (L[m] + xl - C[k] - xk[:3])
        uv1 = np.array([p.fx * pc[0] / pc[2] + p.cx, p.fy * pc[1] / pc[2] + p.cy])
        uv, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], xk, xl)
        np.testing.assert_allclose(uv, uv1, rtol=1e-12)


def test_jacobian_matches_finite_differences():
    p = synth.make_walk(0, n_kf=20, n_lm=50)
    R, C, L = _refs(p)
    rng = np.random.default_rng(3)
    for f in range(0, p.n_obs, 13):
        k, m = p.obs_kf[f], p.obs_lm[f]
        x = np.concatenate([rng.normal(0, 0.05, 6), rng.normal(0, 0.05, 3)])
        lin = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], x[:6], x[6:], p.obs_uv[f])
        assert lin["active"]
        Jfd = np.zeros((2, 9))
        h = 1e-6
        for i in range(9):
            xp, xm = x.copy(), x.copy()
            xp[i] += h
            xm[i] -= h
            up, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], xp[:6], xp[6:])
            um, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], xm[:6], xm[6:])
            Jfd[:, i] = (up - um) / (2 * h)
        np.testing.assert_allclose(lin["J"], Jfd, rtol=1e-6, atol=1e-6 * np.abs(Jfd).max())
        uv, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], x[:6], x[6:])
        np.testing.assert_allclose(lin["r"], p.obs_uv[f] - uv, rtol=1e-12, atol=1e-9)


def test_information_form_encodes_the_linearised_residual():
    """-1/2 x^T A x + c^T x must equal -1/2 W |r0 - J (x - x0)|^2 up to a
    constant: a sign or term error in eta = J^T W (J x0 + r) breaks it."""
    p = synth.make_circle(0)
    R, C, L = _refs(p)
    rng = np.random.default_rng(4)
    for f in range(0, p.n_obs, 51):
        k, m = p.obs_kf[f], p.obs_lm[f]
        x0 = rng.normal(0, 0.05, 9)
        lin = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], x0[:6], x0[6:], p.obs_uv[f], sigma_px=1.5)
        W = lin["k"] / 1.5 ** 2

        def e_info(x):
            return -0.5 * x @ lin["A"] @ x + lin["c"] @ x

        def e_res(x):
            d = lin["r"] - lin["J"] @ (x - x0)
            return -0.5 * W * d @ d

        xs = [rng.normal(0, 0.1, 9) for _ in range(3)]
        a = [e_info(x) - e_info(xs[0]) for x in xs[1:]]
        b = [e_res(x) - e_res(xs[0]) for x in xs[1:]]
        np.testing.assert_allclose(a, b, rtol=1e-9)
        assert np.linalg.matrix_rank(lin["A"], tol=1e-9 * np.abs(lin["A"]).max()) == 2


def test_factor_behind_camera_is_inactive():
    p = synth.make_circle(0)
    R, C, L = _refs(p)
    k, m = p.obs_kf[0], p.obs_lm[0]
    # move the landmark to the camera centre: depth 0 < z_min
    xl = C[k] - L[m]
    lin = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], np.zeros(6), xl, p.obs_uv[0])
    assert not lin["active"]
    assert np.all(lin["A"] == 0) and np.all(lin["c"] == 0)


# ------------------------------------------------------------------ Huber

def test_huber_weight_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["huber_example"]
    assert oracle.huber_weight(g["M"], g["nsigma"]) == pytest.approx(g["weight"], abs=1e-15)
    N = 2.0
    assert oracle.huber_weight(N, N) == 1.0
    assert oracle.huber_weight(0.3, N) == 1.0
    assert oracle.huber_weight(50.0, 0.0) == 1.0          # disabled
    for M in [2.0001, 3.0, 10.0, 1e3]:
        k = oracle.huber_weight(M, N)
        # Sec. 6: rescaled quadratic cost equals the Huber cost 2 N M - N^2
        assert k * M * M == pytest.approx(2 * N * M - N * N, rel=1e-12)
        assert 0.0 < k < 1.0


def test_huber_weight_enters_information():
    p = synth.make_walk(0, n_kf=20, n_lm=50)
    R, C, L = _refs(p)
    f = int(np.nonzero(p.obs_outlier)[0][0]) if p.obs_outlier.any() else 0
    k, m = p.obs_kf[f], p.obs_lm[f]
    z = p.obs_uv[f] + np.array([40.0, -30.0])
    a = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], np.zeros(6), np.zeros(3), z, huber_nsigma=0.0)
    b = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], np.zeros(6), np.zeros(3), z, huber_nsigma=2.0)
    M = np.linalg.norm(a["r"])
    assert b["k"] == pytest.approx(2 * 2.0 / M - 4.0 / M ** 2)
    np.testing.assert_allclose(b["A"], b["k"] * a["A"], rtol=1e-12)
    np.testing.assert_allclose(b["c"], b["k"] * a["c"], rtol=1e-12)


# ------------------------------------------------------- messages (P4)

@pytest.mark.parametrize("target", [0, 1])
def test_schur_message_equals_covariance_form_marginal(target):
    rng = np.random.default_rng(5 + target)
    J = rng.normal(size=(2, 9))
    A = J.T @ J * 3.0
    c = rng.normal(size=9)
    nb = 3 if target == 0 else 6
    G = rng.normal(size=(nb, nb))
    lam_in = G @ G.T + nb * np.eye(nb)
    eta_in = rng.normal(size=nb)
    lam_out, eta_out = oracle.factor_message(A, c, target, lam_in, eta_in)
    # joint of factor x incoming message, in covariance form
    a_idx = np.arange(0, 6) if target == 0 else np.arange(6, 9)
    b_idx = np.arange(6, 9) if target == 0 else np.arange(0, 6)
    Lj = A.copy()
    Lj[np.ix_(b_idx, b_idx)] += lam_in
    ej = c.copy()
    ej[b_idx] += eta_in
    # A is rank 2, so add a weak prior on block a to make the joint proper;
    # the marginal's information then carries the same prior.
    prior = 0.7 * np.eye(a_idx.size)
    Lj[np.ix_(a_idx, a_idx)] += prior
    Sigma = np.linalg.inv(Lj)
    mu = Sigma @ ej
    Saa = Sigma[np.ix_(a_idx, a_idx)]
    lam_marg = np.linalg.inv(Saa)
    eta_marg = lam_marg @ mu[a_idx]
    np.testing.assert_allclose(lam_out + prior, lam_marg, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(eta_out, eta_marg, rtol=1e-9, atol=1e-9)


# --------------------------------------------------------------- priors

def test_prior_schedule_matches_paper_constants():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    T = g["prior_anneal_iters"]["value"]
    s_end = g["prior_final_scale"]["value"]
    s = [oracle.prior_scale(t, prior_anneal_iters=T, prior_final_scale=s_end) for t in range(T + 5)]
    assert s[0] == 1.0
    assert s[T] == pytest.approx(s_end, rel=1e-14)
    assert all(v == pytest.approx(s_end, rel=1e-14) for v in s[T:])
    ratios = [s[t + 1] / s[t] for t in range(T)]
    np.testing.assert_allclose(ratios, ratios[0], rtol=1e-12)   # geometric
    assert oracle.prior_scale(3, prior_anneal_iters=0, prior_final_scale=s_end) == s_end
    assert oracle.DEFAULTS["damping"] == g["damping"]["value"]
    assert oracle.DEFAULTS["relin_beta"] == g["relin_beta"]["value"]
    assert oracle.DEFAULTS["relin_interval"] == g["relin_interval"]["value"]
    assert oracle.DEFAULTS["undamped_iters"] == g["undamped_iters"]["value"]


def test_prior_diagonal_from_finite_difference_jacobians():
    p = synth.make_circle(0, n_kf=5, n_lm=20)
    o = oracle.Oracle(p)
    Dk, Dl = o.prior_diag()
    R, C, L = _refs(p)
    sk, sl = np.zeros((p.n_kf, 6)), np.zeros((p.n_lm, 3))
    nk, nl = np.zeros(p.n_kf), np.zeros(p.n_lm)
    h = 1e-6
    for f in range(p.n_obs):
        k, m = p.obs_kf[f], p.obs_lm[f]
        Jfd = np.zeros((2, 9))
        for i in range(9):
            xp, xm = np.zeros(9), np.zeros(9)
            xp[i], xm[i] = h, -h
            up, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], xp[:6], xp[6:])
            um, _ = oracle.project(_cam(p), R[k].ravel(), C[k], L[m], xm[:6], xm[6:])
            Jfd[:, i] = (up - um) / (2 * h)
        d = (Jfd ** 2).sum(axis=0)
        sk[k] += d[:6]
        sl[m] += d[6:]
        nk[k] += 1
        nl[m] += 1
    np.testing.assert_allclose(Dk, sk / nk[:, None], rtol=1e-6)
    np.testing.assert_allclose(Dl, sl / nl[:, None], rtol=1e-6)
    # b^0 = prior at scale 1 (plus anchor), mean 0
    kl, ke, ll, le = o.beliefs()
    np.testing.assert_allclose(np.diagonal(kl[1]), Dk[1], rtol=1e-14)
    np.testing.assert_allclose(np.diagonal(kl[0]), Dk[0] * (1 + 1e3), rtol=1e-14)
    assert np.all(ke == 0) and np.all(le == 0)


# ---------------------------------------------------- dense references

def _dense_system(p, o, prior_scale, anchor_scale=1e3):
    """H x = b of the linearised problem at the chart origin, assembled from
    the oracle's per-factor (A, c) at x0 = 0 plus the prior diagonals."""
    R, C, L = _refs(p)
    nk = p.n_kf
    N = 6 * nk + 3 * p.n_lm
    Dk, Dl = o.prior_diag()
    H = np.zeros((N, N))
    b = np.zeros(N)
    P = prior_scale * np.concatenate([Dk.ravel(), Dl.ravel()])
    for a in p.anchor_kf:
        P[6 * a:6 * a + 6] += anchor_scale * Dk[a]
    H[np.diag_indices(N)] += P
    for f in range(p.n_obs):
        k, m = p.obs_kf[f], p.obs_lm[f]
        lin = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], np.zeros(6), np.zeros(3), p.obs_uv[f],
                               **{kk: o.params[kk] for kk in ("huber_nsigma", "sigma_px", "z_min")})
        idx = np.r_[6 * k:6 * k + 6, 6 * nk + 3 * m:6 * nk + 3 * m + 3]
        H[np.ix_(idx, idx)] += lin["A"]
        b[idx] += lin["c"]
    return H, b


def test_tree_is_exact_for_means_and_covariances():
    """P1: on a loop-free graph, linear GBP reaches the exact marginals
    (means and covariances) after a diameter's worth of iterations (Sec. 3.2)."""
    p = synth.make_chain(4)
    o = oracle.Oracle(p, linear=1, damping=0.0, prior_anneal_iters=0, prior_final_scale=0.01)
    o.iterate(20)
    H, b = _dense_system(p, o, 0.01)
    x = np.linalg.solve(H, b)
    Sigma = np.linalg.inv(H)
    kf, lm = o.means()
    nk = p.n_kf
    np.testing.assert_allclose(np.concatenate([kf.ravel(), lm.ravel()]), x, rtol=1e-9, atol=1e-12)
    kl, _, ll, _ = o.beliefs()
    for v in range(nk):
        np.testing.assert_allclose(np.linalg.inv(kl[v]), Sigma[6 * v:6 * v + 6, 6 * v:6 * v + 6], rtol=1e-7,
                                   atol=1e-9 * np.abs(Sigma).max())
    for v in range(p.n_lm):
        i = 6 * nk + 3 * v
        np.testing.assert_allclose(np.linalg.inv(ll[v]), Sigma[i:i + 3, i:i + 3], rtol=1e-7,
                                   atol=1e-9 * np.abs(Sigma).max())


@pytest.mark.parametrize("damping", [0.0, 0.4])
def test_loopy_linear_means_equal_dense_solve(damping):
    """P2: on a loopy graph linear GBP means converge to the exact solve
    (Sec. 3.2, Weiss and Freeman); damping never moves the fixed point."""
    p = synth.make_circle(0, n_kf=4, n_lm=12)
    o = oracle.Oracle(p, linear=1, damping=damping, prior_anneal_iters=0, prior_final_scale=0.01)
    it, d = o.run_to_convergence(1e-15, 40000, chunk=100)
    assert d < 1e-12
    H, b = _dense_system(p, o, 0.01)
    x = np.linalg.solve(H, b)
    kf, lm = o.means()
    np.testing.assert_allclose(np.concatenate([kf.ravel(), lm.ravel()]), x, rtol=1e-7, atol=1e-9)


def test_nonlinear_fixed_point_is_gauss_newton_stationary():
    """P3: relinearised GBP stops where one Gauss-Newton step of the full
    objective (Sec. 4, eq. residuals) with the final priors is zero."""
    p = synth.make_circle(1, n_kf=5, n_lm=25)
    o = oracle.Oracle(p, relin_beta=0.0, relin_interval=10)
    it, d = o.run_to_convergence(1e-14, 40000, chunk=10)
    assert d < 1e-12
    kf, lm = o.means()
    x = np.concatenate([kf.ravel(), lm.ravel()])
    R, C, L = _refs(p)
    nk = p.n_kf
    N = x.size
    Dk, Dl = o.prior_diag()
    P = 0.01 * np.concatenate([Dk.ravel(), Dl.ravel()])
    for a in p.anchor_kf:
        P[6 * a:6 * a + 6] += 1e3 * Dk[a]
    H = np.diag(P)
    g = -P * x
    for f in range(p.n_obs):
        k, m = p.obs_kf[f], p.obs_lm[f]
        lin = oracle.linearise(_cam(p), R[k].ravel(), C[k], L[m], kf[k], lm[m], p.obs_uv[f])
        idx = np.r_[6 * k:6 * k + 6, 6 * nk + 3 * m:6 * nk + 3 * m + 3]
        H[np.ix_(idx, idx)] += lin["A"]
        g[idx] += lin["k"] * lin["J"].T @ lin["r"]
    step = np.linalg.solve(H, g)
    assert np.abs(step).max() < 1e-8
    assert N == 6 * nk + 3 * p.n_lm


def test_information_matrices_symmetric_psd():
    """P5: messages and beliefs stay symmetric positive (semi)definite."""
    p = synth.make_walk(0, n_kf=15, n_lm=120)
    o = oracle.Oracle(p, huber_nsigma=2.0)
    o.iterate(40)
    mk, _, ml, _ = o.messages()
    kl, _, ll, _ = o.beliefs()
    for M in (mk, ml):
        np.testing.assert_allclose(M, np.swapaxes(M, 1, 2), rtol=1e-10, atol=1e-9 * np.abs(M).max())
        ev = np.linalg.eigvalsh(M)
        assert (ev[:, 0] >= -1e-10 * np.maximum(ev[:, -1], 1)).all()
    for M in (kl, ll):
        assert (np.linalg.eigvalsh(M)[:, 0] > 0).all()


def test_noise_free_problem_recovers_ground_truth():
    """P7: exact measurements + fixed scale (two anchored keyframes at their
    true poses) + vanishing priors: the MAP is the ground truth."""
    p = synth.make_circle(2, noise_px=0.0, rot_sigma=0.01, pos_sigma=0.02, lm_sigma=0.03, anchors=(0, 1))
    o = oracle.Oracle(p, prior_final_scale=1e-7, relin_beta=0.0)
    o.iterate(1500)
    kf, lm = o.world()
    np.testing.assert_allclose(lm, p.lm_true, atol=2e-6)
    np.testing.assert_allclose(kf, p.kf_Rt_true, atol=2e-6)
    assert o.are()[0] < 1e-3


def test_are_definition():
    p = synth.make_circle(0)
    o = oracle.Oracle(p)
    are, n = o.are()
    pc = np.einsum("nij,nj->ni", p.kf_Rt_init[p.obs_kf, :9].reshape(-1, 3, 3), p.lm_init[p.obs_lm]) \
        + p.kf_Rt_init[p.obs_kf, 9:]
    uv = np.stack([p.fx * pc[:, 0] / pc[:, 2] + p.cx, p.fy * pc[:, 1] / pc[:, 2] + p.cy], axis=1)
    assert n == p.n_obs
    assert are == pytest.approx(np.linalg.norm(uv - p.obs_uv, axis=1).mean(), rel=1e-12)
    v, _ = o.are_vs(p.kf_Rt_init, p.lm_init)
    assert v == pytest.approx(0.0, abs=1e-9)
    q = copy.deepcopy(p)
    q.obs_uv = uv
    assert oracle.Oracle(q).are()[0] == pytest.approx(0.0, abs=1e-9)


def test_circle_converges_near_optimum():
    p = synth.make_circle(0)
    o = oracle.Oracle(p)
    o.iterate(200)
    are, _ = o.are()
    # 1 px noise: the optimum reprojection error is about sigma sqrt(pi/2) ~ 1.2 px less the fitted dof
    assert 0.8 < are < 1.2


def test_invalid_input_rejected():
    p = synth.make_circle(0, n_kf=4, n_lm=10)
    q = copy.deepcopy(p)
    q.obs_kf = q.obs_kf.copy()
    q.obs_kf[0] = 99
    with pytest.raises(ValueError):
        oracle.Oracle(q)


def test_relinearisation_threshold_never_met_equals_linear_mode():
    """Sec. 5: a factor relinearises only when the adjacent beliefs moved more
    than beta from its linearisation point; beta = infinity is linear GBP."""
    p = synth.make_circle(0, n_kf=5, n_lm=20)
    a = oracle.Oracle(p, relin_beta=1e30)
    b = oracle.Oracle(p, linear=1)
    a.iterate(60)
    b.iterate(60)
    for x, y in zip(a.means(), b.means()):
        np.testing.assert_array_equal(x, y)


# ------------------------------------------------ schedule (Sec. 5, Sec. 8)
#
# The relinearisation gate, the undamped hold after a (re)linearisation, the
# damping of eta only and the held-message rule are comparisons and branches:
# each pin below fails when one of them is flipped (< for <=), shifted by an
# iteration, or applied to the wrong quantity.

@pytest.mark.parametrize("hold", [0, 1, 3, 8])
def test_damping_starts_exactly_after_the_undamped_hold(hold):
    """Sec. 8: messages stay undamped for the first iterations after a
    (re)linearisation; the first message is never damped (nothing to damp
    towards).  In linear mode every factor is linearised at t = 0, so runs
    with d = 0 and d = 0.4 agree bit for bit for exactly max(hold, 1)
    iterations and part on the next."""
    p = synth.make_circle(0, n_kf=5, n_lm=30)
    n_same = max(hold, 1)
    a = oracle.Oracle(p, linear=1, damping=0.0, undamped_iters=hold)
    b = oracle.Oracle(p, linear=1, damping=0.4, undamped_iters=hold)
    a.iterate(n_same)
    b.iterate(n_same)
    for x, y in zip(a.means() + a.messages(), b.means() + b.messages()):
        np.testing.assert_array_equal(x, y)
    a.iterate(1)
    b.iterate(1)
    assert np.abs(a.means()[1] - b.means()[1]).max() > 1e-9
    # Lambda is never damped: the precision messages still agree
    np.testing.assert_array_equal(a.messages()[0], b.messages()[0])
    np.testing.assert_array_equal(a.messages()[2], b.messages()[2])


@pytest.mark.parametrize("interval,n_iters", [(10, 10), (10, 11), (10, 35), (7, 29), (7, 30), (1, 5)])
def test_relinearisation_count_with_beta_zero(interval, n_iters):
    """Sec. 5 / Sec. 8: with beta = 0 every factor relinearises as soon as the
    interval allows -- at t = interval, 2 interval, ... (iterations numbered
    from 0) -- so after N iterations the count is n_f * floor((N - 1) /
    interval) and every factor's t_lin is the last such multiple."""
    p = synth.make_circle(0, n_kf=5, n_lm=30)
    o = oracle.Oracle(p, relin_beta=0.0, relin_interval=interval)
    o.iterate(n_iters)
    k = (n_iters - 1) // interval
    assert o.relinearisations() == p.n_obs * k
    np.testing.assert_array_equal(o.relin_iters(), np.full(p.n_obs, k * interval))


def test_relinearisation_needs_movement_strictly_beyond_beta():
    """Sec. 5: a factor relinearises when its variables moved further than
    beta.  Measurements equal to the projections at the initial estimate
    leave every mean exactly at its chart origin, so even beta = 0 never
    triggers a relinearisation."""
    p = synth.make_circle(0, n_kf=5, n_lm=30)
    R, C, _ = _refs(p)
    q = copy.deepcopy(p)
    q.obs_uv = np.array([oracle.project(_cam(p), R[k].ravel(), C[k], p.lm_init[m], np.zeros(6), np.zeros(3))[0]
                         for k, m in zip(p.obs_kf, p.obs_lm)])
    o = oracle.Oracle(q, relin_beta=0.0)
    o.iterate(35)
    kf, lm = o.means()
    assert np.abs(kf).max() == 0.0 and np.abs(lm).max() == 0.0
    assert o.relinearisations() == 0
    np.testing.assert_array_equal(o.relin_iters(), 0)


def test_tree_covariances_exact_while_damped_means_are_not():
    """Sec. 5: damping acts on eta only, so on a tree the precisions still
    become exact after a diameter's worth of iterations (Sec. 3.2) while the
    damped means are still on their way."""
    p = synth.make_chain(4)
    kw = dict(linear=1, prior_anneal_iters=0, prior_final_scale=0.01, undamped_iters=1)
    o = oracle.Oracle(p, damping=0.4, **kw)
    o.iterate(8)
    H, b = _dense_system(p, o, 0.01)
    x = np.linalg.solve(H, b)
    Sigma = np.linalg.inv(H)
    nk = p.n_kf
    kl, _, ll, _ = o.beliefs()
    for v in range(nk):
        np.testing.assert_allclose(np.linalg.inv(kl[v]), Sigma[6 * v:6 * v + 6, 6 * v:6 * v + 6], rtol=1e-7,
                                   atol=1e-9 * np.abs(Sigma).max())
    for v in range(p.n_lm):
        i = 6 * nk + 3 * v
        np.testing.assert_allclose(np.linalg.inv(ll[v]), Sigma[i:i + 3, i:i + 3], rtol=1e-7,
                                   atol=1e-9 * np.abs(Sigma).max())
    kf, lm = o.means()
    err = np.abs(np.concatenate([kf.ravel(), lm.ravel()]) - x).max()
    assert err > 1e-6 * np.abs(x).max()
    # and undamped the means are exact by then too
    u = oracle.Oracle(p, damping=0.0, **kw)
    u.iterate(8)
    kf, lm = u.means()
    np.testing.assert_allclose(np.concatenate([kf.ravel(), lm.ravel()]), x, rtol=1e-9, atol=1e-12)


def test_message_with_indefinite_incoming_precision_is_held():
    """The Schur complement of Sec. 5 needs a positive definite incoming
    precision.  A hand-built state where one factor's incoming precision
    from its landmark is indefinite keeps that message at its previous
    value, counts it, and sends every other message normally."""
    p = synth.make_circle(0, n_kf=5, n_lm=30)
    o = oracle.Oracle(p, linear=1)
    o.iterate(3)
    mk, ek, ml, el = (a.copy() for a in o.messages())
    counts = np.bincount(p.obs_lm, minlength=p.n_lm)
    m = int(np.argmax(counts >= 2))
    f, g = np.flatnonzero(p.obs_lm == m)[:2]
    kl, _, ll, _ = o.beliefs()
    others = ll[m] - ml[f] - ml[g]                  # prior(t) + the remaining messages
    big = 1e3 * np.trace(ll[m])
    ml[f] = ml[f] + big * np.eye(3)                 # keeps the belief positive definite
    ml[g] = -others - 1e-3 * big * np.eye(3)        # f's incoming precision: others + ml[g] < 0
    o.set_messages(mk, ek, ml, el)
    inc = o.beliefs()[2][m] - ml[f]
    assert np.linalg.eigvalsh(inc)[0] < 0
    held0 = o.held_messages()
    o.iterate(1)
    assert o.held_messages() - held0 == 1
    mk1, ek1, ml1, el1 = o.messages()
    np.testing.assert_array_equal(mk1[f], mk[f])    # kept, not zeroed or recomputed
    np.testing.assert_array_equal(ek1[f], ek[f])
    changed = [h for h in range(p.n_obs) if h != f and not np.array_equal(mk1[h], mk[h])]
    assert len(changed) == p.n_obs - 1


def test_held_message_defers_its_factors_relinearisation():
    """A kept message is only meaningful with the linearisation it was formed
    at, so a factor holding a message does not relinearise in that
    iteration even when the schedule is due (beta = 0, t = interval): every
    other factor relinearises, the held one keeps t_lin = 0 and does so in
    the next iteration."""
    p = synth.make_circle(0, n_kf=5, n_lm=30)
    o = oracle.Oracle(p, relin_beta=0.0, relin_interval=10)
    o.iterate(10)
    mk, ek, ml, el = (a.copy() for a in o.messages())
    m = int(np.argmax(np.bincount(p.obs_lm, minlength=p.n_lm) >= 2))
    f, g = np.flatnonzero(p.obs_lm == m)[:2]
    ll = o.beliefs()[2]
    others = ll[m] - ml[f] - ml[g]
    big = 1e3 * np.trace(ll[m])
    ml[f] = ml[f] + big * np.eye(3)
    ml[g] = -others - 1e-3 * big * np.eye(3)
    o.set_messages(mk, ek, ml, el)
    o.iterate(1)
    tl = o.relin_iters()
    assert o.held_messages() == 1
    assert tl[f] == 0 and (np.delete(tl, f) == 10).all()
    assert o.relinearisations() == p.n_obs - 1


def test_openmp_build_gives_the_same_bits():
    """The OpenMP build (factors of an iteration and variables of a belief
    update in parallel, every sum in the same order) is the oracle itself:
    bit for bit the single-threaded results, relinearisations included."""
    if not oracle.omp_available():
        pytest.skip("no OpenMP compiler")
    p = synth.make_walk(1, n_kf=30, n_lm=400)
    a = oracle.Oracle(p, huber_nsigma=2.0)
    b = oracle.Oracle(p, huber_nsigma=2.0, omp=True)
    a.iterate(45)
    b.iterate(45)
    for x, y in zip(a.means() + a.messages(), b.means() + b.messages()):
        np.testing.assert_array_equal(x, y)
    assert a.relinearisations() == b.relinearisations() > 0


# ------------------------------------------------------- incremental (Sec. 9.2)

def test_added_keyframe_and_points_start_where_the_rule_puts_them():
    """Sec. 9.2 leaves the initial values of added variables to the front
    end; the rule here: the new keyframe at the latest keyframe's current
    estimate, each new point 1 m in front of it on the ray that first
    observes it."""
    p = synth.make_walk(2, n_kf=30, n_lm=500, smooth=True)
    init, steps = synth.stream_plan(p, 10)
    o = oracle.Oracle(init)
    o.iterate(25)
    # steps before the first one that brings new points
    n = 0
    while steps[n].n_new_lm == 0:
        o.add_keyframe(steps[n].obs_lm, steps[n].obs_uv, n_new_lm=0)
        o.iterate(5)
        n += 1
    kf_before, lm_before = o.world()
    n_lm0 = lm_before.shape[0]
    st = steps[n]
    k = o.add_keyframe(st.obs_lm, st.obs_uv, n_new_lm=st.n_new_lm)
    assert k == kf_before.shape[0] and st.n_new_lm > 0
    kf, lm = o.world()
    # new keyframe = the latest keyframe's current estimate; old variables untouched
    np.testing.assert_allclose(kf[k], kf_before[k - 1], atol=1e-12)
    np.testing.assert_allclose(kf[:k], kf_before, atol=0)
    np.testing.assert_allclose(lm[:n_lm0], lm_before, atol=0)
    R, t = kf[k, :9].reshape(3, 3), kf[k, 9:]
    for j in range(n_lm0, n_lm0 + st.n_new_lm):
        i = int(np.nonzero(st.obs_lm == j)[0][0])
        pc = R @ lm[j] + t
        assert pc[2] == pytest.approx(1.0, abs=1e-12)
        uv = np.array([p.fx * pc[0] / pc[2] + p.cx, p.fy * pc[1] / pc[2] + p.cy])
        np.testing.assert_allclose(uv, st.obs_uv[i], atol=1e-9)


def test_incremental_fixed_point_is_gauss_newton_stationary():
    """After keyframes are added and the graph converges, the means satisfy
    the Gauss-Newton stationarity of the grown problem (objective of Sec. 4
    with the priors at their final scale)."""
    p = synth.make_circle(5, n_kf=7, n_lm=30)
    init, steps = synth.stream_plan(p, 4)
    o = oracle.Oracle(init, relin_beta=0.0, relin_interval=10)
    o.iterate(20)
    for st in steps:
        o.add_keyframe(st.obs_lm, st.obs_uv, n_new_lm=st.n_new_lm,
                       new_lm_xyz=st.new_lm_true + 0.05 if st.n_new_lm else None)
        o.iterate(15)
    it, d = o.run_to_convergence(1e-14, 60000, chunk=10)
    assert d < 1e-12
    kf, lm = o.means()
    nk, nl, nf = o.sizes()
    # the grown graph's observations in the order the oracle stores them
    obs_kf = np.concatenate([init.obs_kf] + [np.full(st.obs_lm.size, init.n_kf + i) for i, st in enumerate(steps)])
    obs_lm = np.concatenate([init.obs_lm] + [st.obs_lm for st in steps])
    obs_uv = np.concatenate([init.obs_uv] + [st.obs_uv for st in steps])
    assert obs_kf.size == nf
    # references = initial values the oracle used
    Rw, lw = o.world()
    mu_k, mu_l = o.means()
    refs = []
    for v in range(nk):
        w = mu_k[v, 3:]
        Rv = Rw[v, :9].reshape(3, 3)
        Rref = Rotation.from_rotvec(w).as_matrix().T @ Rv
        cref = -Rv.T @ Rw[v, 9:] - mu_k[v, :3]
        refs.append((Rref, cref))
    lref = lw - mu_l
    Dk, Dl = o.prior_diag()
    x = np.concatenate([kf.ravel(), lm.ravel()])
    P = 0.01 * np.concatenate([Dk.ravel(), Dl.ravel()])
    for a in init.anchor_kf:
        P[6 * a:6 * a + 6] += 1e3 * Dk[a]
    H = np.diag(P)
    gvec = -P * x
    cam = _cam(p)
    for f in range(nf):
        k, m = obs_kf[f], obs_lm[f]
        lin = oracle.linearise(cam, refs[k][0].ravel(), refs[k][1], lref[m], kf[k], lm[m], obs_uv[f])
        idx = np.r_[6 * k:6 * k + 6, 6 * nk + 3 * m:6 * nk + 3 * m + 3]
        H[np.ix_(idx, idx)] += lin["A"]
        gvec[idx] += lin["k"] * lin["J"].T @ lin["r"]
    step = np.linalg.solve(H, gvec)
    assert np.abs(step).max() < 1e-7
