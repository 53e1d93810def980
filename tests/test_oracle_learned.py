"""Pins for the oracle's learned-damping schedule (no counterpart in the
paper: a per-factor d in place of the fixed d of Sec. 5 / Sec. 8).

Each pin rebuilds the quantity from other pieces: the network against the
numpy reference network; the 16 features from the oracle's public messages,
beliefs and linearisation; the damping targets by brute-force search over d;
the schedule through its special cases (a constant network is the fixed
schedule; damping never moves the linear fixed point; recording does not
change the iteration)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2003_03134_gb300 import synth


def _scaled_params(seed):
    p = mlp.unpack(mlp.init_params(seed))
    rng = np.random.default_rng(seed + 1)
    p["W3"] = rng.normal(0.0, 0.5, 64)
    p["b1"] = rng.normal(0.0, 0.2, 64)
    p["b2"] = rng.normal(0.0, 0.2, 64)
    return mlp.pack(p)


def test_network_matches_numpy_reference():
    p = _scaled_params(0)
    X = np.random.default_rng(1).normal(size=(100, 16))
    ref, _ = mlp.forward(p, X)
    got = np.array([oracle.net_forward(p, x) for x in X])
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


def _constant_net(d):
    p = mlp.unpack(mlp.init_params(2))
    p["W3"][:] = 0.0
    p["b3"][:] = np.log(d / (0.9 - d))
    return mlp.pack(p)


def test_constant_network_is_the_fixed_schedule():
    """W3 = 0 makes every d_f = 0.9 sigmoid(b3); the learned schedule then
    is the fixed one with that d (same undamped hold after relinearising)."""
    p = synth.make_walk(3, n_kf=15, n_lm=150)
    net = _constant_net(0.3)
    d = oracle.net_forward(net, np.zeros(16))
    assert abs(d - 0.3) < 1e-12
    a = oracle.Oracle(p, huber_nsigma=2.0, damping=d)
    b = oracle.Oracle(p, huber_nsigma=2.0, damping=d)
    b.set_damping_net(net)
    a.iterate(60)
    b.iterate(60)
    for x, y in zip(a.means(), b.means()):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-12)
    assert a.relinearisations() == b.relinearisations()


def test_learned_damping_keeps_the_linear_fixed_point():
    """Damping changes the path, never the fixed point (linear GBP).  Priors
    end at 1/10 of a measurement so that both runs converge in a few hundred
    iterations."""
    p = synth.make_walk(3, n_kf=10, n_lm=80)
    a = oracle.Oracle(p, linear=1, prior_final_scale=0.1)
    b = oracle.Oracle(p, linear=1, prior_final_scale=0.1)
    b.set_damping_net(_scaled_params(5))
    assert a.run_to_convergence(1e-11, 3000, chunk=20)[1] < 1e-11
    assert b.run_to_convergence(1e-11, 3000, chunk=20)[1] < 1e-11
    for x, y in zip(a.means(), b.means()):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-8)


def test_recording_does_not_change_the_iteration():
    p = synth.make_walk(4, n_kf=12, n_lm=120)
    a = oracle.Oracle(p, huber_nsigma=2.0)
    b = oracle.Oracle(p, huber_nsigma=2.0)
    b.capture_messages()
    a.iterate(25)
    b.iterate_record(25)
    for x, y in zip(a.means(), b.means()):
        np.testing.assert_array_equal(x, y)


def test_record_needs_a_reference():
    o = oracle.Oracle(synth.make_circle(0))
    with pytest.raises(RuntimeError):
        o.iterate_record(1)


def _brute_force_damping(sides):
    """argmin over a fine grid of d in [0, 0.9] of the sum over the sides
    (nw, old, ref) of |(1-d) nw + d old - ref|^2 / |old - nw|^2."""
    grid = np.linspace(0.0, 0.9, 9001)
    total = np.zeros_like(grid)
    for nw, old, ref in sides:
        cand = (1.0 - grid)[:, None] * nw[None, :] + grid[:, None] * old[None, :]
        total += ((cand - ref[None, :]) ** 2).sum(axis=1) / ((old - nw) @ (old - nw))
    return grid[np.argmin(total)]


def test_features_and_targets_from_public_pieces():
    """Linear mode (every factor linearised at the initial point, t_lin = 0)
    with damping from the second iteration on: the undamped new messages are
    recovered from two consecutive message snapshots, and every feature and
    target is recomputed from them."""
    p = synth.make_walk(5, n_kf=12, n_lm=100)
    prm = dict(linear=1, undamped_iters=1, huber_nsigma=2.0)
    d = oracle.DEFAULTS["damping"]
    ref = oracle.Oracle(p, **prm)
    ref.run_to_convergence(1e-10, 3000, chunk=20)
    _, rk, _, rl = ref.messages()
    o = oracle.Oracle(p, **prm)
    o.set_reference_messages(rk, rl)

    nf = p.n_obs
    Rt = p.kf_Rt_init
    M = np.zeros(nf)
    k = np.zeros(nf)
    cam = (p.fx, p.fy, p.cx, p.cy)
    for f in range(nf):
        R = Rt[p.obs_kf[f], :9].reshape(3, 3)
        c = -R.T @ Rt[p.obs_kf[f], 9:]
        lin = oracle.linearise(cam, R.ravel(), c, p.lm_init[p.obs_lm[f]], np.zeros(6), np.zeros(3),
                               p.obs_uv[f], **prm)
        if lin["active"]:
            M[f] = np.linalg.norm(lin["r"])
            k[f] = lin["k"]
    assert (k < 1).any(), "the case should exercise the Huber weight"
    deg_k = np.bincount(p.obs_kf, minlength=p.n_kf)[p.obs_kf]
    deg_l = np.bincount(p.obs_lm, minlength=p.n_lm)[p.obs_lm]

    def rel(a, b):
        return np.linalg.norm(a - b, axis=1) / (np.linalg.norm(a, axis=1) + np.linalg.norm(b, axis=1) + 1e-30)

    def cos(a, b):
        return (a * b).sum(axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1) + 1e-30)

    hist = np.zeros((nf, 4))
    ek_prev, el_prev = np.zeros((nf, 6)), np.zeros((nf, 3))
    n_checked = 0
    for t in range(12):
        lk0, ek0, ll0, el0 = o.messages()
        bkl, _, bll, _ = o.beliefs()
        X, T = o.iterate_record(1)
        X, T = X[0], T[0]
        lk1, ek1, ll1, el1 = o.messages()
        dd = d if t >= 1 else 0.0
        nk = (ek1 - dd * ek0) / (1.0 - dd)
        nl = (el1 - dd * el0) / (1.0 - dd)
        tr_lk = np.trace(lk1, axis1=1, axis2=2)
        tr_ll = np.trace(ll1, axis1=1, axis2=2)
        tr_pk = np.trace(bkl[p.obs_kf] - lk0, axis1=1, axis2=2)
        tr_pl = np.trace(bll[p.obs_lm] - ll0, axis1=1, axis2=2)
        ck, cm = rel(nk, ek0), rel(nl, el0)
        want = np.zeros((nf, 16))
        want[:, 0] = np.log1p(M) / 3.0
        want[:, 1] = k
        want[:, 2] = tr_lk / (tr_lk + tr_pk + 1e-30)
        want[:, 3] = tr_ll / (tr_ll + tr_pl + 1e-30)
        # keyframe-side step cosine: only once the three messages share one
        # linearisation (t - t_lin >= 2; linear mode: t_lin = 0)
        want[:, 4], want[:, 5:7] = ck, hist[:, 0:2]
        want[:, 7] = cos(nk - ek0, ek0 - ek_prev) if t >= 2 else 0.0
        want[:, 8], want[:, 9:11], want[:, 11] = cm, hist[:, 2:4], cos(nl - el0, el0 - el_prev)
        want[:, 12] = np.log1p(deg_k) / 5.0
        want[:, 13] = np.log1p(deg_l) / 3.0
        want[:, 14] = min(t, 50) / 50.0
        want[:, 15] = min(t, 50) / 50.0
        np.testing.assert_allclose(X, want, rtol=0, atol=1e-7)
        hist = np.stack([ck, hist[:, 0], cm, hist[:, 2]], axis=1)
        ek_prev, el_prev = ek0, el0

        for f in range(nf):
            if t == 0 or k[f] == 0.0:
                assert T[f] == -1.0
                continue
            sides = []
            for nw, old, r in ((nk[f], ek0[f], rk[f]), (nl[f], el0[f], rl[f])):
                u = old - nw
                if u @ u > 1e-10 * (nw @ nw + old @ old):
                    sides.append((nw, old, r))
            expect = _brute_force_damping(sides) if sides else -1.0
            assert abs(T[f] - expect) <= 2e-4, (t, f, T[f], expect)
            n_checked += 1
    assert n_checked > 1000
