"""GPU learned damping (network inference fused into the factor kernel, the
record schedule's features and targets) against the FP64 oracle.

Parity has three parts.  (1) A constant network (W3 = 0) turns the learned
schedule into the fixed schedule with d = its output, which the oracle
computes exactly: FP32 tolerance as for fixed damping, TOL32 = 1e-5
relative per variable.  (2) The features and
targets recorded on the GPU against the oracle's, row by row: features to
2e-4 absolute (FP32 messages), targets to 0.02 where both messages clearly
changed (a target is a ratio of differences of messages, so FP32 rounding
of the messages shows up in it).  (3) A general network: the GPU's BF16
network differs from the oracle's FP64 one by up to ~0.01 in d, so the
trajectories agree loosely; the fixed point does not depend on damping, so
at convergence they agree to TOL32 again."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2003_03134_gb300 import build, gbp, learned, synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
DET = dict(relin_beta=0.0, relin_interval=10)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    gbp.lib()
    return t


def rel_err(kf, lm, okf, olm):
    ek = np.linalg.norm(kf - okf, axis=1) / np.maximum(np.linalg.norm(okf, axis=1), 1.0)
    el = np.linalg.norm(lm - olm, axis=1) / np.maximum(np.linalg.norm(olm, axis=1), 1.0)
    return np.concatenate([ek, el])


def constant_net(d):
    p = mlp.unpack(mlp.init_params(2))
    p["W3"][:] = 0.0
    p["b3"][:] = np.log(d / (0.9 - d))
    return mlp.pack(p)


def scaled_net(seed):
    p = mlp.unpack(mlp.init_params(seed))
    rng = np.random.default_rng(seed + 1)
    p["W3"] = rng.normal(0.0, 0.5, 64)
    p["b1"] = rng.normal(0.0, 0.2, 64)
    p["b2"] = rng.normal(0.0, 0.2, 64)
    return mlp.pack(p).astype(np.float32).astype(np.float64)


def gpu_output(torch, net, x=None):
    """The GPU network's prediction for one feature row."""
    X = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    if x is not None:
        X[0] = torch.from_numpy(np.asarray(x, dtype=np.float32))
    y = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.forward(X.data_ptr(), 1, y.data_ptr())
    torch.cuda.synchronize()
    return float(y.cpu()[0])


def test_learned_schedule_needs_a_network(torch):
    g = gbp.Graph(synth.make_circle(0), damping_mode=1)
    with pytest.raises(gbp.GBPError) as e:
        g.iterate(5)
    assert e.value.status == gbp.GBP_ESTATE
    with pytest.raises(gbp.GBPError):
        g.autotune(4)
    g.set_params(damping_mode=0)
    g.iterate(5)
    g.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_constant_network_matches_oracle(torch, mode):
    p = synth.make_walk(2, n_kf=25, n_lm=300)
    net = gbp.DampingNet(constant_net(0.3))
    d = gpu_output(torch, net)
    assert abs(d - 0.3) < 1e-3
    g = gbp.Graph(p, huber_nsigma=2.0, damping_mode=1, launch_mode=mode, **DET)
    g.set_damping_model(net)
    g.iterate(80)
    kf, lm = g.beliefs()
    st = g.stats()
    o = oracle.Oracle(p, huber_nsigma=2.0, damping=d, **DET)
    o.iterate(80)
    okf, olm = o.world()
    e = rel_err(kf, lm, okf, olm)
    assert e.max() <= TOL32, (e.max(), np.median(e))
    assert abs(st["are"] - o.are()[0]) <= 1e-3
    g.close()
    net.close()


def test_constant_network_fp64_matches_oracle_tightly(torch):
    p = synth.make_walk(3, n_kf=15, n_lm=150)
    net = gbp.DampingNet(constant_net(0.25))
    d = gpu_output(torch, net)
    g = gbp.Graph(p, huber_nsigma=2.0, damping_mode=1, precision_mode=2)
    g.set_damping_model(net)
    g.iterate(100)
    kf, lm = g.beliefs()
    o = oracle.Oracle(p, huber_nsigma=2.0, damping=d)
    o.iterate(100)
    okf, olm = o.world()
    assert rel_err(kf, lm, okf, olm).max() < 1e-8
    assert g.stats()["relinearisations"] == o.relinearisations()
    g.close()


def test_learned_launch_modes_are_bitwise_equal(torch):
    p = synth.make_walk(4, n_kf=30, n_lm=400)
    net = gbp.DampingNet(scaled_net(3))
    out = []
    for mode in (1, 2):
        g = gbp.Graph(p, huber_nsigma=2.0, damping_mode=1, launch_mode=mode)
        g.set_damping_model(net)
        g.iterate(45)
        out.append(g.beliefs())
        g.close()
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    net.close()


def test_general_network_tracks_oracle_and_shares_its_fixed_point(torch):
    p = synth.make_walk(3, n_kf=10, n_lm=80)
    w = scaled_net(5)
    net = gbp.DampingNet(w)
    prm = dict(linear=1, prior_final_scale=0.1)
    g = gbp.Graph(p, damping_mode=1, **prm)
    g.set_damping_model(net)
    o = oracle.Oracle(p, **prm)
    o.set_damping_net(w)
    g.iterate(30)
    o.iterate(30)
    e = rel_err(*g.beliefs(), *o.world())
    assert e.max() <= 1e-2 and np.median(e) <= 1e-3, (e.max(), np.median(e))
    g.iterate(2000)
    o.run_to_convergence(1e-11, 3000, chunk=20)
    e = rel_err(*g.beliefs(), *o.world())
    assert e.max() <= TOL32, e.max()
    g.close()
    net.close()


def _record_pair(torch, p, n_conv, n_rec, prm):
    g = gbp.Graph(p, **prm)
    g.iterate(n_conv)
    g.capture_messages()
    g.reset()
    nf = p.n_obs
    X = torch.full((n_rec, nf, 16), -7.0, dtype=torch.float32, device="cuda")
    T = torch.full((n_rec, nf), -7.0, dtype=torch.float32, device="cuda")
    g.record(n_rec, X.data_ptr(), T.data_ptr())
    torch.cuda.synchronize()
    order = g.factor_order()
    gX = np.empty((n_rec, nf, 16))
    gT = np.empty((n_rec, nf))
    gX[:, order] = X.cpu().numpy()
    gT[:, order] = T.cpu().numpy()
    kf, lm = g.beliefs()
    g.close()
    ref = oracle.Oracle(p, **prm)
    ref.iterate(n_conv)
    _, rk, _, rl = ref.messages()
    o = oracle.Oracle(p, **prm)
    o.set_reference_messages(rk, rl)
    oX, oT = o.iterate_record(n_rec)
    return gX, gT, oX, oT, (kf, lm), o.world()


def test_recorded_features_and_targets_match_oracle(torch):
    p = synth.make_walk(5, n_kf=20, n_lm=250)
    gX, gT, oX, oT, gw, ow = _record_pair(torch, p, 150, 20, dict(huber_nsigma=2.0, **DET))
    assert (gX != -7.0).all() and (gT != -7.0).all()
    err = np.abs(gX - oX)
    # every feature but the step cosines (7, 11) is compared everywhere.  A
    # cosine's error is about the messages' FP32 trajectory error (~1e-5 of
    # |eta|, the parity tolerance) over the step lengths: with both steps
    # above 1e-2 of |eta| it stays below ~2e-3
    plain = [j for j in range(16) if j not in (7, 11)]
    assert err[..., plain].max() <= 2e-4, np.unravel_index(err[..., plain].argmax(), err[..., plain].shape)
    for j, a, b in ((7, 4, 5), (11, 8, 9)):
        big = (oX[..., a] > 1e-2) & (oX[..., b] > 1e-2)
        assert big.sum() > 1000
        assert err[..., j][big].max() <= 5e-3, err[..., j][big].max()
        assert np.median(err[..., j][big]) <= 1e-4
    # recording runs the fixed schedule unchanged: bitwise the plain run's beliefs
    g = gbp.Graph(p, huber_nsigma=2.0, **DET)
    g.iterate(20)
    for a, b in zip(g.beliefs(), gw):
        np.testing.assert_array_equal(a, b)
    g.close()
    # targets never used by the learned schedule are flagged on both sides
    hold = oracle.DEFAULTS["undamped_iters"]
    never = (oX[..., 14] < hold / 50.0 - 1e-9) | (oX[..., 1] == 0.0)
    assert (oT[never] == -1.0).all() and (gT[never] == -1.0).all()
    clear = (oT >= 0) & (oX[..., 4] > 1e-2) & (oX[..., 8] > 1e-2)
    assert clear.sum() > 1000
    dT = np.abs(gT[clear] - oT[clear])
    assert dT.max() <= 0.02, dT.max()
    assert np.median(dT) <= 1e-3


def test_record_arguments(torch):
    p = synth.make_circle(0)
    g = gbp.Graph(p)
    X = torch.zeros((2, p.n_obs, 16), dtype=torch.float32, device="cuda")
    T = torch.zeros((2, p.n_obs), dtype=torch.float32, device="cuda")
    with pytest.raises(gbp.GBPError) as e:
        g.record(2, X.data_ptr(), T.data_ptr())
    assert e.value.status == gbp.GBP_ESTATE
    g.capture_messages()
    with pytest.raises(gbp.GBPError) as e:
        g.record(1, X.data_ptr() + 4, T.data_ptr())
    assert e.value.status == gbp.GBP_EINVAL
    g.record(2, X.data_ptr(), T.data_ptr())
    assert g.stats()["iterations"] == 2
    g.close()


@pytest.mark.parametrize("seed", [0, 2])
def test_trained_network_gain(torch, seed):
    """What the shipped network (trained on problems with seeds 10000-10999)
    gains on held-out paper-scale problems: fewer iterations to 0.01 px of
    average reprojection error against the converged solution, no more
    iterations to 0.1 px or 1 px, and the same final error."""
    net = gbp.DampingNet(learned.trained_params())
    r = learned.compare(torch, synth.make_walk(seed=seed), net)
    fx, lr = r["fixed"], r["learned"]
    print(seed, {k: (fx[k], lr[k]) for k in ("iters", "ms")})
    assert lr["iters"]["0.01"] <= 0.85 * fx["iters"]["0.01"]
    assert lr["iters"]["0.1"] <= fx["iters"]["0.1"]
    assert lr["iters"]["1.0"] <= fx["iters"]["1.0"]
    assert abs(lr["final"]["are"] - fx["final"]["are"]) <= 1e-2
    net.close()


def test_trained_network_reaches_the_fixed_damping_beliefs(torch):
    """Damping does not move the fixed point.  With relinearisation at every
    10th iteration (no threshold) the FP32 iteration ends in a small limit
    cycle -- relinearising at rounded means perturbs the weakly constrained
    points by ~1e-5 each period -- so the comparison is made at the same
    phase of that cycle and against its own amplitude: the learned end state
    lies within twice the fixed schedule's half-period drift (and at least
    within TOL32) of the fixed end state, with the same ARE to 1e-3 px.
    Priors end at 1/10 of a measurement (not 1/100) so that the weakly
    observed directions converge within the 4000 iterations."""
    p = synth.make_walk(1, n_kf=40, n_lm=600)
    net = gbp.DampingNet(learned.trained_params())
    fixed = gbp.Graph(p, huber_nsigma=2.0, prior_final_scale=0.1, **DET)
    fixed.iterate(4000)
    f_end = fixed.beliefs()
    f_are = fixed.stats()["are"]
    fixed.iterate(5)
    drift = rel_err(*fixed.beliefs(), *f_end).max()
    fixed.close()
    g = gbp.Graph(p, huber_nsigma=2.0, prior_final_scale=0.1, damping_mode=1, **DET)
    g.set_damping_model(net)
    g.iterate(4000)
    e = rel_err(*g.beliefs(), *f_end)
    assert e.max() <= max(TOL32, 2.0 * drift), (e.max(), drift)
    assert abs(g.stats()["are"] - f_are) <= 1e-3
    g.close()
    net.close()


def test_stream_learned_against_fixed():
    """The incremental stream (one keyframe every 20 iterations, growing to
    500 keyframes and ~8000 points; new keyframes at the latest pose, new
    points at 1 m along their first ray).  On the stream where both
    schedules keep tracking (seed 1: the error of the growing graph settles
    near the noise-and-outlier floor) the learned schedule keeps it at least
    as low as fixed d = 0.4 on most steps.  On the other seeds the 1 m depth
    of new points is far from their true depth (1-10 m) and is corrected only
    slowly from baselines of 8 cm per keyframe, the misplaced points pull the
    keyframes, and the graph drifts under either schedule, so no ordering is
    asserted there (test_streams_track_with_new_points_near_their_depth shows
    that the drift is the initialisation's)."""
    import torch
    init, steps = synth.make_stream(1)
    net = gbp.DampingNet(learned.trained_params())
    r = learned.stream_compare(torch, net, init, steps, per_step=20)
    fx, lr = r["fixed"], r["learned"]
    print({k: (fx[k], lr[k]) for k in ("mean_are", "final_are", "device_ms")})
    a, b = np.array(fx["are_per_step"]), np.array(lr["are_per_step"])
    assert np.isfinite(a).all() and np.isfinite(b).all()
    assert fx["final_are"] < 10.0
    assert lr["mean_are"] <= fx["mean_are"]
    assert (b <= a).mean() >= 0.75
    net.close()


@pytest.mark.parametrize("seed", [0, 2, 3])
def test_streams_track_with_new_points_near_their_depth(seed):
    """The streams that drift with the 1 m rule track under both schedules
    when each new point starts within ~5 cm of its true position: the error
    of the growing graph stays near the noise-and-outlier floor (~7 px) over
    all 490 steps.  So their drift comes from the new points' initial depth,
    not from the iteration."""
    import torch
    init, steps = synth.make_stream(seed)
    rng = np.random.default_rng(seed)
    xyz = [st.new_lm_true + rng.normal(0.0, 0.05, st.new_lm_true.shape) for st in steps]
    net = gbp.DampingNet(learned.trained_params())
    r = learned.stream_compare(torch, net, init, steps, per_step=20, new_lm_xyz=xyz)
    fx, lr = r["fixed"], r["learned"]
    print(seed, {k: (fx[k], lr[k]) for k in ("mean_are", "final_are", "device_ms")})
    for s in (fx, lr):
        a = np.array(s["are_per_step"])
        assert np.isfinite(a).all()
        assert s["final_are"] < 10.0 and a.max() < 20.0
    net.close()
