"""One graph split across ranks (paper_2003_03134_gb300.split).

CPU: the partition's invariants, and the split iteration run as 2 and 4
gloo processes -- each rank's part solved by the oracle restricted to that
part, the boundary records exchanged host-staged -- bit for bit equal to the
whole graph solved by the oracle in one process.  GPU: every part on one
GPU in turn (records handed over in memory) bit for bit equal to the whole
graph on that GPU."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2003_03134_gb300 import split, synth


def _loop(n_kf=120, n_lm=3000, seed=0):
    """A small stand-in of the 2000-keyframe loop: two laps, so loop closures
    put landmarks on keyframe segments far apart in the sequence."""
    return synth.make_loop(seed=seed, n_kf=n_kf, n_lm=n_lm, radius=8.0)


@pytest.mark.parametrize("kf_split", ["spatial", "sequence"])
@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_partition_invariants(world, kf_split):
    p = _loop()
    q, new_of_old, parts = split.partition(p, world, kf_split=kf_split)
    # a relabelling of the same problem: every observation keeps its pose, point and pixel
    np.testing.assert_array_equal(q.lm_init[new_of_old], p.lm_init)
    np.testing.assert_array_equal(q.obs_lm, new_of_old[p.obs_lm])
    np.testing.assert_array_equal(q.kf_Rt_init[q.obs_kf], p.kf_Rt_init[p.obs_kf])
    np.testing.assert_array_equal(q.kf_Rt_true[q.obs_kf], p.kf_Rt_true[p.obs_kf])
    np.testing.assert_array_equal(q.obs_uv, p.obs_uv)
    np.testing.assert_array_equal(np.sort(q.kf_Rt_init[q.anchor_kf], axis=0), np.sort(p.kf_Rt_init[p.anchor_kf], axis=0))
    if kf_split == "sequence":
        np.testing.assert_array_equal(q.obs_kf, p.obs_kf)
    # contiguous keyframe segments and landmark ranges covering everything once
    assert parts[0].kf_range[0] == 0 and parts[-1].kf_range[1] == p.n_kf
    assert parts[0].lm_range[0] == 0 and parts[-1].lm_range[1] == p.n_lm
    for a, b in zip(parts, parts[1:]):
        assert a.kf_range[1] == b.kf_range[0] and a.lm_range[1] == b.lm_range[0]
    np.testing.assert_array_equal(np.sort(np.concatenate([r.factors for r in parts])), np.arange(p.n_obs))
    owner_k = np.repeat(np.arange(world), [r.kf_range[1] - r.kf_range[0] for r in parts])
    for r in parts:
        # a rank's factors are those of its landmarks, whose majority of observers it owns
        assert np.all((q.obs_lm[r.factors] >= r.lm_range[0]) & (q.obs_lm[r.factors] < r.lm_range[1]))
        for m in range(r.lm_range[0], r.lm_range[1], 97):
            votes = np.bincount(owner_k[q.obs_kf[q.obs_lm == m]], minlength=world)
            assert votes[r.rank] == votes.max()
        # every boundary message goes to its keyframe's owner, and comes back as beliefs
        for s, obs in r.send_msgs.items():
            assert np.all(owner_k[q.obs_kf[obs]] == s)
            np.testing.assert_array_equal(parts[s].recv_msgs[r.rank], obs)
            np.testing.assert_array_equal(parts[s].send_kfs[r.rank], r.recv_kfs[s])
    if world > 1:
        assert sum(len(o) for r in parts for o in r.send_msgs.values()) > 0
        # no rank idle, none with more than twice its share of factors
        n = np.array([len(r.factors) for r in parts])
        assert n.min() > 0 and n.max() <= 2 * p.n_obs / world


def test_spatial_split_keeps_loop_closures_on_one_rank():
    """On two laps of a loop, contiguous segments of the sequence put the
    two visits of every place on different ranks; spatial groups do not."""
    p = _loop()
    seq = split.boundary_stats(split.partition(p, 4, kf_split="sequence")[2])
    spa = split.boundary_stats(split.partition(p, 4, kf_split="spatial")[2])
    assert spa["messages"] < 0.5 * seq["messages"]


def test_spatial_groups_balance_weight():
    rng = np.random.default_rng(0)
    c = rng.normal(size=(500, 3)) * [10, 3, 1]
    w = rng.integers(1, 20, size=500).astype(float)
    for world in (2, 3, 5, 8):
        groups = split.spatial_groups(c, w, world)
        assert len(groups) == world
        np.testing.assert_array_equal(np.sort(np.concatenate(groups)), np.arange(500))
        share = np.array([w[g].sum() for g in groups]) / w.sum()
        assert np.all(np.abs(share - 1 / world) < 0.05)


class OracleEngine:
    """A rank's part solved by the FP64 oracle restricted to it (test only)."""

    msg_width = 42     # the message to the keyframe: Lambda 36, eta 6
    kf_width = 48      # a keyframe belief: Lambda 36, eta 6, mean 6

    def __init__(self, problem, part, **params):
        self.o = oracle.Oracle(problem, **params)
        fm = np.zeros(problem.n_obs, np.uint8)
        fm[part.factors] = 1
        vm = np.zeros(problem.n_kf + problem.n_lm, np.uint8)
        vm[part.kf_range[0]:part.kf_range[1]] = 1
        vm[problem.n_kf + part.lm_range[0]:problem.n_kf + part.lm_range[1]] = 1
        self.o.set_part(fm, vm)

    def factor_phase(self):
        self.o.factor_phase()

    def belief_phase(self):
        self.o.belief_phase()

    def get_messages(self, obs):
        lam, eta = self.o.new_kf_messages(obs)
        return np.concatenate([lam, eta], axis=1)

    def put_messages(self, obs, recs):
        self.o.put_new_kf_messages(obs, recs[:, :36], recs[:, 36:])

    def get_keyframes(self, kfs):
        return self.o.kf_beliefs(kfs)

    def put_keyframes(self, kfs, recs):
        self.o.put_kf_beliefs(kfs, recs)

    def means(self):
        return self.o.means()


PARAMS = dict(huber_nsigma=2.0)
N_ITERS = 25


def test_split_oracle_in_one_process_equals_whole_graph():
    p = _loop()
    q, _, parts = split.partition(p, 3)
    ranks = [split.SplitRank(OracleEngine(q, r, **PARAMS), r) for r in parts]
    split.run_local(ranks, N_ITERS)
    kf, lm = split.gather_means(parts, [r.engine.means() for r in ranks])
    whole = oracle.Oracle(q, **PARAMS)
    whole.iterate(N_ITERS)
    okf, olm = whole.means()
    np.testing.assert_array_equal(kf, okf)
    np.testing.assert_array_equal(lm, olm)


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _loop()
        q, _, parts = split.partition(p, world)
        eng = OracleEngine(q, parts[rank], **PARAMS)
        split.run_distributed(split.SplitRank(eng, parts[rank]), N_ITERS, eng.msg_width, eng.kf_width,
                              torch.float64)
        means = [None] * world
        dist.all_gather_object(means, eng.means())
        if rank == 0:
            kf, lm = split.gather_means(parts, means)
            np.save(os.path.join(out_dir, "kf.npy"), kf)
            np.save(os.path.join(out_dir, "lm.npy"), lm)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_split_across_gloo_ranks_equals_whole_graph(tmp_path, world):
    """The split iteration on `world` CPU processes, boundary records sent
    point to point over gloo, gives the single-process run's bits."""
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    oracle.build()
    tmp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                        start_method="spawn")
    p = _loop()
    q, _, _ = split.partition(p, world)
    whole = oracle.Oracle(q, **PARAMS)
    whole.iterate(N_ITERS)
    okf, olm = whole.means()
    np.testing.assert_array_equal(np.load(tmp_path / "kf.npy"), okf)
    np.testing.assert_array_equal(np.load(tmp_path / "lm.npy"), olm)


@pytest.mark.gpu
@pytest.mark.parametrize("world,factor_shape", [(2, -1), (4, -1), (2, 4)])
def test_split_parts_on_one_gpu_equal_whole_graph(world, factor_shape):
    """Every rank's part on this GPU, the ranks stepped in turn with the
    records handed over in memory: the whole graph's bits (FP32, the paper's
    schedule, with relinearisations), also with the factor kernel that
    defers FP64 tiles to a second kernel."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_03134_gb300 import build, gbp
    build.build()
    p = _loop()
    q, _, parts = split.partition(p, world)
    ranks = [split.SplitRank(split.GpuEngine(q, r, factor_shape=factor_shape, **PARAMS), r) for r in parts]
    n = 40
    split.run_local(ranks, n)
    kf, lm = split.gather_means(parts, [r.engine.means() for r in ranks])
    g = gbp.Graph(q, launch_mode=2, factor_shape=factor_shape, **PARAMS)
    g.iterate(n)
    gkf, glm = g.means()
    st = g.stats()
    g.close()
    for r in ranks:
        r.engine.close()
    assert st["relinearisations"] > 0
    np.testing.assert_array_equal(kf, gkf)
    np.testing.assert_array_equal(lm, glm)
