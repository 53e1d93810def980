"""Sharding of independent problems across ranks: the partition rule on its
own, and the multi-rank path as two gloo processes on the CPU (each rank
takes its share of the batched workload, the shares cover every problem
exactly once, and the timing reduction gives the slowest rank's time and
the total work)."""
import os
import socket

import numpy as np
import pytest

from paper_2003_03134_gb300 import shard


def _sizes(n=256, seed=0):
    rng = np.random.default_rng(seed)
    return rng.integers(1000, 50000, n)


@pytest.mark.parametrize("n_ranks", [1, 2, 3, 8])
def test_partition_covers_every_problem_once(n_ranks):
    s = _sizes()
    parts = shard.partition(s, n_ranks)
    assert len(parts) == n_ranks
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(s)))


@pytest.mark.parametrize("n_ranks", [2, 4, 8])
def test_partition_is_balanced(n_ranks):
    """LPT: the busiest rank carries at most the average load plus one
    problem, and at most 4/3 of the optimum (bounded below by the average)."""
    s = _sizes(seed=n_ranks)
    ld = shard.loads(s, shard.partition(s, n_ranks))
    avg = s.sum() / n_ranks
    assert max(ld) <= avg + s.max()
    assert max(ld) <= 4.0 / 3.0 * max(avg, s.max()) + 1


def test_partition_small_cases():
    assert shard.partition([5, 1, 3], 2) == [[0], [1, 2]]
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([7, 7, 7, 7], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def test_partition_is_deterministic():
    s = _sizes(seed=5)
    assert shard.partition(s, 4) == shard.partition(list(s), 4)


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank_main(rank, world, port, sizes, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.partition(sizes, world)[rank]
        units = float(sum(int(sizes[i]) for i in mine))
        ms = 10.0 + rank          # a slower rank 1
        t, u = shard.reduce_timing(ms, units)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([t, u, len(mine)] + sorted(i for g in gathered for i in g), dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    sizes = [int(x) for x in _sizes(64, seed=9)]
    port = _free_port()
    tmp.start_processes(_rank_main, args=(2, port, sizes, str(tmp_path)), nprocs=2, join=True,
                        start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    # both ranks agree on the reduced figures: slowest time, total work
    assert r0[0] == r1[0] == 11.0
    assert r0[1] == r1[1] == float(sum(sizes))
    # the gathered shares cover every problem exactly once
    assert list(r0[3:].astype(int)) == list(range(len(sizes)))
    assert r0[2] + r1[2] == len(sizes)
    assert torch is not None


def test_reduce_timing_without_a_group():
    pytest.importorskip("torch")
    assert shard.reduce_timing(3.0, 7.0) == (3.0, 7.0)
