"""One graph split across ranks.

The paper runs a graph on one IPU and names multi-chip scaling as the way to
larger problems (Sec. 10).  Here a large graph (the 2000-keyframe loop) is
cut into parts, one per rank:

* ``partition``: keyframes in groups of about equal factor counts, one per
  rank -- by default spatial groups (recursive bisection of the initial
  camera centres along the widest axis), so that a place the camera
  revisits (a loop closure) stays on one rank; or contiguous segments of the
  sequence.  Each landmark goes to the rank that owns the majority of the
  keyframes observing it (ties to the lowest rank), and with it all of its
  factors.  Keyframes and landmarks are renumbered so that each rank's are
  contiguous (a relabelling of the same problem).
* ``SplitRank``: one rank's side of an iteration, over an *engine* that runs
  the rank's part -- its factors' messages (factor phase), its variables'
  beliefs (belief phase) -- and reads and writes boundary records:

    1. factor phase of iteration t on the rank's factors;
    2. the new message to the keyframe of every rank factor whose keyframe
       another rank owns goes to that owner (``send_msgs`` / ``recv_msgs``);
    3. belief phase on the rank's keyframes and landmarks;
    4. the beliefs of the rank's keyframes that other ranks' factors observe
       go to those ranks (``send_kfs`` / ``recv_kfs``).

  The owner of a keyframe receives its factors' messages themselves, not
  partial sums, and sums every message in the order the whole graph would:
  the split run gives the whole graph's bits.
* Drivers: ``run_local`` steps every rank of one process in turn (the
  exchange is a hand-over in memory; used to run all parts on one GPU),
  ``run_distributed`` runs one rank per process and exchanges the records,
  host-staged, with point-to-point sends of ``torch.distributed`` (gloo on
  CPU tensors; no collective on the data path besides the final gather).
* ``GpuEngine``: a rank's part on a GPU through the C ABI
  (``gbp_set_partition``, ``gbp_split_phase``, ``gbp_get/put_split_records``).
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field

import numpy as np

from . import gbp


@dataclass
class Part:
    rank: int
    world: int
    kf_range: tuple            # [k0, k1): keyframes whose beliefs this rank forms
    lm_range: tuple            # [l0, l1): landmarks (renumbered) whose factors and beliefs it forms
    factors: np.ndarray        # observation indices of its factors
    send_msgs: dict = field(default_factory=dict)   # rank -> observations (its factors on that rank's keyframes)
    recv_msgs: dict = field(default_factory=dict)   # rank -> observations (that rank's factors on my keyframes)
    send_kfs: dict = field(default_factory=dict)    # rank -> my keyframes its factors observe
    recv_kfs: dict = field(default_factory=dict)    # rank -> its keyframes my factors observe


def kf_owner(n_kf: int, world: int) -> np.ndarray:
    """Contiguous, equal segments of the keyframe sequence."""
    return (np.arange(n_kf, dtype=np.int64) * world) // max(n_kf, 1)


def camera_centres(kf_Rt: np.ndarray) -> np.ndarray:
    """c = -R^T t of each (R | t) world-to-camera pose."""
    R = kf_Rt[:, :9].reshape(-1, 3, 3)
    return -np.einsum("kji,kj->ki", R, kf_Rt[:, 9:])


def spatial_groups(centres: np.ndarray, weight: np.ndarray, world: int) -> list:
    """Recursive coordinate bisection: split the keyframes at the weighted
    median of the widest axis of their bounding box, the weight shared out in
    proportion to the ranks on each side, until there is one group per rank.
    Each group lists its keyframes in increasing order."""
    def rec(ids, w):
        if w == 1 or ids.size <= 1:
            return [ids] + [ids[:0]] * (w - 1)
        c = centres[ids]
        ax = int(np.argmax(c.max(axis=0) - c.min(axis=0)))
        o = ids[np.argsort(c[:, ax], kind="stable")]
        w1 = w // 2
        cw = np.cumsum(weight[o])
        cut = int(np.searchsorted(cw, cw[-1] * w1 / w)) + 1
        cut = min(max(cut, 1), o.size - 1)
        return rec(np.sort(o[:cut]), w1) + rec(np.sort(o[cut:]), w - w1)
    return rec(np.arange(centres.shape[0]), world)


def partition(problem, world: int, kf_split: str = "spatial"):
    """(renumbered problem, landmark permutation old -> new, [Part per rank]).
    ``kf_split``: "spatial" (``spatial_groups`` weighted by observation
    counts) or "sequence" (``kf_owner``).  With "sequence" the keyframes keep
    their numbers."""
    if kf_split == "spatial" and world > 1:
        counts = np.bincount(problem.obs_kf, minlength=problem.n_kf).astype(np.float64)
        groups = spatial_groups(camera_centres(problem.kf_Rt_init), counts, world)
        order_k = np.concatenate(groups)                      # new keyframe i = old order_k[i]
        sizes = np.array([g.size for g in groups])
        own_k = np.repeat(np.arange(world), sizes)
    elif kf_split in ("spatial", "sequence"):
        order_k = np.arange(problem.n_kf)
        own_k = kf_owner(problem.n_kf, world)
    else:
        raise ValueError(f"unknown kf_split {kf_split!r}")
    new_k_of_old = np.empty(problem.n_kf, dtype=np.int64)
    new_k_of_old[order_k] = np.arange(problem.n_kf)
    obs_kf = new_k_of_old[problem.obs_kf]
    votes = np.zeros((problem.n_lm, world), dtype=np.int64)
    np.add.at(votes, (problem.obs_lm, own_k[obs_kf]), 1)
    own_l = np.argmax(votes, axis=1)                       # majority, ties to the lowest rank
    order = np.argsort(own_l, kind="stable")               # new landmark i = old order[i]
    new_of_old = np.empty(problem.n_lm, dtype=np.int64)
    new_of_old[order] = np.arange(problem.n_lm)
    q = copy.copy(problem)
    q.kf_Rt_true = problem.kf_Rt_true[order_k]
    q.kf_Rt_init = problem.kf_Rt_init[order_k]
    q.obs_kf = obs_kf.astype(np.int32)
    q.anchor_kf = np.sort(new_k_of_old[problem.anchor_kf]).astype(np.int32)
    q.lm_true = problem.lm_true[order]
    q.lm_init = problem.lm_init[order]
    q.obs_lm = new_of_old[problem.obs_lm].astype(np.int32)
    own_l = own_l[order]
    lm_bounds = np.searchsorted(own_l, np.arange(world + 1))
    kf_bounds = np.searchsorted(own_k, np.arange(world + 1))
    f_rank = own_l[q.obs_lm]                                 # rank of each factor (its landmark's)
    k_rank = own_k[q.obs_kf]                                 # owner of its keyframe
    parts = []
    for r in range(world):
        p = Part(r, world, (int(kf_bounds[r]), int(kf_bounds[r + 1])), (int(lm_bounds[r]), int(lm_bounds[r + 1])),
                 np.flatnonzero(f_rank == r))
        for s in range(world):
            if s == r:
                continue
            out = np.flatnonzero((f_rank == r) & (k_rank == s))
            inc = np.flatnonzero((f_rank == s) & (k_rank == r))
            if out.size:
                p.send_msgs[s] = out
                p.recv_kfs[s] = np.unique(q.obs_kf[out])
            if inc.size:
                p.recv_msgs[s] = inc
                p.send_kfs[s] = np.unique(q.obs_kf[inc])
        parts.append(p)
    return q, new_of_old, parts


def boundary_stats(parts) -> dict:
    """Records each iteration exchanges: messages to keyframes of another
    rank and keyframe beliefs sent back, in total and for the busiest rank."""
    msgs = [sum(len(o) for o in p.send_msgs.values()) for p in parts]
    kfs = [sum(len(o) for o in p.send_kfs.values()) for p in parts]
    return {"messages": int(sum(msgs)), "keyframe_beliefs": int(sum(kfs)),
            "max_rank_messages": int(max(msgs)), "max_rank_keyframe_beliefs": int(max(kfs)),
            "factors_per_rank": [int(len(p.factors)) for p in parts]}


class SplitRank:
    """One rank's side of the split iteration over an engine with
    factor_phase(), belief_phase(), get/put_messages(obs[, recs]) and
    get/put_keyframes(kfs[, recs])."""

    def __init__(self, engine, part: Part):
        self.engine = engine
        self.part = part

    def phase_a(self) -> dict:
        self.engine.factor_phase()
        return {s: self.engine.get_messages(obs) for s, obs in self.part.send_msgs.items()}

    def deliver_a(self, incoming: dict):
        for s, recs in incoming.items():
            self.engine.put_messages(self.part.recv_msgs[s], recs)

    def phase_b(self) -> dict:
        self.engine.belief_phase()
        return {s: self.engine.get_keyframes(kfs) for s, kfs in self.part.send_kfs.items()}

    def deliver_b(self, incoming: dict):
        for s, recs in incoming.items():
            self.engine.put_keyframes(self.part.recv_kfs[s], recs)


def run_local(ranks, n_iters: int):
    """Every rank of this process in lockstep; the exchanges are hand-overs."""
    for _ in range(n_iters):
        out = [r.phase_a() for r in ranks]
        for r in ranks:
            r.deliver_a({s: out[s][r.part.rank] for s in range(len(ranks)) if r.part.rank in out[s]})
        out = [r.phase_b() for r in ranks]
        for r in ranks:
            r.deliver_b({s: out[s][r.part.rank] for s in range(len(ranks)) if r.part.rank in out[s]})


def _exchange(send: dict, recv_shapes: dict, dtype, group=None):
    """Point-to-point exchange of host arrays with every peer (torch.distributed)."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], {}
    for s, shape in recv_shapes.items():
        bufs[s] = torch.empty(shape, dtype=dtype)
        reqs.append(dist.irecv(bufs[s], src=s, group=group))
    keep = []
    for s, arr in send.items():
        t = torch.from_numpy(np.ascontiguousarray(arr))
        keep.append(t)
        reqs.append(dist.isend(t, dst=s, group=group))
    for q in reqs:
        q.wait()
    return {s: b.numpy() for s, b in bufs.items()}


def run_distributed(rank: SplitRank, n_iters: int, msg_width: int, kf_width: int, dtype, group=None):
    """One rank per process: the same iteration, records sent host-staged to
    the peers that need them."""
    p = rank.part
    shapes_a = {s: (len(obs), msg_width) for s, obs in p.recv_msgs.items()}
    shapes_b = {s: (len(kfs), kf_width) for s, kfs in p.recv_kfs.items()}
    for _ in range(n_iters):
        rank.deliver_a(_exchange(rank.phase_a(), shapes_a, dtype, group))
        rank.deliver_b(_exchange(rank.phase_b(), shapes_b, dtype, group))


class GpuEngine:
    """A rank's part on a GPU (FP32 path, fixed damping schedule): the whole
    renumbered problem's layout, with this part's factors and beliefs."""

    msg_width = gbp.GBP_SPLIT_MSG_FLOATS
    kf_width = gbp.GBP_SPLIT_KF_FLOATS

    def __init__(self, problem, part: Part, stream=None, **params):
        self.graph = gbp.Graph(problem, stream=stream, launch_mode=2, **params)
        gbp.gbp_set_partition(self.graph.h, part.kf_range, part.lm_range)

    def factor_phase(self):
        gbp.gbp_split_phase(self.graph.h, 0)

    def belief_phase(self):
        gbp.gbp_split_phase(self.graph.h, 1)

    def get_messages(self, obs):
        return gbp.gbp_get_split_records(self.graph.h, 0, obs)

    def put_messages(self, obs, recs):
        gbp.gbp_put_split_records(self.graph.h, 0, obs, recs)

    def get_keyframes(self, kfs):
        return gbp.gbp_get_split_records(self.graph.h, 1, kfs)

    def put_keyframes(self, kfs, recs):
        gbp.gbp_put_split_records(self.graph.h, 1, kfs, recs)

    def means(self):
        return self.graph.means()

    def close(self):
        self.graph.close()


def gather_means(parts, means):
    """The whole graph's chart means from each rank's (kf_mu, lm_mu): every
    variable from the rank that owns it."""
    kf = np.array(means[0][0], copy=True)
    lm = np.array(means[0][1], copy=True)
    for p, (k, m) in zip(parts, means):
        kf[p.kf_range[0]:p.kf_range[1]] = k[p.kf_range[0]:p.kf_range[1]]
        lm[p.lm_range[0]:p.lm_range[1]] = m[p.lm_range[0]:p.lm_range[1]]
    return kf, lm
