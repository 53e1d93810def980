"""Training and evaluation driver of the per-factor damping network.

The network and its features are described in include/gbp.h (it replaces
the fixed damping factor d of Sec. 5 / Sec. 8 by a per-factor prediction;
the paper has no such network).  Every arithmetic step -- GBP iterations,
features, damping targets, forward, backward and Adam -- runs in libgbp's
CUDA kernels; this module only moves device buffers around (PyTorch tensors
for memory, random minibatch indices) and keeps the loop.

Training data come from GBP itself: for a batch of synthetic problems the
solver runs to convergence, its converged messages become the reference,
and a rerun from the start with the fixed schedule records, per factor and
iteration, the 16 features and the damping that would have brought each
new message closest to the reference.
"""
from __future__ import annotations

import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import gbp, synth

N_FEAT = gbp.GBP_MLP_NFEAT
N_PARAM = gbp.GBP_MLP_NPARAM
D_FIXED = 0.4        # the paper's d (Sec. 8)

# solver settings of the paper-scale configuration (Huber at 2 sigma, the
# paper's relinearisation and damping schedule)
SOLVER = dict(huber_nsigma=2.0)

# weights trained by ``python -m paper_2003_03134_gb300.train_damping``
# (1000 problems, seeds 10000-10999; log in damping_net.json)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "damping_net.npy")


def trained_params() -> np.ndarray:
    return np.load(WEIGHTS).astype(np.float32)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal hidden layers, a small output layer and b3 such that the
    untrained network predicts the paper's d = 0.4 everywhere."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.standard_normal((N_FEAT, 64)) * np.sqrt(2.0 / N_FEAT)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    W3 = rng.standard_normal(64) * (0.1 / 8.0)
    b3 = np.log(D_FIXED / (0.9 - D_FIXED))
    flat = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [b3]])
    assert flat.size == N_PARAM
    return flat.astype(np.float32)


@dataclass
class Samples:
    """Recorded (features, target) rows on the device; ``valid`` indexes the
    rows with a target (>= 0)."""
    X: object
    T: object
    valid: object
    n_factors: int
    iters: int


def record(torch, problems, conv_iters: int = 1500, record_iters: int = 80, conv_tol: float = 1e-6,
           stream=None, **solver) -> Samples:
    """Run the batch of problems to convergence, take its messages as the
    reference, restart and record ``record_iters`` iterations."""
    prm = dict(SOLVER, **solver)
    g = gbp.Graph(list(problems) if len(problems) > 1 else problems[0], stream=stream,
                  conv_tol=conv_tol, iterations=conv_iters, **prm)
    g.iterate(0)
    g.capture_messages()
    g.reset()
    nf = gbp.gbp_get_sizes(g.h)[2]
    X = torch.empty((record_iters * nf, N_FEAT), dtype=torch.float32, device="cuda")
    T = torch.empty(record_iters * nf, dtype=torch.float32, device="cuda")
    g.record(record_iters, X.data_ptr(), T.data_ptr())
    torch.cuda.synchronize()
    g.close()
    valid = torch.nonzero(T >= 0).view(-1).to(torch.int32)
    return Samples(X, T, valid, nf, record_iters)


@dataclass
class TrainLog:
    chunks: list = field(default_factory=list)


def train(torch, net: gbp.DampingNet, problem_chunks, steps_per_chunk: int = 300, batch: int = 4096,
          lr: float = 1e-3, seed: int = 0, record_kw=None, log: TrainLog | None = None, verbose=False):
    """Streamed training: record one chunk of problems, take
    ``steps_per_chunk`` Adam steps on random minibatches of its rows, move on."""
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    record_kw = record_kw or {}
    for ci, problems in enumerate(problem_chunks):
        t0 = time.perf_counter()
        s = record(torch, problems, **record_kw)
        n = int(s.valid.numel())
        if n == 0:
            continue
        losses = []
        for step in range(steps_per_chunk):
            pick = torch.randint(0, n, (batch,), generator=gen, device="cuda")
            idx = s.valid[pick].contiguous()
            want = step == steps_per_chunk - 1 or step == 0
            loss = net.train_step(s.X.data_ptr(), s.T.data_ptr(), batch, lr, idx_ptr=idx.data_ptr(), want_loss=want)
            if want:
                losses.append(loss)
        torch.cuda.synchronize()
        entry = dict(chunk=ci, rows=n, factors=s.n_factors, loss_first=losses[0], loss_last=losses[-1],
                     seconds=time.perf_counter() - t0)
        if log is not None:
            log.chunks.append(entry)
        if verbose:
            print(entry, flush=True)
        del s
    return log


def evaluate_loss(torch, net: gbp.DampingNet, s: Samples, max_rows: int = 1 << 22):
    """(network loss, loss of the constant d = 0.4) over up to max_rows valid rows."""
    idx = s.valid[:max_rows].contiguous()
    n = int(idx.numel())
    Xs = s.X.index_select(0, idx.long()).contiguous()
    Ts = s.T.index_select(0, idx.long()).contiguous()
    loss, _ = net.gradient(Xs.data_ptr(), Ts.data_ptr(), n)
    const = float(((Ts - D_FIXED) ** 2).mean())
    return loss, const


def iterations_to(g: gbp.Graph, thresholds, max_iters: int = 2000, conv_tol: float = 1e-6, check: int = 1):
    """Iterations from reset until ARE against the graph's reference drops
    below each threshold (px), and until max |dmu| < conv_tol."""
    g.reset()
    out = {float(th): None for th in thresholds}
    conv = None
    it = 0
    while it < max_iters:
        g.iterate(check)
        it += check
        st = g.stats()
        for th in out:
            if out[th] is None and st["are_ref"] < th:
                out[th] = it
        if conv is None and st["max_dmu"] < conv_tol:
            conv = it
        if conv is not None and all(v is not None for v in out.values()):
            break
    return out, conv


def time_iterations(torch, g: gbp.Graph, n: int, repeats: int = 5, flush=None) -> float:
    """Median device time (ms) of n iterations from reset."""
    if not n:
        return 0.0
    ts = []
    stream = torch.cuda.current_stream()
    for _ in range(repeats):
        if flush is not None:
            flush.fill_(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g.reset()
        a.record(stream)
        g.iterate(n)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def compare(torch, problem, net: gbp.DampingNet, thresholds=(1.0, 0.1, 0.01), max_iters=2000, conv_tol=1e-6,
            stream=None, launch_mode=0, reference=None, **solver):
    """Fixed d = 0.4 against the learned schedule on one problem: iterations
    and device milliseconds to each ARE threshold against ``reference``
    (world poses and points; default: the converged fixed-damping solution)
    and to convergence."""
    prm = dict(SOLVER, **solver)
    if reference is None:
        ref = gbp.Graph(problem, stream=stream, conv_tol=conv_tol, iterations=max_iters * 2, **prm)
        ref.iterate(0)
        reference = ref.beliefs()
        ref.close()
    kf_ref, lm_ref = reference
    res = {}
    for name, mode in (("fixed", 0), ("learned", 1)):
        g = gbp.Graph(problem, stream=stream, damping_mode=mode, launch_mode=launch_mode, **prm)
        if mode:
            g.set_damping_model(net)
        g.set_reference(kf_ref, lm_ref)
        its, conv = iterations_to(g, thresholds, max_iters, conv_tol)
        st = g.stats()   # where the search stopped: convergence or max_iters
        r = {"iters": {str(k): v for k, v in its.items()}, "iters_to_conv": conv,
             "final": {"iteration": st["iterations"], "are": st["are"], "are_ref": st["are_ref"]}}
        r["ms"] = {str(k): (time_iterations(torch, g, v) if v else None) for k, v in its.items()}
        r["ms_to_conv"] = time_iterations(torch, g, conv) if conv else None
        res[name] = r
        g.close()
    return res


def stream_compare(torch, net: gbp.DampingNet, init, steps, per_step: int = 20, stream=None, new_lm_xyz=None,
                   **solver):
    """The incremental stream of Sec. 9.2 (one keyframe added every
    ``per_step`` iterations) with fixed d = 0.4 and with the learned
    schedule: per step the ARE of the current graph after its iterations,
    and the device time of all iterations (CUDA events around each step's
    gbp_iterate; gbp_add_keyframe's host re-layout is the same for both and
    not included).  new_lm_xyz: per step the initial positions of its new
    points, or None for the library's rule (1 m along the first ray)."""
    prm = dict(SOLVER, **solver)
    out = {}
    cur = torch.cuda.current_stream()
    for name, mode in (("fixed", 0), ("learned", 1)):
        g = gbp.Graph(init, stream=stream, damping_mode=mode, **prm)
        if mode:
            g.set_damping_model(net)
        ares, ms = [], 0.0
        for i in range(len(steps) + 1):
            if i:
                st = steps[i - 1]
                xyz = None if new_lm_xyz is None or not st.n_new_lm else new_lm_xyz[i - 1]
                g.add_keyframe(st.obs_lm, st.obs_uv, n_new_lm=st.n_new_lm, new_lm_xyz=xyz)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cur)
            g.iterate(per_step)
            b.record(cur)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
            ares.append(g.stats()["are"])
        out[name] = {"are_per_step": ares, "mean_are": float(np.mean(ares)), "final_are": ares[-1],
                     "device_ms": ms, "iterations": per_step * (len(steps) + 1)}
        g.close()
    return out
