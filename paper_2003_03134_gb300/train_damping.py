"""Train the per-factor damping network on GBP trajectories of synthetic
batched problems (walk problems of 10-200 keyframes and 100-5000 points,
each seeded by its index), entirely on the GPU.

    python -m paper_2003_03134_gb300.train_damping [--problems 1000]
        [--first-seed 10000] [--chunk 25] [--steps 300] [--batch 4096]
        [--lr 1e-3] [--record-iters 80] [--out paper_2003_03134_gb300/damping_net.npy]

Writes the trained parameters (float32, the flat layout of include/gbp.h)
and, beside them, a JSON log of the per-chunk losses and the held-out loss
against the constant d = 0.4.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import build, gbp, learned, synth

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "damping_net.npy")
HELD_OUT_SEED = 20000   # evaluation problems, disjoint from the training seeds


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--problems", type=int, default=1000)
    ap.add_argument("--first-seed", type=int, default=10000)
    ap.add_argument("--chunk", type=int, default=25)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--record-iters", type=int, default=80)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_OUT)
    a = ap.parse_args(argv)

    import torch
    build.build()
    gbp.lib()
    t0 = time.perf_counter()
    net = gbp.DampingNet(learned.init_params(a.init_seed))

    def chunks():
        for c in range(0, a.problems, a.chunk):
            yield synth.make_batch(min(a.chunk, a.problems - c), first_seed=a.first_seed + c)

    log = learned.TrainLog()
    learned.train(torch, net, chunks(), steps_per_chunk=a.steps, batch=a.batch, lr=a.lr,
                  seed=a.init_seed, record_kw=dict(record_iters=a.record_iters), log=log, verbose=True)
    held = learned.record(torch, synth.make_batch(4, first_seed=HELD_OUT_SEED), record_iters=a.record_iters)
    loss, const = learned.evaluate_loss(torch, net, held)
    w = net.params
    np.save(a.out, w)
    summary = dict(problems=a.problems, first_seed=a.first_seed, chunk=a.chunk, steps_per_chunk=a.steps,
                   batch=a.batch, lr=a.lr, record_iters=a.record_iters, seconds=time.perf_counter() - t0,
                   held_out_seeds=[HELD_OUT_SEED, HELD_OUT_SEED + 3], held_out_loss=loss,
                   held_out_loss_constant_0_4=const, chunks=log.chunks)
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "chunks"}))


if __name__ == "__main__":
    main()
