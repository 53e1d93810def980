"""Robustness experiments of Sec. 9.3 and Sec. 9.4 on synthetic problems,
run through the batched GPU path.

* ``convergence_basin`` (Sec. 9.3): the share of problems that reach a mean
  reprojection error below 1.5 px (the paper's success criterion) as the
  noise on the keyframes' initial positions grows.  Each noise level is one
  batch of independent problems (problem i seeded by i) solved by one launch
  per iteration (``gbp_create_batch``); every problem's ARE comes from
  ``gbp_get_problem_are``.
* ``outlier_classification`` (Sec. 9.4): a problem in which a share of the
  data associations are wrong.  After each checkpoint, measurements whose
  reprojection error is in the linear regime of the Huber loss (error > N
  sigma, Sec. 6) are classified as outliers; precision and recall against the
  generator's labels, and the ARE of the correct measurements.
* ``huber_ablation`` (Sec. 9.4): the converged ARE of the correct
  measurements with and without the Huber loss for growing shares of wrong
  associations.
* ``lm_convergence_basin``: the basin trials solved by the project's CPU
  Levenberg-Marquardt baseline (``paper_2003_03134_gb300.lm``), the
  comparison the paper makes against Ceres.

The paper runs these on TUM sequences; these synthetic problems stand in for
them (30-keyframe and 20-keyframe video-like tracks, ``synth.make_walk`` with
``smooth=True``).  ``python -m paper_2003_03134_gb300.experiments`` runs all
three and prints one JSON object.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import gbp, synth

SUCCESS_PX = 1.5   # Sec. 9.1 / 9.3: converged once ARE < 1.5 px


def basin_problem(seed: int, pos_sigma: float, n_kf: int = 30, n_lm: int = 400):
    """One trial of the convergence-basin experiment: a 30-keyframe
    video-like track, no outliers, keyframe positions perturbed by
    ``pos_sigma`` (m), rotations by 0.02 rad, points by 0.1 m."""
    return synth.make_walk(seed=seed, n_kf=n_kf, n_lm=n_lm, outlier_frac=0.0, pos_sigma=pos_sigma, rot_sigma=0.02,
                           lm_sigma=0.1, smooth=True, name=f"basin{seed}")


def _make_basin(args):
    return basin_problem(*args)


def _problems(fn, args_list):
    import multiprocessing as mp
    try:
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            return pool.map(fn, args_list)
    except Exception:
        return [fn(a) for a in args_list]


def convergence_basin(noise_levels=(0.02, 0.07, 0.15, 0.3, 0.5, 0.8), trials=100, max_iters=1000, check_every=25,
                      stream=None, huber_nsigma=2.0):
    """Per noise level: the share of ``trials`` problems whose ARE fell below
    1.5 px within ``max_iters`` iterations, and the median iterations of the
    successful ones (to the ``check_every`` grid)."""
    out = []
    for sigma in noise_levels:
        probs = _problems(_make_basin, [(s, sigma) for s in range(trials)])
        g = gbp.Graph(probs, stream=stream, huber_nsigma=huber_nsigma, launch_mode=2)
        first = np.full(trials, -1)
        done = 0
        while done < max_iters and (first < 0).any():
            g.iterate(check_every)
            done += check_every
            are, _, _ = g.problem_are()
            hit = (are < SUCCESS_PX) & (first < 0)
            first[hit] = done
        g.close()
        ok = first >= 0
        out.append({"pos_sigma_m": sigma, "trials": trials, "success": float(ok.mean()),
                    "median_iters": float(np.median(first[ok])) if ok.any() else None})
    return out


def _lm_trial(args):
    """One trial with the CPU Levenberg-Marquardt baseline: iterations until
    ARE < 1.5 px (or -1 if it converged above it / ran out of iterations)."""
    seed, sigma, max_iters, huber_nsigma = args
    from .lm import LM, reprojection_error
    p = basin_problem(seed, sigma)
    lm = LM(p, huber_nsigma=huber_nsigma)
    while lm.iterations < max_iters and not lm.converged:
        lm.step(1)
        if reprojection_error(p, *lm.world()) < SUCCESS_PX:
            return lm.iterations
    return -1


def lm_convergence_basin(noise_levels=(0.02, 0.07, 0.15, 0.3, 0.5, 0.8), trials=100, max_iters=100, huber_nsigma=2.0):
    """The same trials solved by the CPU Levenberg-Marquardt baseline (the
    paper's comparison in Sec. 9.3 is Ceres, an LM solver)."""
    out = []
    for sigma in noise_levels:
        its = np.array(_problems(_lm_trial, [(s, sigma, max_iters, huber_nsigma) for s in range(trials)]))
        ok = its >= 0
        out.append({"pos_sigma_m": sigma, "trials": trials, "success": float(ok.mean()),
                    "median_iters": float(np.median(its[ok])) if ok.any() else None})
    return out


def classify(err, labels, huber_nsigma, sigma_px=1.0):
    """Measurements in the Huber loss's linear regime (err > N sigma) are the
    outlier class; returns (precision, recall, number flagged).  Precision is
    1 when nothing is flagged; recall is 1 when there are no outliers."""
    err = np.asarray(err)
    labels = np.asarray(labels, bool)
    flagged = (err > huber_nsigma * sigma_px) & (err >= 0)
    tp = int((flagged & labels).sum())
    n_flag, n_pos = int(flagged.sum()), int(labels.sum())
    precision = tp / n_flag if n_flag else 1.0
    recall = tp / n_pos if n_pos else 1.0
    return precision, recall, n_flag


def outlier_problem(seed: int = 0, bad_frac: float = 0.03, n_kf: int = 20, n_lm: int = 300):
    """A 20-keyframe video-like track with a share of wrong data associations
    (Sec. 9.4: 3%) and no other outliers."""
    return synth.make_walk(seed=seed, n_kf=n_kf, n_lm=n_lm, outlier_frac=0.0, bad_assoc_frac=bad_frac, smooth=True,
                           pos_sigma=0.07, rot_sigma=0.02, lm_sigma=0.1, name=f"assoc{seed}")


def outlier_classification(p=None, checkpoints=(1, 5, 10, 20, 50, 100, 200, 300, 500, 800), huber_nsigma=2.0,
                           stream=None):
    """Precision and recall of the Huber-regime outlier classification and
    the ARE over all / correct measurements at each checkpoint."""
    p = p if p is not None else outlier_problem()
    g = gbp.Graph(p, stream=stream, huber_nsigma=huber_nsigma)
    rows, done = [], 0
    for c in checkpoints:
        g.iterate(c - done)
        done = c
        err = g.residuals()
        prec, rec, n_flag = classify(err, p.obs_outlier, huber_nsigma)
        ok = err >= 0
        rows.append({"iteration": c, "precision": prec, "recall": rec, "flagged": n_flag,
                     "are": float(err[ok].mean()), "are_inliers": float(err[ok & ~p.obs_outlier].mean())})
    g.close()
    return {"problem": p.name, "observations": p.n_obs, "wrong_associations": int(p.obs_outlier.sum()),
            "huber_nsigma": huber_nsigma, "checkpoints": rows}


def huber_ablation(fracs=(0.0, 0.01, 0.03, 0.05, 0.1), seeds=(0, 1, 2), iters=1000, stream=None):
    """Converged ARE of the correct measurements with the Huber loss (N = 2)
    and without it, per share of wrong associations (median over seeds)."""
    out = []
    for frac in fracs:
        row = {"bad_frac": frac}
        for label, n in (("huber", 2.0), ("no_huber", 0.0)):
            vals = []
            for s in seeds:
                p = outlier_problem(seed=s, bad_frac=frac)
                g = gbp.Graph(p, stream=stream, huber_nsigma=n)
                g.iterate(iters)
                err = g.residuals()
                g.close()
                ok = err >= 0
                vals.append(float(err[ok & ~p.obs_outlier].mean()))
            row[label] = float(np.median(vals))
            row[label + "_converged"] = float(np.mean(np.array(vals) < SUCCESS_PX))
        out.append(row)
    return out


def main():
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    res = {"convergence_basin": convergence_basin(stream=stream),
           "convergence_basin_lm": lm_convergence_basin(),
           "outlier_classification": outlier_classification(stream=stream),
           "huber_ablation": huber_ablation(stream=stream)}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
