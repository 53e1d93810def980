"""Seeded synthetic bundle-adjustment problems.

This module is the input generator shared by the CUDA path's tests and bench
and by the oracle's tests.  It holds none of the belief-propagation
arithmetic: it places cameras and points, decides which keyframes observe
which points, projects the ground truth through a pinhole camera to make
measurements, adds pixel noise and outliers, and perturbs an initial estimate.
Every random draw comes from ``numpy.random.Generator(PCG64(seed))``.

The workloads stand in for the paper's TUM/KITTI bundle-adjustment problems
(Sec. 9, Table 1), which are not available: sizes follow Table 1 (fr3teddy:
125 keyframes, 1919 points) and the camera follows a 640x480 pinhole.

Pose convention: a keyframe pose is ``Rt = [R (row-major, 9), t (3)]`` mapping
world points into the camera frame, ``x_cam = R x_world + t`` (Sec. 4, the
measurement function pi(R l + t)).  Camera axes: x right, y down, z forward.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

__all__ = ["Problem", "StreamStep", "make_circle", "make_walk", "make_loop", "make_batch",
           "make_chain", "make_stream", "stream_plan", "concat", "subgraph", "workload"]


@dataclass
class Problem:
    name: str
    seed: int
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    kf_Rt_true: np.ndarray      # (n_kf, 12) float64
    kf_Rt_init: np.ndarray      # (n_kf, 12) float64
    lm_true: np.ndarray         # (n_lm, 3) float64
    lm_init: np.ndarray         # (n_lm, 3) float64
    obs_kf: np.ndarray          # (n_obs,) int32
    obs_lm: np.ndarray          # (n_obs,) int32
    obs_uv: np.ndarray          # (n_obs, 2) float64, pixels
    obs_outlier: np.ndarray     # (n_obs,) bool, generator label
    anchor_kf: np.ndarray       # (n_anchor,) int32
    params: dict = field(default_factory=dict)

    @property
    def n_kf(self) -> int:
        return int(self.kf_Rt_true.shape[0])

    @property
    def n_lm(self) -> int:
        return int(self.lm_true.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs_kf.shape[0])

    def intrinsics(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


# ---------------------------------------------------------------------------
# camera placement helpers (data synthesis only)

def _look_rotation(forward: np.ndarray, up: np.ndarray) -> np.ndarray:
    """World->camera rotation whose optical axis is ``forward`` and whose image
    'up' direction is ``up`` (camera y points down in the image)."""
    z = forward / np.linalg.norm(forward)
    y = -(up - np.dot(up, z) * z)
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    return np.stack([x, y, z])


def _pack(R: np.ndarray, center: np.ndarray) -> np.ndarray:
    t = -R @ center
    return np.concatenate([R.reshape(-1), t])


def _camera_points(Rt: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Camera-frame coordinates of points X (n,3) in every keyframe:
    returns (n_kf, n, 3)."""
    R = Rt[:, :9].reshape(-1, 3, 3)
    t = Rt[:, 9:]
    return np.einsum("kij,nj->kni", R, X) + t[:, None, :]


def _pixels(pc: np.ndarray, fx, fy, cx, cy) -> np.ndarray:
    return np.stack([fx * pc[..., 0] / pc[..., 2] + cx,
                     fy * pc[..., 1] / pc[..., 2] + cy], axis=-1)


def _visible(pc, fx, fy, cx, cy, w, h, min_depth):
    z = pc[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = _pixels(pc, fx, fy, cx, cy)
    return (z > min_depth) & (uv[..., 0] >= 0) & (uv[..., 0] < w) & \
        (uv[..., 1] >= 0) & (uv[..., 1] < h)


def _weighted_subsets(rng, weights: np.ndarray, counts: np.ndarray):
    """For each row, draw ``counts[row]`` distinct columns without replacement
    with probability proportional to ``weights`` (zero weight = never), by
    the Gumbel-top-k construction of successive weighted sampling: the
    columns of the ``counts[row]`` largest log-weight + Gumbel keys, in
    column order."""
    with np.errstate(divide="ignore"):
        logw = np.where(weights > 0, np.log(np.maximum(weights, 1e-300)), -np.inf)
    g = rng.gumbel(size=weights.shape)
    keys = logw + g
    n_rows, n_cols = keys.shape
    counts = np.asarray(counts, dtype=np.int64)
    if n_rows == 0 or counts.sum() == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    cmax = int(counts.max())
    # the cmax largest keys of every row (keys are continuous: no ties), then
    # their order, then the first counts[row] of them
    if cmax < n_cols:
        top = np.argpartition(-keys, cmax - 1, axis=1)[:, :cmax]
    else:
        top = np.tile(np.arange(n_cols), (n_rows, 1))
    tk = np.take_along_axis(keys, top, axis=1)
    top = np.take_along_axis(top, np.argsort(-tk, axis=1, kind="stable"), axis=1)
    take = np.arange(top.shape[1])[None, :] < counts[:, None]
    sel = np.where(take, top, n_cols)          # columns not taken sort last
    sel = np.sort(sel, axis=1)
    rows = np.repeat(np.arange(n_rows, dtype=np.int64), counts)
    cols = sel[np.arange(sel.shape[1])[None, :] < counts[:, None]].astype(np.int64)
    return rows, cols


def _perturb_init(rng, kf_true, lm_true, rot_sigma, pos_sigma, lm_sigma, anchors):
    n_kf = kf_true.shape[0]
    kf_init = kf_true.copy()
    for i in range(n_kf):
        if i in anchors:
            continue
        R = kf_true[i, :9].reshape(3, 3)
        t = kf_true[i, 9:]
        center = -R.T @ t
        dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, 3)).as_matrix()
        Rn = dR @ R
        cn = center + rng.normal(0.0, pos_sigma, 3)
        kf_init[i] = _pack(Rn, cn)
    lm_init = lm_true + rng.normal(0.0, lm_sigma, lm_true.shape)
    return kf_init, lm_init


def _finish(name, seed, cam, kf_true, kf_init, lm_true, lm_init, obs_kf, obs_lm,
            uv, outlier, anchors, params, min_init_depth=0.05):
    """Sort observations by (landmark, keyframe) and drop any whose initial
    depth is not positive enough (the library rejects those at creation)."""
    fx, fy, cx, cy, w, h = cam
    order = np.lexsort((obs_kf, obs_lm))
    obs_kf, obs_lm, uv, outlier = obs_kf[order], obs_lm[order], uv[order], outlier[order]
    R = kf_init[obs_kf, :9].reshape(-1, 3, 3)
    t = kf_init[obs_kf, 9:]
    pc = np.einsum("nij,nj->ni", R, lm_init[obs_lm]) + t
    keep = pc[:, 2] > 2.0 * min_init_depth
    return Problem(name=name, seed=seed, fx=fx, fy=fy, cx=cx, cy=cy, width=w, height=h,
                   kf_Rt_true=kf_true, kf_Rt_init=kf_init, lm_true=lm_true, lm_init=lm_init,
                   obs_kf=obs_kf[keep].astype(np.int32), obs_lm=obs_lm[keep].astype(np.int32),
                   obs_uv=uv[keep].astype(np.float64), obs_outlier=outlier[keep].astype(bool),
                   anchor_kf=np.asarray(sorted(anchors), dtype=np.int32), params=dict(params))


CAMERA = (500.0, 500.0, 320.0, 240.0, 640, 480)


# ---------------------------------------------------------------------------
# workloads

def make_circle(seed: int = 0, n_kf: int = 10, n_lm: int = 100, radius: float = 2.0,
                obs_range=(3, 6), noise_px: float = 1.0, rot_sigma: float = 0.05,
                pos_sigma: float = 0.1, lm_sigma: float = 0.1, anchors=(0,)) -> Problem:
    """Small ring of keyframes around a 1 m cube of points (oracle-sized)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fx, fy, cx, cy, w, h = CAMERA
    kf = []
    for i in range(n_kf):
        a = 2.0 * np.pi * i / n_kf
        c = np.array([radius * np.cos(a), radius * np.sin(a), 0.0])
        R = _look_rotation(-c, np.array([0.0, 0.0, 1.0]))
        kf.append(_pack(R, c))
    kf_true = np.array(kf)
    lms, obs_kf, obs_lm = [], [], []
    while len(lms) < n_lm:
        X = rng.uniform(-0.5, 0.5, 3)
        vis = np.nonzero(_visible(_camera_points(kf_true, X[None])[:, 0], fx, fy, cx, cy, w, h, 0.1))[0]
        if vis.size < obs_range[0]:
            continue
        c = int(rng.integers(obs_range[0], obs_range[1] + 1))
        c = min(c, vis.size)
        sel = np.sort(rng.choice(vis, size=c, replace=False))
        j = len(lms)
        lms.append(X)
        obs_kf.extend(sel.tolist())
        obs_lm.extend([j] * c)
    lm_true = np.array(lms)
    obs_kf = np.array(obs_kf, dtype=np.int64)
    obs_lm = np.array(obs_lm, dtype=np.int64)
    pc = np.einsum("nij,nj->ni", kf_true[obs_kf, :9].reshape(-1, 3, 3), lm_true[obs_lm]) + kf_true[obs_kf, 9:]
    uv = _pixels(pc, fx, fy, cx, cy) + rng.normal(0.0, noise_px, (obs_kf.size, 2))
    outlier = np.zeros(obs_kf.size, bool)
    kf_init, lm_init = _perturb_init(rng, kf_true, lm_true, rot_sigma, pos_sigma, lm_sigma, set(anchors))
    params = dict(damping=0.4, huber_nsigma=0.0, sigma_px=1.0, iterations=200)
    return _finish(f"circle{n_kf}x{n_lm}", seed, CAMERA, kf_true, kf_init, lm_true, lm_init,
                   obs_kf, obs_lm, uv, outlier, anchors, params)


def _smooth_track(rng, n_kf, step=0.08, turn_sigma_deg=1.0, max_turn_deg=8.0):
    """Camera centres and headings of a video-like track: constant step,
    heading driven by an AR(1) turn rate capped at max_turn_deg per keyframe,
    steered back toward the middle of [2, 8]^2 near its edges."""
    pos = rng.uniform(3.0, 7.0, 2)
    theta = rng.uniform(0, 2 * np.pi)
    omega = 0.0
    out = []
    for _ in range(n_kf):
        out.append((pos.copy(), theta))
        omega = 0.9 * omega + rng.normal(0.0, np.radians(turn_sigma_deg))
        edge = min(pos[0] - 2.0, 8.0 - pos[0], pos[1] - 2.0, 8.0 - pos[1])
        if edge < 1.5:
            to_c = np.arctan2(5.0 - pos[1], 5.0 - pos[0])
            err = (to_c - theta + np.pi) % (2 * np.pi) - np.pi
            omega += 0.15 * err
        omega = float(np.clip(omega, -np.radians(max_turn_deg), np.radians(max_turn_deg)))
        theta += omega
        pos = np.clip(pos + step * np.array([np.cos(theta), np.sin(theta)]), 2.0, 8.0)
    return out


def make_walk(seed: int = 0, n_kf: int = 125, n_lm: int = 1919, obs_range=(4, 15),
              outlier_frac: float = 0.02, noise_px: float = 1.0, rot_sigma: float = 0.05,
              pos_sigma: float = 0.1, lm_sigma: float = 0.1, anchors=(0,),
              name: str | None = None, smooth: bool = False, bad_assoc_frac: float = 0.0) -> Problem:
    """Keyframes on a smooth random walk (height 1.5 m, AR(1) velocity,
    heading along the velocity, horizontal optical axis) inside a
    10 x 10 x 3 m volume of points; each point seen by 4-15 keyframes drawn
    with visibility weight exp(-depth / 3 m); 2% outlier pixels.  With
    ``smooth`` the keyframes follow a video-like track instead (8 cm steps,
    a few degrees of turn per keyframe; see _smooth_track), as a SLAM front
    end would select them.  ``bad_assoc_frac`` of the (inlier) observations
    become wrong data associations: the pixel of another point seen by the
    same keyframe (labelled as outliers; drawn after everything else, so 0
    leaves the problem unchanged)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fx, fy, cx, cy, w, h = CAMERA
    kf = []
    if smooth:
        for pos, theta in _smooth_track(rng, n_kf):
            R = _look_rotation(np.array([np.cos(theta), np.sin(theta), 0.0]), np.array([0.0, 0.0, 1.0]))
            kf.append(_pack(R, np.array([pos[0], pos[1], 1.5])))
    else:
        pos = rng.uniform(2.0, 8.0, 2)
        ang = rng.uniform(0, 2 * np.pi)
        v = 0.1 * np.array([np.cos(ang), np.sin(ang)])
        for _ in range(n_kf):
            heading = np.array([v[0], v[1], 0.0])
            R = _look_rotation(heading, np.array([0.0, 0.0, 1.0]))
            kf.append(_pack(R, np.array([pos[0], pos[1], 1.5])))
            v = 0.9 * v + rng.normal(0.0, 0.05, 2)
            if np.linalg.norm(v) < 1e-3:
                v = v + 1e-3
            pos = pos + v
            for d in range(2):
                if pos[d] < 2.0:
                    pos[d] = 4.0 - pos[d]
                    v[d] = abs(v[d])
                elif pos[d] > 8.0:
                    pos[d] = 16.0 - pos[d]
                    v[d] = -abs(v[d])
    kf_true = np.array(kf)
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([10.0, 10.0, 3.0])
    accepted, vis_rows = [], []
    tries = 0
    while sum(a.shape[0] for a in accepted) < n_lm:
        tries += 1
        if tries > 2000:
            raise RuntimeError("landmark rejection sampling did not finish")
        X = rng.uniform(lo, hi, (4096, 3))
        pc = _camera_points(kf_true, X)                       # (n_kf, n, 3)
        vis = _visible(pc, fx, fy, cx, cy, w, h, 0.5)         # (n_kf, n)
        ok = vis.sum(axis=0) >= obs_range[0]
        accepted.append(X[ok])
        vis_rows.append(vis[:, ok].T)
    lm_true = np.concatenate(accepted)[:n_lm]
    vis = np.concatenate(vis_rows)[:n_lm]
    depth = _camera_points(kf_true, lm_true)[..., 2].T        # (n_lm, n_kf)
    weights = np.where(vis, np.exp(-depth / 3.0), 0.0)
    counts = rng.integers(obs_range[0], obs_range[1] + 1, n_lm)
    counts = np.minimum(counts, vis.sum(axis=1))
    obs_lm, obs_kf = _weighted_subsets(rng, weights, counts)
    pc = np.einsum("nij,nj->ni", kf_true[obs_kf, :9].reshape(-1, 3, 3), lm_true[obs_lm]) + kf_true[obs_kf, 9:]
    uv = _pixels(pc, fx, fy, cx, cy) + rng.normal(0.0, noise_px, (obs_kf.size, 2))
    outlier = rng.uniform(size=obs_kf.size) < outlier_frac
    n_out = int(outlier.sum())
    uv[outlier] = np.stack([rng.uniform(0, w, n_out), rng.uniform(0, h, n_out)], axis=1)
    kf_init, lm_init = _perturb_init(rng, kf_true, lm_true, rot_sigma, pos_sigma, lm_sigma, set(anchors))
    if bad_assoc_frac > 0.0:
        uv, outlier = _bad_associations(rng, obs_kf, uv, outlier, bad_assoc_frac)
    params = dict(damping=0.4, huber_nsigma=2.0, sigma_px=1.0, iterations=1000, conv_tol=1e-6)
    return _finish(name or f"walk{n_kf}x{n_lm}", seed, CAMERA, kf_true, kf_init, lm_true, lm_init,
                   obs_kf, obs_lm, uv, outlier, anchors, params)


def _bad_associations(rng, obs_kf, uv, outlier, frac):
    """Wrong correspondences: a ``frac`` share of the inlier observations take
    the pixel of another observation of the same keyframe."""
    uv = uv.copy()
    outlier = outlier.copy()
    pick = (rng.uniform(size=obs_kf.size) < frac) & ~outlier
    by_kf = {}
    for i, k in enumerate(obs_kf):
        by_kf.setdefault(int(k), []).append(i)
    src = uv.copy()
    for i in np.flatnonzero(pick):
        same = by_kf[int(obs_kf[i])]
        if len(same) < 2:
            continue
        j = i
        while j == i:
            j = same[int(rng.integers(len(same)))]
        uv[i] = src[j]
        outlier[i] = True
    return uv, outlier


def make_loop(seed: int = 0, n_kf: int = 2000, n_lm: int = 200_000, loops: int = 2,
              radius: float = 30.0, obs_range=(5, 15), outlier_frac: float = 0.02,
              noise_px: float = 1.0, rot_sigma: float = 0.05, pos_sigma: float = 0.1,
              lm_sigma: float = 0.1, anchors=(0,)) -> Problem:
    """Large looping trajectory (``loops`` laps of a 30 m circle with a
    random-walk wobble); points in an annulus around the path; revisits on the
    second lap give loop closures.  About 10 observations per point."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fx, fy, cx, cy, w, h = CAMERA
    wobble = np.zeros(3)
    kf = []
    for i in range(n_kf):
        a = 2.0 * np.pi * loops * i / n_kf
        wobble = 0.95 * wobble + rng.normal(0.0, [0.05, 0.05, 0.02])
        c = np.array([radius * np.cos(a), radius * np.sin(a), 1.5]) + wobble
        tangent = np.array([-np.sin(a), np.cos(a), 0.0])
        yaw = rng.normal(0.0, 0.03)
        fwd = np.cos(yaw) * tangent + np.sin(yaw) * np.array([np.cos(a), np.sin(a), 0.0])
        R = _look_rotation(fwd, np.array([0.0, 0.0, 1.0]))
        kf.append(_pack(R, c))
    kf_true = np.array(kf)
    accepted, counts_all, pairs = [], [], []
    n_acc = 0
    tries = 0
    while n_acc < n_lm:
        tries += 1
        if tries > 4000:
            raise RuntimeError("landmark rejection sampling did not finish")
        m = 2048
        r = np.sqrt(rng.uniform((radius - 12.0) ** 2, (radius + 12.0) ** 2, m))
        th = rng.uniform(0, 2 * np.pi, m)
        X = np.stack([r * np.cos(th), r * np.sin(th), rng.uniform(0.0, 5.0, m)], axis=1)
        pc = _camera_points(kf_true, X)
        vis = _visible(pc, fx, fy, cx, cy, w, h, 1.0) & (pc[..., 2] < 25.0)
        ok = vis.sum(axis=0) >= obs_range[0]
        X, vis, depth = X[ok], vis[:, ok].T, pc[..., 2][:, ok].T
        take = min(X.shape[0], n_lm - n_acc)
        X, vis, depth = X[:take], vis[:take], depth[:take]
        weights = np.where(vis, np.exp(-depth / 10.0), 0.0)
        cnt = np.minimum(rng.integers(obs_range[0], obs_range[1] + 1, take), vis.sum(axis=1))
        rows, cols = _weighted_subsets(rng, weights, cnt)
        pairs.append((rows + n_acc, cols))
        accepted.append(X)
        n_acc += take
    lm_true = np.concatenate(accepted)
    obs_lm = np.concatenate([p[0] for p in pairs])
    obs_kf = np.concatenate([p[1] for p in pairs])
    pc = np.einsum("nij,nj->ni", kf_true[obs_kf, :9].reshape(-1, 3, 3), lm_true[obs_lm]) + kf_true[obs_kf, 9:]
    uv = _pixels(pc, fx, fy, cx, cy) + rng.normal(0.0, noise_px, (obs_kf.size, 2))
    outlier = rng.uniform(size=obs_kf.size) < outlier_frac
    n_out = int(outlier.sum())
    uv[outlier] = np.stack([rng.uniform(0, w, n_out), rng.uniform(0, h, n_out)], axis=1)
    kf_init, lm_init = _perturb_init(rng, kf_true, lm_true, rot_sigma, pos_sigma, lm_sigma, set(anchors))
    params = dict(damping=0.4, huber_nsigma=2.0, sigma_px=1.0, iterations=200)
    return _finish(f"loop{n_kf}x{n_lm}", seed, CAMERA, kf_true, kf_init, lm_true, lm_init,
                   obs_kf, obs_lm, uv, outlier, anchors, params)


def make_batch(n_problems: int = 256, first_seed: int = 0, kf_range=(10, 200),
               lm_range=(100, 5000)) -> list[Problem]:
    """Independent walk problems of uneven size; problem i is seeded by
    ``first_seed + i`` and draws its keyframe and point counts uniformly."""
    out = []
    for i in range(n_problems):
        seed = first_seed + i
        rng = np.random.Generator(np.random.PCG64(seed))
        n_kf = int(rng.integers(kf_range[0], kf_range[1] + 1))
        n_lm = int(rng.integers(lm_range[0], lm_range[1] + 1))
        out.append(make_walk(seed=seed, n_kf=n_kf, n_lm=n_lm, name=f"batch{seed}"))
    return out


def make_chain(n_kf: int = 3, seed: int = 0, noise_px: float = 1.0) -> Problem:
    """Tree-shaped graph kf0-lm0-kf1-lm1-...-kf(n-1): every point is seen by
    exactly two consecutive keyframes, so the factor graph has no loops."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fx, fy, cx, cy, w, h = CAMERA
    kf = []
    for i in range(n_kf):
        c = np.array([0.3 * i, 0.0, 0.0])
        R = _look_rotation(np.array([0.0, 0.0, 1.0]), np.array([0.0, -1.0, 0.0]))
        kf.append(_pack(R, c))
    kf_true = np.array(kf)
    lm_true = np.array([[0.3 * j + 0.15, 0.1 * (-1) ** j, 3.0 + 0.2 * j] for j in range(n_kf - 1)])
    obs_kf, obs_lm = [], []
    for j in range(n_kf - 1):
        obs_kf += [j, j + 1]
        obs_lm += [j, j]
    obs_kf = np.array(obs_kf)
    obs_lm = np.array(obs_lm)
    pc = np.einsum("nij,nj->ni", kf_true[obs_kf, :9].reshape(-1, 3, 3), lm_true[obs_lm]) + kf_true[obs_kf, 9:]
    uv = _pixels(pc, fx, fy, cx, cy) + rng.normal(0.0, noise_px, (obs_kf.size, 2))
    kf_init, lm_init = _perturb_init(rng, kf_true, lm_true, 0.02, 0.05, 0.05, set())
    params = dict(damping=0.0, huber_nsigma=0.0, sigma_px=1.0, iterations=20)
    return _finish(f"chain{n_kf}", seed, CAMERA, kf_true, kf_init, lm_true, lm_init,
                   obs_kf, obs_lm, uv, np.zeros(obs_kf.size, bool), (), params)


@dataclass
class StreamStep:
    kf: int                    # keyframe index in the growing graph
    obs_lm: np.ndarray         # (n,) int32 landmark indices in the growing graph
    obs_uv: np.ndarray         # (n, 2) pixels
    n_new_lm: int              # landmarks first seen by this keyframe (the last n_new_lm indices)
    kf_Rt_true: np.ndarray     # (12,) ground truth pose of the new keyframe
    new_lm_true: np.ndarray    # (n_new_lm, 3) ground truth of the new landmarks


def stream_plan(p: Problem, start_kf: int):
    """Split a problem into an initial graph (keyframes < start_kf and the
    points they see) and one step per later keyframe, landmarks renumbered in
    order of first appearance (Sec. 9.2 incremental SLAM)."""
    first = np.full(p.n_lm, p.n_kf, dtype=np.int64)
    np.minimum.at(first, p.obs_lm, p.obs_kf)
    order = np.lexsort((np.arange(p.n_lm), first))            # by first observing keyframe
    order = order[first[order] < p.n_kf]
    new_id = np.full(p.n_lm, -1, dtype=np.int64)
    new_id[order] = np.arange(order.size)
    init_lm = order[first[order] < start_kf]
    sel = p.obs_kf < start_kf
    init = Problem(name=p.name + f"_first{start_kf}", seed=p.seed, fx=p.fx, fy=p.fy, cx=p.cx, cy=p.cy,
                   width=p.width, height=p.height, kf_Rt_true=p.kf_Rt_true[:start_kf],
                   kf_Rt_init=p.kf_Rt_init[:start_kf], lm_true=p.lm_true[init_lm], lm_init=p.lm_init[init_lm],
                   obs_kf=p.obs_kf[sel].astype(np.int32), obs_lm=new_id[p.obs_lm[sel]].astype(np.int32),
                   obs_uv=p.obs_uv[sel], obs_outlier=p.obs_outlier[sel],
                   anchor_kf=p.anchor_kf[p.anchor_kf < start_kf], params=dict(p.params))
    steps = []
    for k in range(start_kf, p.n_kf):
        idx = np.nonzero(p.obs_kf == k)[0]
        lm_new = order[first[order] == k]
        steps.append(StreamStep(kf=k, obs_lm=new_id[p.obs_lm[idx]].astype(np.int32), obs_uv=p.obs_uv[idx],
                                n_new_lm=int(lm_new.size), kf_Rt_true=p.kf_Rt_true[k], new_lm_true=p.lm_true[lm_new]))
    return init, steps


def make_stream(seed: int = 0, n_kf: int = 500, n_lm: int = 8000, start_kf: int = 10):
    """Incremental-SLAM stream over one video-like walk (smooth track, a few
    degrees and 8 cm between keyframes): the initial graph and the steps
    that add one keyframe each (see stream_plan)."""
    p = make_walk(seed=seed, n_kf=n_kf, n_lm=n_lm, obs_range=(4, 15), name=f"stream{n_kf}x{n_lm}", smooth=True)
    return stream_plan(p, start_kf)


def concat(problems: list[Problem], name: str | None = None) -> Problem:
    """Several independent problems as one disconnected graph: keyframe,
    landmark and observation arrays are stacked with index offsets (a batch
    of problems for one launch).  All problems must share the camera."""
    kf_off = np.cumsum([0] + [p.n_kf for p in problems])
    lm_off = np.cumsum([0] + [p.n_lm for p in problems])
    p0 = problems[0]
    cat = lambda attr: np.concatenate([getattr(p, attr) for p in problems])
    return Problem(name=name or f"batch{len(problems)}", seed=p0.seed, fx=p0.fx, fy=p0.fy, cx=p0.cx, cy=p0.cy,
                   width=p0.width, height=p0.height, kf_Rt_true=cat("kf_Rt_true"), kf_Rt_init=cat("kf_Rt_init"),
                   lm_true=cat("lm_true"), lm_init=cat("lm_init"),
                   obs_kf=np.concatenate([p.obs_kf + kf_off[i] for i, p in enumerate(problems)]).astype(np.int32),
                   obs_lm=np.concatenate([p.obs_lm + lm_off[i] for i, p in enumerate(problems)]).astype(np.int32),
                   obs_uv=cat("obs_uv"), obs_outlier=cat("obs_outlier"),
                   anchor_kf=np.concatenate([p.anchor_kf + kf_off[i] for i, p in enumerate(problems)]).astype(np.int32),
                   params=dict(p0.params))


def subgraph(p: Problem, n_kf: int, min_obs: int = 2) -> Problem:
    """The part of ``p`` seen by its first ``n_kf`` keyframes: those
    keyframes, every point observed at least ``min_obs`` times by them, and
    those observations, re-indexed (anchors among the kept keyframes stay
    anchored)."""
    m = p.obs_kf < n_kf
    cnt = np.bincount(p.obs_lm[m], minlength=p.n_lm)
    keep_lm = np.flatnonzero(cnt >= min_obs)
    remap = np.full(p.n_lm, -1, dtype=np.int64)
    remap[keep_lm] = np.arange(keep_lm.size)
    keep = m & (remap[p.obs_lm] >= 0)
    return Problem(name=f"{p.name}_kf{n_kf}", seed=p.seed, fx=p.fx, fy=p.fy, cx=p.cx, cy=p.cy,
                   width=p.width, height=p.height, kf_Rt_true=p.kf_Rt_true[:n_kf].copy(),
                   kf_Rt_init=p.kf_Rt_init[:n_kf].copy(), lm_true=p.lm_true[keep_lm].copy(),
                   lm_init=p.lm_init[keep_lm].copy(), obs_kf=p.obs_kf[keep].astype(np.int32),
                   obs_lm=remap[p.obs_lm[keep]].astype(np.int32), obs_uv=p.obs_uv[keep].copy(),
                   obs_outlier=p.obs_outlier[keep].copy(),
                   anchor_kf=p.anchor_kf[p.anchor_kf < n_kf].astype(np.int32), params=dict(p.params))


def workload(name: str, seed: int = 0) -> Problem:
    """Named workloads: 'circle' (10 kf / 100 points / ~450 factors),
    'walk' (125 kf / 1919 points / ~15k factors), 'loop' (2000 kf / 200k
    points / ~2M factors)."""
    if name == "circle":
        return make_circle(seed=seed)
    if name == "walk":
        return make_walk(seed=seed)
    if name == "loop":
        return make_loop(seed=seed)
    raise KeyError(name)
