"""Levenberg-Marquardt bundle adjustment with a dense Schur complement, on the
CPU: the comparison baseline of the paper's timing experiments (Sec. 9.1),
written for this project (``lm_ba.c``; plain single-threaded C).

It minimises the energy of GBP's factors -- reprojection errors
under the Huber loss (Sec. 6), the weak priors of Sec. 4 at their final
strength (Sec. 8) and the anchor of the first keyframe -- in the same chart
(every variable perturbs its initial value).  ``LM(problem).solve()`` runs to
convergence; ``step`` runs single iterations for timing curves.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lm_ba.c")
_LIB = os.path.join(_HERE, "liblm_ba.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lm_ba.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp, _SRC,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("n_kf", C.c_int), ("n_lm", C.c_int), ("n_obs", C.c_int), ("n_anchor", C.c_int),
                ("Rref", C.POINTER(C.c_double)), ("cref", C.POINTER(C.c_double)), ("lref", C.POINTER(C.c_double)),
                ("obs_kf", C.POINTER(C.c_int)), ("obs_lm", C.POINTER(C.c_int)), ("obs_uv", C.POINTER(C.c_double)),
                ("anchor_kf", C.POINTER(C.c_int)),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("sigma", C.c_double), ("huber_n", C.c_double), ("z_min", C.c_double),
                ("prior_scale", C.c_double), ("anchor_scale", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.lm_create.restype = C.c_void_p
        L.lm_create.argtypes = [C.POINTER(_Problem)]
        L.lm_destroy.argtypes = [C.c_void_p]
        L.lm_iterate.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.lm_cost.restype = C.c_double
        L.lm_cost.argtypes = [C.c_void_p]
        L.lm_converged.argtypes = [C.c_void_p]
        L.lm_state.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def reprojection_error(p, kf_Rt, lm_xyz, mask=None, z_min=0.05):
    """Mean |z - pi(R X + t)| over the observations (optionally masked) whose
    point lies at least z_min in front of its camera (Sec. 9.1's ARE)."""
    R = kf_Rt[p.obs_kf, :9].reshape(-1, 3, 3)
    pc = np.einsum("nij,nj->ni", R, lm_xyz[p.obs_lm]) + kf_Rt[p.obs_kf, 9:]
    ok = pc[:, 2] >= z_min
    if mask is not None:
        ok &= mask
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = np.stack([p.fx * pc[:, 0] / pc[:, 2] + p.cx, p.fy * pc[:, 1] / pc[:, 2] + p.cy], axis=1)
    return float(np.linalg.norm(uv[ok] - p.obs_uv[ok], axis=1).mean()) if ok.any() else 0.0


class LM:
    """One problem (a ``synth.Problem``); parameters as GBP's: huber_nsigma,
    sigma_px, z_min, prior_final_scale, anchor_scale."""

    def __init__(self, p, huber_nsigma=0.0, sigma_px=1.0, z_min=0.05, prior_final_scale=0.01, anchor_scale=1e3):
        Rt = np.ascontiguousarray(p.kf_Rt_init, dtype=np.float64)
        R = Rt[:, :9].reshape(-1, 3, 3)
        self._R = np.ascontiguousarray(R.reshape(-1, 9))
        self._c = np.ascontiguousarray(-np.einsum("kji,kj->ki", R, Rt[:, 9:]))
        self._l = np.ascontiguousarray(p.lm_init, dtype=np.float64)
        self._ok = np.ascontiguousarray(p.obs_kf, dtype=np.int32)
        self._ol = np.ascontiguousarray(p.obs_lm, dtype=np.int32)
        self._uv = np.ascontiguousarray(p.obs_uv, dtype=np.float64)
        self._an = np.ascontiguousarray(p.anchor_kf, dtype=np.int32)
        self.n_kf, self.n_lm = p.n_kf, p.n_lm
        prob = _Problem(p.n_kf, p.n_lm, p.n_obs, int(self._an.size), _d(self._R), _d(self._c), _d(self._l),
                        _i(self._ok), _i(self._ol), _d(self._uv), _i(self._an), p.fx, p.fy, p.cx, p.cy,
                        float(sigma_px), float(huber_nsigma), float(z_min), float(prior_final_scale),
                        float(anchor_scale))
        self._h = C.c_void_p(lib().lm_create(C.byref(prob)))
        self.iterations = 0

    def step(self, n: int = 1, tol: float = 1e-10) -> int:
        k = lib().lm_iterate(self._h, int(n), float(tol))
        self.iterations += k
        return k

    def solve(self, max_iters: int = 100, tol: float = 1e-10) -> int:
        while self.iterations < max_iters and not self.converged:
            if self.step(1, tol) == 0:
                break
        return self.iterations

    @property
    def converged(self) -> bool:
        return bool(lib().lm_converged(self._h))

    @property
    def cost(self) -> float:
        return lib().lm_cost(self._h)

    def world(self):
        kf, lm = np.zeros((self.n_kf, 12)), np.zeros((self.n_lm, 3))
        lib().lm_state(self._h, _d(kf), _d(lm))
        return kf, lm

    def close(self):
        if getattr(self, "_h", None):
            lib().lm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
