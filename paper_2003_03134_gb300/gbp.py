"""Python binding of libgbp (include/gbp.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; all GBP work runs in the CUDA kernels behind
``libgbp.so``.  Loading fails loudly when the library is missing: there is no
CPU fallback.

Arrays: poses ``kf_Rt`` are (n_kf, 12) float64 (R row-major, t; world to
camera), points (n_lm, 3) float64, observations int32 indices and (n_obs, 2)
float64 pixels.  ``stream`` is a ``cudaStream_t`` as an int (for example
``torch.cuda.current_stream().cuda_stream``) or None for the default stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbp.so")

GBP_OK, GBP_EINVAL, GBP_ENOMEM, GBP_ECUDA, GBP_EDIVERGED, GBP_ETIMEOUT, GBP_ESTATE = range(7)


class GBPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class gbp_intrinsics(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32)]


class gbp_params(C.Structure):
    _fields_ = [("damping", C.c_float), ("huber_nsigma", C.c_float), ("sigma_px", C.c_float),
                ("iterations", C.c_int32), ("conv_tol", C.c_float), ("check_every", C.c_int32),
                ("prior_final_scale", C.c_float), ("prior_anneal_iters", C.c_int32),
                ("anchor_scale", C.c_float), ("z_min", C.c_float), ("relin_beta", C.c_float),
                ("relin_interval", C.c_int32), ("undamped_iters", C.c_int32),
                ("fp64_pivot_ratio", C.c_float), ("precision_mode", C.c_int32), ("linear", C.c_int32),
                ("launch_mode", C.c_int32), ("damping_mode", C.c_int32), ("factor_shape", C.c_int32),
                ("persistent_shape", C.c_int32), ("fp64_exact_cavity", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


GBP_MAX_TUNING_CANDIDATES = 12


class gbp_tuning(C.Structure):
    _fields_ = [("launch_mode", C.c_int32), ("factor_shape", C.c_int32), ("persistent_shape", C.c_int32),
                ("factor_threads", C.c_int32), ("factor_min_blocks", C.c_int32),
                ("persistent_min_blocks", C.c_int32), ("tile_factors", C.c_int32), ("n_candidates", C.c_int32),
                ("cand_mode", C.c_int32 * GBP_MAX_TUNING_CANDIDATES),
                ("cand_shape", C.c_int32 * GBP_MAX_TUNING_CANDIDATES),
                ("cand_ms", C.c_double * GBP_MAX_TUNING_CANDIDATES)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_[:8]}
        d["candidates"] = [{"launch_mode": self.cand_mode[i], "shape": self.cand_shape[i], "ms": self.cand_ms[i]}
                           for i in range(self.n_candidates)]
        return d


class gbp_problem_desc(C.Structure):
    _fields_ = [("n_kf", C.c_int32), ("kf_Rt", C.POINTER(C.c_double)), ("n_lm", C.c_int32),
                ("lm_xyz", C.POINTER(C.c_double)), ("n_obs", C.c_int32), ("obs_kf", C.POINTER(C.c_int32)),
                ("obs_lm", C.POINTER(C.c_int32)), ("obs_uv", C.POINTER(C.c_double)), ("n_anchor", C.c_int32),
                ("anchor_kf", C.POINTER(C.c_int32))]


class gbp_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("max_dmu", C.c_float), ("are", C.c_double),
                ("are_ref", C.c_double), ("n_are", C.c_int32), ("huber_count", C.c_int32),
                ("fp64_fallbacks", C.c_int32), ("relinearisations", C.c_int32), ("launch_mode", C.c_int32),
                ("kernel_launches", C.c_int64), ("held_messages", C.c_int32),
                ("fp64_resums", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)
_lib = None

# exported names, in header order
EXPORTS = ["gbp_default_params", "gbp_create_graph", "gbp_set_params", "gbp_get_params", "gbp_iterate",
           "gbp_reset", "gbp_get_beliefs", "gbp_get_means", "gbp_set_reference", "gbp_add_keyframe",
           "gbp_get_stats", "gbp_get_sizes", "gbp_profile_iterations", "gbp_destroy_graph", "gbp_status_string",
           "gbp_last_error", "gbp_reprojection_error_noalloc", "gbp_autotune", "gbp_create_batch",
           "gbp_get_batch_info", "gbp_get_problem_are", "gbp_mlp_create", "gbp_mlp_set_params",
           "gbp_mlp_get_params", "gbp_mlp_forward", "gbp_mlp_gradient", "gbp_mlp_train_step", "gbp_mlp_destroy",
           "gbp_set_damping_model", "gbp_capture_messages", "gbp_get_factor_order", "gbp_record_iterations",
           "gbp_get_relin_iters", "gbp_get_tuning", "gbp_get_residuals", "gbp_set_partition", "gbp_split_phase",
           "gbp_get_split_records", "gbp_put_split_records"]
GBP_SPLIT_MSG_FLOATS = 20
GBP_SPLIT_KF_FLOATS = 56
GBP_MLP_NFEAT = 16
GBP_MLP_NPARAM = 5313
GBP_NOALLOC_MAX_OBS = 1 << 20


def lib() -> C.CDLL:
    """Load libgbp.so (built by ``paper_2003_03134_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgbp.so not found at {LIB_PATH}: build it with "
                           "`python -m paper_2003_03134_gb300.build` (there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.gbp_default_params.argtypes = [C.POINTER(gbp_params)]
    L.gbp_default_params.restype = None
    L.gbp_create_graph.argtypes = [C.POINTER(gbp_intrinsics), C.c_int32, _D, C.c_int32, _D, C.c_int32, _I, _I, _D,
                                   C.c_int32, _I, vp, C.POINTER(vp)]
    L.gbp_set_params.argtypes = [vp, C.POINTER(gbp_params)]
    L.gbp_get_params.argtypes = [vp, C.POINTER(gbp_params)]
    L.gbp_iterate.argtypes = [vp, C.c_int32, _I]
    L.gbp_reset.argtypes = [vp]
    L.gbp_get_beliefs.argtypes = [vp, _D, _D, _D, _D]
    L.gbp_get_means.argtypes = [vp, _D, _D]
    L.gbp_set_reference.argtypes = [vp, _D, _D]
    L.gbp_add_keyframe.argtypes = [vp, _D, C.c_int32, _D, C.c_int32, _I, _D, _I]
    L.gbp_get_stats.argtypes = [vp, C.POINTER(gbp_stats)]
    L.gbp_get_sizes.argtypes = [vp, _I, _I, _I]
    L.gbp_get_relin_iters.argtypes = [vp, _I]
    L.gbp_get_residuals.argtypes = [vp, _D]
    L.gbp_set_partition.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
    L.gbp_split_phase.argtypes = [vp, C.c_int32]
    L.gbp_get_split_records.argtypes = [vp, C.c_int32, C.c_int32, _I, C.POINTER(C.c_float)]
    L.gbp_put_split_records.argtypes = [vp, C.c_int32, C.c_int32, _I, C.POINTER(C.c_float)]
    L.gbp_profile_iterations.argtypes = [vp, C.c_int32, _D]
    L.gbp_autotune.argtypes = [vp, C.c_int32, _I, _D]
    L.gbp_get_tuning.argtypes = [vp, C.POINTER(gbp_tuning)]
    L.gbp_create_batch.argtypes = [C.POINTER(gbp_intrinsics), C.c_int32, C.POINTER(gbp_problem_desc), vp,
                                   C.POINTER(vp)]
    L.gbp_get_batch_info.argtypes = [vp, _I, _I, _I, _I]
    L.gbp_get_problem_are.argtypes = [vp, _D, _I, _I]
    L.gbp_destroy_graph.argtypes = [vp]
    L.gbp_destroy_graph.restype = None
    L.gbp_status_string.argtypes = [C.c_int]
    L.gbp_status_string.restype = C.c_char_p
    L.gbp_last_error.argtypes = [vp]
    L.gbp_last_error.restype = C.c_char_p
    L.gbp_reprojection_error_noalloc.argtypes = [C.POINTER(gbp_intrinsics), C.c_double, C.c_int32, vp, C.c_int32, vp,
                                                 C.c_int32, vp, vp, vp, vp, vp]
    _F = C.POINTER(C.c_float)
    L.gbp_mlp_create.argtypes = [_F, vp, C.POINTER(vp)]
    L.gbp_mlp_set_params.argtypes = [vp, _F]
    L.gbp_mlp_get_params.argtypes = [vp, _F]
    L.gbp_mlp_forward.argtypes = [vp, vp, C.c_int32, vp]
    L.gbp_mlp_gradient.argtypes = [vp, vp, vp, C.c_int32, _F, _D]
    L.gbp_mlp_train_step.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_float, _F]
    L.gbp_mlp_destroy.argtypes = [vp]
    L.gbp_mlp_destroy.restype = None
    L.gbp_set_damping_model.argtypes = [vp, vp]
    L.gbp_capture_messages.argtypes = [vp]
    L.gbp_record_iterations.argtypes = [vp, C.c_int32, vp, vp]
    L.gbp_get_factor_order.argtypes = [vp, _I]
    _lib = L
    return L


def _check(status: int, handle=None):
    if status != GBP_OK:
        L = lib()
        what = L.gbp_status_string(status).decode()
        detail = L.gbp_last_error(handle).decode() if handle else ""
        raise GBPError(status, f"{what}: {detail}" if detail else what)


def _f64(a, cols=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_I)


# ---------------------------------------------------------------------------
# entry points

def gbp_default_params() -> gbp_params:
    p = gbp_params()
    lib().gbp_default_params(C.byref(p))
    return p


def gbp_create_graph(intrinsics, kf_Rt, lm_xyz, obs_kf, obs_lm, obs_uv, anchor_kf=(), stream=None) -> int:
    fx, fy, cx, cy, w, h = intrinsics
    intr = gbp_intrinsics(fx, fy, cx, cy, int(w), int(h))
    kf = _f64(kf_Rt, 12)
    lm = _f64(lm_xyz, 3)
    ok, ol = _i32(obs_kf), _i32(obs_lm)
    uv = _f64(obs_uv, 2)
    an = _i32(anchor_kf)
    out = C.c_void_p()
    st = lib().gbp_create_graph(C.byref(intr), kf.shape[0], _dp(kf), lm.shape[0], _dp(lm), ok.size, _ip(ok),
                                _ip(ol), _dp(uv), an.size, _ip(an), C.c_void_p(stream or 0), C.byref(out))
    _check(st)
    return out.value


def gbp_create_batch(intrinsics, problems, stream=None) -> int:
    """problems: sequence of objects with kf_Rt_init, lm_init, obs_kf, obs_lm,
    obs_uv, anchor_kf (e.g. synth.Problem)."""
    fx, fy, cx, cy, w, h = intrinsics
    intr = gbp_intrinsics(fx, fy, cx, cy, int(w), int(h))
    keep = []
    descs = (gbp_problem_desc * len(problems))()
    for i, p in enumerate(problems):
        kf, lm = _f64(p.kf_Rt_init, 12), _f64(p.lm_init, 3)
        ok, ol, uv, an = _i32(p.obs_kf), _i32(p.obs_lm), _f64(p.obs_uv, 2), _i32(p.anchor_kf)
        keep += [kf, lm, ok, ol, uv, an]
        descs[i] = gbp_problem_desc(kf.shape[0], _dp(kf), lm.shape[0], _dp(lm), ok.size, _ip(ok), _ip(ol), _dp(uv),
                                    an.size, _ip(an))
    out = C.c_void_p()
    st = lib().gbp_create_batch(C.byref(intr), len(problems), descs, C.c_void_p(stream or 0), C.byref(out))
    _check(st)
    return out.value


def gbp_get_batch_info(g: int):
    n = C.c_int32()
    _check(lib().gbp_get_batch_info(g, C.byref(n), None, None, None), g)
    kf = np.zeros(n.value + 1, np.int32)
    lm = np.zeros(n.value + 1, np.int32)
    obs = np.zeros(max(n.value, 1), np.int32)
    _check(lib().gbp_get_batch_info(g, C.byref(n), _ip(kf), _ip(lm), _ip(obs)), g)
    return kf, lm, obs[:n.value]


def gbp_get_problem_are(g: int):
    kf, _, _ = gbp_get_batch_info(g)
    n = kf.size - 1
    are = np.zeros(max(n, 1))
    cnt = np.zeros(max(n, 1), np.int32)
    hub = np.zeros(max(n, 1), np.int32)
    _check(lib().gbp_get_problem_are(g, _dp(are), _ip(cnt), _ip(hub)), g)
    return are[:n], cnt[:n], hub[:n]


def gbp_set_params(g: int, params: gbp_params) -> None:
    _check(lib().gbp_set_params(g, C.byref(params)), g)


def gbp_get_params(g: int) -> gbp_params:
    p = gbp_params()
    _check(lib().gbp_get_params(g, C.byref(p)), g)
    return p


def gbp_iterate(g: int, n_iters: int = 0) -> int:
    done = C.c_int32(0)
    _check(lib().gbp_iterate(g, int(n_iters), C.byref(done)), g)
    return done.value


def gbp_reset(g: int) -> None:
    _check(lib().gbp_reset(g), g)


def gbp_get_sizes(g: int):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().gbp_get_sizes(g, C.byref(a), C.byref(b), C.byref(c)), g)
    return a.value, b.value, c.value


def gbp_get_beliefs(g: int, covariances: bool = False):
    n_kf, n_lm, _ = gbp_get_sizes(g)
    kf = np.zeros((n_kf, 12))
    lm = np.zeros((n_lm, 3))
    kc = np.zeros((n_kf, 6, 6)) if covariances else None
    lc = np.zeros((n_lm, 3, 3)) if covariances else None
    _check(lib().gbp_get_beliefs(g, _dp(kf), _dp(lm), _dp(kc), _dp(lc)), g)
    return (kf, lm, kc, lc) if covariances else (kf, lm)


def gbp_get_means(g: int):
    n_kf, n_lm, _ = gbp_get_sizes(g)
    kf = np.zeros((n_kf, 6))
    lm = np.zeros((n_lm, 3))
    _check(lib().gbp_get_means(g, _dp(kf), _dp(lm)), g)
    return kf, lm


def gbp_set_reference(g: int, ref_kf_Rt, ref_lm_xyz) -> None:
    if ref_kf_Rt is None:
        _check(lib().gbp_set_reference(g, None, None), g)
        return
    a, b = _f64(ref_kf_Rt, 12), _f64(ref_lm_xyz, 3)
    _check(lib().gbp_set_reference(g, _dp(a), _dp(b)), g)


def gbp_add_keyframe(g: int, kf_Rt_init, new_lm_xyz, n_new_lm: int, obs_lm, obs_uv) -> int:
    kf = None if kf_Rt_init is None else _f64(kf_Rt_init).reshape(12)
    nl = None if new_lm_xyz is None else _f64(new_lm_xyz, 3)
    ol = _i32(obs_lm)
    uv = _f64(obs_uv, 2)
    idx = C.c_int32(-1)
    _check(lib().gbp_add_keyframe(g, _dp(kf), int(n_new_lm), _dp(nl), ol.size, _ip(ol), _dp(uv), C.byref(idx)), g)
    return idx.value


def gbp_get_relin_iters(g: int) -> np.ndarray:
    """Iteration of each observation's last (re)linearisation (observation order)."""
    n = gbp_get_sizes(g)[2]
    t = np.zeros(n, dtype=np.int32)
    _check(lib().gbp_get_relin_iters(g, _ip(t)), g)
    return t


def gbp_get_residuals(g: int) -> np.ndarray:
    """Reprojection error of every observation at the current means
    (observation order), -1 where the point is closer than z_min."""
    e = np.zeros(gbp_get_sizes(g)[2])
    _check(lib().gbp_get_residuals(g, _dp(e)), g)
    return e


def gbp_set_partition(g: int, kf_range, lm_range) -> None:
    """This graph's part of a graph split across ranks (None: the whole graph)."""
    if lm_range is None:
        _check(lib().gbp_set_partition(g, 0, 0, 0, -1), g)
    else:
        _check(lib().gbp_set_partition(g, int(kf_range[0]), int(kf_range[1]), int(lm_range[0]), int(lm_range[1])), g)


def gbp_split_phase(g: int, phase: int) -> None:
    _check(lib().gbp_split_phase(g, int(phase)), g)


def gbp_get_split_records(g: int, kind: int, index) -> np.ndarray:
    idx = _i32(index)
    width = GBP_SPLIT_MSG_FLOATS if kind == 0 else GBP_SPLIT_KF_FLOATS
    out = np.zeros((idx.size, width), dtype=np.float32)
    _check(lib().gbp_get_split_records(g, int(kind), idx.size, _ip(idx), out.ctypes.data_as(C.POINTER(C.c_float))), g)
    return out


def gbp_put_split_records(g: int, kind: int, index, recs) -> None:
    idx = _i32(index)
    width = GBP_SPLIT_MSG_FLOATS if kind == 0 else GBP_SPLIT_KF_FLOATS
    r = np.ascontiguousarray(recs, dtype=np.float32).reshape(idx.size, width)
    _check(lib().gbp_put_split_records(g, int(kind), idx.size, _ip(idx), r.ctypes.data_as(C.POINTER(C.c_float))), g)


def gbp_get_stats(g: int) -> gbp_stats:
    s = gbp_stats()
    _check(lib().gbp_get_stats(g, C.byref(s)), g)
    return s


def gbp_autotune(g: int, n_trial: int = 8):
    """Time both launch modes; returns (chosen mode, ms/iteration of mode 1, of mode 2)."""
    chosen = C.c_int32(0)
    ms = np.zeros(2)
    _check(lib().gbp_autotune(g, int(n_trial), C.byref(chosen), _dp(ms)), g)
    return chosen.value, float(ms[0]), float(ms[1])


def gbp_get_tuning(g: int) -> dict:
    t = gbp_tuning()
    _check(lib().gbp_get_tuning(g, C.byref(t)), g)
    return t.as_dict()


def gbp_profile_iterations(g: int, n_iters: int):
    """(mean device ms per iteration in the current launch mode, mean ms of one factor-kernel launch)."""
    out = np.zeros(2)
    _check(lib().gbp_profile_iterations(g, int(n_iters), _dp(out)), g)
    return float(out[0]), float(out[1])


def gbp_reprojection_error_noalloc(intrinsics, z_min, n_kf, kf_Rt_ptr, n_lm, lm_xyz_ptr, n_obs, obs_kf_ptr,
                                   obs_lm_ptr, obs_uv_ptr, out_ptr, stream=None) -> None:
    """Average reprojection error of caller-owned device arrays (raw device
    pointers as ints) into out_ptr[0:2] = (mean error px, count), with no
    allocation: for callers that cannot allocate device memory at that
    point.  Observations with an out-of-range index are left out.
    Asynchronous on ``stream``."""
    fx, fy, cx, cy, w, h = intrinsics
    intr = gbp_intrinsics(fx, fy, cx, cy, int(w), int(h))
    _check(lib().gbp_reprojection_error_noalloc(C.byref(intr), float(z_min), int(n_kf), kf_Rt_ptr, int(n_lm),
                                                lm_xyz_ptr, int(n_obs), obs_kf_ptr, obs_lm_ptr, obs_uv_ptr, out_ptr,
                                                C.c_void_p(stream or 0)))


def gbp_destroy_graph(g: int) -> None:
    if g:
        lib().gbp_destroy_graph(g)


# --- learned damping network (device arrays are passed as raw pointers) ---

def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def gbp_mlp_create(params, stream=None) -> int:
    w = _f32(params, GBP_MLP_NPARAM)
    out = C.c_void_p()
    _check(lib().gbp_mlp_create(w.ctypes.data_as(C.POINTER(C.c_float)), C.c_void_p(stream or 0), C.byref(out)))
    return out.value


def gbp_mlp_set_params(net: int, params) -> None:
    w = _f32(params, GBP_MLP_NPARAM)
    _check(lib().gbp_mlp_set_params(net, w.ctypes.data_as(C.POINTER(C.c_float))))


def gbp_mlp_get_params(net: int) -> np.ndarray:
    w = np.empty(GBP_MLP_NPARAM, dtype=np.float32)
    _check(lib().gbp_mlp_get_params(net, w.ctypes.data_as(C.POINTER(C.c_float))))
    return w


def gbp_mlp_forward(net: int, X_ptr: int, count: int, y_ptr: int) -> None:
    """Predictions for ``count`` rows of device features (count x 16 float32)
    into device ``y`` (count float32); asynchronous."""
    _check(lib().gbp_mlp_forward(net, X_ptr, int(count), y_ptr))


def gbp_mlp_gradient(net: int, X_ptr: int, target_ptr: int, count: int):
    """(loss, gradient as a float32 vector of GBP_MLP_NPARAM) of the mean
    squared error over ``count`` device rows."""
    g = np.empty(GBP_MLP_NPARAM, dtype=np.float32)
    loss = C.c_double()
    _check(lib().gbp_mlp_gradient(net, X_ptr, target_ptr, int(count), g.ctypes.data_as(C.POINTER(C.c_float)),
                                  C.byref(loss)))
    return loss.value, g


def gbp_mlp_train_step(net: int, X_ptr: int, target_ptr: int, idx_ptr, count: int, lr: float,
                       want_loss: bool = False):
    """One Adam step on rows ``idx`` (device int32 pointer, or None for rows
    0..count) of device X / target.  Returns the minibatch loss when
    ``want_loss`` (synchronising), else None (asynchronous)."""
    loss = C.c_float()
    _check(lib().gbp_mlp_train_step(net, X_ptr, target_ptr, idx_ptr or None, int(count), float(lr),
                                    C.byref(loss) if want_loss else None))
    return float(loss.value) if want_loss else None


def gbp_mlp_destroy(net: int) -> None:
    if net:
        lib().gbp_mlp_destroy(net)


def gbp_set_damping_model(g: int, net) -> None:
    """Copy the network's weights into graph ``g`` (``net`` None removes them)."""
    _check(lib().gbp_set_damping_model(g, net or None), g)


def gbp_capture_messages(g: int) -> None:
    _check(lib().gbp_capture_messages(g), g)


def gbp_get_factor_order(g: int) -> np.ndarray:
    """Caller observation index of each internal factor (the record rows)."""
    n = gbp_get_sizes(g)[2]
    out = np.zeros(n, dtype=np.int32)
    _check(lib().gbp_get_factor_order(g, _ip(out)), g)
    return out


def gbp_record_iterations(g: int, n_iters: int, X_ptr: int, target_ptr: int) -> None:
    """Run ``n_iters`` iterations with the fixed schedule, writing n_iters x
    n_obs feature rows (16 float32 each) to device ``X`` and damping targets
    to device ``target``."""
    _check(lib().gbp_record_iterations(g, int(n_iters), X_ptr, target_ptr), g)


# ---------------------------------------------------------------------------

class Graph:
    """Owning wrapper around one gbp_graph handle.  ``problem`` is one
    problem or a list of problems (a batch, see gbp_create_batch)."""

    def __init__(self, problem, stream=None, **params):
        self.problem = problem
        if isinstance(problem, (list, tuple)):
            self.h = gbp_create_batch(problem[0].intrinsics(), problem, stream)
        else:
            self.h = gbp_create_graph(problem.intrinsics(), problem.kf_Rt_init, problem.lm_init, problem.obs_kf,
                                      problem.obs_lm, problem.obs_uv, problem.anchor_kf, stream)
        if params:
            self.set_params(**params)

    def batch_info(self):
        return gbp_get_batch_info(self.h)

    def problem_are(self):
        return gbp_get_problem_are(self.h)

    def set_params(self, **kw):
        p = gbp_get_params(self.h)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        gbp_set_params(self.h, p)

    @property
    def params(self) -> dict:
        return gbp_get_params(self.h).as_dict()

    def iterate(self, n: int = 0) -> int:
        return gbp_iterate(self.h, n)

    def reset(self):
        gbp_reset(self.h)

    def beliefs(self, covariances=False):
        return gbp_get_beliefs(self.h, covariances)

    def means(self):
        return gbp_get_means(self.h)

    def stats(self) -> dict:
        return gbp_get_stats(self.h).as_dict()

    def profile(self, n: int):
        return gbp_profile_iterations(self.h, n)

    def relin_iters(self) -> np.ndarray:
        return gbp_get_relin_iters(self.h)

    def residuals(self) -> np.ndarray:
        return gbp_get_residuals(self.h)

    def autotune(self, n_trial: int = 8):
        return gbp_autotune(self.h, n_trial)

    def tuning(self) -> dict:
        return gbp_get_tuning(self.h)

    def set_reference(self, kf_Rt, lm_xyz):
        gbp_set_reference(self.h, kf_Rt, lm_xyz)

    def add_keyframe(self, obs_lm, obs_uv, kf_Rt_init=None, n_new_lm=0, new_lm_xyz=None) -> int:
        return gbp_add_keyframe(self.h, kf_Rt_init, new_lm_xyz, n_new_lm, obs_lm, obs_uv)

    def set_damping_model(self, net):
        """``net``: a DampingNet (its current weights are copied) or None."""
        gbp_set_damping_model(self.h, net.h if net is not None else None)

    def capture_messages(self):
        gbp_capture_messages(self.h)

    def record(self, n_iters: int, X_ptr: int, target_ptr: int):
        gbp_record_iterations(self.h, n_iters, X_ptr, target_ptr)

    def factor_order(self) -> np.ndarray:
        return gbp_get_factor_order(self.h)

    def close(self):
        if getattr(self, "h", None):
            gbp_destroy_graph(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DampingNet:
    """Owning wrapper around one gbp_mlp handle."""

    def __init__(self, params, stream=None):
        self.h = gbp_mlp_create(params, stream)

    @property
    def params(self) -> np.ndarray:
        return gbp_mlp_get_params(self.h)

    def set_params(self, params):
        gbp_mlp_set_params(self.h, params)

    def forward(self, X_ptr: int, count: int, y_ptr: int):
        gbp_mlp_forward(self.h, X_ptr, count, y_ptr)

    def gradient(self, X_ptr: int, target_ptr: int, count: int):
        return gbp_mlp_gradient(self.h, X_ptr, target_ptr, count)

    def train_step(self, X_ptr: int, target_ptr: int, count: int, lr: float, idx_ptr=None, want_loss=False):
        return gbp_mlp_train_step(self.h, X_ptr, target_ptr, idx_ptr, count, lr, want_loss)

    def close(self):
        if getattr(self, "h", None):
            gbp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
