"""FP64 CPU oracle for GBP bundle adjustment -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library; the
two only see the same seeded inputs from ``paper_2003_03134_gb300.synth``.

``build()`` compiles ``gbp_oracle.c`` with gcc into ``liboracle_gbp.so`` next
to it, and the same source with OpenMP into ``liboracle_gbp_omp.so`` (factors
of an iteration, and variables of a belief update, run in parallel with the
same arithmetic in the same order, so its results are bit for bit those of
the single-threaded build); ``Oracle`` wraps one graph through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gbp.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_gbp_omp.so")
_lib = None
_lib_omp = None


def _compile(out, extra, force):
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gbp_oracle.h"))):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99, -O2, no fast-math) if out of date, and
    its OpenMP build (skipped if the compiler has no OpenMP)."""
    _compile(_LIB, ["-Wno-unknown-pragmas"], force)
    try:
        _compile(_LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass
    return _LIB


def omp_available() -> bool:
    build()
    return os.path.exists(_LIB_OMP)


class _Cam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("damping", C.c_double), ("huber_nsigma", C.c_double), ("sigma_px", C.c_double),
                ("prior_final_scale", C.c_double), ("prior_anneal_iters", C.c_int),
                ("anchor_scale", C.c_double), ("z_min", C.c_double), ("linear", C.c_int),
                ("relin_beta", C.c_double), ("relin_interval", C.c_int), ("undamped_iters", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib(omp: bool = False):
    """The oracle's ctypes handle; omp=True: its OpenMP build (threads from
    OMP_NUM_THREADS, default all cores)."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            if not omp_available():
                raise RuntimeError("the oracle's OpenMP build is not available")
            _lib_omp = _declare(C.CDLL(_LIB_OMP))
        return _lib_omp
    if _lib is None:
        build()
        _lib = _declare(C.CDLL(_LIB))
    return _lib


def _declare(L):
    if True:
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Cam), C.POINTER(_Params), C.c_int, _D, C.c_int, _D,
                                 C.c_int, _I, _I, _D, C.c_int, _I]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_iterate.argtypes = [C.c_void_p, C.c_int, _D]
        L.orc_iterations_done.argtypes = [C.c_void_p]
        L.orc_get_means.argtypes = [C.c_void_p, _D, _D]
        L.orc_get_world.argtypes = [C.c_void_p, _D, _D]
        L.orc_get_beliefs.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.orc_get_prior_diag.argtypes = [C.c_void_p, _D, _D]
        L.orc_get_messages.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.orc_are.restype = C.c_double
        L.orc_are.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte), _I]
        L.orc_are_vs.restype = C.c_double
        L.orc_are_vs.argtypes = [C.c_void_p, _D, _D, _I]
        L.orc_huber_count.argtypes = [C.c_void_p]
        L.orc_relinearisations.argtypes = [C.c_void_p]
        L.orc_add_keyframe.argtypes = [C.c_void_p, _D, C.c_int, _D, C.c_int, _I, _D]
        L.orc_sizes.argtypes = [C.c_void_p, _I, _I, _I]
        L.orc_relinearisations.restype = C.c_long
        L.orc_held_messages.argtypes = [C.c_void_p]
        L.orc_held_messages.restype = C.c_long
        L.orc_so3_exp.argtypes = [_D, _D]
        L.orc_so3_left_jacobian.argtypes = [_D, _D]
        L.orc_huber_weight.restype = C.c_double
        L.orc_huber_weight.argtypes = [C.c_double, C.c_double]
        L.orc_prior_scale.restype = C.c_double
        L.orc_prior_scale.argtypes = [C.POINTER(_Params), C.c_int]
        L.orc_project.restype = C.c_double
        L.orc_project.argtypes = [C.POINTER(_Cam), _D, _D, _D, _D, _D, _D]
        L.orc_linearise.argtypes = [C.POINTER(_Cam), C.POINTER(_Params), _D, _D, _D, _D, _D, _D,
                                    _D, _D, _D, _D, _D]
        L.orc_factor_message.argtypes = [_D, _D, C.c_int, _D, _D, _D, _D]
        L.orc_net_forward.restype = C.c_double
        L.orc_net_forward.argtypes = [_D, _D]
        L.orc_set_damping_net.argtypes = [C.c_void_p, _D]
        L.orc_set_reference_messages.argtypes = [C.c_void_p, _D]
        L.orc_set_reference_messages.restype = None
        L.orc_iterate_record.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.orc_get_relin_iters.argtypes = [C.c_void_p, _I]
        L.orc_get_relin_iters.restype = None
        L.orc_set_messages.argtypes = [C.c_void_p, _D, _D, _D, _D]
        _U = C.POINTER(C.c_ubyte)
        L.orc_set_part.argtypes = [C.c_void_p, _U, _U]
        L.orc_factor_phase.argtypes = [C.c_void_p]
        L.orc_belief_phase.argtypes = [C.c_void_p, _D]
        for name in ("orc_get_new_kf_messages", "orc_put_new_kf_messages"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, _I, _D, _D]
            getattr(L, name).restype = None
        for name in ("orc_get_kf_beliefs", "orc_put_kf_beliefs"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, _I, _D]
            getattr(L, name).restype = None
    return L


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


DEFAULTS = dict(damping=0.4, huber_nsigma=0.0, sigma_px=1.0, prior_final_scale=0.01,
                prior_anneal_iters=10, anchor_scale=1e3, z_min=0.05, linear=0,
                relin_beta=0.01, relin_interval=10, undamped_iters=8)


def make_params(**kw) -> _Params:
    p = dict(DEFAULTS)
    for k, v in kw.items():
        if k in p:
            p[k] = v
    return _Params(float(p["damping"]), float(p["huber_nsigma"]), float(p["sigma_px"]),
                   float(p["prior_final_scale"]), int(p["prior_anneal_iters"]), float(p["anchor_scale"]),
                   float(p["z_min"]), int(p["linear"]), float(p["relin_beta"]), int(p["relin_interval"]),
                   int(p["undamped_iters"]))


def make_cam(fx, fy, cx, cy) -> _Cam:
    return _Cam(float(fx), float(fy), float(cx), float(cy))


# ---------------------------------------------------------------------------
# unit pieces

def so3_exp(w):
    w = _f64(w)
    R = np.zeros(9)
    lib().orc_so3_exp(_dp(w), _dp(R))
    return R.reshape(3, 3)


def so3_left_jacobian(w):
    w = _f64(w)
    J = np.zeros(9)
    lib().orc_so3_left_jacobian(_dp(w), _dp(J))
    return J.reshape(3, 3)


def huber_weight(M, nsigma):
    return lib().orc_huber_weight(float(M), float(nsigma))


def prior_scale(t, **kw):
    p = make_params(**kw)
    return lib().orc_prior_scale(C.byref(p), int(t))


def project(cam, Rref, cref, lref, xk, xl):
    uv = np.zeros(2)
    c = make_cam(*cam)
    Rref, cref, lref, xk, xl = (_f64(a) for a in (Rref, cref, lref, xk, xl))
    depth = lib().orc_project(C.byref(c), _dp(Rref), _dp(cref), _dp(lref), _dp(xk), _dp(xl), _dp(uv))
    return uv, depth


def linearise(cam, Rref, cref, lref, xk, xl, z, **kw):
    c = make_cam(*cam)
    p = make_params(**kw)
    J, r, k, A, cv = np.zeros(18), np.zeros(2), np.zeros(1), np.zeros(81), np.zeros(9)
    Rref, cref, lref, xk, xl, z = (_f64(a) for a in (Rref, cref, lref, xk, xl, z))
    active = lib().orc_linearise(C.byref(c), C.byref(p), _dp(Rref), _dp(cref), _dp(lref), _dp(xk), _dp(xl),
                                 _dp(z), _dp(J), _dp(r), _dp(k), _dp(A), _dp(cv))
    return dict(active=bool(active), J=J.reshape(2, 9), r=r, k=float(k[0]), A=A.reshape(9, 9), c=cv)


def factor_message(A, c, target, lam_in, eta_in):
    A, c, lam_in, eta_in = _f64(A), _f64(c), _f64(lam_in), _f64(eta_in)
    na = 6 if target == 0 else 3
    lam_out, eta_out = np.zeros(na * na), np.zeros(na)
    rc = lib().orc_factor_message(_dp(A), _dp(c), int(target), _dp(lam_in), _dp(eta_in), _dp(lam_out), _dp(eta_out))
    if rc != 0:
        raise np.linalg.LinAlgError("matrix to invert is not positive definite")
    return lam_out.reshape(na, na), eta_out


N_FEAT, N_NET_PARAMS = 16, 5313


def net_forward(params, x) -> float:
    """The damping network's output for one feature row (FP64, in C)."""
    p, xv = _f64(params), _f64(x)
    assert p.size == N_NET_PARAMS and xv.size == N_FEAT
    return lib().orc_net_forward(_dp(p), _dp(xv))


# ---------------------------------------------------------------------------

class Oracle:
    """One GBP graph in the FP64 oracle."""

    def __init__(self, problem, anchors=None, omp=False, **params):
        """omp=True runs the OpenMP build (same results, all cores)."""
        self.p = problem
        self._L = lib(omp)
        self._cam = make_cam(problem.fx, problem.fy, problem.cx, problem.cy)
        self._prm = make_params(**params)
        self.params = dict(DEFAULTS, **{k: v for k, v in params.items() if k in DEFAULTS})
        self._kf = _f64(problem.kf_Rt_init)
        self._lm = _f64(problem.lm_init)
        self._ok = np.ascontiguousarray(problem.obs_kf, dtype=np.int32)
        self._ol = np.ascontiguousarray(problem.obs_lm, dtype=np.int32)
        self._uv = _f64(problem.obs_uv)
        anc = problem.anchor_kf if anchors is None else anchors
        self._anc = np.ascontiguousarray(anc, dtype=np.int32)
        h = self._L.orc_create(C.byref(self._cam), C.byref(self._prm), problem.n_kf, _dp(self._kf),
                             problem.n_lm, _dp(self._lm), problem.n_obs, _ip(self._ok), _ip(self._ol),
                             _dp(self._uv), int(self._anc.size), _ip(self._anc))
        if not h:
            raise ValueError("oracle rejected the problem")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and getattr(self, "_L", None) is not None:
            self._L.orc_destroy(h)
            self._h = None

    def iterate(self, n: int) -> float:
        d = C.c_double(0.0)
        if self._L.orc_iterate(self._h, int(n), C.byref(d)) != 0:
            raise FloatingPointError("a belief stopped being positive definite")
        return d.value

    def run_to_convergence(self, tol: float, max_iters: int, chunk: int = 1):
        it = 0
        d = np.inf
        while it < max_iters:
            d = self.iterate(chunk)
            it += chunk
            if d < tol:
                break
        return it, d

    @property
    def t(self) -> int:
        return self._L.orc_iterations_done(self._h)

    def means(self):
        nk, nl, _ = self.sizes()
        kf, lm = np.zeros((nk, 6)), np.zeros((nl, 3))
        self._L.orc_get_means(self._h, _dp(kf), _dp(lm))
        return kf, lm

    def world(self):
        nk, nl, _ = self.sizes()
        kf, lm = np.zeros((nk, 12)), np.zeros((nl, 3))
        self._L.orc_get_world(self._h, _dp(kf), _dp(lm))
        return kf, lm

    def beliefs(self):
        nk, nl, _ = self.sizes()
        kl, ke = np.zeros((nk, 6, 6)), np.zeros((nk, 6))
        ll, le = np.zeros((nl, 3, 3)), np.zeros((nl, 3))
        self._L.orc_get_beliefs(self._h, _dp(kl), _dp(ke), _dp(ll), _dp(le))
        return kl, ke, ll, le

    def prior_diag(self):
        nk, nl, _ = self.sizes()
        kd, ld = np.zeros((nk, 6)), np.zeros((nl, 3))
        self._L.orc_get_prior_diag(self._h, _dp(kd), _dp(ld))
        return kd, ld

    def messages(self):
        n = self.sizes()[2]
        a, b, c, d = np.zeros((n, 6, 6)), np.zeros((n, 6)), np.zeros((n, 3, 3)), np.zeros((n, 3))
        self._L.orc_get_messages(self._h, _dp(a), _dp(b), _dp(c), _dp(d))
        return a, b, c, d

    def are(self, mask=None):
        cnt = C.c_int(0)
        if mask is None:
            v = self._L.orc_are(self._h, None, C.byref(cnt))
        else:
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            v = self._L.orc_are(self._h, m.ctypes.data_as(C.POINTER(C.c_ubyte)), C.byref(cnt))
        return v, cnt.value

    def are_vs(self, ref_kf_Rt, ref_lm):
        cnt = C.c_int(0)
        a, b = _f64(ref_kf_Rt), _f64(ref_lm)
        v = self._L.orc_are_vs(self._h, _dp(a), _dp(b), C.byref(cnt))
        return v, cnt.value

    def huber_count(self) -> int:
        return self._L.orc_huber_count(self._h)

    def add_keyframe(self, obs_lm, obs_uv, kf_Rt_init=None, n_new_lm=0, new_lm_xyz=None) -> int:
        ol = np.ascontiguousarray(obs_lm, dtype=np.int32)
        uv = _f64(obs_uv)
        kf = None if kf_Rt_init is None else _f64(kf_Rt_init)
        nl = None if new_lm_xyz is None else _f64(new_lm_xyz)
        r = self._L.orc_add_keyframe(self._h, None if kf is None else _dp(kf), int(n_new_lm),
                                   None if nl is None else _dp(nl), ol.size, _ip(ol), _dp(uv))
        if r < 0:
            raise ValueError("oracle rejected the keyframe")
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._L.orc_sizes(self._h, C.byref(a), C.byref(b), C.byref(c))
        self.n_kf, self.n_lm, self.n_obs = a.value, b.value, c.value
        return r

    def sizes(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        self._L.orc_sizes(self._h, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def relinearisations(self) -> int:
        return self._L.orc_relinearisations(self._h)

    def relin_iters(self) -> np.ndarray:
        """Iteration of each factor's last (re)linearisation, observation order."""
        t = np.zeros(self.sizes()[2], dtype=np.int32)
        self._L.orc_get_relin_iters(self._h, _ip(t))
        return t

    def set_messages(self, mk_lam, mk_eta, ml_lam, ml_eta):
        """Test hook: replace the current messages (the layout of messages())
        and recompute the beliefs from them."""
        n = self.sizes()[2]
        a, b = _f64(mk_lam).reshape(n, 36), _f64(mk_eta).reshape(n, 6)
        c, d = _f64(ml_lam).reshape(n, 9), _f64(ml_eta).reshape(n, 3)
        if self._L.orc_set_messages(self._h, _dp(a), _dp(b), _dp(c), _dp(d)) != 0:
            raise FloatingPointError("a belief is not positive definite")

    # one graph solved in parts (multi-rank split)
    def set_part(self, fac_mask, var_mask):
        """Compute only these factors' messages and these variables' beliefs
        (keyframes then landmarks); None = all."""
        U = C.POINTER(C.c_ubyte)
        self._fm = None if fac_mask is None else np.ascontiguousarray(fac_mask, dtype=np.uint8)
        self._vm = None if var_mask is None else np.ascontiguousarray(var_mask, dtype=np.uint8)
        self._L.orc_set_part(self._h, None if self._fm is None else self._fm.ctypes.data_as(U),
                             None if self._vm is None else self._vm.ctypes.data_as(U))

    def factor_phase(self):
        if self._L.orc_factor_phase(self._h) != 0:
            raise RuntimeError("the factor phase runs the fixed schedule only")

    def belief_phase(self) -> float:
        d = C.c_double(0.0)
        if self._L.orc_belief_phase(self._h, C.byref(d)) != 0:
            raise FloatingPointError("a belief stopped being positive definite")
        return d.value

    def new_kf_messages(self, factors):
        f = np.ascontiguousarray(factors, dtype=np.int32)
        lam, eta = np.zeros((f.size, 36)), np.zeros((f.size, 6))
        self._L.orc_get_new_kf_messages(self._h, f.size, _ip(f), _dp(lam), _dp(eta))
        return lam, eta

    def put_new_kf_messages(self, factors, lam, eta):
        f = np.ascontiguousarray(factors, dtype=np.int32)
        self._L.orc_put_new_kf_messages(self._h, f.size, _ip(f), _dp(_f64(lam)), _dp(_f64(eta)))

    def kf_beliefs(self, kfs):
        k = np.ascontiguousarray(kfs, dtype=np.int32)
        rec = np.zeros((k.size, 48))
        self._L.orc_get_kf_beliefs(self._h, k.size, _ip(k), _dp(rec))
        return rec

    def put_kf_beliefs(self, kfs, rec):
        k = np.ascontiguousarray(kfs, dtype=np.int32)
        self._L.orc_put_kf_beliefs(self._h, k.size, _ip(k), _dp(_f64(rec)))

    def held_messages(self) -> int:
        return self._L.orc_held_messages(self._h)

    # learned damping
    def set_damping_net(self, params):
        """Learned schedule with these network parameters; None: fixed schedule."""
        if params is None:
            self._L.orc_set_damping_net(self._h, None)
            return
        self._net = _f64(params)
        if self._net.size != N_NET_PARAMS or self._L.orc_set_damping_net(self._h, _dp(self._net)) != 0:
            raise ValueError("bad network parameters")

    def set_reference_messages(self, mk_eta, ml_eta):
        """Reference eta of the damping targets: (n_obs, 6) messages to the
        keyframes and (n_obs, 3) to the landmarks."""
        self._ref = np.ascontiguousarray(np.concatenate([_f64(mk_eta).reshape(-1, 6), _f64(ml_eta).reshape(-1, 3)],
                                                        axis=1))
        self._L.orc_set_reference_messages(self._h, _dp(self._ref))

    def capture_messages(self):
        """The current messages become the reference."""
        _, mk_eta, _, ml_eta = self.messages()
        self.set_reference_messages(mk_eta, ml_eta)

    def iterate_record(self, n: int):
        """n iterations of the fixed schedule; returns features (n, n_obs, 16)
        and damping targets (n, n_obs) in observation order."""
        nf = self.sizes()[2]
        X, T = np.zeros((n, nf, N_FEAT)), np.zeros((n, nf))
        rc = self._L.orc_iterate_record(self._h, int(n), _dp(X), _dp(T))
        if rc == -2:
            raise RuntimeError("no reference messages set")
        if rc != 0:
            raise FloatingPointError("a belief stopped being positive definite")
        return X, T
