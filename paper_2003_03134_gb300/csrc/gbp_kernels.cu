// gbp_kernels.cu -- CUDA kernels (sm_103a) of one synchronous GBP iteration
// for bundle adjustment (Ortiz et al., "Bundle Adjustment on a Graph
// Processor", CVPR 2020), templated on the storage/arithmetic type R
// (float: the fast path with an FP64 fallback; double: a full-precision
// mode).
//
// Iteration t (Sec. 5, synchronous schedule):
//   factor kernel  -- a warp per tile of whole landmarks, a lane per factor:
//                     both incoming messages, the relinearisation test
//                     (Sec. 5, Sec. 8), the Jacobian and residual at the
//                     factor's linearisation point, the Huber weight
//                     (Sec. 6), both factor-to-variable messages (eqs.
//                     messageeta, messagelambda), damping of eta (Sec. 5,
//                     Sec. 8); the beliefs of the landmarks inside the tile.
//   belief kernel  -- a block (small graphs) or a warp per keyframe: a
//                     fixed-order reduction of its messages, expanded from
//                     their compact form: prior(t+1) + sum of messages
//                     (eqs. beliefeta, belieflambda), its Cholesky factor
//                     and mean.
// No atomics touch floating-point sums: every reduction has a fixed order,
// so results are bitwise reproducible.
//
// Message arithmetic.  A factor's information is rank 2: Lambda_f = W J^T J
// and eta_f = W J^T y with y = J x0 + r (Sec. 4).  Marginalising block b
// (incoming precision P_b = Lambda_belief_b - Lambda_msg_b and vector
// q_b = eta_belief_b - eta_msg_b) out of the product of the factor and the
// incoming message gives, by the matrix inversion lemma, exactly
//   Lambda_{f->a} = J_a^T M J_a,  eta_{f->a} = J_a^T g,  M = W N,  g = M (y - s)
// with Q = J_b P_b^-1 J_b^T (2x2), s = J_b P_b^-1 q_b, N = (I + W Q)^-1.
// This equals the printed Schur complement A_aa - A_ab (A_bb + P_b)^-1 A_ba
// and never forms a 9x9 matrix.  Messages are stored as (M, g): 5 numbers
// per side.  Damping eta (Sec. 5) damps g, since a factor's J changes only
// when it relinearises, and messages are never damped then (Sec. 8).  The
// keyframe's incoming precision B - J^T M J is never formed: with B's
// Cholesky factor L (computed once per keyframe by the belief kernel) every
// quantity reduces to 2x2 ones (KfSide), so no factor factorises a 6x6.
#include "gbp_internal.h"
#include "gbp_mlp.cuh"

#include <math.h>

#include <algorithm>
#include <utility>

namespace gbp {

// ------------------------------------------------------------------------
// small dense helpers

__host__ __device__ constexpr int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

// 1/x: correctly rounded reciprocal in FP32 (cheaper than a division),
// plain division in FP64.
template <typename R>
__device__ __forceinline__ R rcp(R x) {
    if constexpr (sizeof(R) == 4) return __frcp_rn(x);
    else return R(1) / x;
}

// (sqrt(s), 1/sqrt(s)) for s > 0.  FP32: hardware reciprocal square root
// refined by one Newton-Raphson step y <- y (3 - s y^2) / 2; FP64: exact.
template <typename R>
__device__ __forceinline__ void sqrt_pair(R s, R& d, R& id) {
    if constexpr (sizeof(R) == 4) {
        float y = rsqrtf(fmaxf(s, 1.17549435e-38f));
        y = y * (1.5f - 0.5f * s * y * y);
        id = y;
        d = s * y;
    } else {
        d = sqrt(fmax(s, R(0)));
        id = R(1) / d;
    }
}

// In-place Cholesky of a packed lower-triangular n x n SPD matrix.
// On return A holds L (packed) and inv_d[i] = 1 / L_ii.  Returns false if a
// pivot is not positive and finite; pivot_ratio = min pivot / max pivot.
// Columns (and rows of the substitutions) recurse on a template index so
// that every loop bound is a compile-time constant and the packed matrix
// stays in registers.
template <typename R, int n, int j>
struct CholCol {
    static __device__ __forceinline__ void run(R* A, R* inv_d, R& pmin, R& pmax, bool& ok) {
        if constexpr (j < n) {
            R s = A[pk(j, j)];
#pragma unroll
            for (int p = 0; p < j; ++p) s -= A[pk(j, p)] * A[pk(j, p)];
            ok = ok && (s > R(0)) && isfinite(s);
            if (j == 0) { pmin = s; pmax = s; }
            pmin = fmin(pmin, s);
            pmax = fmax(pmax, s);
            R d, id;
            sqrt_pair<R>(s, d, id);
            A[pk(j, j)] = d;
            inv_d[j] = id;
#pragma unroll
            for (int i = j + 1; i < n; ++i) {
                R t = A[pk(i, j)];
#pragma unroll
                for (int p = 0; p < j; ++p) t -= A[pk(i, p)] * A[pk(j, p)];
                A[pk(i, j)] = t * id;
            }
            CholCol<R, n, j + 1>::run(A, inv_d, pmin, pmax, ok);
        }
    }
};

template <typename R, int n>
__device__ __forceinline__ bool chol_packed(R* A, R* inv_d, R& pivot_ratio) {
    R pmin = R(0), pmax = R(0);
    bool ok = true;
    CholCol<R, n, 0>::run(A, inv_d, pmin, pmax, ok);
    pivot_ratio = ok ? pmin * rcp(pmax) : R(0);
    return ok;
}

template <typename R, int n, int i>
struct FwdRow {
    static __device__ __forceinline__ void run(const R* L, const R* inv_d, R* b) {
        if constexpr (i < n) {
            R s = b[i];
#pragma unroll
            for (int p = 0; p < i; ++p) s -= L[pk(i, p)] * b[p];
            b[i] = s * inv_d[i];
            FwdRow<R, n, i + 1>::run(L, inv_d, b);
        }
    }
};

// b <- L^-1 b (forward substitution with a packed Cholesky factor)
template <typename R, int n>
__device__ __forceinline__ void fwd_solve(const R* L, const R* inv_d, R* b) {
    FwdRow<R, n, 0>::run(L, inv_d, b);
}

template <typename R, int n, int i>
struct BwdRow {
    static __device__ __forceinline__ void run(const R* L, const R* inv_d, R* b) {
        if constexpr (i >= 0) {
            R s = b[i];
#pragma unroll
            for (int p = i + 1; p < n; ++p) s -= L[pk(p, i)] * b[p];
            b[i] = s * inv_d[i];
            BwdRow<R, n, i - 1>::run(L, inv_d, b);
        }
    }
};

// b <- L^-T b (backward substitution)
template <typename R, int n>
__device__ __forceinline__ void bwd_solve(const R* L, const R* inv_d, R* b) {
    BwdRow<R, n, n - 1>::run(L, inv_d, b);
}

// ------------------------------------------------------------------------
// rotations: E = Exp(w) = I + a W + b W^2 and the left Jacobian
// Jl(w) = I + b W + c W^2, W = [w]x, W^2 = w w^T - |w|^2 I.
// b = (1 - cos th)/th^2 is evaluated as 2 sin^2(th/2)/th^2 and
// c = (th - sin th)/th^3 by its Taylor series below th = 0.5, which keeps
// both accurate in FP32.

template <typename R>
__device__ __forceinline__ void so3_exp_jl(const R w[3], R E[9], R J[9]) {
    R th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    R a, b, c;
    if (th2 < R(0.25)) {
        // |w| < 0.5: Taylor series of sin(x)/x, (1 - cos x)/x^2 and
        // (x - sin x)/x^3 in x^2; the first omitted term is below 3e-11
        a = R(1) + th2 * (R(-1.0 / 6.0) + th2 * (R(1.0 / 120.0) + th2 * (R(-1.0 / 5040.0) + th2 * R(1.0 / 362880.0))));
        b = R(0.5) + th2 * (R(-1.0 / 24.0) + th2 * (R(1.0 / 720.0) + th2 * (R(-1.0 / 40320.0) + th2 * R(1.0 / 3628800.0))));
        c = R(1.0 / 6.0) + th2 * (R(-1.0 / 120.0) + th2 * (R(1.0 / 5040.0) +
            th2 * (R(-1.0 / 362880.0) + th2 * R(1.0 / 39916800.0))));
    } else {
        R th = sqrt(th2);
        R st = sin(th), sh = sin(R(0.5) * th);
        a = st / th;
        b = R(2) * sh * sh / th2;
        c = (th - st) / (th2 * th);
    }
    // W^2 = w w^T - th2 I
    R W2[9] = {w[0] * w[0] - th2, w[0] * w[1], w[0] * w[2],
               w[1] * w[0], w[1] * w[1] - th2, w[1] * w[2],
               w[2] * w[0], w[2] * w[1], w[2] * w[2] - th2};
    R W[9] = {R(0), -w[2], w[1], w[2], R(0), -w[0], -w[1], w[0], R(0)};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        E[i] = a * W[i] + b * W2[i];
        J[i] = b * W[i] + c * W2[i];
    }
    E[0] += R(1); E[4] += R(1); E[8] += R(1);
    J[0] += R(1); J[4] += R(1); J[8] += R(1);
}

// ------------------------------------------------------------------------
// linearisation of one reprojection factor at x0 = [dc dw | dl] (Sec. 4)
// in the chart R_k = Exp(dw) Rref_k, c_k = cref_k + dc, l_m = lref_m + dl,
// h = pi(R_k (l_m - c_k)).  Output: Jk (2x6, columns dc then dw),
// Jl (2x3) = -Jk[:, 0:3], y = J x0 + r, W = k / sigma^2 (0 if inactive).

template <typename R>
struct Lin {
    R Jk[2][6];
    R Jl[2][3];
    R y[2];
    R W;
    R r2;   // |r|^2 (pixels^2)
};

// Rr: the keyframe's reference rotation in R; dlc = lref - cref, subtracted
// in double before rounding to R (the large world coordinates cancel there).
template <typename R>
__device__ __forceinline__ void linearise_ref(const KParams<R>& P, const R Rr[9], const R dlc[3], const R x0[9],
                                              R zu, R zv, Lin<R>& L) {
    R w[3] = {x0[3], x0[4], x0[5]};
    R E[9], Jw[9];
    so3_exp_jl(w, E, Jw);
    R Rm[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rm[i * 3 + j] = E[i * 3 + 0] * Rr[0 * 3 + j] + E[i * 3 + 1] * Rr[1 * 3 + j] + E[i * 3 + 2] * Rr[2 * 3 + j];
    R d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = dlc[i] + (x0[6 + i] - x0[i]);
    R p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) p[i] = Rm[i * 3 + 0] * d[0] + Rm[i * 3 + 1] * d[1] + Rm[i * 3 + 2] * d[2];

    if (!(p[2] >= P.z_min)) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int j = 0; j < 6; ++j) L.Jk[a][j] = R(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) L.Jl[a][j] = R(0);
            L.y[a] = R(0);
        }
        L.W = R(0);
        L.r2 = R(0);
        return;
    }
    const R fx = P.fx, fy = P.fy;
    R iz = rcp(p[2]);
    R u = fx * p[0] * iz, v = fy * p[1] * iz;
    R r0 = zu - (u + P.cx);
    R r1 = zv - (v + P.cy);
    // d pi / d p rows
    R q[2][3] = {{fx * iz, R(0), -u * iz}, {R(0), fy * iz, -v * iz}};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        // d p / d dl = Rm  ->  Jl = q Rm ;  d p / d dc = -Rm
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            R s = q[a][0] * Rm[0 * 3 + j] + q[a][1] * Rm[1 * 3 + j] + q[a][2] * Rm[2 * 3 + j];
            L.Jl[a][j] = s;
            L.Jk[a][j] = -s;
        }
        // d p / d dw = -[p]x Jl(dw):  q (-[p]x) = -(q x p)^T ... as a row: -(q cross p)
        R cx_ = q[a][1] * p[2] - q[a][2] * p[1];
        R cy_ = q[a][2] * p[0] - q[a][0] * p[2];
        R cz_ = q[a][0] * p[1] - q[a][1] * p[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) L.Jk[a][3 + j] = -(cx_ * Jw[0 * 3 + j] + cy_ * Jw[1 * 3 + j] + cz_ * Jw[2 * 3 + j]);
    }
    // Huber weight (Sec. 6) on the Mahalanobis distance M = |r| / sigma
    R r2 = r0 * r0 + r1 * r1;
    R k = R(1);
    if (P.huber_n > R(0)) {
        R M = sqrt(r2) * P.inv_sigma;
        R N = P.huber_n;
        if (M > N) {
            R iM = rcp(M);
            k = R(2) * N * iM - (N * N) * (iM * iM);
        }
    }
    L.W = k * P.inv_sigma2;
    L.r2 = r2;
    // y = J x0 + r ;  J x0 = Jk[:,0:3] (dc - dl) + Jk[:,3:6] dw
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        R s = (a == 0 ? r0 : r1);
#pragma unroll
        for (int j = 0; j < 3; ++j) s += L.Jk[a][j] * (x0[j] - x0[6 + j]) + L.Jk[a][3 + j] * x0[3 + j];
        L.y[a] = s;
    }
}

template <typename R>
__device__ __forceinline__ void load_refs(const double* __restrict__ Rref, const double* __restrict__ cref,
                                          const double* __restrict__ lref, R Rr[9], R dlc[3]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Rr[i] = R(Rref[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) dlc[i] = R(lref[i] - cref[i]);
}

template <typename R>
__device__ __forceinline__ void linearise(const KParams<R>& P, const double* __restrict__ Rref,
                                          const double* __restrict__ cref, const double* __restrict__ lref,
                                          const R x0[9], R zu, R zv, Lin<R>& L) {
    R Rr[9], dlc[3];
    load_refs<R>(Rref, cref, lref, Rr, dlc);
    linearise_ref<R>(P, Rr, dlc, x0, zu, zv, L);
}

// ------------------------------------------------------------------------
// messages in compact form.  A factor's information is W J^T J with J the
// 2 x 9 Jacobian, so each factor-to-variable message is J_a^T M J_a (M a
// symmetric 2 x 2) with eta J_a^T g.  Marginalising block b with incoming
// precision P_b and vector q_b (Sec. 5) gives, by the matrix inversion lemma,
//   Q = J_b P_b^-1 J_b^T,  s = J_b P_b^-1 q_b,  N = (I + W Q)^-1,
//   M = W N,  g = M (y - s).
// This equals the printed Schur complement A_aa - A_ab (A_bb + P_b)^-1 A_ba.

template <typename R> struct Vec4;
template <> struct Vec4<float> { typedef float4 T; };
template <> struct Vec4<double> { typedef double4_32a T; };

template <typename R, int N>
__device__ __forceinline__ void load_rec(const R* __restrict__ src, R* dst) {
    static_assert(N % 4 == 0, "record length");
    typedef typename Vec4<R>::T V;
    const V* s = reinterpret_cast<const V*>(src);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        V v = s[i];
        dst[4 * i + 0] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
    }
}

template <typename R, int N>
__device__ __forceinline__ void store_rec(R* dst, const R* src) {
    typedef typename Vec4<R>::T V;
    V* d = reinterpret_cast<V*>(dst);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        V v;
        v.x = src[4 * i + 0]; v.y = src[4 * i + 1]; v.z = src[4 * i + 2]; v.w = src[4 * i + 3];
        d[i] = v;
    }
}

// L2-coherent loads (bypass L1) for data that other SMs write during the
// same launch (the persistent kernel runs many iterations in one launch).
template <typename R, int N>
__device__ __forceinline__ void load_rec_cg(const R* src, R* dst) {
    if constexpr (sizeof(R) == 4) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            float4 v = __ldcg(s4 + i);
            dst[4 * i + 0] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
        }
    } else {
        const double2* s2 = reinterpret_cast<const double2*>(src);
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            double2 v = __ldcg(s2 + i);
            dst[2 * i + 0] = v.x; dst[2 * i + 1] = v.y;
        }
    }
}

// An iteration index kept in a Real slot of a record, by its bits.
template <typename R>
__device__ __forceinline__ R int_bits(int v) {
    if constexpr (sizeof(R) == 4) return __int_as_float(v);
    else return __longlong_as_double((long long)v);
}
template <typename R>
__device__ __forceinline__ int bits_int(R v) {
    if constexpr (sizeof(R) == 4) return __float_as_int(v);
    else return (int)__double_as_longlong(v);
}

// Lambda = J^T M J (packed n x n) and eta = J^T g of a compact message.
// Explicitly rounded multiply and fused multiply-add: the compiler may not
// contract or split these, so an expansion rounds the same way in every
// kernel it is inlined into, whatever the register budget.
template <typename R>
__device__ __forceinline__ R mul_rn(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}
template <typename R>
__device__ __forceinline__ R fma_rn(R a, R b, R c) {
    if constexpr (sizeof(R) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}

template <typename R, int n>
__device__ __forceinline__ void expand_msg(const R J[2][n], R M00, R M01, R M11, R g0, R g1, R* lam, R* eta) {
    R ua[n], va[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        ua[i] = fma_rn(M00, J[0][i], mul_rn(M01, J[1][i]));
        va[i] = fma_rn(M01, J[0][i], mul_rn(M11, J[1][i]));
        eta[i] = fma_rn(J[0][i], g0, mul_rn(J[1][i], g1));
    }
#pragma unroll
    for (int i = 0; i < n; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) lam[pk(i, j)] = fma_rn(ua[i], J[0][j], mul_rn(va[i], J[1][j]));
}

// tr(J^T M J) and J^T g of a compact message (learned-damping features).
template <typename R, int n>
__device__ __forceinline__ R msg_trace(const R J[2][n], R M00, R M01, R M11) {
    R a = R(0), b = R(0), c = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        a += J[0][i] * J[0][i];
        b += J[0][i] * J[1][i];
        c += J[1][i] * J[1][i];
    }
    return M00 * a + R(2) * M01 * b + M11 * c;
}
template <typename R, int n>
__device__ __forceinline__ void msg_eta(const R J[2][n], R g0, R g1, R* eta) {
#pragma unroll
    for (int i = 0; i < n; ++i) eta[i] = J[0][i] * g0 + J[1][i] * g1;
}

// Whether keyframe k's belief is formed in this graph (always, unless the
// graph is one rank's part of a split graph).
template <typename R>
__device__ __forceinline__ bool kf_in_part(const DevGraph<R>& g, int k) {
    return k >= g.kf_item_off && k < g.kf_item_off + g.kf_item_n;
}

// A factor's lin record (SoA rows y0, y1, W, |r|^2): its linearisation
// between relinearisations, with the keyframe Jacobian block in kj.
template <typename R>
__device__ __forceinline__ void store_lin(const DevGraph<R>& g, int f, const Lin<R>& L) {
    const size_t n_f = g.n_f;
    g.lin[f] = L.y[0];
    g.lin[n_f + f] = L.y[1];
    g.lin[2 * n_f + f] = L.W;
    g.lin[3 * n_f + f] = L.r2;
}

// A keyframe Jacobian block record (row 0, then row 1).
template <typename R>
__device__ __forceinline__ void store_jac(R* dst, const R J[2][6]) {
    R jr[KJ];
#pragma unroll
    for (int i = 0; i < 6; ++i) { jr[i] = J[0][i]; jr[6 + i] = J[1][i]; }
    store_rec<R, KJ>(dst, jr);
}

// M = W (I + W Q)^-1 and g = M (y - s); out = {M00, M01, M11, g0, g1}.
template <typename C>
__device__ __forceinline__ void compact_from_Qs(C Q00, C Q01, C Q11, C s0, C s1, const C y[2], C W, C* out) {
    const C a00 = C(1) + W * Q00, a01 = W * Q01, a11 = C(1) + W * Q11;
    const C idet = rcp(a00 * a11 - a01 * a01);
    const C N00 = a11 * idet, N01 = -a01 * idet, N11 = a00 * idet;
    const C M00 = W * N00, M01 = W * N01, M11 = W * N11;
    const C e0 = y[0] - s0, e1 = y[1] - s1;
    out[0] = M00;
    out[1] = M01;
    out[2] = M11;
    out[3] = M00 * e0 + M01 * e1;
    out[4] = M01 * e0 + M11 * e1;
}

// Compact message from an explicit incoming precision: Lb, inv_d its
// Cholesky factor (chol_packed), qb the incoming vector, Jb the Jacobian
// block of the marginalised variable.
template <typename C, int nb>
__device__ __forceinline__ void message_chol(const C* Lb, const C* inv_d, const C* qb, const C Jb[2][nb],
                                             const C y[2], C W, C* out) {
    C V0[nb], V1[nb], u[nb];
#pragma unroll
    for (int i = 0; i < nb; ++i) { V0[i] = Jb[0][i]; V1[i] = Jb[1][i]; u[i] = qb[i]; }
    fwd_solve<C, nb>(Lb, inv_d, V0);
    fwd_solve<C, nb>(Lb, inv_d, V1);
    fwd_solve<C, nb>(Lb, inv_d, u);
    C Q00 = C(0), Q01 = C(0), Q11 = C(0), s0 = C(0), s1 = C(0);
#pragma unroll
    for (int i = 0; i < nb; ++i) {
        Q00 += V0[i] * V0[i];
        Q01 += V0[i] * V1[i];
        Q11 += V1[i] * V1[i];
        s0 += V0[i] * u[i];
        s1 += V1[i] * u[i];
    }
    compact_from_Qs<C>(Q00, Q01, Q11, s0, s1, y, W, out);
}

// v <- L^-1 v with a keyframe belief's stored factor (packed lower, 1/L_ii
// on the diagonal), kept in registers.
template <typename R>
__device__ __forceinline__ void fwd_solve_stored(const R* Ls, R* v) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        R s = v[i];
#pragma unroll
        for (int p = 0; p < i; ++p) s -= Ls[pk(i, p)] * v[p];
        v[i] = s * Ls[pk(i, i)];
    }
}

// The keyframe side of a factor in the basis of its stored messages
// (Jacobian block Jo): with the keyframe belief B = L L^T, its mean mu and
// the factor's previous message to the keyframe Jo^T Mo Jo (eta Jo^T go),
// the incoming precision is P = B - Jo^T Mo Jo.  With Vo = L^-1 Jo^T,
// G = Vo^T Vo = Jo B^-1 Jo^T and a = Jo mu - G go:
//   P^-1 = B^-1 + B^-1 Jo^T (I - Mo G)^-1 Mo Jo B^-1,
// so every quantity of the message to the landmark reduces to 2 x 2 ones,
// and P is positive definite iff both eigenvalues of I - Mo G are positive
// (B being so); det(I - Mo G) is the share of B's precision volume left.
template <typename R>
struct KfSide {
    R G00, G01, G11;       // G = Vo^T Vo
    R a0, a1;              // Jo mu - G go
    R K00, K01, K11;       // K = (I - Mo G)^-1 Mo (symmetric)
    R det;                 // det(I - Mo G)
    bool pd;               // P positive definite
};

template <typename R>
__device__ __forceinline__ void kf_side(const R* Ls, const R* mu, const R Jo[2][6], const R* mo, KfSide<R>& s) {
    R V0[6], V1[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) { V0[i] = Jo[0][i]; V1[i] = Jo[1][i]; }
    fwd_solve_stored<R>(Ls, V0);
    fwd_solve_stored<R>(Ls, V1);
    R G00 = R(0), G01 = R(0), G11 = R(0), jm0 = R(0), jm1 = R(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        G00 += V0[i] * V0[i];
        G01 += V0[i] * V1[i];
        G11 += V1[i] * V1[i];
        jm0 += Jo[0][i] * mu[i];
        jm1 += Jo[1][i] * mu[i];
    }
    s.G00 = G00; s.G01 = G01; s.G11 = G11;
    const R M00 = mo[0], M01 = mo[1], M11 = mo[2];
    s.a0 = jm0 - (G00 * mo[3] + G01 * mo[4]);
    s.a1 = jm1 - (G01 * mo[3] + G11 * mo[4]);
    // D = I - M G
    const R D00 = R(1) - (M00 * G00 + M01 * G01), D01 = -(M00 * G01 + M01 * G11);
    const R D10 = -(M01 * G00 + M11 * G01), D11 = R(1) - (M01 * G01 + M11 * G11);
    const R det = D00 * D11 - D01 * D10;
    s.det = det;
    s.pd = det > R(0) && D00 + D11 > R(0);
    // K = D^-1 M = adj(D) M / det
    const R id = s.pd ? rcp(det) : R(0);
    s.K00 = (D11 * M00 - D01 * M01) * id;
    s.K01 = (D11 * M01 - D01 * M11) * id;
    s.K11 = (-D10 * M01 + D00 * M11) * id;
}

// Compact message to the landmark from KfSide when the basis is unchanged:
//   Q = G + G K G,  s = a + G K a.
template <typename R>
__device__ __forceinline__ void message_to_landmark(const KfSide<R>& s, const R y[2], R W, R* out) {
    const R Y00 = s.G00 * s.K00 + s.G01 * s.K01, Y01 = s.G00 * s.K01 + s.G01 * s.K11;
    const R Y10 = s.G01 * s.K00 + s.G11 * s.K01, Y11 = s.G01 * s.K01 + s.G11 * s.K11;
    compact_from_Qs<R>(s.G00 + (Y00 * s.G00 + Y01 * s.G01), s.G01 + (Y00 * s.G01 + Y01 * s.G11),
                       s.G11 + (Y10 * s.G01 + Y11 * s.G11), s.a0 + (Y00 * s.a0 + Y01 * s.a1),
                       s.a1 + (Y10 * s.a0 + Y11 * s.a1), y, W, out);
}

// ------------------------------------------------------------------------
// Rare paths, kept out of line so that their state does not weigh on the
// register allocation of the common path: arguments and results by value.

// What a linearisation needs besides the factor's x0: the keyframe's
// reference rotation and the factor's point-minus-centre difference, both
// rounded to R on the host, the pixel and the camera and noise parameters.
template <typename R>
struct LinArgs {
    const R* Rr;
    R dlc0, dlc1, dlc2;
    R zu, zv;
    R fx, fy, cx, cy, inv_sigma2, inv_sigma, huber_n, z_min;
};

template <typename R>
__device__ __forceinline__ LinArgs<R> lin_args(const KParams<R>& P, const DevGraph<R>& g, int k, int f) {
    const size_t n_f = (size_t)g.n_f;
    return LinArgs<R>{g.kf_Rr + (size_t)k * 9, g.f_dlc[f], g.f_dlc[n_f + f], g.f_dlc[2 * n_f + f],
                      g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], P.fx, P.fy, P.cx, P.cy, P.inv_sigma2, P.inv_sigma,
                      P.huber_n, P.z_min};
}

template <typename R>
__device__ __forceinline__ void lin_from_args(const LinArgs<R>& A, const R* x0, Lin<R>& L) {
    KParams<R> P{};
    P.fx = A.fx; P.fy = A.fy; P.cx = A.cx; P.cy = A.cy;
    P.inv_sigma2 = A.inv_sigma2; P.inv_sigma = A.inv_sigma; P.huber_n = A.huber_n; P.z_min = A.z_min;
    R Rr[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rr[i] = A.Rr[i];
    const R dlc[3] = {A.dlc0, A.dlc1, A.dlc2};
    linearise_ref<R>(P, Rr, dlc, x0, A.zu, A.zv, L);
}

template <typename R> struct Arr9 { R v[9]; };
template <typename R> struct Arr12 { R v[12]; };
template <typename R> struct Msg5 { R v[5]; };

// A factor's linearisation at x0 (its first; out of line, since it happens
// once per linearisation point while the stored one serves every other
// iteration).
template <typename R>
__device__ __noinline__ Lin<R> linearise_at(Arr9<R> x0, LinArgs<R> A) {
    Lin<R> L;
    lin_from_args<R>(A, x0.v, L);
    return L;
}

// A relinearisation in this iteration: the factor's linearisation at its
// new point x0n, and its message to the landmark in that new basis from the
// keyframe side computed in the old basis Jo (KfSide), by the two-basis form
//   Q = Gnn + Gno K Gno^T,  s = an + Gno K a,  Gno = Vn^T Vo,  an = Jn mu - Gno go.
template <typename R>
struct Rebased {
    Lin<R> L;
    R cl[5];
};

template <typename R>
__device__ __noinline__ Rebased<R> rebase(const R* kbp, Arr12<R> Jo, R go0, R go1, R a0, R a1, R K00, R K01, R K11,
                                          bool form_lm, Arr9<R> x0n, LinArgs<R> A) {
    Rebased<R> out;
    lin_from_args<R>(A, x0n.v, out.L);
    for (int i = 0; i < 5; ++i) out.cl[i] = R(0);
    if (!form_lm) return out;
    R Ls[KB_A];
    load_rec_cg<R, KB_A>(kbp, Ls);
    const R* mu = Ls + KB_MU;
    R Vo[2][6], Vn[2][6];
    for (int i = 0; i < 6; ++i) {
        Vo[0][i] = Jo.v[i]; Vo[1][i] = Jo.v[6 + i];
        Vn[0][i] = out.L.Jk[0][i]; Vn[1][i] = out.L.Jk[1][i];
    }
    fwd_solve_stored<R>(Ls, Vo[0]);
    fwd_solve_stored<R>(Ls, Vo[1]);
    fwd_solve_stored<R>(Ls, Vn[0]);
    fwd_solve_stored<R>(Ls, Vn[1]);
    R Gn00 = R(0), Gn01 = R(0), Gn11 = R(0), X00 = R(0), X01 = R(0), X10 = R(0), X11 = R(0), jm0 = R(0), jm1 = R(0);
    for (int i = 0; i < 6; ++i) {
        Gn00 += Vn[0][i] * Vn[0][i];
        Gn01 += Vn[0][i] * Vn[1][i];
        Gn11 += Vn[1][i] * Vn[1][i];
        X00 += Vn[0][i] * Vo[0][i];
        X01 += Vn[0][i] * Vo[1][i];
        X10 += Vn[1][i] * Vo[0][i];
        X11 += Vn[1][i] * Vo[1][i];
        jm0 += out.L.Jk[0][i] * mu[i];
        jm1 += out.L.Jk[1][i] * mu[i];
    }
    const R an0 = jm0 - (X00 * go0 + X01 * go1), an1 = jm1 - (X10 * go0 + X11 * go1);
    const R Y00 = X00 * K00 + X01 * K01, Y01 = X00 * K01 + X01 * K11;
    const R Y10 = X10 * K00 + X11 * K01, Y11 = X10 * K01 + X11 * K11;
    compact_from_Qs<R>(Gn00 + (Y00 * X00 + Y01 * X01), Gn01 + (Y00 * X10 + Y01 * X11), Gn11 + (Y10 * X10 + Y11 * X11),
                       an0 + (Y00 * a0 + Y01 * a1), an1 + (Y10 * a0 + Y11 * a1), out.L.y, out.L.W, out.cl);
    return out;
}

// FP64 redo for an incoming precision the FP32 arithmetic cannot take: the
// incoming precision formed in FP64 from FP32 state; *_ok decides whether it
// is positive definite, *_message (same decision) forms the compact message
// (M00, M01, M11, g0, g1) in FP64 from the factor's FP32 linearisation (its
// Jacobian and residual are well conditioned; the incoming precision is
// what FP32 cannot take).  The decision uses iteration-t state only, so it
// is taken before the relinearisation test and the message formed after it.

template <typename R>
__device__ __forceinline__ void widen_lin(const Lin<R>& L, Lin<double>& D) {
    for (int a = 0; a < 2; ++a) {
        for (int j = 0; j < 6; ++j) D.Jk[a][j] = double(L.Jk[a][j]);
        for (int j = 0; j < 3; ++j) D.Jl[a][j] = double(L.Jl[a][j]);
        D.y[a] = double(L.y[a]);
    }
    D.W = double(L.W);
    D.r2 = double(L.r2);
}

// Message to the keyframe: the landmark's incoming precision as the FP32
// path formed it (P 6, q 3).
template <typename R>
__device__ __noinline__ bool lm_incoming_ok64(Arr9<R> pq) {
    double A[6], inv_d[3], ratio;
    for (int i = 0; i < 6; ++i) A[i] = double(pq.v[i]);
    return chol_packed<double, 3>(A, inv_d, ratio);
}

template <typename R>
__device__ __noinline__ Msg5<R> lm_message64(Arr9<R> pq, Lin<R> Lf) {
    double P[6], inv_d[3], q[3], ratio;
    for (int i = 0; i < 6; ++i) P[i] = double(pq.v[i]);
    for (int i = 0; i < 3; ++i) q[i] = double(pq.v[6 + i]);
    chol_packed<double, 3>(P, inv_d, ratio);
    Lin<double> L;
    widen_lin<R>(Lf, L);
    double o[5];
    message_chol<double, 3>(P, inv_d, q, L.Jl, L.y, L.W, o);
    Msg5<R> out;
    for (int i = 0; i < 5; ++i) out.v[i] = R(o[i]);
    return out;
}

// Message to the landmark: the keyframe's incoming precision b^t - m^t in
// FP64, formed once per factor and iteration and kept (packed A 21, q 6,
// then A's Cholesky factor in place and its inverse diagonal 6) for both
// uses, the decision and the message, so that the message sees the state
// the decision saw.  First from the belief record's Lambda, eta and the
// factor's previous message (its compact record and Jacobian block, exactly
// what the belief summed).  If that is not positive definite (the FP32
// belief's rounding, summed over ~100 messages, can leave the difference
// indefinite where this message dominates a direction), the incoming
// message is summed again exactly from its parts: the keyframe's prior at
// iteration t plus every other factor's current message, a loop over the
// keyframe's contiguous slots [i0, i1) of buffers this iteration only reads.
constexpr int KC64 = 33;   // A 21, q 6, inv_d 6

template <typename R>
__device__ __forceinline__ void expand_slot64(const R* recs, const R* jac, int j, double* lam, double* eta) {
    const R* rec = recs + (size_t)j * KREC;
    const R* jr = jac + (size_t)j * KJ;
    double J[2][6];
    for (int i = 0; i < 6; ++i) { J[0][i] = double(__ldcg(jr + i)); J[1][i] = double(__ldcg(jr + 6 + i)); }
    expand_msg<double, 6>(J, double(__ldcg(rec)), double(__ldcg(rec + 1)), double(__ldcg(rec + 2)),
                          double(__ldcg(rec + 3)), double(__ldcg(rec + 4)), lam, eta);
}

__device__ __forceinline__ bool chol_kc64(double* A, const double* q, double* c) {
    double inv_d[6], ratio;
    const bool ok = chol_packed<double, 6>(A, inv_d, ratio);
    for (int i = 0; i < 21; ++i) c[i] = A[i];
    for (int i = 0; i < 6; ++i) { c[21 + i] = q[i]; c[27 + i] = inv_d[i]; }
    return ok;
}

// b^t - m^t from the belief record kb and this factor's slot
template <typename R>
__device__ __noinline__ bool kf_incoming_self64(const R* kb, const R* recs, const R* jac, int self, double* c) {
    double lam[21], eta[6], A[21], q[6];
    expand_slot64<R>(recs, jac, self, lam, eta);
    for (int i = 0; i < 21; ++i) A[i] = double(__ldcg(kb + KB_LAM + i)) - lam[i];
    for (int i = 0; i < 6; ++i) q[i] = double(__ldcg(kb + KB_ETA + i)) - eta[i];
    return chol_kc64(A, q, c);
}

// prior(t) (as b^t added it, in the kernel's precision; its mean is the
// chart origin) plus the messages of slots [i0, i1) other than self
template <typename R>
__device__ __noinline__ bool kf_resum64(const R* recs, const R* jac, int i0, int i1, int self, R s, const R* D,
                                        const R* Aa, R anchor_scale, R inv_sigma2, double* c) {
    double A[21], q[6], lam[21], eta[6];
    for (int i = 0; i < 21; ++i) A[i] = 0.0;
    for (int i = 0; i < 6; ++i) {
        A[pk(i, i)] = double((s * D[i] + anchor_scale * Aa[i]) * inv_sigma2);
        q[i] = 0.0;
    }
    for (int j = i0; j < i1; ++j) {
        if (j == self) continue;
        expand_slot64<R>(recs, jac, j, lam, eta);
        for (int i = 0; i < 21; ++i) A[i] += lam[i];
        for (int i = 0; i < 6; ++i) q[i] += eta[i];
    }
    return chol_kc64(A, q, c);
}

template <typename R>
__device__ __noinline__ Msg5<R> kf_message64(const double* c, Lin<R> Lf) {
    Lin<double> L;
    widen_lin<R>(Lf, L);
    double o[5];
    message_chol<double, 6>(c, c + 27, c + 21, L.Jk, L.y, L.W, o);
    Msg5<R> out;
    for (int i = 0; i < 5; ++i) out.v[i] = R(o[i]);
    return out;
}


__device__ __forceinline__ void raise_error(int32_t* ctl, int where) {
    if (atomicCAS(&ctl[CTL_ERR], 0, 1) == 0) ctl[CTL_ERR_WHERE] = where;
}

// ------------------------------------------------------------------------
// shared pieces of the belief updates

// Sec. 8: prior scale at iteration t (geometric anneal to the final scale),
// tabulated on the host.
template <typename R>
__device__ __forceinline__ R prior_scale(const KParams<R>& P, int t) {
    t = t < 0 ? 0 : t;
    return P.prior_s[t < P.prior_T ? t : P.prior_T];
}

// A variable's prior anneals from the iteration it was added at (Sec. 9.2:
// keyframes and points added during incremental SLAM start at measurement
// scale like the initial ones).
template <typename R>
__device__ __forceinline__ R kf_prior_scale(const DevGraph<R>& g, const KParams<R>& P, int k, int t) {
    return prior_scale(P, t - g.kf_birth[k]);
}
template <typename R>
__device__ __forceinline__ R lm_prior_scale(const DevGraph<R>& g, const KParams<R>& P, int m, int t) {
    return prior_scale(P, t - g.lm_birth[m]);
}

template <typename R, int n>
__device__ __forceinline__ bool solve_mean(R* lam_packed_copy, const R* eta, R* mu, R& ratio) {
    R inv_d[n];
    bool ok = chol_packed<R, n>(lam_packed_copy, inv_d, ratio);
#pragma unroll
    for (int i = 0; i < n; ++i) mu[i] = eta[i];
    fwd_solve<R, n>(lam_packed_copy, inv_d, mu);
    bwd_solve<R, n>(lam_packed_copy, inv_d, mu);
    return ok;
}

// FP64 redo of a belief mean: reads Lambda (packed) and eta from the
// belief record in global memory and writes mu back into it.
template <typename R, int n>
__device__ __noinline__ bool solve_mean_fp64(R* rec) {
    constexpr int p = n * (n + 1) / 2;
    double A[p], e[n], m[n], ratio;
    for (int i = 0; i < p; ++i) A[i] = double(rec[i]);
    for (int i = 0; i < n; ++i) e[i] = double(rec[p + i]);
    bool ok = solve_mean<double, n>(A, e, m, ratio);
    for (int i = 0; i < n; ++i) rec[p + n + i] = R(m[i]);
    return ok;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Landmark belief b^{t+1} = s(t+1) D + sum of messages (eqs. beliefeta /
// belieflambda) and its mean; writes the record, returns |dmu|_inf.
template <typename R>
__device__ __forceinline__ float finish_landmark(const DevGraph<R>& g, const KParams<R>& P, int m, R s, const R* sum,
                                                 const R* mu_old, R* out_bel) {
    R lam[6], eta[3], mu[3], work[6], ratio;
    const R isig2 = P.inv_sigma2;
#pragma unroll
    for (int j = 0; j < 6; ++j) lam[j] = sum[j];
#pragma unroll
    for (int j = 0; j < 3; ++j) eta[j] = sum[6 + j];
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[pk(i, i)] += s * g.lm_D[m * 3 + i] * isig2;
#pragma unroll
    for (int j = 0; j < 6; ++j) work[j] = lam[j];
    bool ok = solve_mean<R, 3>(work, eta, mu, ratio);
    R out[LBEL];
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = lam[j];
#pragma unroll
    for (int j = 0; j < 3; ++j) { out[6 + j] = eta[j]; out[9 + j] = mu[j]; }
    R* rec = out_bel + (size_t)m * LBEL;
    store_rec<R, LBEL>(rec, out);
    if (sizeof(R) == 4 && P.fallback && !ok) {
        ok = solve_mean_fp64<R, 3>(rec);
#pragma unroll
        for (int i = 0; i < 3; ++i) mu[i] = rec[9 + i];
        atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
    }
    float dmu = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (!isfinite(mu[i])) ok = false;
        dmu = fmaxf(dmu, float(fabs(mu[i] - mu_old[i])));
    }
    if (!ok) raise_error(g.ctl, g.n_kf + m);
    return dmu;
}

// A keyframe belief record from Lambda and eta: the Cholesky factor (1/L_ii
// on its diagonal), the mean, tr Lambda, Lambda and eta.  Returns false if
// Lambda is not positive definite; *ratio receives the pivot ratio.
template <typename R>
__device__ __forceinline__ bool kf_record(const R* lam, const R* eta, R* out, R& ratio) {
    R Lw[21], inv[6], mu[6];
#pragma unroll
    for (int j = 0; j < 21; ++j) Lw[j] = lam[j];
    const bool ok = chol_packed<R, 6>(Lw, inv, ratio);
#pragma unroll
    for (int i = 0; i < 6; ++i) mu[i] = eta[i];
    fwd_solve<R, 6>(Lw, inv, mu);
    bwd_solve<R, 6>(Lw, inv, mu);
#pragma unroll
    for (int j = 0; j < 21; ++j) out[KB_L + j] = Lw[j];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        out[KB_L + pk(i, i)] = inv[i];
        out[KB_MU + i] = mu[i];
        out[KB_ETA + i] = eta[i];
    }
    out[KB_TR] = lam[0] + lam[2] + lam[5] + lam[9] + lam[14] + lam[20];
#pragma unroll
    for (int j = 0; j < 21; ++j) out[KB_LAM + j] = lam[j];
    out[KBEL - 1] = R(0);
    return ok;
}

// FP64 redo of a keyframe record's factor and mean (rounded back to R).
template <typename R>
__device__ __noinline__ bool kf_record_fp64(R* out) {
    double lam[21], eta[6], o[KBEL], ratio;
    for (int j = 0; j < 21; ++j) lam[j] = double(out[KB_LAM + j]);
    for (int i = 0; i < 6; ++i) eta[i] = double(out[KB_ETA + i]);
    const bool ok = kf_record<double>(lam, eta, o, ratio);
    for (int j = 0; j < 21; ++j) out[KB_L + j] = R(o[KB_L + j]);
    for (int i = 0; i < 6; ++i) out[KB_MU + i] = R(o[KB_MU + i]);
    return ok;
}

// Keyframe belief b^{t+1} = s(t+1) D + anchor + sum of messages and its
// mean from the (already reduced) sums; writes the record to out and
// returns |dmu|_inf against mu_old.
// prior[i] = (s(t+1) D_i + anchor_scale A_i) / sigma^2, formed by the caller.
template <typename R>
__device__ __forceinline__ float finish_keyframe(const DevGraph<R>& g, const KParams<R>& P, int k, const R* prior,
                                                 const R* sum, const R* mu_old, R* out_bel) {
    R lam[21], eta[6], ratio;
#pragma unroll
    for (int j = 0; j < 21; ++j) lam[j] = sum[j];
#pragma unroll
    for (int j = 0; j < 6; ++j) eta[j] = sum[21 + j];
#pragma unroll
    for (int i = 0; i < 6; ++i) lam[pk(i, i)] += prior[i];
    R out[KBEL];
    bool ok = kf_record<R>(lam, eta, out, ratio);
    R* rec = out_bel + (size_t)k * KBEL;
    store_rec<R, KBEL>(rec, out);
    R mu[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) mu[i] = out[KB_MU + i];
    if (sizeof(R) == 4 && P.fallback && (!ok || ratio < P.pivot_ratio)) {
        // the stored record's Lambda and eta, factorised again in FP64
        ok = kf_record_fp64<R>(rec);
#pragma unroll
        for (int i = 0; i < 6; ++i) mu[i] = rec[KB_MU + i];
        atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
    }
    float dmu = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (!isfinite(mu[i])) ok = false;
        dmu = fmaxf(dmu, float(fabs(mu[i] - mu_old[i])));
    }
    if (!ok) raise_error(g.ctl, k);
    return dmu;
}

// The record of a belief that is the prior alone (diagonal p), mean 0.
template <typename R>
__device__ __forceinline__ void kf_prior_record(const R* p, R* out) {
#pragma unroll
    for (int j = 0; j < KBEL; ++j) out[j] = R(0);
    R tr = R(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        R d, id;
        sqrt_pair<R>(p[i], d, id);
        out[KB_L + pk(i, i)] = id;
        out[KB_LAM + pk(i, i)] = p[i];
        tr += p[i];
    }
    out[KB_TR] = tr;
}


// Keyframe messages are double-buffered by iteration parity: iteration t
// reads m^t from buffer t & 1 and writes m^{t+1} to the other buffer
// (mk_redirect, when set, receives the writes instead).
template <typename R>
__device__ __forceinline__ const R* mk_read(const DevGraph<R>& g, int t) { return (t & 1) ? g.mk2 : g.mk; }
template <typename R>
__device__ __forceinline__ R* mk_write(const DevGraph<R>& g, int t) {
    return g.mk_redirect ? g.mk_redirect : ((t & 1) ? g.mk : g.mk2);
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Compensated summation (Knuth's TwoSum): hi + lo carries a running sum
// with the rounding error of every addition kept in lo, so a sum of many
// FP32 terms comes out within about one rounding of its exact value, in
// whatever order the terms are added.
template <typename R>
__device__ __forceinline__ void two_sum_add(R& hi, R& lo, R x) {
    const R s = hi + x;
    const R bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Sum NV (a power of two, <= 32) values over the 32 lanes of a warp, as
// (hi, lo) pairs.  Offsets 16 .. NV exchange every value (butterfly); the
// remaining levels halve: at offset h a lane keeps the upper or the lower
// half of its values (by lane bit h), sends the other half to its partner
// and adds the partner's copy of the half it keeps -- 31 shuffle pairs in
// all for 32 values.  On return lane l holds the total of value l % NV in
// hi[0], lo[0].  Every total is formed by one fixed tree, so the result
// does not depend on the lane that holds it.
template <typename R, int NV>
__device__ __forceinline__ void warp_transpose_sum(R (&hi)[NV], R (&lo)[NV], int lane) {
    static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV");
#pragma unroll
    for (int o = 16; o >= NV; o >>= 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const R rh = __shfl_xor_sync(0xffffffffu, hi[i], o);
            const R rl = __shfl_xor_sync(0xffffffffu, lo[i], o);
            two_sum_add(hi[i], lo[i], rh);
            lo[i] += rl;
        }
    }
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            R kh = up ? hi[h + i] : hi[i], kl = up ? lo[h + i] : lo[i];
            const R sh = up ? hi[i] : hi[h + i], sl = up ? lo[i] : lo[h + i];
            const R rh = __shfl_xor_sync(0xffffffffu, sh, h);
            const R rl = __shfl_xor_sync(0xffffffffu, sl, h);
            two_sum_add(kh, kl, rh);
            kl += rl;
            hi[i] = kh;
            lo[i] = kl;
        }
    }
}

// The same transposing reduction without compensation (one shuffle and
// one addition per step): lane l receives the total of value l % NV.
template <typename R, int NV>
__device__ __forceinline__ R warp_transpose_sum_plain(R (&v)[NV], int lane) {
#pragma unroll
    for (int o = 16; o >= NV; o >>= 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const R keep = up ? v[h + i] : v[i];
            const R send = up ? v[i] : v[h + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

__device__ __forceinline__ int dmu_slot(int t) { return (t & 1) ? CTL_DMU_ACC1 : CTL_DMU_ACC; }

__device__ __forceinline__ void dmu_atomic_max_slot(int32_t* ctl, int slot, float v) {
    if (!(v >= 0.0f)) v = INFINITY;
    atomicMax(reinterpret_cast<unsigned int*>(&ctl[slot]), __float_as_uint(v));
}

// ------------------------------------------------------------------------
// Learned damping.  Features of factor f at iteration t (all O(1)); for each
// message side, eta_new is this iteration's undamped message, eta_old = m^t
// and eta_prev = m^{t-1}:
//   0  log(1 + M) / 3, M = |r| / sigma (Mahalanobis residual, Sec. 6)
//   1  Huber weight k (Sec. 6; 0 for a factor behind the camera)
//   2  tr Lambda_{f->k} / (tr Lambda_{f->k} + tr P_k), P_k the keyframe's incoming precision
//   3  the same for the landmark
//   4  |eta_new - eta_old| / (|eta_new| + |eta_old|) of the message to the keyframe
//   5, 6  its values at iterations t - 1 and t - 2
//   7  cosine between eta_new - eta_old and eta_old - eta_prev (0 if either is 0):
//      negative when the message oscillates, positive when it moves steadily
//   8-11 the same four for the message to the landmark
//   12 log(1 + deg k) / 5,  13 log(1 + deg m) / 3
//   14 min(t - t_lin, 50) / 50,  15 min(t - t_birth(m), 50) / 50
// Target (record mode): the damping d in [0, 0.9] minimising
//   sum_s |(1 - d) eta_new,s + d eta_old,s - eta_inf,s|^2 / |eta_old,s - eta_new,s|^2
// over the sides s where eta_old != eta_new, eta_inf the reference (the
// run's converged message): each term is |u_s|^-2 times a parabola in d with
// vertex d_s = <u_s, eta_inf,s - eta_new,s> / |u_s|^2 (u_s = eta_old,s -
// eta_new,s), so the minimiser is clip(mean_s d_s, 0, 0.9).

// Square roots and quotients of the learned schedule's features.  In the
// FP32 path the features are network inputs rounded to BF16 (8 significant
// bits), so they take the hardware approximations (rsqrt, fast divide:
// ~2 ulp of FP32) instead of the correctly rounded sequences, which sat on
// every factor warp's path to the network.  x * rsqrt(max(x, 1e-30)) is
// sqrt(x) for x >= 1e-30 and below 1e-15 otherwise (0 at x = 0).
__device__ __forceinline__ float feat_sqrt(float x) { return x * rsqrtf(fmaxf(x, 1e-30f)); }

template <typename R, int n>
__device__ __forceinline__ float rel_change(const R* nw, const R* old) {
    R dd = R(0), a = R(0), b = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        dd += (nw[i] - old[i]) * (nw[i] - old[i]);
        a += nw[i] * nw[i];
        b += old[i] * old[i];
    }
    if constexpr (sizeof(R) == 4)
        return __fdividef(feat_sqrt(dd), feat_sqrt(a) + feat_sqrt(b) + 1e-30f);
    else
        return float(sqrt(dd) / (sqrt(a) + sqrt(b) + R(1e-30)));
}

template <typename R, int n>
__device__ __forceinline__ float step_cosine(const R* nw, const R* old, const R* prev) {
    R ab = R(0), aa = R(0), bb = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const R a = nw[i] - old[i], b = old[i] - prev[i];
        ab += a * b;
        aa += a * a;
        bb += b * b;
    }
    if constexpr (sizeof(R) == 4)
        return __fdividef(ab, feat_sqrt(aa) * feat_sqrt(bb) + 1e-30f);
    else
        return float(ab / (sqrt(aa) * sqrt(bb) + R(1e-30)));
}

// Vertex of one side's parabola (unclipped); valid = the side's message changed.
template <typename R, int n>
__device__ __forceinline__ float damping_vertex(const R* nw, const R* old, const R* inf, bool& valid) {
    R uu = R(0), uv = R(0), nn = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const R u = old[i] - nw[i];
        uu += u * u;
        uv += u * (inf[i] - nw[i]);
        nn += nw[i] * nw[i] + old[i] * old[i];
    }
    valid = uu > R(1e-10) * nn && uu > R(0);
    return valid ? float(uv / uu) : 0.0f;
}

// Shared memory of the learned schedule: the network's packed weights and
// per-warp activation tiles (BF16 bits).
template <int MODE>
struct MlpSmem {
    int unused;
};
template <>
struct MlpSmem<DAMP_LEARNED> {
    uint32_t frag[FWD_FRAG_WORDS];
    float bias[MLP_BIAS_WORDS];
    alignas(16) uint16_t x[FACTOR_BLOCK / 32][32 * XS];
};

template <int MODE, typename R>
__device__ __forceinline__ void mlp_load(const KParams<R>& P, MlpSmem<MODE>& S) {
    if constexpr (MODE == DAMP_LEARNED) {
        for (int i = threadIdx.x; i < FWD_FRAG_WORDS; i += blockDim.x) S.frag[i] = P.mlp_frag[i];
        for (int i = threadIdx.x; i < MLP_BIAS_WORDS; i += blockDim.x) S.bias[i] = P.mlp_bias[i];
        __syncthreads();
    }
}

// 16-byte asynchronous global-to-shared copies (cp.async, through L2).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The per-phase factor kernel starts the weight copy at launch and waits for
// it (every warp of the block, once) just before the network, so the copy
// overlaps the message arithmetic instead of preceding it.
template <int MODE, typename R>
__device__ __forceinline__ void mlp_load_async(const KParams<R>& P, MlpSmem<MODE>& S) {
    if constexpr (MODE == DAMP_LEARNED) {
        for (int c = threadIdx.x; c < FWD_FRAG_WORDS / 4; c += blockDim.x) cp_async16(S.frag + 4 * c, P.mlp_frag + 4 * c);
        for (int c = threadIdx.x; c < MLP_BIAS_WORDS / 4; c += blockDim.x) cp_async16(S.bias + 4 * c, P.mlp_bias + 4 * c);
        cp_async_commit();
    }
}
__device__ __forceinline__ void mlp_load_wait() {
    cp_async_wait_all();
    __syncthreads();
}

// One factor's messages once both incoming precisions are known (Lm, im:
// the landmark side's FP32 Cholesky factor; ks: the keyframe side): the
// FP64 redo where FP32 cannot take an incoming precision (FP64 = true),
// the kept messages, the relinearisation test and the linearisation at the
// new point, and both new messages in compact form (ck to the keyframe, cl
// to the landmark), in the basis of L.
template <typename R, bool FP64>
__device__ __forceinline__ void form_messages(const DevGraph<R>& g, const KParams<R>& P, int f, int k, int slot, int t,
                                              int& tl, bool due, bool active, const R* kbp, Lin<R>& L,
                                              const KfSide<R>& ks, const R* mo, const R* cml, const R* kmu,
                                              const R* lb_mu, const R* x0, const R* Pm, const R* qm, const R* Lm,
                                              const R* im, bool& ok_m, bool& ok_k, R* ck, R* cl) {
    const int n_f = g.n_f;
    // FP64 where FP32 cannot take an incoming precision (decided here, from
    // iteration-t state only; the messages are formed after the
    // relinearisation test)
    bool m64 = false, k64 = false;
    double kc[KC64];   // the keyframe's FP64 incoming precision, formed once for both uses
    if (FP64 && sizeof(R) == 4 && P.fallback && active) {
        if (!ok_m) {
            Arr9<R> pq;
#pragma unroll
            for (int i = 0; i < 6; ++i) pq.v[i] = Pm[i];
#pragma unroll
            for (int i = 0; i < 3; ++i) pq.v[6 + i] = qm[i];
            ok_m = lm_incoming_ok64<R>(pq);
            m64 = ok_m;
            // kept for the FP64 message in this factor's (per-iteration)
            // expanded-message slot, which is rewritten below
            if (m64)
#pragma unroll
                for (int i = 0; i < 9; ++i) g.mlx[(size_t)i * n_f + f] = pq.v[i];
            atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
        }
        if (!(ks.det >= P.cav_ratio)) {
            const R* recs = mk_read(g, t);
            // the sum from its parts needs all of the keyframe's messages on this rank
            const bool exact = P.exact_cavity && kf_in_part(g, k);
            ok_k = !exact && kf_incoming_self64<R>(kbp, recs, g.kj, slot, kc);
            if (!ok_k && kf_in_part(g, k)) {
                ok_k = kf_resum64<R>(recs, g.kj, g.kf_off[k], g.kf_off[k + 1], slot, kf_prior_scale(g, P, k, t),
                                     g.kf_D + (size_t)k * 6, g.kf_A + (size_t)k * 6, P.anchor_scale, P.inv_sigma2,
                                     kc);
                atomicAdd(&g.ctl[CTL_RESUMS], 1);
            }
            k64 = ok_k;
            atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
        }
    }
    if (active && !ok_m) atomicAdd(&g.ctl[CTL_HELD], 1);
    if (active && !ok_k) atomicAdd(&g.ctl[CTL_HELD], 1);

    // 3. Sec. 5 / Sec. 8: relinearise when the adjacent means moved more than
    // beta from the linearisation point, at most every relin_interval
    // iterations -- unless a message of this factor is kept this iteration
#pragma unroll
    for (int i = 0; i < NML; ++i) cl[i] = cml[i];   // kept unless formed below
    bool rebased = false;
    if (due && ok_m && ok_k) {
        R d2 = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) d2 += (kmu[i] - x0[i]) * (kmu[i] - x0[i]);
#pragma unroll
        for (int i = 0; i < 3; ++i) d2 += (lb_mu[i] - x0[6 + i]) * (lb_mu[i] - x0[6 + i]);
        if (d2 > P.relin_beta * P.relin_beta) {
            Arr9<R> xn;
            Arr12<R> Jo;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                xn.v[i] = kmu[i];
                Jo.v[i] = L.Jk[0][i];
                Jo.v[6 + i] = L.Jk[1][i];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) xn.v[6 + i] = lb_mu[i];
#pragma unroll
            for (int i = 0; i < 9; ++i) g.x0[(size_t)i * n_f + f] = xn.v[i];
            tl = t;
            g.tlin[f] = t;
            atomicAdd(&g.ctl[CTL_RELINS], 1);
            rebased = true;
            const Rebased<R> rb = rebase<R>(kbp, Jo, mo[3], mo[4], ks.a0, ks.a1, ks.K00, ks.K01, ks.K11, !k64, xn,
                                            lin_args<R>(P, g, k, f));
            L = rb.L;
            store_lin<R>(g, f, L);
            store_jac<R>(g.kjs + (size_t)slot * KJ, L.Jk);
            if (!kf_in_part(g, k)) store_jac<R>(g.kj + (size_t)slot * KJ, L.Jk);
            if (!k64)
#pragma unroll
                for (int i = 0; i < NML; ++i) cl[i] = rb.cl[i];
        }
    }

    // 4. the new messages (compact), in the basis of L
    if (!ok_m) {
#pragma unroll
        for (int i = 0; i < NML; ++i) ck[i] = mo[i];
    } else if (m64) {
        Arr9<R> pq;
#pragma unroll
        for (int i = 0; i < 9; ++i) pq.v[i] = g.mlx[(size_t)i * n_f + f];
        const Msg5<R> o = lm_message64<R>(pq, L);
#pragma unroll
        for (int i = 0; i < NML; ++i) ck[i] = o.v[i];
    } else {
        message_chol<R, 3>(Lm, im, qm, L.Jl, L.y, L.W, ck);
    }
    if (ok_k) {
        if (k64) {
            const Msg5<R> o = kf_message64<R>(kc, L);
#pragma unroll
            for (int i = 0; i < NML; ++i) cl[i] = o.v[i];
        } else if (!rebased) {
            message_to_landmark<R>(ks, L.y, L.W, cl);
        }
    }

}

// Damping of eta (Sec. 5), i.e. of g, in the fixed schedule -- the message
// sent in the iteration of a (re)linearisation and the next damp_hold - 1
// are undamped (Sec. 8) -- then the stores: the keyframe record (with the
// t_lin of its basis), the landmark message, and for a landmark split
// across tiles the expanded one.  sum receives the expanded landmark
// message for the tile's landmark sums.
template <typename R>
__device__ __forceinline__ void damp_store_fixed(const DevGraph<R>& g, const KParams<R>& P, int f, int slot, int t,
                                                 int tl, bool whole, bool ok_m, bool ok_k, R* ck, R* cl, const R* mo,
                                                 const R* cml, const Lin<R>& L, R* sum) {
    const int n_f = g.n_f;
    if (t - tl >= P.damp_hold) {
        const R d = P.damping;
        if (ok_m) {
            ck[3] = (R(1) - d) * ck[3] + d * mo[3];
            ck[4] = (R(1) - d) * ck[4] + d * mo[4];
        }
        if (ok_k) {
            cl[3] = (R(1) - d) * cl[3] + d * cml[3];
            cl[4] = (R(1) - d) * cl[4] + d * cml[4];
        }
    }
    R rec[KREC];
#pragma unroll
    for (int i = 0; i < NML; ++i) rec[i] = ck[i];
    rec[KREC_TL] = int_bits<R>(tl);
    rec[6] = R(0);
    rec[7] = R(0);
    store_rec<R, KREC>(mk_write(g, t) + (size_t)slot * KREC, rec);
#pragma unroll
    for (int i = 0; i < NML; ++i) g.ml_out[(size_t)i * n_f + f] = cl[i];
    expand_msg<R, 3>(L.Jl, cl[0], cl[1], cl[2], cl[3], cl[4], sum, sum + 6);
    if (!whole)
#pragma unroll
        for (int i = 0; i < 9; ++i) g.mlx[(size_t)i * n_f + f] = sum[i];
}

// ------------------------------------------------------------------------
// Phase A: one warp, one tile of whole landmarks (at most 32 factors,
// consecutive in landmark order), one lane per factor.  For each factor:
//   1. its linearisation at x0 (the basis its stored messages are in);
//   2. both incoming precisions (Sec. 5): the landmark's as prior(t) plus
//      the other factors' previous messages (segmented warp scans, no
//      cancellation), the keyframe's through the belief's stored Cholesky
//      factor (KfSide); an FP64 redo where FP32 cannot take them;
//   3. the relinearisation test (Sec. 5, Sec. 8), skipped by a factor one of
//      whose messages must be kept (its incoming precision is not positive
//      definite), then the linearisation at the new point;
//   4. both new messages in compact form, the Huber weight (Sec. 6) inside W;
//   5. damping of g, i.e. of eta (Sec. 5), after the undamped hold (Sec. 8);
// then the landmark messages of the tile are summed per landmark by a
// segmented warp scan (fixed lane order) and each landmark's last lane forms
// its belief b^{t+1} and mean (a landmark wholly inside a tile is read by no
// other warp).  Returns this lane's max |dmu|.
// MODE selects the damping schedule (DampMode); the learned schedule
// evaluates the network for the warp's 32 factors at once on the tensor
// cores, between forming the messages and damping them.

// DEFER (fixed FP32 schedule): a tile with a factor whose incoming
// precision FP32 cannot take is not worked here -- it stores nothing and is
// listed for factor_deferred_kernel, which works it with the FP64 redo --
// so that this kernel carries no state for the FP64 path.
template <typename R, int MODE, bool DEFER = false>
__device__ __forceinline__ float tile_work(const DevGraph<R>& g, const KParams<R>& P, int tile, int t, int lane,
                                           MlpSmem<MODE>& S, bool weights_pending = false) {
    const int n_f = g.n_f;
    const int ts = g.tile_start[tile], te = g.tile_start[tile + 1];
    const int f = ts + lane;
    const bool active = f < te;
    constexpr bool FEAT = MODE != DAMP_FIXED;

    // Every load of the common path is issued in two waves before anything
    // is stored: the factor's own entries (wave 1), then what they index
    // (wave 2).  A store in between (the first linearisation writes the
    // lin record and the keyframe block) would keep later loads behind it.
    int m = -1, lo = 0, hi = 0, k = 0, slot = 0, tl = 0, lbirth = 0;
    R cml[NML];          // this factor's previous message to the landmark (compact)
    R lin4[NLIN];        // y0, y1, W, |r|^2 of its stored linearisation
#pragma unroll
    for (int i = 0; i < NML; ++i) cml[i] = R(0);
#pragma unroll
    for (int i = 0; i < NLIN; ++i) lin4[i] = R(0);
    if (active) {
        m = g.fm[f];
        k = g.fk[f];
        slot = g.kpos[f];
        tl = g.tlin[f];
#pragma unroll
        for (int i = 0; i < NML; ++i) cml[i] = g.ml[(size_t)i * n_f + f];
#pragma unroll
        for (int i = 0; i < NLIN; ++i) lin4[i] = g.lin[(size_t)i * n_f + f];
    }
    // the linearisation point is needed for a factor's first linearisation
    // and for the relinearisation test once the interval allows one
    const bool fresh = active && tl == t;
    const bool due = active && !P.linear && t - tl >= P.relin_interval;
    const R* kbp = g.kf_bel + (size_t)k * KBEL;
    R x0[9];
    R jr[KJ];            // the stored keyframe block of the factor's messages
    R kb[KB_A];          // the keyframe belief's Cholesky factor, mean and trace
    R mo[KREC];          // the previous message to the keyframe (compact record)
    R lb_mu[3];          // the landmark's mean mu^t
    R lD[3];             // the landmark's prior diagonal
    if (active) {
        lo = g.lm_off[m];
        hi = g.lm_off[m + 1];
        lbirth = g.lm_birth[m];
        // the keyframe block is moved into kj by the belief phase, on another
        // SM within one persistent launch: read through L2, as the beliefs
        load_rec_cg<R, KJ>(g.kj + (size_t)slot * KJ, jr);
        load_rec_cg<R, KB_A>(kbp, kb);
        load_rec<R, KREC>(mk_read(g, t) + (size_t)slot * KREC, mo);
        const R* lbp = g.lm_bel + (size_t)m * LBEL;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            lb_mu[i] = __ldcg(lbp + 9 + i);
            lD[i] = g.lm_D[m * 3 + i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < KJ; ++i) jr[i] = R(0);
#pragma unroll
        for (int i = 0; i < KB_A; ++i) kb[i] = R(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) kb[pk(i, i)] = R(1);
#pragma unroll
        for (int i = 0; i < KREC; ++i) mo[i] = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) { lb_mu[i] = R(0); lD[i] = R(0); }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) x0[i] = (fresh || due) ? g.x0[(size_t)i * n_f + f] : R(0);
    // The learned schedule reads a factor's features only where it damps
    // (t - t_lin >= damp_hold), and those read the history written in the
    // two iterations before; earlier in the hold the features are neither
    // formed nor stored (t_lin as stored: a relinearisation in this
    // iteration only moves the factor back into its hold).  The record
    // schedule writes every active factor's features.  Their loads join the
    // second wave: g of m^{t-1} to the keyframe (still in the buffer this
    // iteration writes), the history, the keyframe's degree.
    const bool need_feat = active && (MODE != DAMP_LEARNED || t - tl >= P.damp_hold - 2);
    R pr_g0 = R(0), pr_g1 = R(0);
    float h[HIST];
    int deg_k = 0;
    if constexpr (FEAT) {
        if (need_feat) {
            const R* pp = mk_write(g, t) + (size_t)slot * KREC;
            pr_g0 = pp[3];
            pr_g1 = pp[4];
#pragma unroll
            for (int j = 0; j < HIST; ++j) h[j] = g.hist[(size_t)j * n_f + f];
            deg_k = g.kf_off[k + 1] - g.kf_off[k];
        } else {
#pragma unroll
            for (int j = 0; j < HIST; ++j) h[j] = 0.0f;
        }
    }
    const bool whole = active && lo >= ts && hi <= te;
    const int seg0 = whole ? lo - ts : lane;
    const int seg1 = whole ? hi - ts - 1 : lane;
    // the scans below need steps d < the longest landmark segment of the
    // tile; the steps they skip would add nothing
    const int seg_max = __reduce_max_sync(0xffffffffu, unsigned(seg1 - seg0 + 1));

    // 1. the factor's linearisation (Sec. 4), the basis of its stored
    // messages: computed at its first iteration, else as stored when it was
    // taken -- the keyframe block J_k from the slot's kj record (the landmark
    // block is -J_k[:, 0:3]), y, W and |r|^2 from the factor's lin record
    Lin<R> L;
    if (fresh) {
        Arr9<R> xv;
#pragma unroll
        for (int i = 0; i < 9; ++i) xv.v[i] = x0[i];
        L = linearise_at<R>(xv, lin_args<R>(P, g, k, f));
        store_lin<R>(g, f, L);
        store_jac<R>(g.kjs + (size_t)slot * KJ, L.Jk);
        // a keyframe of another rank's part: no belief phase here moves the
        // staged block, so the factor keeps its own copy up to date
        if (!kf_in_part(g, k)) store_jac<R>(g.kj + (size_t)slot * KJ, L.Jk);
    } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            L.Jk[0][j] = jr[j];
            L.Jk[1][j] = jr[6 + j];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            L.Jl[0][j] = -jr[j];
            L.Jl[1][j] = -jr[6 + j];
        }
        L.y[0] = lin4[0];
        L.y[1] = lin4[1];
        L.W = lin4[2];
        L.r2 = lin4[3];
    }

    // 2a. keyframe incoming precision b^t - m^t through the belief's factor
    R kmu[6];            // the keyframe's mean mu^t
    KfSide<R> ks;
    kf_side<R>(kb, kb + KB_MU, L.Jk, mo, ks);
#pragma unroll
    for (int i = 0; i < 6; ++i) kmu[i] = kb[KB_MU + i];
    const R tr_b = kb[KB_TR];
    bool ok_k = ks.pd;

    // learned / record schedules: quantities of the previous messages, in
    // their basis, before a relinearisation replaces it
    R ek_old[6], ek_prev[6], em_old[3];
    R tr_pk = R(0), tr_pm = R(0);
    if constexpr (FEAT) {
        if (need_feat) {
            msg_eta<R, 6>(L.Jk, mo[3], mo[4], ek_old);
            msg_eta<R, 6>(L.Jk, pr_g0, pr_g1, ek_prev);
            tr_pk = tr_b - msg_trace<R, 6>(L.Jk, mo[0], mo[1], mo[2]);
        } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) { ek_old[i] = R(0); ek_prev[i] = R(0); }
        }
    }

    // 2b. landmark incoming precision.  For a landmark wholly inside the
    // tile: prior(t) plus the exclusive prefix and suffix sums of the other
    // factors' previous messages, which equals b^t - m^t without the
    // cancellation of subtracting one message from the belief.
    R mlo[9];            // this factor's previous landmark message, expanded
    expand_msg<R, 3>(L.Jl, cml[0], cml[1], cml[2], cml[3], cml[4], mlo, mlo + 6);
    if constexpr (FEAT) {
#pragma unroll
        for (int i = 0; i < 3; ++i) em_old[i] = mlo[6 + i];
    }
    R Pm[6], qm[3];
    {
        R fw[9], bw[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) { fw[j] = mlo[j]; bw[j] = mlo[j]; }
        for (int d = 1; d < seg_max; d <<= 1) {
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                R o = __shfl_up_sync(0xffffffffu, fw[j], d);
                if (lane - d >= seg0) fw[j] += o;
                R u = __shfl_down_sync(0xffffffffu, bw[j], d);
                if (lane + d <= seg1) bw[j] += u;
            }
        }
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            R pre = __shfl_up_sync(0xffffffffu, fw[j], 1);
            R suf = __shfl_down_sync(0xffffffffu, bw[j], 1);
            const R cv = (lane - 1 >= seg0 ? pre : R(0)) + (lane + 1 <= seg1 ? suf : R(0));
            if (j < 6) Pm[j] = cv;
            else qm[j - 6] = cv;
        }
    }
    if (active) {
        const R* lbp = g.lm_bel + (size_t)m * LBEL;
        if (whole) {
            const R sp = prior_scale(P, t - lbirth) * P.inv_sigma2;
#pragma unroll
            for (int i = 0; i < 3; ++i) Pm[pk(i, i)] += sp * lD[i];
        } else {
            // a landmark split across tiles: its belief divided by this message
            R lb[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) lb[i] = __ldcg(lbp + i);
#pragma unroll
            for (int i = 0; i < 6; ++i) Pm[i] = lb[i] - mlo[i];
#pragma unroll
            for (int i = 0; i < 3; ++i) qm[i] = lb[6 + i] - mlo[6 + i];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) Pm[i] = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) { Pm[pk(i, i)] = R(1); qm[i] = R(0); }   // idle lanes: any positive definite matrix
    }
    if constexpr (FEAT) tr_pm = Pm[0] + Pm[2] + Pm[5];
    R Lm[6], im[3], rm;
#pragma unroll
    for (int i = 0; i < 6; ++i) Lm[i] = Pm[i];
    bool ok_m = chol_packed<R, 3>(Lm, im, rm);

    // 3, 4 and 5
    R ck[NML], cl[NML];  // the new messages: to the keyframe, to the landmark
    R sum[9];            // the new landmark message, expanded
    if constexpr (DEFER) {
        static_assert(MODE == DAMP_FIXED && sizeof(R) == 4, "deferral: fixed FP32 schedule");
        // a tile with a factor that needs the FP64 redo is left to
        // factor_deferred_kernel: nothing of it is stored here (a first
        // linearisation above stores what the deferred run stores again)
        const bool needs64 = P.fallback && active && (!ok_m || !(ks.det >= P.cav_ratio));
        if (__any_sync(0xffffffffu, needs64)) {
            if (lane == 0) {
                const int i = atomicAdd(&g.ctl[CTL_DEFER_N0 + (t & 1)], 1);
                if (i < g.n_tiles) g.deferred[i] = tile;
            }
            return 0.0f;
        }
        if (active) {
            form_messages<R, false>(g, P, f, k, slot, t, tl, due, active, kbp, L, ks, mo, cml, kmu, lb_mu, x0, Pm, qm,
                                    Lm, im, ok_m, ok_k, ck, cl);
            damp_store_fixed<R>(g, P, f, slot, t, tl, whole, ok_m, ok_k, ck, cl, mo, cml, L, sum);
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) sum[i] = R(0);
        }
    } else {
        form_messages<R, true>(g, P, f, k, slot, t, tl, due, active, kbp, L, ks, mo, cml, kmu, lb_mu, x0, Pm, qm, Lm,
                               im, ok_m, ok_k, ck, cl);
        // features of the learned schedule and targets of the record schedule
        float feat[N_FEAT];
#pragma unroll
        for (int i = 0; i < N_FEAT; ++i) feat[i] = 0.0f;
        R ek_new[6], em_new[3];
        if constexpr (FEAT) {
            if (need_feat) {
                msg_eta<R, 6>(L.Jk, ck[3], ck[4], ek_new);
                msg_eta<R, 3>(L.Jl, cl[3], cl[4], em_new);
                const float tr_lk = float(msg_trace<R, 6>(L.Jk, ck[0], ck[1], ck[2]));
                const float tr_lm = float(msg_trace<R, 3>(L.Jl, cl[0], cl[1], cl[2]));
                const float M = float(sqrt(L.r2) * P.inv_sigma);
                const float cfk = rel_change<R, 6>(ek_new, ek_old);
                const float cfm = rel_change<R, 3>(em_new, em_old);
                const R em_prev[3] = {R(h[4]), R(h[5]), R(h[6])};
                feat[0] = log1pf(M) * (1.0f / 3.0f);
                if constexpr (sizeof(R) == 4) {
                    feat[1] = __fdividef(L.W, P.inv_sigma2);
                    feat[2] = __fdividef(tr_lk, tr_lk + tr_pk + 1e-30f);
                    feat[3] = __fdividef(tr_lm, tr_lm + tr_pm + 1e-30f);
                } else {
                    feat[1] = float(L.W / P.inv_sigma2);
                    feat[2] = tr_lk / (tr_lk + float(tr_pk) + 1e-30f);
                    feat[3] = tr_lm / (tr_lm + float(tr_pm) + 1e-30f);
                }
                feat[4] = cfk;
                feat[5] = h[0];
                feat[6] = h[1];
                // the three keyframe messages share one basis only from t_lin + 2 on
                feat[7] = t - tl >= 2 ? step_cosine<R, 6>(ek_new, ek_old, ek_prev) : 0.0f;
                feat[8] = cfm;
                feat[9] = h[2];
                feat[10] = h[3];
                feat[11] = step_cosine<R, 3>(em_new, em_old, em_prev);
                feat[12] = log1pf(float(deg_k)) * 0.2f;
                feat[13] = log1pf(float(hi - lo)) * (1.0f / 3.0f);
                feat[14] = float(min(t - tl, 50)) * 0.02f;
                feat[15] = float(min(t - lbirth, 50)) * 0.02f;
                const float hn[HIST] = {cfk, h[0], cfm, h[2], float(em_old[0]), float(em_old[1]), float(em_old[2]), 0.0f};
#pragma unroll
                for (int j = 0; j < HIST; ++j) g.hist[(size_t)j * n_f + f] = hn[j];
                if constexpr (MODE == DAMP_RECORD) {
                    R ik[6], imm[3];
#pragma unroll
                    for (int i = 0; i < 6; ++i) ik[i] = g.eta_inf[(size_t)i * n_f + f];
#pragma unroll
                    for (int i = 0; i < 3; ++i) imm[i] = g.eta_inf[(size_t)(6 + i) * n_f + f];
                    bool vk, vm;
                    const float dk = damping_vertex<R, 6>(ek_new, ek_old, ik, vk);
                    const float dm = damping_vertex<R, 3>(em_new, em_old, imm, vm);
                    float target = (vk || vm) ? fminf(fmaxf((dk * float(vk) + dm * float(vm)) /
                                                            float(int(vk) + int(vm)), 0.0f), MLP_DMAX)
                                              : -1.0f;
                    // samples the learned schedule never damps: the hold after
                    // a (re)linearisation, a factor behind the camera
                    if (t - tl < P.damp_hold || !(L.W > R(0))) target = -1.0f;
                    float4* xo = reinterpret_cast<float4*>(g.rec_X + (size_t)f * N_FEAT);
#pragma unroll
                    for (int j = 0; j < N_FEAT / 4; ++j)
                        xo[j] = make_float4(feat[4 * j], feat[4 * j + 1], feat[4 * j + 2], feat[4 * j + 3]);
                    g.rec_T[f] = target;
                }
            }
        }

        // 5. damping of eta (Sec. 5), i.e. of g: the message sent in the
        // iteration of a (re)linearisation and the next damp_hold - 1 are
        // undamped (Sec. 8); the learned schedule damps after the network
        if constexpr (MODE != DAMP_LEARNED) {
            if (active && t - tl >= P.damp_hold) {
                const R d = P.damping;
                if (ok_m) {
                    ck[3] = (R(1) - d) * ck[3] + d * mo[3];
                    ck[4] = (R(1) - d) * ck[4] + d * mo[4];
                }
                if (ok_k) {
                    cl[3] = (R(1) - d) * cl[3] + d * cml[3];
                    cl[4] = (R(1) - d) * cl[4] + d * cml[4];
                }
            }
        }
        if constexpr (MODE == DAMP_LEARNED) {
            // the network for the warp's 32 factors (inactive lanes: zero rows),
            // then g damped by each factor's own d wherever the fixed schedule
            // would damp (after the undamped hold of Sec. 8)
            const int w = threadIdx.x >> 5;
            const bool damp_f = active && t - tl >= P.damp_hold;
            if (weights_pending) mlp_load_wait();   // uniform per block: every warp of the block passes here once
            if (__any_sync(0xffffffffu, damp_f)) {   // uniform per warp: skipped while every lane is in its hold
                __nv_bfloat16* xt = reinterpret_cast<__nv_bfloat16*>(S.x[w]);
#pragma unroll
                for (int j = 0; j < N_FEAT; j += 2)
                    *reinterpret_cast<uint32_t*>(xt + lane * XS + j) = pack_bf16(feat[j], feat[j + 1]);
                __syncwarp();
                const float z3 = mlp_forward_regs(S.frag, S.bias, xt, lane);
                __syncwarp();   // the tile is rewritten by the warp's next tile
                float dl = mlp_output(z3);
                if (!(dl >= 0.0f && dl <= MLP_DMAX)) dl = float(P.damping);
                if (damp_f) {
                    const R dd = R(dl);
                    if (ok_m) {
                        ck[3] = (R(1) - dd) * ck[3] + dd * mo[3];
                        ck[4] = (R(1) - dd) * ck[4] + dd * mo[4];
                    }
                    if (ok_k) {
                        cl[3] = (R(1) - dd) * cl[3] + dd * cml[3];
                        cl[4] = (R(1) - dd) * cl[4] + dd * cml[4];
                    }
                }
            }
        }

        // stores: the keyframe record (with the t_lin of its basis), the new
        // basis for the belief phase when it changed, the landmark message
        if (active) {
            R rec[KREC];
#pragma unroll
            for (int i = 0; i < NML; ++i) rec[i] = ck[i];
            rec[KREC_TL] = int_bits<R>(tl);
            rec[6] = R(0);
            rec[7] = R(0);
            store_rec<R, KREC>(mk_write(g, t) + (size_t)slot * KREC, rec);
#pragma unroll
            for (int i = 0; i < NML; ++i) g.ml_out[(size_t)i * n_f + f] = cl[i];
            expand_msg<R, 3>(L.Jl, cl[0], cl[1], cl[2], cl[3], cl[4], sum, sum + 6);
            if (!whole)
#pragma unroll
                for (int i = 0; i < 9; ++i) g.mlx[(size_t)i * n_f + f] = sum[i];
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) sum[i] = R(0);
        }
    }

    // landmarks wholly inside the tile: segmented inclusive scan over the
    // lanes holding the same landmark (landmark ranges are contiguous)
    for (int d = 1; d < seg_max; d <<= 1) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            R o = __shfl_up_sync(0xffffffffu, sum[j], d);
            if (lane - d >= seg0) sum[j] += o;
        }
    }
    float dmu = 0.0f;
    if (whole && lane == hi - ts - 1) {
        dmu = finish_landmark<R>(g, P, m, prior_scale(P, t + 1 - lbirth), sum, lb_mu, g.lm_bel_out);
    }
    return dmu;
}



// ------------------------------------------------------------------------
// Phase B: one group of threads per work item -- one warp, or the whole
// block for small graphs (g.b_warps = FACTOR_BLOCK / 32), where a warp per
// item would leave SMs idle.  Item b in [0, n_kf): keyframe b -- a
// fixed-order reduction of its messages, stored contiguously in the
// keyframe's CSR order: thread i of the group takes entries i, i + group
// size, ...; then the group's sums (group_total) reach the group's first
// thread, which forms the belief.  In the block mapping (small graphs) only
// a thread's own one or two additions round plainly and every addition
// after them is compensated, so an FP32 belief is its messages' sum to
// within about one rounding more; the warp mapping (large graphs, where a
// lane adds ~5-10 entries itself) keeps a plain tree.  Then one item per landmark
// split across tiles (the same over its factors' landmark messages), then
// groups of variables without factors (prior-only beliefs).  Every thread
// of the group calls it with the same item; returns max |dmu| in the
// group's first thread.

// Totals of NVAL values (NV >= NVAL, a power of two) over the group, into
// out[] of the group's first thread.  A warp: a plain transposing tree.  A
// block: a compensated transposing tree per warp, then NVAL threads add the
// warps' (hi, lo) sums, compensated, in warp order.
template <typename R, int NV, int NVAL, int W>
__device__ __forceinline__ void group_total(R (&v)[NV], R (&out)[NVAL]) {
    constexpr int NW = FACTOR_BLOCK / 32;
    __shared__ R part_hi[NW][32], part_lo[NW][32], total[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (W == 1) {
        // many items: a plain tree (the warp's own few entries per lane
        // dominate the rounding anyway), kept cheap for large graphs
        const R t = warp_transpose_sum_plain<R, NV>(v, lane);
#pragma unroll
        for (int j = 0; j < NVAL; ++j) out[j] = __shfl_sync(0xffffffffu, t, j);
    } else {
        R lo[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) lo[j] = R(0);
        warp_transpose_sum<R, NV>(v, lo, lane);
        if (lane < NVAL) {
            part_hi[warp][lane] = v[0];
            part_lo[warp][lane] = lo[0];
        }
        __syncthreads();
        if (threadIdx.x < NVAL) {
            R h = part_hi[0][threadIdx.x], l = part_lo[0][threadIdx.x];
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                two_sum_add(h, l, part_hi[w][threadIdx.x]);
                l += part_lo[w][threadIdx.x];
            }
            total[threadIdx.x] = h + l;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int j = 0; j < NVAL; ++j) out[j] = total[j];
        }
    }
}

// W: warps per item (g.b_warps)
template <typename R, int W>
__device__ __forceinline__ float phase_b_item(const DevGraph<R>& g, const KParams<R>& P, int item, int t) {
    const int gsize = 32 * W;
    const int tg = threadIdx.x & (gsize - 1);   // thread within the group
    float dmu = 0.0f;
    if (item < g.kf_item_n) {
        const int k = g.kf_item_off + item;
        const R* msgs = mk_write(g, t);
        // the first thread's own inputs first, so their loads overlap the reduction
        R prior[6], mu_old[6];
        if (tg == 0) {
            const R sp = kf_prior_scale(g, P, k, t + 1);
            const R* old = g.kf_bel + (size_t)k * KBEL;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                prior[i] = (sp * g.kf_D[k * 6 + i] + P.anchor_scale * g.kf_A[k * 6 + i]) * P.inv_sigma2;
                mu_old[i] = __ldcg(old + KB_MU + i);
            }
        }
        R hi[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) hi[j] = R(0);
        const int b0 = g.kf_off[k], b1 = g.kf_off[k + 1];
        // BU entries per thread at a time: their loads are all issued before
        // any of them is summed (the summation order stays entry by entry)
        constexpr int BU = 4;
        for (int i0 = b0 + tg; i0 < b1; i0 += BU * gsize) {
            // the compact message m^{t+1} and the Jacobian block it is in: the
            // staged new block when its factor (re)linearised in iteration t
            // (which then becomes the slot's block)
            R rec[BU][KREC], jr[BU][KJ];
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                const int i = i0 + u * gsize;
                if (i < b1) {
                    load_rec_cg<R, KREC>(msgs + (size_t)i * KREC, rec[u]);
                    load_rec_cg<R, KJ>(g.kj + (size_t)i * KJ, jr[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                const int i = i0 + u * gsize;
                if (i < b1) {
                    if (bits_int<R>(rec[u][KREC_TL]) == t) {
                        load_rec_cg<R, KJ>(g.kjs + (size_t)i * KJ, jr[u]);
                        store_rec<R, KJ>(g.kj + (size_t)i * KJ, jr[u]);
                    }
                    const R J[2][6] = {{jr[u][0], jr[u][1], jr[u][2], jr[u][3], jr[u][4], jr[u][5]},
                                       {jr[u][6], jr[u][7], jr[u][8], jr[u][9], jr[u][10], jr[u][11]}};
                    R lam[21], eta[6];
                    expand_msg<R, 6>(J, rec[u][0], rec[u][1], rec[u][2], rec[u][3], rec[u][4], lam, eta);
#pragma unroll
                    for (int j = 0; j < 21; ++j) hi[j] += lam[j];
#pragma unroll
                    for (int j = 0; j < 6; ++j) hi[21 + j] += eta[j];
                }
            }
        }
        R acc[27];
        group_total<R, 32, 27, W>(hi, acc);
        if (tg == 0) dmu = finish_keyframe<R>(g, P, k, prior, acc, mu_old, g.kf_bel_out);
    } else if (item < g.kf_item_n + g.big_item_n) {
        const int m = g.big_lm[g.big_item_off + item - g.kf_item_n];
        R hi[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) hi[j] = R(0);
        const int b0 = g.lm_off[m], b1 = g.lm_off[m + 1];
        for (int f = b0 + tg; f < b1; f += gsize) {
#pragma unroll
            for (int j = 0; j < 9; ++j) hi[j] += __ldcg(g.mlx + (size_t)j * g.n_f + f);
        }
        R acc[9];
        group_total<R, 16, 9, W>(hi, acc);
        if (tg == 0) {
            const R* old = g.lm_bel + (size_t)m * LBEL;
            R mu_old[3] = {__ldcg(old + 9), __ldcg(old + 10), __ldcg(old + 11)};
            dmu = finish_landmark<R>(g, P, m, lm_prior_scale(g, P, m, t + 1), acc, mu_old, g.lm_bel_out);
        }
    } else {
        // variables without factors: prior-only beliefs, mean 0
        const int i = (item - g.kf_item_n - g.big_item_n) * gsize + tg;
        if (i < g.n_orphan) {
            const int v = g.orphan[i];
            const R isig2 = P.inv_sigma2;
            if (v < g.n_kf) {
                R p[6], out[KBEL];
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    p[q] = (kf_prior_scale(g, P, v, t + 1) * g.kf_D[v * 6 + q] + P.anchor_scale * g.kf_A[v * 6 + q]) *
                           isig2;
                kf_prior_record<R>(p, out);
                store_rec<R, KBEL>(g.kf_bel_out + (size_t)v * KBEL, out);
            } else {
                const int mm = v - g.n_kf;
                R out[LBEL];
#pragma unroll
                for (int j = 0; j < LBEL; ++j) out[j] = R(0);
#pragma unroll
                for (int q = 0; q < 3; ++q) out[pk(q, q)] = lm_prior_scale(g, P, mm, t + 1) * g.lm_D[mm * 3 + q] * isig2;
                store_rec<R, LBEL>(g.lm_bel_out + (size_t)mm * LBEL, out);
            }
        }
    }
    return dmu;
}

// phase-B work items, and the blocks that hold them at one item per group
template <typename R>
__host__ __device__ inline int phase_b_items(const DevGraph<R>& g) {
    return g.kf_item_n + g.big_item_n + (g.n_orphan + 32 * g.b_warps - 1) / (32 * g.b_warps);
}
template <typename R>
__host__ __device__ inline int phase_b_blocks(const DevGraph<R>& g) {
    constexpr int WPB = FACTOR_BLOCK / 32;
    return (phase_b_items(g) * g.b_warps + WPB - 1) / WPB;
}
// the item of this thread's group when block b holds items from b * items-per-block
__device__ __forceinline__ int phase_b_item_of(int W, int block) {
    return W == FACTOR_BLOCK / 32 ? block : block * (FACTOR_BLOCK / 32) + (int(threadIdx.x) >> 5);
}

// ------------------------------------------------------------------------
// Two-kernel iteration (the launch-per-phase path).

// Programmatic dependent launch: the per-phase kernels let the next kernel
// in the stream launch once all of their blocks are past their main work
// (so only one kernel waits ahead), and wait for the previous kernel's
// completion (and its memory) before they read anything it writes.  Without
// the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename R, int MODE, int NT, bool DEFER>
__device__ __forceinline__ void factor_body(const DevGraph<R>& g, const KParams<R>& P) {
    __shared__ __align__(16) MlpSmem<MODE> S;
    mlp_load_async<MODE>(P, S);   // network weights do not change between iterations
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    const int t = g.ctl[CTL_ITER];
    float dmu = 0.0f;
    if (tile < g.n_tiles)   // uniform per warp
        dmu = tile_work<R, MODE, DEFER>(g, P, g.tile_off + tile, t, lane, S, MODE == DAMP_LEARNED);
    else if constexpr (MODE == DAMP_LEARNED) mlp_load_wait();   // the block's barrier, for warps without a tile
    pdl_allow_next();
    dmu = warp_max(dmu);
    if (lane == 0 && dmu > 0.0f) dmu_atomic_max_slot(g.ctl, dmu_slot(t), dmu);
    // the belief kernel of this iteration reads t from CTL_ITER_B: the belief
    // kernel of t - 1 has finished and that of t starts after this kernel
    if (blockIdx.x == 0 && threadIdx.x == 0) g.ctl[CTL_ITER_B] = t;
}

// NT threads per block, and at least MINB blocks per SM (the register budget
// per thread; 1 = no constraint).  Each warp does one tile whatever the
// shape, so every shape gives bitwise identical results; the FP32 fixed
// schedule is instantiated in several shapes for the autotuner.
template <typename R, int MODE, int NT, int MINB, bool DEFER = false>
__global__ void __launch_bounds__(NT, MINB) factor_kernel(const __grid_constant__ DevGraph<R> g,
                                                          const __grid_constant__ KParams<R> P) {
    factor_body<R, MODE, NT, DEFER>(g, P);
}

// The tiles that factor_kernel<..., DEFER = true> left in this iteration
// (a factor of theirs needs the FP64 redo), worked with it: warps walk the
// list.  No store of theirs happened before, so they see the same state.
// The last block to finish clears the list for the next use of its slot.
template <typename R>
__global__ void __launch_bounds__(FACTOR_BLOCK) factor_deferred_kernel(const __grid_constant__ DevGraph<R> g,
                                                                       const __grid_constant__ KParams<R> P) {
    constexpr int WPB = FACTOR_BLOCK / 32;
    MlpSmem<DAMP_FIXED> S;
    pdl_wait_prev();
    const int lane = threadIdx.x & 31;
    const int t = g.ctl[CTL_ITER];
    const int slot = CTL_DEFER_N0 + (t & 1);
    const int n = min(g.ctl[slot], g.n_tiles);
    float dmu = 0.0f;
    for (int i = blockIdx.x * WPB + (threadIdx.x >> 5); i < n; i += gridDim.x * WPB)
        dmu = fmaxf(dmu, tile_work<R, DAMP_FIXED, false>(g, P, g.deferred[i], t, lane, S));
    pdl_allow_next();
    dmu = warp_max(dmu);
    if (lane == 0 && dmu > 0.0f) dmu_atomic_max_slot(g.ctl, dmu_slot(t), dmu);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&g.ctl[CTL_DEFER_DONE], 1) == int(gridDim.x) - 1) {
            g.ctl[slot] = 0;
            g.ctl[CTL_DEFER_DONE] = 0;
        }
    }
}

// BW = g.b_warps (warps per belief item), one instantiation per mapping
template <typename R, int BW>
__global__ void __launch_bounds__(FACTOR_BLOCK) belief_kernel(DevGraph<R> g, KParams<R> P) {
    pdl_wait_prev();
    const int t = g.ctl[CTL_ITER_B];
    // close the iteration from one thread: the factor kernel of t has
    // finished and that of t + 1 starts only after this kernel, so the
    // counter it reads and the |dmu| slot it fills are free to set now
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g.ctl[CTL_ITER] = t + 1;
        g.ctl[dmu_slot(t + 1)] = 0;
    }
    float dmu = 0.0f;
    const int item = phase_b_item_of(BW, blockIdx.x);
    if (item < phase_b_items(g)) dmu = phase_b_item<R, BW>(g, P, item, t);   // uniform per group
    pdl_allow_next();
    // max is order independent: the atomic on non-negative float bits is deterministic
    if (dmu > 0.0f) dmu_atomic_max_slot(g.ctl, dmu_slot(t), dmu);
}

// ------------------------------------------------------------------------
// Persistent iteration kernel: one cooperative launch runs up to n_iters
// iterations; the two phases are separated by a grid barrier.  The barrier's
// wait is bounded: after ~1 s without progress the block records a timeout
// (CTL_ERR = 2) and every block leaves the loop.

constexpr long long BARRIER_SPIN_LIMIT = 10000000;   // x ~100 ns sleeps

__device__ __forceinline__ bool grid_barrier(int32_t* ctl, int nblocks, int* flag_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int32_t* vgen = ctl + CTL_BAR_GEN;
        volatile int32_t* verr = ctl + CTL_ERR;
        const int gen = *vgen;
        __threadfence();
        const int arrived = atomicAdd(&ctl[CTL_BAR_COUNT], 1);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&ctl[CTL_BAR_COUNT], 0);
            __threadfence();
            atomicAdd(&ctl[CTL_BAR_GEN], 1);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (*verr == 2 || ++spins > BARRIER_SPIN_LIMIT) {
                    atomicCAS(&ctl[CTL_ERR], 0, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *flag_sh = ok && (*verr != 2);
    }
    __syncthreads();
    return *flag_sh;
}

// BW = g.b_warps (warps per belief item): a separate instantiation per
// mapping, so that the block mapping's barriers and shared-memory reduction
// do not weigh on the register allocation of the warp mapping's kernel.
// MINB: at least this many blocks per SM (the register budget; 1 = none),
// a launch shape the autotuner chooses for the FP32 fixed schedule.
template <typename R, int MODE, int BW, int MINB>
__global__ void __launch_bounds__(FACTOR_BLOCK, MINB)
    persistent_kernel(const __grid_constant__ DevGraph<R> g, const __grid_constant__ KParams<R> P, int n_iters,
                      float conv_tol, int check_every) {
    __shared__ int flag_sh;
    __shared__ __align__(16) MlpSmem<MODE> S;
    mlp_load<MODE>(P, S);
    constexpr int WPB = FACTOR_BLOCK / 32;
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * WPB + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * WPB;
    const int nb = gridDim.x;
    const int t0 = __ldcg(&g.ctl[CTL_ITER]);
    const int items = phase_b_items(g);
    int done = 0;
    float last = 0.0f;
    for (int it = 0; it < n_iters; ++it) {
        const int t = t0 + it;
        // phase A: factors and landmarks wholly inside a tile
        float dmu = 0.0f;
        for (int tile = gwarp; tile < g.n_tiles; tile += nwarps)
            dmu = fmaxf(dmu, tile_work<R, MODE>(g, P, g.tile_off + tile, t, lane, S));
        dmu = warp_max(dmu);
        if (lane == 0 && dmu > 0.0f) dmu_atomic_max_slot(g.ctl, dmu_slot(t), dmu);
        if (!grid_barrier(g.ctl, nb, &flag_sh)) break;
        // phase B: keyframes, split landmarks, orphans
        if (blockIdx.x == 0 && threadIdx.x == 0) g.ctl[dmu_slot(t + 1)] = 0;   // every block has read it
        float d2 = 0.0f;
        // a block per item, or a warp per item (see phase_b_item)
        constexpr bool per_block = BW == WPB;
        const int stride = per_block ? nb : nwarps;
        for (int item = per_block ? int(blockIdx.x) : gwarp; item < items; item += stride)
            d2 = fmaxf(d2, phase_b_item<R, BW>(g, P, item, t));
        if (d2 > 0.0f) dmu_atomic_max_slot(g.ctl, dmu_slot(t), d2);   // groups' first threads
        if (!grid_barrier(g.ctl, nb, &flag_sh)) break;
        done = it + 1;
        last = __int_as_float(__ldcg(&g.ctl[dmu_slot(t)]));
        if (conv_tol > 0.0f && done % check_every == 0 && last < conv_tol) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g.ctl[CTL_ITER] = t0 + done;
        g.ctl[CTL_DMU_LAST] = __float_as_int(last);
        g.ctl[CTL_ITERS_RUN] = done;
    }
}

// Beliefs of iteration 0: b^0 = prior(0) (+ anchor), mean 0.
template <typename R>
__global__ void init_beliefs_kernel(DevGraph<R> g, KParams<R> P) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const R isig2 = P.inv_sigma2;
    if (v < g.n_kf) {
        const R s = kf_prior_scale(g, P, v, g.kf_birth[v]);
        R p[6], out[KBEL];
#pragma unroll
        for (int i = 0; i < 6; ++i) p[i] = (s * g.kf_D[v * 6 + i] + P.anchor_scale * g.kf_A[v * 6 + i]) * isig2;
        kf_prior_record<R>(p, out);
        store_rec<R, KBEL>(g.kf_bel + (size_t)v * KBEL, out);
    } else if (v < g.n_kf + g.n_lm) {
        const int m = v - g.n_kf;
        const R s = lm_prior_scale(g, P, m, g.lm_birth[m]);
        R out[LBEL];
#pragma unroll
        for (int j = 0; j < LBEL; ++j) out[j] = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) out[pk(i, i)] = s * g.lm_D[m * 3 + i] * isig2;
        store_rec<R, LBEL>(g.lm_bel + (size_t)m * LBEL, out);
    }
}

// ------------------------------------------------------------------------
// prior generation (Sec. 4 / Sec. 8): per-variable mean over its factors of
// diag(J_v^T J_v) at the factors' linearisation points (the references, at
// creation) with Huber weight 1 and sigma = 1.

template <typename R>
__global__ void __launch_bounds__(FACTOR_BLOCK) prior_factor_kernel(DevGraph<R> g, KParams<R> P, R* tmp_k, R* tmp_l) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.n_f) return;
    const int k = g.fk[f], m = g.fm[f];
    KParams<R> Q = P;
    Q.huber_n = R(0);
    Q.inv_sigma2 = R(1);
    Q.inv_sigma = R(1);
    R x0[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x0[i] = g.x0[(size_t)i * g.n_f + f];
    Lin<R> L;
    linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x0,
                 g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);
#pragma unroll
    for (int j = 0; j < 6; ++j) tmp_k[(size_t)j * g.n_f + f] = L.W * (L.Jk[0][j] * L.Jk[0][j] + L.Jk[1][j] * L.Jk[1][j]);
#pragma unroll
    for (int j = 0; j < 3; ++j) tmp_l[(size_t)j * g.n_f + f] = L.W * (L.Jl[0][j] * L.Jl[0][j] + L.Jl[1][j] * L.Jl[1][j]);
}

template <typename R, int n>
__device__ __forceinline__ void finish_prior(R* D, int deg) {
    R mx = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) {
        if (deg > 0) D[i] /= R(deg);
        mx = fmax(mx, D[i]);
    }
#pragma unroll
    for (int i = 0; i < n; ++i) {
        if (mx <= R(0)) D[i] = R(1);
        else if (D[i] < R(1e-9) * mx) D[i] = R(1e-9) * mx;
    }
}

template <typename R>
__global__ void prior_reduce_kernel(DevGraph<R> g, const R* tmp_k, const R* tmp_l, R* kf_D, R* lm_D) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < g.n_kf) {
        R D[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        const int b0 = g.kf_off[v], b1 = g.kf_off[v + 1];
        for (int i = b0; i < b1; ++i) {
            const int f = g.kf_list[i];
#pragma unroll
            for (int j = 0; j < 6; ++j) D[j] += tmp_k[(size_t)j * g.n_f + f];
        }
        finish_prior<R, 6>(D, b1 - b0);
#pragma unroll
        for (int j = 0; j < 6; ++j) kf_D[v * 6 + j] = D[j];
    } else if (v < g.n_kf + g.n_lm) {
        const int m = v - g.n_kf;
        R D[3] = {R(0), R(0), R(0)};
        const int b0 = g.lm_off[m], b1 = g.lm_off[m + 1];
        for (int f = b0; f < b1; ++f) {
#pragma unroll
            for (int j = 0; j < 3; ++j) D[j] += tmp_l[(size_t)j * g.n_f + f];
        }
        finish_prior<R, 3>(D, b1 - b0);
#pragma unroll
        for (int j = 0; j < 3; ++j) lm_D[m * 3 + j] = D[j];
    }
}

// ------------------------------------------------------------------------
// metrics: average reprojection error (Sec. 9.1) at the current means, its
// distance to reference projections, Huber-regime count.  Two-pass fixed
// order reduction through per-block partials.

template <typename R>
__global__ void __launch_bounds__(METRIC_BLOCK) metrics_kernel(DevGraph<R> g, KParams<R> P, double* partials) {
    __shared__ double red[4][METRIC_BLOCK];
    const int tid = threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f = blockIdx.x * METRIC_BLOCK + tid; f < g.n_f; f += gridDim.x * METRIC_BLOCK) {
        const int k = g.fk[f], m = g.fm[f];
        const R* kb = g.kf_bel + (size_t)k * KBEL;
        const R* lb = g.lm_bel + (size_t)m * LBEL;
        R x[9] = {kb[KB_MU], kb[KB_MU + 1], kb[KB_MU + 2], kb[KB_MU + 3], kb[KB_MU + 4], kb[KB_MU + 5],
                   lb[9], lb[10], lb[11]};
        KParams<R> Q = P;
        Q.huber_n = R(0);
        Lin<R> L;
        linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x,
                     g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);
        if (L.W > R(0)) {
            double e = sqrt(double(L.r2));
            v[0] += e;
            v[2] += 1.0;
            if (P.huber_n > R(0) && e * double(P.inv_sigma) > double(P.huber_n)) v[3] += 1.0;
        }
    }
    for (int j = 0; j < 4; ++j) red[j][tid] = v[j];
    __syncthreads();
    for (int st = METRIC_BLOCK / 2; st > 0; st >>= 1) {
        if (tid < st)
            for (int j = 0; j < 4; ++j) red[j][tid] += red[j][tid + st];
        __syncthreads();
    }
    if (tid == 0)
        for (int j = 0; j < 4; ++j) partials[(size_t)j * gridDim.x + blockIdx.x] = red[j][0];
}

// reference-projection distance needs the residual vector, not only |r|:
// recompute h(mu) per factor
template <typename R>
__global__ void __launch_bounds__(METRIC_BLOCK) metrics_ref_kernel(DevGraph<R> g, KParams<R> P, double* partials) {
    __shared__ double red[2][METRIC_BLOCK];
    const int tid = threadIdx.x;
    double acc = 0.0, cnt = 0.0;
    for (int f = blockIdx.x * METRIC_BLOCK + tid; f < g.n_f; f += gridDim.x * METRIC_BLOCK) {
        const int k = g.fk[f], m = g.fm[f];
        const R* kb = g.kf_bel + (size_t)k * KBEL;
        const R* lb = g.lm_bel + (size_t)m * LBEL;
        R x[9] = {kb[KB_MU], kb[KB_MU + 1], kb[KB_MU + 2], kb[KB_MU + 3], kb[KB_MU + 4], kb[KB_MU + 5],
                   lb[9], lb[10], lb[11]};
        KParams<R> Q = P;
        Q.huber_n = R(0);
        Lin<R> L;
        // with z = reference pixel the residual is ref - h(mu)
        R ru = g.uv_ref[2 * (size_t)f], rv = g.uv_ref[2 * (size_t)f + 1];
        linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x, ru, rv, L);
        if (L.W > R(0) && isfinite(ru)) {
            acc += sqrt(double(L.r2));
            cnt += 1.0;
        }
    }
    red[0][tid] = acc;
    red[1][tid] = cnt;
    __syncthreads();
    for (int st = METRIC_BLOCK / 2; st > 0; st >>= 1) {
        if (tid < st) {
            red[0][tid] += red[0][tid + st];
            red[1][tid] += red[1][tid + st];
        }
        __syncthreads();
    }
    if (tid == 0) {
        partials[(size_t)4 * gridDim.x + blockIdx.x] = red[0][0];
        partials[(size_t)5 * gridDim.x + blockIdx.x] = red[1][0];
    }
}

// Per-problem reprojection statistics of a batch: one block per problem
// over its contiguous factor range, fixed-order block reduction.
// out[3p] = sum of errors, out[3p+1] = count, out[3p+2] = Huber-regime count.
template <typename R>
__global__ void __launch_bounds__(METRIC_BLOCK) problem_metrics_kernel(DevGraph<R> g, KParams<R> P,
                                                                       const int32_t* prob_f0, double* out) {
    __shared__ double red[3][METRIC_BLOCK];
    const int tid = threadIdx.x, p = blockIdx.x;
    double v[3] = {0.0, 0.0, 0.0};
    for (int f = prob_f0[p] + tid; f < prob_f0[p + 1]; f += METRIC_BLOCK) {
        const int k = g.fk[f], m = g.fm[f];
        const R* kb = g.kf_bel + (size_t)k * KBEL;
        const R* lb = g.lm_bel + (size_t)m * LBEL;
        R x[9] = {kb[KB_MU], kb[KB_MU + 1], kb[KB_MU + 2], kb[KB_MU + 3], kb[KB_MU + 4], kb[KB_MU + 5],
                   lb[9], lb[10], lb[11]};
        KParams<R> Q = P;
        Q.huber_n = R(0);
        Lin<R> L;
        linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x,
                     g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);
        if (L.W > R(0)) {
            double e = sqrt(double(L.r2));
            v[0] += e;
            v[1] += 1.0;
            if (P.huber_n > R(0) && e * double(P.inv_sigma) > double(P.huber_n)) v[2] += 1.0;
        }
    }
    for (int j = 0; j < 3; ++j) red[j][tid] = v[j];
    __syncthreads();
    for (int st = METRIC_BLOCK / 2; st > 0; st >>= 1) {
        if (tid < st)
            for (int j = 0; j < 3; ++j) red[j][tid] += red[j][tid + st];
        __syncthreads();
    }
    if (tid == 0)
        for (int j = 0; j < 3; ++j) out[3 * (size_t)p + j] = red[j][0];
}

// Per-factor reprojection error |z - h(mu)| at the current means (Sec. 9.1),
// -1 for a point closer than z_min to its camera.
template <typename R>
__global__ void __launch_bounds__(METRIC_BLOCK) residual_kernel(DevGraph<R> g, KParams<R> P, double* out) {
    const int f = blockIdx.x * METRIC_BLOCK + threadIdx.x;
    if (f >= g.n_f) return;
    const int k = g.fk[f], m = g.fm[f];
    const R* kb = g.kf_bel + (size_t)k * KBEL;
    const R* lb = g.lm_bel + (size_t)m * LBEL;
    R x[9] = {kb[KB_MU], kb[KB_MU + 1], kb[KB_MU + 2], kb[KB_MU + 3], kb[KB_MU + 4], kb[KB_MU + 5],
              lb[9], lb[10], lb[11]};
    KParams<R> Q = P;
    Q.huber_n = R(0);
    Lin<R> L;
    linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x,
                 g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);
    out[f] = L.W > R(0) ? sqrt(double(L.r2)) : -1.0;
}

__global__ void metrics_finish_kernel(const double* partials, int nb, int with_ref, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < 6; ++j) {
        if (j >= 4 && !with_ref) break;
        for (int b = 0; b < nb; ++b) s[j] += partials[(size_t)j * nb + b];
    }
    out[MET_N_ARE] = s[2];
    out[MET_ARE] = s[2] > 0 ? s[0] / s[2] : 0.0;
    out[MET_HUBER] = s[3];
    out[MET_ARE_REF] = with_ref ? (s[5] > 0 ? s[4] / s[5] : 0.0) : -1.0;
}

// ------------------------------------------------------------------------
// launchers

int metrics_blocks(int n_f) {
    int b = (n_f + METRIC_BLOCK - 1) / METRIC_BLOCK;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return b;
}

// One launch, with programmatic stream serialisation when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), int blocks, int threads, cudaStream_t s, bool pdl, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename R, int MODE, int NT, int MINB, bool DEFER = false>
cudaError_t launch_factor_shape(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s, bool pdl) {
    constexpr int wpb = NT / 32;
    const int blocks = std::max(1, (g.n_tiles + wpb - 1) / wpb);   // >= 1: it also publishes the iteration index
    cudaError_t e = launch_ex(factor_kernel<R, MODE, NT, MINB, DEFER>, blocks, NT, s, pdl, g, p);
    if constexpr (DEFER) {
        // deferred tiles are rare: a few hundred warps walk the list
        constexpr int wpd = FACTOR_BLOCK / 32;
        const int nb = std::max(1, std::min((g.n_tiles + wpd - 1) / wpd, 608));
        if (e == cudaSuccess) e = launch_ex(factor_deferred_kernel<R>, nb, FACTOR_BLOCK, s, pdl, g, p);
    }
    return e;
}

template <typename R>
cudaError_t launch_factor(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s, int mode, bool pdl, int shape) {
    if (mode == DAMP_LEARNED) return launch_factor_shape<R, DAMP_LEARNED, 128, 1>(g, p, s, pdl);
    if (mode == DAMP_RECORD) return launch_factor_shape<R, DAMP_RECORD, 128, 1>(g, p, s, pdl);
    if constexpr (sizeof(R) == 4) {
        switch (shape) {
            case 1: return launch_factor_shape<R, DAMP_FIXED, 128, 3>(g, p, s, pdl);
            case 2: return launch_factor_shape<R, DAMP_FIXED, 128, 4>(g, p, s, pdl);
            case 3: return launch_factor_shape<R, DAMP_FIXED, 64, 1>(g, p, s, pdl);
            case 4: return launch_factor_shape<R, DAMP_FIXED, 128, 4, true>(g, p, s, pdl);
            case 5: return launch_factor_shape<R, DAMP_FIXED, 128, 3, true>(g, p, s, pdl);
            default: break;
        }
    }
    return launch_factor_shape<R, DAMP_FIXED, 128, 1>(g, p, s, pdl);
}

template <typename R>
cudaError_t launch_belief(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s, bool pdl) {
    int blocks = phase_b_blocks(g);
    if (blocks < 1) blocks = 1;
    if (g.b_warps == FACTOR_BLOCK / 32)
        return launch_ex(belief_kernel<R, FACTOR_BLOCK / 32>, blocks, FACTOR_BLOCK, s, pdl, g, p);
    return launch_ex(belief_kernel<R, 1>, blocks, FACTOR_BLOCK, s, pdl, g, p);
}

// the persistent kernel for this graph's belief mapping and damping
// schedule (one launch shape)
template <typename R, int BW>
const void* persistent_fn_bw(int mode, int) {
    if (mode == DAMP_LEARNED) return reinterpret_cast<const void*>(persistent_kernel<R, DAMP_LEARNED, BW, 1>);
    return reinterpret_cast<const void*>(persistent_kernel<R, DAMP_FIXED, BW, 1>);
}

template <typename R>
const void* persistent_fn(const DevGraph<R>& g, int mode, int shape) {
    constexpr int WPB = FACTOR_BLOCK / 32;
    return g.b_warps == WPB ? persistent_fn_bw<R, WPB>(mode, shape) : persistent_fn_bw<R, 1>(mode, shape);
}

template <typename R>
int persistent_grid(const DevGraph<R>& g, int mode, int shape) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_fn(g, mode, shape), FACTOR_BLOCK, 0);
    if (e != cudaSuccess || per_sm <= 0) return 0;
    constexpr int wpb = FACTOR_BLOCK / 32;
    const int cap = sms * per_sm;
    const int want = std::max((g.n_tiles + wpb - 1) / wpb, phase_b_blocks(g));
    return std::max(1, std::min(cap, want));
}

template <typename R>
cudaError_t launch_persistent(const DevGraph<R>& g, const KParams<R>& p, int n_iters, float conv_tol,
                              int check_every, int grid, cudaStream_t s, int mode, int shape) {
    DevGraph<R> gg = g;
    KParams<R> pp = p;
    void* args[] = {&gg, &pp, &n_iters, &conv_tol, &check_every};
    return cudaLaunchCooperativeKernel(persistent_fn(g, mode, shape), dim3(grid), dim3(FACTOR_BLOCK), args, 0, s);
}

// The current messages' eta in factor order (keyframe side 6, landmark side
// 3; SoA 9 x n_f): the reference of the record schedule's damping targets.
// Both messages of a factor are in the basis of its current Jacobian, whose
// keyframe block the slot's kj record holds (the landmark block is minus its
// first three columns).
template <typename R>
__global__ void capture_messages_kernel(DevGraph<R> g, const R* __restrict__ mk_cur, R* __restrict__ eta_inf) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.n_f) return;
    const size_t n_f = g.n_f;
    const R* rec = mk_cur + (size_t)g.kpos[f] * KREC;
    const R* jr = g.kj + (size_t)g.kpos[f] * KJ;
    const R J[2][6] = {{jr[0], jr[1], jr[2], jr[3], jr[4], jr[5]}, {jr[6], jr[7], jr[8], jr[9], jr[10], jr[11]}};
    const R Jl[2][3] = {{-jr[0], -jr[1], -jr[2]}, {-jr[6], -jr[7], -jr[8]}};
    R ek[6], el[3];
    msg_eta<R, 6>(J, rec[3], rec[4], ek);
    msg_eta<R, 3>(Jl, g.ml[3 * n_f + f], g.ml[4 * n_f + f], el);
#pragma unroll
    for (int i = 0; i < 6; ++i) eta_inf[i * n_f + f] = ek[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) eta_inf[(6 + i) * n_f + f] = el[i];
}

template <typename R>
cudaError_t launch_capture_messages(const DevGraph<R>& g, int t, R* eta_inf, cudaStream_t s) {
    if (g.n_f == 0) return cudaSuccess;
    // after t completed iterations the current messages m^t are in buffer t & 1
    const R* mk_cur = (t & 1) ? g.mk2 : g.mk;
    capture_messages_kernel<R><<<(g.n_f + 255) / 256, 256, 0, s>>>(g, mk_cur, eta_inf);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s) {
    int nv = g.n_kf + g.n_lm;
    if (nv > 0) init_beliefs_kernel<R><<<(nv + 127) / 128, 128, 0, s>>>(g, p);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prior(const DevGraph<R>& g, const KParams<R>& p, R* tmp_k, R* tmp_l, R* kf_D, R* lm_D,
                         cudaStream_t s) {
    if (g.n_f > 0) prior_factor_kernel<R><<<(g.n_f + FACTOR_BLOCK - 1) / FACTOR_BLOCK, FACTOR_BLOCK, 0, s>>>(g, p, tmp_k, tmp_l);
    int nv = g.n_kf + g.n_lm;
    if (nv > 0) prior_reduce_kernel<R><<<(nv + 127) / 128, 128, 0, s>>>(g, tmp_k, tmp_l, kf_D, lm_D);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_metrics(const DevGraph<R>& g, const KParams<R>& p, double* partials, int nb, double* out,
                           cudaStream_t s) {
    metrics_kernel<R><<<nb, METRIC_BLOCK, 0, s>>>(g, p, partials);
    if (g.uv_ref) metrics_ref_kernel<R><<<nb, METRIC_BLOCK, 0, s>>>(g, p, partials);
    metrics_finish_kernel<<<1, 32, 0, s>>>(partials, nb, g.uv_ref != nullptr, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_problem_metrics(const DevGraph<R>& g, const KParams<R>& p, const int32_t* prob_f0, int n_problems,
                                   double* out, cudaStream_t s) {
    if (n_problems > 0) problem_metrics_kernel<R><<<n_problems, METRIC_BLOCK, 0, s>>>(g, p, prob_f0, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_residuals(const DevGraph<R>& g, const KParams<R>& p, double* out, cudaStream_t s) {
    if (g.n_f > 0) residual_kernel<R><<<(g.n_f + METRIC_BLOCK - 1) / METRIC_BLOCK, METRIC_BLOCK, 0, s>>>(g, p, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// One graph split across ranks: the records a rank exchanges between the
// phases of an iteration.  Message records (kind 0), per factor: its
// compact message to the keyframe of iteration t+1 (KREC) and its staged
// Jacobian block (KJ) -- what the keyframe's owner needs to sum it.
// Keyframe records (kind 1): the belief record (KBEL).

constexpr int SPLIT_MSG = KREC + KJ;

template <typename R>
__global__ void split_records_kernel(DevGraph<R> g, int kind, int put, int n, const int32_t* __restrict__ idx,
                                     float* io) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (kind == 0) {
        const int t = g.ctl[CTL_ITER];
        const size_t slot = (size_t)g.kpos[idx[i]];
        R* rec = mk_write(g, t) + slot * KREC;
        R* jr = g.kjs + slot * KJ;
        float* o = io + (size_t)i * SPLIT_MSG;
        for (int j = 0; j < KREC; ++j) {
            if (put) rec[j] = R(o[j]);
            else o[j] = float(rec[j]);
        }
        for (int j = 0; j < KJ; ++j) {
            if (put) jr[j] = R(o[KREC + j]);
            else o[KREC + j] = float(jr[j]);
        }
    } else {
        R* rec = g.kf_bel + (size_t)idx[i] * KBEL;
        float* o = io + (size_t)i * KBEL;
        for (int j = 0; j < KBEL; ++j) {
            if (put) rec[j] = R(o[j]);
            else o[j] = float(rec[j]);
        }
    }
}

template <typename R>
cudaError_t launch_split_records(const DevGraph<R>& g, int kind, int put, int n, const int32_t* idx, float* io,
                                 cudaStream_t s) {
    if (n > 0) split_records_kernel<R><<<(n + 127) / 128, 128, 0, s>>>(g, kind, put, n, idx, io);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Re-layout after a keyframe is added (incremental SLAM): the per-factor
// state of the grown graph gathered on the device from the previous
// layout's buffers.  src_f[f]: the previous internal index of the new
// layout's factor f, or -1 for a factor of the new keyframe.
//   phase 0: linearisation points -- kept, or for a new factor the current
//            means (its keyframe's chart origin and its landmark's mean,
//            or 0 for a new landmark);
//   phase 1: t_lin, the stored linearisation, the landmark message, the
//            learned schedule's history, and by keyframe slot the Jacobian
//            block and both message buffers -- kept, or empty and t_lin = t.

template <typename R>
__global__ void relayout_kernel(DevGraph<R> nw, RelayoutSrc<R> o, int phase) {
    const int F1 = nw.n_f, F0 = o.n_f;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < F1; f += gridDim.x * blockDim.x) {
        const int src = o.src_f[f];
        if (phase == 0) {
            if (src >= 0) {
                for (int i = 0; i < 9; ++i) nw.x0[(size_t)i * F1 + f] = o.x0[(size_t)i * F0 + src];
            } else {
                const int m = nw.fm[f];
                for (int i = 0; i < 6; ++i) nw.x0[(size_t)i * F1 + f] = R(0);
                for (int i = 0; i < 3; ++i)
                    nw.x0[(size_t)(6 + i) * F1 + f] = m < o.n_lm ? o.lm_bel[(size_t)m * LBEL + 9 + i] : R(0);
            }
            continue;
        }
        const int slot = nw.kpos[f];
        R* mk_cur = (o.t & 1) ? nw.mk2 : nw.mk;
        R* mk_oth = (o.t & 1) ? nw.mk : nw.mk2;
        if (src >= 0) {
            const int os = o.kpos[src];
            nw.tlin[f] = o.tlin[src];
            for (int i = 0; i < NML; ++i) nw.ml[(size_t)i * F1 + f] = o.ml[(size_t)i * F0 + src];
            for (int i = 0; i < NLIN; ++i) nw.lin[(size_t)i * F1 + f] = o.lin[(size_t)i * F0 + src];
            for (int i = 0; i < HIST; ++i) nw.hist[(size_t)i * F1 + f] = o.hist[(size_t)i * F0 + src];
            for (int i = 0; i < KJ; ++i) nw.kj[(size_t)slot * KJ + i] = o.kj[(size_t)os * KJ + i];
            for (int i = 0; i < KREC; ++i) {
                mk_cur[(size_t)slot * KREC + i] = o.mk_cur[(size_t)os * KREC + i];
                mk_oth[(size_t)slot * KREC + i] = o.mk_oth[(size_t)os * KREC + i];
            }
        } else {
            nw.tlin[f] = o.t;
            for (int i = 0; i < NML; ++i) nw.ml[(size_t)i * F1 + f] = R(0);
            for (int i = 0; i < NLIN; ++i) nw.lin[(size_t)i * F1 + f] = R(0);
            for (int i = 0; i < HIST; ++i) nw.hist[(size_t)i * F1 + f] = 0.0f;
            for (int i = 0; i < KJ; ++i) nw.kj[(size_t)slot * KJ + i] = R(0);
            for (int i = 0; i < KREC; ++i) {
                mk_cur[(size_t)slot * KREC + i] = R(0);
                mk_oth[(size_t)slot * KREC + i] = R(0);
            }
        }
    }
}

template <typename R>
cudaError_t launch_relayout(const DevGraph<R>& nw, const RelayoutSrc<R>& o, int phase, cudaStream_t s) {
    const int blocks = std::max(1, std::min((nw.n_f + 255) / 256, 1024));
    relayout_kernel<R><<<blocks, 256, 0, s>>>(nw, o, phase);
    return cudaGetLastError();
}

#define GBP_INSTANTIATE(R)                                                                                 \
    template cudaError_t launch_factor<R>(const DevGraph<R>&, const KParams<R>&, cudaStream_t, int, bool, int); \
    template cudaError_t launch_capture_messages<R>(const DevGraph<R>&, int, R*, cudaStream_t);            \
    template cudaError_t launch_init<R>(const DevGraph<R>&, const KParams<R>&, cudaStream_t);              \
    template cudaError_t launch_belief<R>(const DevGraph<R>&, const KParams<R>&, cudaStream_t, bool);      \
    template cudaError_t launch_problem_metrics<R>(const DevGraph<R>&, const KParams<R>&, const int32_t*, int, double*, cudaStream_t); \
    template int persistent_grid<R>(const DevGraph<R>&, int, int);                                         \
    template cudaError_t launch_persistent<R>(const DevGraph<R>&, const KParams<R>&, int, float, int, int, cudaStream_t, int, int); \
    template cudaError_t launch_prior<R>(const DevGraph<R>&, const KParams<R>&, R*, R*, R*, R*, cudaStream_t); \
    template cudaError_t launch_metrics<R>(const DevGraph<R>&, const KParams<R>&, double*, int, double*, cudaStream_t); \
    template cudaError_t launch_residuals<R>(const DevGraph<R>&, const KParams<R>&, double*, cudaStream_t); \
    template cudaError_t launch_split_records<R>(const DevGraph<R>&, int, int, int, const int32_t*, float*, cudaStream_t); \
    template cudaError_t launch_relayout<R>(const DevGraph<R>&, const RelayoutSrc<R>&, int, cudaStream_t);

GBP_INSTANTIATE(float)
GBP_INSTANTIATE(double)

}  // namespace gbp
