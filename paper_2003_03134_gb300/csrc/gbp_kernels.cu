// gbp_kernels.cu -- CUDA kernels (sm_103a) of one synchronous GBP iteration
// for bundle adjustment (Ortiz et al., "Bundle Adjustment on a Graph
// Processor", CVPR 2020), templated on the storage/arithmetic type R
// (float: the fast path with an FP64 fallback; double: a full-precision
// mode).
//
// Iteration t (Sec. 5, synchronous schedule):
//   factor kernel  -- one thread per factor: decide relinearisation (Sec. 5,
//                     Sec. 8), rebuild J and the residual at the factor's
//                     linearisation point, Huber weight (Sec. 6), both
//                     factor-to-variable messages (eqs. messageeta,
//                     messagelambda), damping of eta (Sec. 5, Sec. 8).
//   belief kernel  -- one block per keyframe (fixed-order tree reduction
//                     over its CSR list), one thread per landmark (its
//                     contiguous factor range): prior(t+1) + sum of messages
//                     (eqs. beliefeta, belieflambda), Cholesky mean.
// No atomics touch floating-point sums: every reduction has a fixed order,
// so results are bitwise reproducible.
//
// Message arithmetic.  A factor's information is rank 2: Lambda_f = W J^T J
// and eta_f = W J^T y with y = J x0 + r (Sec. 4).  Marginalising block b
// (incoming precision P_b = Lambda_belief_b - Lambda_msg_b and vector
// q_b = eta_belief_b - eta_msg_b) out of the product of the factor and the
// incoming message gives, by the matrix inversion lemma, exactly
//   Lambda_{f->a} = J_a^T (W N) J_a,   eta_{f->a} = J_a^T W N (y - s)
// with Q = J_b P_b^-1 J_b^T (2x2), s = J_b P_b^-1 q_b, N = (I + W Q)^-1.
// This equals the printed Schur complement A_aa - A_ab (A_bb + P_b)^-1 A_ba
// but never subtracts two large matrices, and Q = V^T V with
// V = L_b^-1 J_b^T (Cholesky P_b = L_b L_b^T) is PSD by construction.
#include "gbp_internal.h"

#include <math.h>

namespace gbp {

// ------------------------------------------------------------------------
// small dense helpers

__host__ __device__ constexpr int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

template <typename R>
__device__ __forceinline__ R rsqrt_exact(R x) { return R(1) / sqrt(x); }

// In-place Cholesky of a packed lower-triangular n x n SPD matrix.
// On return A holds L (packed) and inv_d[i] = 1 / L_ii.  Returns false if a
// pivot is not positive and finite; pivot_ratio = min pivot / max pivot.
template <typename R, int n>
__device__ __forceinline__ bool chol_packed(R* A, R* inv_d, R& pivot_ratio) {
    R pmin = R(0), pmax = R(0);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        R s = A[pk(j, j)];
#pragma unroll
        for (int p = 0; p < j; ++p) s -= A[pk(j, p)] * A[pk(j, p)];
        ok = ok && (s > R(0)) && isfinite(s);
        if (j == 0) { pmin = s; pmax = s; }
        pmin = fmin(pmin, s);
        pmax = fmax(pmax, s);
        R d = sqrt(fmax(s, R(0)));
        R id = R(1) / d;
        A[pk(j, j)] = d;
        inv_d[j] = id;
#pragma unroll
        for (int i = j + 1; i < n; ++i) {
            R t = A[pk(i, j)];
#pragma unroll
            for (int p = 0; p < j; ++p) t -= A[pk(i, p)] * A[pk(j, p)];
            A[pk(i, j)] = t * id;
        }
    }
    pivot_ratio = ok ? pmin / pmax : R(0);
    return ok;
}

// b <- L^-1 b (forward substitution with a packed Cholesky factor)
template <typename R, int n>
__device__ __forceinline__ void fwd_solve(const R* L, const R* inv_d, R* b) {
#pragma unroll
    for (int i = 0; i < n; ++i) {
        R s = b[i];
#pragma unroll
        for (int p = 0; p < i; ++p) s -= L[pk(i, p)] * b[p];
        b[i] = s * inv_d[i];
    }
}

// b <- L^-T b (backward substitution)
template <typename R, int n>
__device__ __forceinline__ void bwd_solve(const R* L, const R* inv_d, R* b) {
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
        R s = b[i];
#pragma unroll
        for (int p = i + 1; p < n; ++p) s -= L[pk(p, i)] * b[p];
        b[i] = s * inv_d[i];
    }
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
    if (th2 < R(1e-8)) {
        a = R(1) - th2 / R(6);
        b = R(0.5) - th2 / R(24);
    } else {
        R th = sqrt(th2);
        R sh = sin(R(0.5) * th);
        a = sin(th) / th;
        b = R(2) * sh * sh / th2;
    }
    if (th2 < R(0.25)) {
        c = R(1.0 / 6.0) + th2 * (R(-1.0 / 120.0) + th2 * (R(1.0 / 5040.0) +
            th2 * (R(-1.0 / 362880.0) + th2 * R(1.0 / 39916800.0))));
    } else {
        R th = sqrt(th2);
        c = (th - sin(th)) / (th2 * th);
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

template <typename R>
__device__ __forceinline__ void linearise(const KParams& P, const double* __restrict__ Rref,
                                          const double* __restrict__ cref, const double* __restrict__ lref,
                                          const R x0[9], R zu, R zv, Lin<R>& L) {
    R w[3] = {x0[3], x0[4], x0[5]};
    R E[9], Jw[9];
    so3_exp_jl(w, E, Jw);
    R Rr[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rr[i] = R(Rref[i]);
    R Rm[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Rm[i * 3 + j] = E[i * 3 + 0] * Rr[0 * 3 + j] + E[i * 3 + 1] * Rr[1 * 3 + j] + E[i * 3 + 2] * Rr[2 * 3 + j];
    // the large world coordinates cancel in double before rounding to R
    R d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = R(lref[i] - cref[i]) + (x0[6 + i] - x0[i]);
    R p[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) p[i] = Rm[i * 3 + 0] * d[0] + Rm[i * 3 + 1] * d[1] + Rm[i * 3 + 2] * d[2];

    if (!(p[2] >= R(P.z_min))) {
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
    const R fx = R(P.fx), fy = R(P.fy);
    R iz = R(1) / p[2];
    R u = fx * p[0] * iz, v = fy * p[1] * iz;
    R r0 = zu - (u + R(P.cx));
    R r1 = zv - (v + R(P.cy));
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
    if (P.huber_n > 0.0) {
        R M = sqrt(r2) * R(P.inv_sigma);
        R N = R(P.huber_n);
        if (M > N) k = R(2) * N / M - (N * N) / (M * M);
    }
    L.W = k * R(P.inv_sigma2);
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

// ------------------------------------------------------------------------
// one factor-to-variable message.  Incoming precision Pb (packed nb x nb,
// destroyed), incoming vector qb (nb), Jacobian rows of the marginalised
// block Jb (2 x nb) and of the target block Ja (2 x na).  Output Lambda
// (packed na x na) and eta (na).  Returns false when the Cholesky of Pb
// failed; *ratio receives its pivot ratio.

template <typename C, int na, int nb>
__device__ __forceinline__ bool message(C* Pb, const C* qb, const C Jb[2][nb], const C Ja[2][na], const C y[2],
                                        C W, C* lam, C* eta, C& ratio) {
    C inv_d[nb];
    bool ok = chol_packed<C, nb>(Pb, inv_d, ratio);
    C V0[nb], V1[nb], u[nb];
#pragma unroll
    for (int i = 0; i < nb; ++i) { V0[i] = Jb[0][i]; V1[i] = Jb[1][i]; u[i] = qb[i]; }
    fwd_solve<C, nb>(Pb, inv_d, V0);
    fwd_solve<C, nb>(Pb, inv_d, V1);
    fwd_solve<C, nb>(Pb, inv_d, u);
    C Q00 = C(0), Q01 = C(0), Q11 = C(0), s0 = C(0), s1 = C(0);
#pragma unroll
    for (int i = 0; i < nb; ++i) {
        Q00 += V0[i] * V0[i];
        Q01 += V0[i] * V1[i];
        Q11 += V1[i] * V1[i];
        s0 += V0[i] * u[i];
        s1 += V1[i] * u[i];
    }
    // N = (I + W Q)^-1
    C a00 = C(1) + W * Q00, a01 = W * Q01, a11 = C(1) + W * Q11;
    C idet = C(1) / (a00 * a11 - a01 * a01);
    C N00 = a11 * idet, N01 = -a01 * idet, N11 = a00 * idet;
    C M00 = W * N00, M01 = W * N01, M11 = W * N11;
    C e0 = y[0] - s0, e1 = y[1] - s1;
    C g0 = M00 * e0 + M01 * e1, g1 = M01 * e0 + M11 * e1;
    C ua[na], va[na];
#pragma unroll
    for (int i = 0; i < na; ++i) {
        ua[i] = M00 * Ja[0][i] + M01 * Ja[1][i];
        va[i] = M01 * Ja[0][i] + M11 * Ja[1][i];
        eta[i] = Ja[0][i] * g0 + Ja[1][i] * g1;
    }
#pragma unroll
    for (int i = 0; i < na; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) lam[pk(i, j)] = ua[i] * Ja[0][j] + va[i] * Ja[1][j];
    return ok;
}

// The same message in FP64 from FP32 inputs (the fallback for an
// ill-conditioned FP32 factorisation).
template <typename R, int na, int nb>
__device__ __noinline__ bool message_fp64(const R* Pb_in, const R* qb, const R Jb[2][nb], const R Ja[2][na],
                                          const R y[2], R W, R* lam, R* eta) {
    double Pb[nb * (nb + 1) / 2], q[nb], jb[2][nb], ja[2][na], yy[2], l[na * (na + 1) / 2], e[na], ratio;
    for (int i = 0; i < nb * (nb + 1) / 2; ++i) Pb[i] = double(Pb_in[i]);
    for (int i = 0; i < nb; ++i) { q[i] = double(qb[i]); jb[0][i] = double(Jb[0][i]); jb[1][i] = double(Jb[1][i]); }
    for (int i = 0; i < na; ++i) { ja[0][i] = double(Ja[0][i]); ja[1][i] = double(Ja[1][i]); }
    yy[0] = double(y[0]);
    yy[1] = double(y[1]);
    bool ok = message<double, na, nb>(Pb, q, jb, ja, yy, double(W), l, e, ratio);
    for (int i = 0; i < na * (na + 1) / 2; ++i) lam[i] = R(l[i]);
    for (int i = 0; i < na; ++i) eta[i] = R(e[i]);
    return ok;
}

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

__device__ __forceinline__ void raise_error(int32_t* ctl, int where) {
    if (atomicCAS(&ctl[CTL_ERR], 0, 1) == 0) ctl[CTL_ERR_WHERE] = where;
}

// ------------------------------------------------------------------------
// factor kernel

template <typename R>
__global__ void __launch_bounds__(FACTOR_BLOCK) factor_kernel(DevGraph<R> g, KParams P) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.n_f) return;
    const int n_f = g.n_f;
    const int t = g.ctl[CTL_ITER];
    const int k = g.fk[f], m = g.fm[f];

    R kb[KBEL], lb[LBEL];
    load_rec<R, KBEL>(g.kf_bel + (size_t)k * KBEL, kb);
    load_rec<R, LBEL>(g.lm_bel + (size_t)m * LBEL, lb);

    R x0[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x0[i] = g.x0[(size_t)i * n_f + f];
    int tl = g.tlin[f];

    // Sec. 5 / Sec. 8: relinearise when the adjacent means moved more than
    // beta from the linearisation point, at most every relin_interval
    // iterations.
    if (!P.linear && t - tl >= P.relin_interval) {
        R mu[9] = {kb[27], kb[28], kb[29], kb[30], kb[31], kb[32], lb[9], lb[10], lb[11]};
        R d2 = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) d2 += (mu[i] - x0[i]) * (mu[i] - x0[i]);
        if (sqrt(d2) > R(P.relin_beta)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                x0[i] = mu[i];
                g.x0[(size_t)i * n_f + f] = mu[i];
            }
            tl = t;
            g.tlin[f] = t;
            atomicAdd(&g.ctl[CTL_RELINS], 1);
        }
    }

    Lin<R> L;
    linearise<R>(P, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x0,
                 g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);

    // previous messages m^t
    R mk[KREC];
    load_rec<R, KREC>(g.mk + (size_t)f * KREC, mk);
    R ml[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) ml[i] = g.ml[(size_t)i * n_f + f];

    // ---- message to the keyframe: marginalise the landmark ----
    // incoming = landmark belief / this factor's previous message to it
    R Pm[6], qm[3];
#pragma unroll
    for (int i = 0; i < 6; ++i) Pm[i] = lb[i] - ml[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) qm[i] = lb[6 + i] - ml[6 + i];
    R Pm_copy[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) Pm_copy[i] = Pm[i];
    R lam_k[21], eta_k[6], ratio_m;
    bool ok_m = message<R, 6, 3>(Pm, qm, L.Jl, L.Jk, L.y, L.W, lam_k, eta_k, ratio_m);

    // ---- message to the landmark: marginalise the keyframe (6x6) ----
    R Pk[21], qk[6];
#pragma unroll
    for (int i = 0; i < 21; ++i) Pk[i] = kb[i] - mk[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) qk[i] = kb[21 + i] - mk[21 + i];
    R Pk_copy[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) Pk_copy[i] = Pk[i];
    R lam_m[6], eta_m[3], ratio_k;
    bool ok_k = message<R, 3, 6>(Pk, qk, L.Jk, L.Jl, L.y, L.W, lam_m, eta_m, ratio_k);

    if (sizeof(R) == 4 && P.fallback) {
        if (!ok_k || ratio_k < R(P.pivot_ratio)) {
            ok_k = message_fp64<R, 3, 6>(Pk_copy, qk, L.Jk, L.Jl, L.y, L.W, lam_m, eta_m);
            atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
        }
        if (!ok_m) {
            ok_m = message_fp64<R, 6, 3>(Pm_copy, qm, L.Jl, L.Jk, L.y, L.W, lam_k, eta_k);
            atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
        }
    }
    if (!ok_k || !ok_m) raise_error(g.ctl, n_f > 0 ? -1 - f : -1);

    // damping of eta (Sec. 5); undamped in the iteration of a (re)linearisation
    // and for the next damp_hold - 1 iterations (Sec. 8)
    if (t - tl >= P.damp_hold) {
        const R d = R(P.damping);
#pragma unroll
        for (int i = 0; i < 6; ++i) eta_k[i] = (R(1) - d) * eta_k[i] + d * mk[21 + i];
#pragma unroll
        for (int i = 0; i < 3; ++i) eta_m[i] = (R(1) - d) * eta_m[i] + d * ml[6 + i];
    }

    R out[KREC];
#pragma unroll
    for (int i = 0; i < 21; ++i) out[i] = lam_k[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) out[21 + i] = eta_k[i];
    out[27] = R(0);
    store_rec<R, KREC>(g.mk_out + (size_t)f * KREC, out);
#pragma unroll
    for (int i = 0; i < 6; ++i) g.ml_out[(size_t)i * n_f + f] = lam_m[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) g.ml_out[(size_t)(6 + i) * n_f + f] = eta_m[i];
}

// ------------------------------------------------------------------------
// belief kernel: blocks [0, n_kf) one keyframe each; then one thread per
// landmark.  Forms b^{t+1} = prior(t+1) + sum of messages and its mean.

// Sec. 8: prior scale at iteration t (geometric anneal to prior_final).
__device__ __forceinline__ double prior_scale(const KParams& P, int t) {
    if (P.prior_anneal <= 0) return P.prior_final;
    int tt = t < P.prior_anneal ? t : P.prior_anneal;
    return pow(P.prior_final, double(tt) / double(P.prior_anneal));
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

template <typename R, int n>
__device__ __noinline__ bool solve_mean_fp64(const R* lam, const R* eta, R* mu) {
    double A[n * (n + 1) / 2], e[n], m[n], ratio;
    for (int i = 0; i < n * (n + 1) / 2; ++i) A[i] = double(lam[i]);
    for (int i = 0; i < n; ++i) e[i] = double(eta[i]);
    bool ok = solve_mean<double, n>(A, e, m, ratio);
    for (int i = 0; i < n; ++i) mu[i] = R(m[i]);
    return ok;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename R>
__global__ void __launch_bounds__(BELIEF_BLOCK) belief_kernel(DevGraph<R> g, KParams P) {
    __shared__ R red[27][BELIEF_BLOCK];
    __shared__ float wmax[BELIEF_BLOCK / 32];
    __shared__ int is_last;
    const int tid = threadIdx.x;
    const int t1 = g.ctl[CTL_ITER] + 1;
    const R s = R(prior_scale(P, t1));
    const R isig2 = R(P.inv_sigma2);
    float dmu = 0.0f;

    if ((int)blockIdx.x < g.n_kf) {
        const int k = blockIdx.x;
        R acc[27];
#pragma unroll
        for (int j = 0; j < 27; ++j) acc[j] = R(0);
        const int b0 = g.kf_off[k], b1 = g.kf_off[k + 1];
        for (int i = b0 + tid; i < b1; i += BELIEF_BLOCK) {
            R rec[KREC];
            load_rec<R, KREC>(g.mk + (size_t)g.kf_list[i] * KREC, rec);
#pragma unroll
            for (int j = 0; j < 27; ++j) acc[j] += rec[j];
        }
#pragma unroll
        for (int j = 0; j < 27; ++j) red[j][tid] = acc[j];
        __syncthreads();
        for (int st = BELIEF_BLOCK / 2; st > 0; st >>= 1) {
            if (tid < st) {
#pragma unroll
                for (int j = 0; j < 27; ++j) red[j][tid] += red[j][tid + st];
            }
            __syncthreads();
        }
        if (tid == 0) {
            R lam[21], eta[6], mu[6], ratio;
#pragma unroll
            for (int j = 0; j < 21; ++j) lam[j] = red[j][0];
#pragma unroll
            for (int j = 0; j < 6; ++j) eta[j] = red[21 + j][0];
#pragma unroll
            for (int i = 0; i < 6; ++i)
                lam[pk(i, i)] += (s * g.kf_D[k * 6 + i] + R(P.anchor_scale) * g.kf_A[k * 6 + i]) * isig2;
            R work[21];
#pragma unroll
            for (int j = 0; j < 21; ++j) work[j] = lam[j];
            bool ok = solve_mean<R, 6>(work, eta, mu, ratio);
            if (sizeof(R) == 4 && P.fallback && (!ok || ratio < R(P.pivot_ratio))) {
                ok = solve_mean_fp64<R, 6>(lam, eta, mu);
                atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
            }
            R* rec = g.kf_bel + (size_t)k * KBEL;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if (!isfinite(mu[i])) ok = false;
                dmu = fmaxf(dmu, float(fabs(mu[i] - rec[27 + i])));
            }
            if (!ok) raise_error(g.ctl, k);
            R out[KBEL];
#pragma unroll
            for (int j = 0; j < 21; ++j) out[j] = lam[j];
#pragma unroll
            for (int j = 0; j < 6; ++j) { out[21 + j] = eta[j]; out[27 + j] = mu[j]; }
            out[33] = out[34] = out[35] = R(0);
            store_rec<R, KBEL>(rec, out);
        }
    } else {
        const int m = (blockIdx.x - g.n_kf) * BELIEF_BLOCK + tid;
        if (m < g.n_lm) {
            R acc[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) acc[j] = R(0);
            const int b0 = g.lm_off[m], b1 = g.lm_off[m + 1];
            for (int f = b0; f < b1; ++f) {
#pragma unroll
                for (int j = 0; j < 9; ++j) acc[j] += g.ml[(size_t)j * g.n_f + f];
            }
            R lam[6], eta[3], mu[3], ratio;
#pragma unroll
            for (int j = 0; j < 6; ++j) lam[j] = acc[j];
#pragma unroll
            for (int j = 0; j < 3; ++j) eta[j] = acc[6 + j];
#pragma unroll
            for (int i = 0; i < 3; ++i) lam[pk(i, i)] += s * g.lm_D[m * 3 + i] * isig2;
            R work[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) work[j] = lam[j];
            bool ok = solve_mean<R, 3>(work, eta, mu, ratio);
            if (sizeof(R) == 4 && P.fallback && !ok) {
                ok = solve_mean_fp64<R, 3>(lam, eta, mu);
                atomicAdd(&g.ctl[CTL_FALLBACKS], 1);
            }
            R* rec = g.lm_bel + (size_t)m * LBEL;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (!isfinite(mu[i])) ok = false;
                dmu = fmaxf(dmu, float(fabs(mu[i] - rec[9 + i])));
            }
            if (!ok) raise_error(g.ctl, g.n_kf + m);
            R out[LBEL];
#pragma unroll
            for (int j = 0; j < 6; ++j) out[j] = lam[j];
#pragma unroll
            for (int j = 0; j < 3; ++j) { out[6 + j] = eta[j]; out[9 + j] = mu[j]; }
            store_rec<R, LBEL>(rec, out);
        }
    }

    // max |dmu| over the grid: max is order independent, so an atomic on
    // the (non-negative) float bits stays deterministic
    dmu = warp_max(dmu);
    if ((tid & 31) == 0) wmax[tid >> 5] = dmu;
    __syncthreads();
    if (tid == 0) {
        float v = 0.0f;
        for (int i = 0; i < BELIEF_BLOCK / 32; ++i) v = fmaxf(v, wmax[i]);
        if (!(v >= 0.0f)) v = INFINITY;
        atomicMax(reinterpret_cast<unsigned int*>(&g.ctl[CTL_DMU_ACC]), __float_as_uint(v));
        __threadfence();
        int ticket = atomicAdd(&g.ctl[CTL_DONE], 1);
        is_last = (ticket == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (is_last && tid == 0) {
        // the last block to finish closes the iteration
        __threadfence();
        int acc = atomicExch(&g.ctl[CTL_DMU_ACC], 0);
        g.ctl[CTL_DMU_LAST] = acc;
        g.ctl[CTL_DONE] = 0;
        g.ctl[CTL_ITER] = t1;
    }
}

// ------------------------------------------------------------------------
// prior generation (Sec. 4 / Sec. 8): per-variable mean over its factors of
// diag(J_v^T J_v) at the reference point with Huber weight 1 and sigma = 1.

template <typename R>
__global__ void __launch_bounds__(FACTOR_BLOCK) prior_factor_kernel(DevGraph<R> g, KParams P, R* tmp_k, R* tmp_l) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= g.n_f) return;
    const int k = g.fk[f], m = g.fm[f];
    KParams Q = P;
    Q.huber_n = 0.0;
    Q.inv_sigma2 = 1.0;
    Q.inv_sigma = 1.0;
    R x0[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x0[i] = R(0);
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
__global__ void __launch_bounds__(METRIC_BLOCK) metrics_kernel(DevGraph<R> g, KParams P, double* partials) {
    __shared__ double red[4][METRIC_BLOCK];
    const int tid = threadIdx.x;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int f = blockIdx.x * METRIC_BLOCK + tid; f < g.n_f; f += gridDim.x * METRIC_BLOCK) {
        const int k = g.fk[f], m = g.fm[f];
        const R* kb = g.kf_bel + (size_t)k * KBEL;
        const R* lb = g.lm_bel + (size_t)m * LBEL;
        R x[9] = {kb[27], kb[28], kb[29], kb[30], kb[31], kb[32], lb[9], lb[10], lb[11]};
        KParams Q = P;
        Q.huber_n = 0.0;
        Lin<R> L;
        linearise<R>(Q, g.kf_R + (size_t)k * 9, g.kf_c + (size_t)k * 3, g.lm_ref + (size_t)m * 3, x,
                     g.z[2 * (size_t)f], g.z[2 * (size_t)f + 1], L);
        if (L.W > R(0)) {
            double e = sqrt(double(L.r2));
            v[0] += e;
            v[2] += 1.0;
            if (P.huber_n > 0.0 && e * P.inv_sigma > P.huber_n) v[3] += 1.0;
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
__global__ void __launch_bounds__(METRIC_BLOCK) metrics_ref_kernel(DevGraph<R> g, KParams P, double* partials) {
    __shared__ double red[2][METRIC_BLOCK];
    const int tid = threadIdx.x;
    double acc = 0.0, cnt = 0.0;
    for (int f = blockIdx.x * METRIC_BLOCK + tid; f < g.n_f; f += gridDim.x * METRIC_BLOCK) {
        const int k = g.fk[f], m = g.fm[f];
        const R* kb = g.kf_bel + (size_t)k * KBEL;
        const R* lb = g.lm_bel + (size_t)m * LBEL;
        R x[9] = {kb[27], kb[28], kb[29], kb[30], kb[31], kb[32], lb[9], lb[10], lb[11]};
        KParams Q = P;
        Q.huber_n = 0.0;
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

template <typename R>
cudaError_t launch_factor(const DevGraph<R>& g, const KParams& p, cudaStream_t s) {
    if (g.n_f == 0) return cudaSuccess;
    factor_kernel<R><<<(g.n_f + FACTOR_BLOCK - 1) / FACTOR_BLOCK, FACTOR_BLOCK, 0, s>>>(g, p);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_belief(const DevGraph<R>& g, const KParams& p, cudaStream_t s) {
    int blocks = g.n_kf + (g.n_lm + BELIEF_BLOCK - 1) / BELIEF_BLOCK;
    if (blocks < 1) blocks = 1;
    belief_kernel<R><<<blocks, BELIEF_BLOCK, 0, s>>>(g, p);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prior(const DevGraph<R>& g, const KParams& p, R* tmp_k, R* tmp_l, R* kf_D, R* lm_D,
                         cudaStream_t s) {
    if (g.n_f > 0) prior_factor_kernel<R><<<(g.n_f + FACTOR_BLOCK - 1) / FACTOR_BLOCK, FACTOR_BLOCK, 0, s>>>(g, p, tmp_k, tmp_l);
    int nv = g.n_kf + g.n_lm;
    if (nv > 0) prior_reduce_kernel<R><<<(nv + 127) / 128, 128, 0, s>>>(g, tmp_k, tmp_l, kf_D, lm_D);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_metrics(const DevGraph<R>& g, const KParams& p, double* partials, int nb, double* out,
                           cudaStream_t s) {
    metrics_kernel<R><<<nb, METRIC_BLOCK, 0, s>>>(g, p, partials);
    if (g.uv_ref) metrics_ref_kernel<R><<<nb, METRIC_BLOCK, 0, s>>>(g, p, partials);
    metrics_finish_kernel<<<1, 32, 0, s>>>(partials, nb, g.uv_ref != nullptr, out);
    return cudaGetLastError();
}

#define GBP_INSTANTIATE(R)                                                                              \
    template cudaError_t launch_factor<R>(const DevGraph<R>&, const KParams&, cudaStream_t);            \
    template cudaError_t launch_belief<R>(const DevGraph<R>&, const KParams&, cudaStream_t);            \
    template cudaError_t launch_prior<R>(const DevGraph<R>&, const KParams&, R*, R*, R*, R*, cudaStream_t); \
    template cudaError_t launch_metrics<R>(const DevGraph<R>&, const KParams&, double*, int, double*, cudaStream_t);

GBP_INSTANTIATE(float)
GBP_INSTANTIATE(double)

}  // namespace gbp
