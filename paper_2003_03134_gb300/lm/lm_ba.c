/*
 * lm_ba.c -- Levenberg-Marquardt bundle adjustment with a dense Schur
 * complement, plain single-threaded C (a CPU comparison baseline; the
 * paper compares GBP against an LM solver with dense Schur elimination and
 * Cholesky, Sec. 9.1).
 *
 * Objective (the energy of GBP's factors, Sec. 4 / Sec. 6 / Sec. 8; with the quadratic
 * loss its minimiser is GBP's fixed point):
 *   E(x) = sum_f rho(|r_f| / sigma) + 1/2 sum_v x_v^T P_v x_v
 *   r_f  = z_f - pi(R_k (l_m - c_k)),  R_k = Exp(w_k) Rref_k,  c_k = cref_k + dc_k,
 *          l_m = lref_m + dl_m      (the chart of every variable: its initial value)
 *   rho  = M^2 / 2 for M <= N, N M - N^2 / 2 beyond (Huber, Sec. 6; N <= 0: quadratic)
 *   P_v  = prior_scale * D_v (+ anchor_scale * D_v on anchored keyframes), D_v the
 *          mean over the variable's factors of diag(J_v^T J_v) / sigma^2 at the
 *          initial point (Sec. 4's priors, at their final strength, Sec. 8)
 * Each LM step linearises every factor, weights it by the Huber IRLS weight
 * rho'(M) / M, forms the normal equations (H + lambda diag(H)) dx = g,
 * eliminates the landmarks (3x3 blocks) into the reduced keyframe system,
 * solves that by dense Cholesky, substitutes back, and keeps the step if E
 * decreased (lambda / 10), else retries with lambda * 10.
 */
#include "lm_ba.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static void* zalloc(size_t n) { return calloc(n ? n : 1, 1); }

static void mat3mul(const double* A, const double* B, double* C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

/* Rodrigues: Exp(w) = I + (sin t / t) [w]x + ((1 - cos t) / t^2) [w]x^2, and the
 * left Jacobian Jl(w) = I + ((1 - cos t) / t^2) [w]x + ((t - sin t) / t^3) [w]x^2 */
static void exp_and_jl(const double w[3], double E[9], double Jl[9])
{
    double t2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], a, b, c;
    if (t2 < 1e-10) {
        a = 1.0 - t2 / 6.0;
        b = 0.5 - t2 / 24.0;
        c = 1.0 / 6.0 - t2 / 120.0;
    } else {
        double t = sqrt(t2);
        a = sin(t) / t;
        b = (1.0 - cos(t)) / t2;
        c = (t - sin(t)) / (t2 * t);
    }
    double W[9] = { 0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0 }, W2[9];
    mat3mul(W, W, W2);
    for (int i = 0; i < 9; ++i) {
        E[i] = a * W[i] + b * W2[i];
        Jl[i] = b * W[i] + c * W2[i];
    }
    for (int i = 0; i < 3; ++i) { E[4 * i] += 1.0; Jl[4 * i] += 1.0; }
}

/* Residual and Jacobian of factor f at the state; J[2][9] = d h / d [dc dw dl]
 * (h the projection), returns 0 if the point is closer than z_min. */
static int factor_lin(const lm_problem* P, const double* xk, const double* xl, int f, double r[2], double J[18])
{
    const int k = P->obs_kf[f], m = P->obs_lm[f];
    double E[9], Jl[9], R[9], d[3], p[3];
    exp_and_jl(xk + 6 * k + 3, E, Jl);
    mat3mul(E, P->Rref + 9 * k, R);
    for (int i = 0; i < 3; ++i) d[i] = P->lref[3 * m + i] + xl[3 * m + i] - P->cref[3 * k + i] - xk[6 * k + i];
    for (int i = 0; i < 3; ++i) p[i] = R[3 * i] * d[0] + R[3 * i + 1] * d[1] + R[3 * i + 2] * d[2];
    if (!(p[2] >= P->z_min)) return 0;
    const double iz = 1.0 / p[2];
    const double u = P->fx * p[0] * iz, v = P->fy * p[1] * iz;
    r[0] = P->obs_uv[2 * f] - (u + P->cx);
    r[1] = P->obs_uv[2 * f + 1] - (v + P->cy);
    /* dpi/dp */
    const double D[2][3] = { { P->fx * iz, 0.0, -u * iz }, { 0.0, P->fy * iz, -v * iz } };
    /* dp/ddl = R, dp/ddc = -R, dp/ddw = -[p]x Jl */
    double Px[9] = { 0.0, -p[2], p[1], p[2], 0.0, -p[0], -p[1], p[0], 0.0 }, PJ[9];
    mat3mul(Px, Jl, PJ);
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double sl = 0.0, sw = 0.0;
            for (int i = 0; i < 3; ++i) {
                sl += D[a][i] * R[3 * i + j];
                sw -= D[a][i] * PJ[3 * i + j];
            }
            J[9 * a + j] = -sl;      /* d/ddc */
            J[9 * a + 3 + j] = sw;   /* d/ddw */
            J[9 * a + 6 + j] = sl;   /* d/ddl */
        }
    return 1;
}

/* Huber: cost rho(M) and IRLS weight rho'(M) / M. */
static double huber_rho(double M, double N) { return (N <= 0.0 || M <= N) ? 0.5 * M * M : N * M - 0.5 * N * N; }
static double huber_w(double M, double N) { return (N <= 0.0 || M <= N) ? 1.0 : N / M; }

static double objective(const lm_problem* P, const double* xk, const double* xl, const double* pk, const double* pl)
{
    double e = 0.0, r[2], J[18];
    for (int f = 0; f < P->n_obs; ++f)
        if (factor_lin(P, xk, xl, f, r, J)) e += huber_rho(sqrt(r[0] * r[0] + r[1] * r[1]) / P->sigma, P->huber_n);
    for (int i = 0; i < 6 * P->n_kf; ++i) e += 0.5 * pk[i] * xk[i] * xk[i];
    for (int i = 0; i < 3 * P->n_lm; ++i) e += 0.5 * pl[i] * xl[i] * xl[i];
    return e;
}

/* Cholesky of a dense symmetric n x n matrix in place (lower), 0 or -1. */
static int chol(int n, double* A)
{
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int p = 0; p < j; ++p) s -= A[(size_t)j * n + p] * A[(size_t)j * n + p];
        if (!(s > 0.0)) return -1;
        s = sqrt(s);
        A[(size_t)j * n + j] = s;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int p = 0; p < j; ++p) t -= A[(size_t)i * n + p] * A[(size_t)j * n + p];
            A[(size_t)i * n + j] = t / s;
        }
    }
    return 0;
}

static void chol_solve(int n, const double* L, double* b)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[(size_t)i * n + p] * b[p];
        b[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int p = i + 1; p < n; ++p) s -= L[(size_t)p * n + i] * b[p];
        b[i] = s / L[(size_t)i * n + i];
    }
}

static int inv3(const double* A, double* B)
{
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (!(det > 0.0)) return -1;
    double id = 1.0 / det;
    B[0] = c00 * id; B[1] = (A[2] * A[7] - A[1] * A[8]) * id; B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id; B[4] = (A[0] * A[8] - A[2] * A[6]) * id; B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id; B[7] = (A[1] * A[6] - A[0] * A[7]) * id; B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
    return 0;
}

/* Prior precisions (diagonal) from the Jacobians at the initial point. */
static void make_priors(const lm_problem* P, const double* xk, const double* xl, double* pk, double* pl)
{
    double* Dk = zalloc(sizeof(double) * 6 * P->n_kf);
    double* Dl = zalloc(sizeof(double) * 3 * P->n_lm);
    int* nk = zalloc(sizeof(int) * P->n_kf);
    int* nl = zalloc(sizeof(int) * P->n_lm);
    double r[2], J[18];
    const double is2 = 1.0 / (P->sigma * P->sigma);
    for (int f = 0; f < P->n_obs; ++f) {
        const int k = P->obs_kf[f], m = P->obs_lm[f];
        nk[k]++;
        nl[m]++;
        if (!factor_lin(P, xk, xl, f, r, J)) continue;
        for (int j = 0; j < 6; ++j) Dk[6 * k + j] += is2 * (J[j] * J[j] + J[9 + j] * J[9 + j]);
        for (int j = 0; j < 3; ++j) Dl[3 * m + j] += is2 * (J[6 + j] * J[6 + j] + J[15 + j] * J[15 + j]);
    }
    for (int v = 0; v < P->n_kf; ++v) {
        double mx = 0.0;
        for (int j = 0; j < 6; ++j) {
            if (nk[v]) Dk[6 * v + j] /= nk[v];
            if (Dk[6 * v + j] > mx) mx = Dk[6 * v + j];
        }
        for (int j = 0; j < 6; ++j) {
            double d = mx <= 0.0 ? 1.0 : (Dk[6 * v + j] < 1e-9 * mx ? 1e-9 * mx : Dk[6 * v + j]);
            pk[6 * v + j] = P->prior_scale * d;
        }
    }
    for (int a = 0; a < P->n_anchor; ++a) {
        const int v = P->anchor_kf[a];
        for (int j = 0; j < 6; ++j) pk[6 * v + j] += P->anchor_scale * (pk[6 * v + j] / P->prior_scale);
    }
    for (int v = 0; v < P->n_lm; ++v) {
        double mx = 0.0;
        for (int j = 0; j < 3; ++j) {
            if (nl[v]) Dl[3 * v + j] /= nl[v];
            if (Dl[3 * v + j] > mx) mx = Dl[3 * v + j];
        }
        for (int j = 0; j < 3; ++j) {
            double d = mx <= 0.0 ? 1.0 : (Dl[3 * v + j] < 1e-9 * mx ? 1e-9 * mx : Dl[3 * v + j]);
            pl[3 * v + j] = P->prior_scale * d;
        }
    }
    free(Dk); free(Dl); free(nk); free(nl);
}

static void lm_world(const lm_problem* P, const double* xk, const double* xl, double* kf_Rt, double* lm_xyz);

struct lm_ctx {
    lm_problem P;              /* with its own copies of the arrays */
    double *xk, *xl, *pk, *pl; /* state (chart) and prior precisions */
    double *Jf, *rf, *wf, *Hll, *Hll_inv, *gl, *Hkl, *S, *H0, *gk, *b, *dl, *xk2, *xl2;
    int *off, *fac;            /* landmark -> factors */
    double lambda, E;
    int converged;
};

static void* dup(const void* src, size_t n)
{
    void* d = zalloc(n);
    if (src && n) memcpy(d, src, n);
    return d;
}

lm_ctx* lm_create(const lm_problem* src)
{
    lm_ctx* c = zalloc(sizeof(lm_ctx));
    lm_problem* P = &c->P;
    *P = *src;
    const int NK = P->n_kf, NL = P->n_lm, NF = P->n_obs, nk6 = 6 * NK;
    P->Rref = dup(src->Rref, sizeof(double) * 9 * NK);
    P->cref = dup(src->cref, sizeof(double) * 3 * NK);
    P->lref = dup(src->lref, sizeof(double) * 3 * NL);
    P->obs_kf = dup(src->obs_kf, sizeof(int) * NF);
    P->obs_lm = dup(src->obs_lm, sizeof(int) * NF);
    P->obs_uv = dup(src->obs_uv, sizeof(double) * 2 * NF);
    P->anchor_kf = dup(src->anchor_kf, sizeof(int) * P->n_anchor);
    c->xk = zalloc(sizeof(double) * nk6);
    c->xl = zalloc(sizeof(double) * 3 * NL);
    c->pk = zalloc(sizeof(double) * nk6);
    c->pl = zalloc(sizeof(double) * 3 * NL);
    make_priors(P, c->xk, c->xl, c->pk, c->pl);
    c->Jf = zalloc(sizeof(double) * 18 * NF);
    c->rf = zalloc(sizeof(double) * 2 * NF);
    c->wf = zalloc(sizeof(double) * NF);
    c->Hll = zalloc(sizeof(double) * 9 * NL);
    c->Hll_inv = zalloc(sizeof(double) * 9 * NL);
    c->gl = zalloc(sizeof(double) * 3 * NL);
    c->Hkl = zalloc(sizeof(double) * 18 * NF);
    c->S = zalloc(sizeof(double) * (size_t)nk6 * nk6);
    c->H0 = zalloc(sizeof(double) * (size_t)nk6 * nk6);
    c->gk = zalloc(sizeof(double) * nk6);
    c->b = zalloc(sizeof(double) * nk6);
    c->dl = zalloc(sizeof(double) * 3 * NL);
    c->xk2 = zalloc(sizeof(double) * nk6);
    c->xl2 = zalloc(sizeof(double) * 3 * NL);
    c->off = zalloc(sizeof(int) * (NL + 1));
    c->fac = zalloc(sizeof(int) * NF);
    for (int f = 0; f < NF; ++f) c->off[P->obs_lm[f] + 1]++;
    for (int v = 0; v < NL; ++v) c->off[v + 1] += c->off[v];
    int* fill = zalloc(sizeof(int) * (NL + 1));
    memcpy(fill, c->off, sizeof(int) * NL);
    for (int f = 0; f < NF; ++f) c->fac[fill[P->obs_lm[f]]++] = f;
    free(fill);
    c->lambda = 1e-4;
    c->E = objective(P, c->xk, c->xl, c->pk, c->pl);
    return c;
}

void lm_destroy(lm_ctx* c)
{
    if (!c) return;
    void* ptrs[] = { (void*)c->P.Rref, (void*)c->P.cref, (void*)c->P.lref, (void*)c->P.obs_kf, (void*)c->P.obs_lm,
                     (void*)c->P.obs_uv, (void*)c->P.anchor_kf, c->xk, c->xl, c->pk, c->pl, c->Jf, c->rf, c->wf,
                     c->Hll, c->Hll_inv, c->gl, c->Hkl, c->S, c->H0, c->gk, c->b, c->dl, c->xk2, c->xl2, c->off,
                     c->fac };
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(c);
}

double lm_cost(const lm_ctx* c) { return c->E; }
int lm_converged(const lm_ctx* c) { return c->converged; }

int lm_iterate(lm_ctx* c, int n, double tol)
{
    const lm_problem* P = &c->P;
    const int NK = P->n_kf, NL = P->n_lm, nk6 = 6 * NK;
    const double is2 = 1.0 / (P->sigma * P->sigma);
    double *xk = c->xk, *xl = c->xl, *pk = c->pk, *pl = c->pl, *H0 = c->H0, *gk = c->gk, *Hll = c->Hll,
           *gl = c->gl, *Hkl = c->Hkl, *S = c->S, *b = c->b, *dl = c->dl, *Hll_inv = c->Hll_inv;
    const int *off = c->off, *fac = c->fac;
    int it;
    for (it = 0; it < n && !c->converged; ++it) {
        /* linearise and weight every factor */
        memset(H0, 0, sizeof(double) * (size_t)nk6 * nk6);
        memset(gk, 0, sizeof(double) * nk6);
        memset(Hll, 0, sizeof(double) * 9 * NL);
        memset(gl, 0, sizeof(double) * 3 * NL);
        for (int f = 0; f < P->n_obs; ++f) {
            double* J = c->Jf + 18 * f;
            double* r = c->rf + 2 * f;
            if (!factor_lin(P, xk, xl, f, r, J)) {
                c->wf[f] = 0.0;
                memset(Hkl + 18 * f, 0, sizeof(double) * 18);
                continue;
            }
            const double w = is2 * huber_w(sqrt(r[0] * r[0] + r[1] * r[1]) / P->sigma, P->huber_n);
            c->wf[f] = w;
            const int k = P->obs_kf[f], m = P->obs_lm[f];
            for (int i = 0; i < 9; ++i) {
                const double gi = w * (J[i] * r[0] + J[9 + i] * r[1]);
                if (i < 6) gk[6 * k + i] += gi;
                else gl[3 * m + i - 6] += gi;
                for (int j = 0; j < 9; ++j) {
                    const double h = w * (J[i] * J[j] + J[9 + i] * J[9 + j]);
                    if (i < 6 && j < 6) H0[(size_t)(6 * k + i) * nk6 + 6 * k + j] += h;
                    else if (i >= 6 && j >= 6) Hll[9 * m + 3 * (i - 6) + (j - 6)] += h;
                    else if (i < 6 && j >= 6) Hkl[18 * f + 3 * i + (j - 6)] = h;
                }
            }
        }
        for (int i = 0; i < nk6; ++i) {
            H0[(size_t)i * nk6 + i] += pk[i];
            gk[i] -= pk[i] * xk[i];
        }
        for (int v = 0; v < NL; ++v)
            for (int i = 0; i < 3; ++i) {
                Hll[9 * v + 4 * i] += pl[3 * v + i];
                gl[3 * v + i] -= pl[3 * v + i] * xl[3 * v + i];
            }
        /* damped steps until one lowers E */
        int accepted = 0;
        for (int tries = 0; tries < 16 && !accepted; ++tries) {
            const double lambda = c->lambda;
            memcpy(S, H0, sizeof(double) * (size_t)nk6 * nk6);
            memcpy(b, gk, sizeof(double) * nk6);
            for (int i = 0; i < nk6; ++i) S[(size_t)i * nk6 + i] *= 1.0 + lambda;
            int bad = 0;
            /* eliminate every landmark: S -= Hkl Hll^-1 Hlk, b -= Hkl Hll^-1 gl */
            for (int v = 0; v < NL && !bad; ++v) {
                double A[9];
                memcpy(A, Hll + 9 * v, sizeof A);
                for (int i = 0; i < 3; ++i) A[4 * i] *= 1.0 + lambda;
                if (inv3(A, Hll_inv + 9 * v) != 0) { bad = 1; break; }
                const double* Ai = Hll_inv + 9 * v;
                double ag[3];
                for (int i = 0; i < 3; ++i) ag[i] = Ai[3 * i] * gl[3 * v] + Ai[3 * i + 1] * gl[3 * v + 1] + Ai[3 * i + 2] * gl[3 * v + 2];
                for (int a = off[v]; a < off[v + 1]; ++a) {
                    const int fa = fac[a], ka = P->obs_kf[fa];
                    const double* Ba = Hkl + 18 * fa;          /* 6x3 */
                    double BA[18];                             /* Ba Ai */
                    for (int i = 0; i < 6; ++i)
                        for (int j = 0; j < 3; ++j)
                            BA[3 * i + j] = Ba[3 * i] * Ai[j] + Ba[3 * i + 1] * Ai[3 + j] + Ba[3 * i + 2] * Ai[6 + j];
                    for (int i = 0; i < 6; ++i) b[6 * ka + i] -= Ba[3 * i] * ag[0] + Ba[3 * i + 1] * ag[1] + Ba[3 * i + 2] * ag[2];
                    for (int c2 = off[v]; c2 < off[v + 1]; ++c2) {
                        const int fb = fac[c2], kb = P->obs_kf[fb];
                        const double* Bb = Hkl + 18 * fb;
                        for (int i = 0; i < 6; ++i)
                            for (int j = 0; j < 6; ++j)
                                S[(size_t)(6 * ka + i) * nk6 + 6 * kb + j] -=
                                    BA[3 * i] * Bb[3 * j] + BA[3 * i + 1] * Bb[3 * j + 1] + BA[3 * i + 2] * Bb[3 * j + 2];
                    }
                }
            }
            if (!bad && chol(nk6, S) == 0) {
                chol_solve(nk6, S, b);                  /* keyframe step */
                for (int v = 0; v < NL; ++v) {          /* landmark step: Hll^-1 (gl - Hlk dk) */
                    double rhs[3] = { gl[3 * v], gl[3 * v + 1], gl[3 * v + 2] };
                    for (int a = off[v]; a < off[v + 1]; ++a) {
                        const int fa = fac[a], ka = P->obs_kf[fa];
                        const double* Ba = Hkl + 18 * fa;
                        for (int j = 0; j < 3; ++j)
                            for (int i = 0; i < 6; ++i) rhs[j] -= Ba[3 * i + j] * b[6 * ka + i];
                    }
                    const double* Ai = Hll_inv + 9 * v;
                    for (int i = 0; i < 3; ++i) dl[3 * v + i] = Ai[3 * i] * rhs[0] + Ai[3 * i + 1] * rhs[1] + Ai[3 * i + 2] * rhs[2];
                }
                for (int i = 0; i < nk6; ++i) c->xk2[i] = xk[i] + b[i];
                for (int i = 0; i < 3 * NL; ++i) c->xl2[i] = xl[i] + dl[i];
                const double E2 = objective(P, c->xk2, c->xl2, pk, pl);
                if (E2 < c->E) {
                    double step = 0.0;
                    for (int i = 0; i < nk6; ++i) step = fmax(step, fabs(b[i]));
                    for (int i = 0; i < 3 * NL; ++i) step = fmax(step, fabs(dl[i]));
                    memcpy(xk, c->xk2, sizeof(double) * nk6);
                    memcpy(xl, c->xl2, sizeof(double) * 3 * NL);
                    const double dE = c->E - E2;
                    c->E = E2;
                    c->lambda = fmax(lambda / 10.0, 1e-12);
                    accepted = 1;
                    if (step < tol || dE < 1e-15 * E2) c->converged = 1;
                    break;
                }
            }
            c->lambda = lambda * 10.0;
        }
        if (!accepted) c->converged = 1;   /* no step lowers E: a minimum to working precision */
    }
    return it;
}

void lm_state(const lm_ctx* c, double* kf_Rt, double* lm_xyz) { lm_world(&c->P, c->xk, c->xl, kf_Rt, lm_xyz); }

static void lm_world(const lm_problem* P, const double* xk, const double* xl, double* kf_Rt, double* lm_xyz)
{
    for (int k = 0; k < P->n_kf; ++k) {
        double E[9], Jl[9], R[9], c[3];
        exp_and_jl(xk + 6 * k + 3, E, Jl);
        mat3mul(E, P->Rref + 9 * k, R);
        for (int i = 0; i < 3; ++i) c[i] = P->cref[3 * k + i] + xk[6 * k + i];
        for (int i = 0; i < 9; ++i) kf_Rt[12 * k + i] = R[i];
        for (int i = 0; i < 3; ++i) kf_Rt[12 * k + 9 + i] = -(R[3 * i] * c[0] + R[3 * i + 1] * c[1] + R[3 * i + 2] * c[2]);
    }
    for (int m = 0; m < P->n_lm; ++m)
        for (int i = 0; i < 3; ++i) lm_xyz[3 * m + i] = P->lref[3 * m + i] + xl[3 * m + i];
}
