/*
 * gbp_oracle.c -- plain single-threaded FP64 GBP for bundle adjustment.
 *
 * TEST INFRASTRUCTURE ONLY (see gbp_oracle.h).  Written for clarity, not
 * speed: full 9x9 factor matrices, explicit Schur complements exactly as
 * printed in the message equations of Sec. 5, plain loops throughout.
 *
 * Paper references used below (Ortiz et al., "Bundle Adjustment on a Graph
 * Processor", CVPR 2020):
 *   Sec. 4   measurement model h = pi(R l + t), linearised factor in
 *            information form: eta = J^T S^-1 (J x0 + z - h(x0)),
 *            Lambda = J^T S^-1 J, J the 2x9 Jacobian.
 *   Sec. 4   priors generated from the Jacobians, 100x weaker than the
 *            measurements; Sec. 8 anneals them from measurement scale to
 *            1/100 over 10 iterations.
 *   Sec. 5   message equations (messageeta / messagelambda), belief
 *            equations (beliefeta / belieflambda), synchronous schedule,
 *            damping of the eta update only.
 *   Sec. 6   Huber rescale: weight 2 N/M - N^2/M^2 when M > N.
 */
#include "gbp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * dense symmetric positive definite solves (row-major n x n, n <= 9)
 * ---------------------------------------------------------------------- */

/* Cholesky factor A = L L^T.  Returns 0, or -1 if A is not positive definite. */
static int cholesky(int n, const double* A, double* L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int p = 0; p < j; ++p) s -= L[i * n + p] * L[j * n + p];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    return 0;
}

/* Solve L L^T x = b. */
static void cholesky_solve(int n, const double* L, const double* b, double* x)
{
    double y[9];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[i * n + p] * y[p];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int p = i + 1; p < n; ++p) s -= L[p * n + i] * x[p];
        x[i] = s / L[i * n + i];
    }
}

/* ------------------------------------------------------------------------
 * rotations
 * ---------------------------------------------------------------------- */

static void skew(const double v[3], double S[9])
{
    S[0] = 0.0;   S[1] = -v[2]; S[2] = v[1];
    S[3] = v[2];  S[4] = 0.0;   S[5] = -v[0];
    S[6] = -v[1]; S[7] = v[0];  S[8] = 0.0;
}

static void matmul3(const double* A, const double* B, double* C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int p = 0; p < 3; ++p) s += A[i * 3 + p] * B[p * 3 + j];
            C[i * 3 + j] = s;
        }
}

/* Rodrigues' formula: Exp(w) = I + a [w]x + b [w]x^2 with
 * a = sin(th)/th, b = (1 - cos(th))/th^2 (Taylor series for small th). */
void orc_so3_exp(const double w[3], double R[9])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-4) {
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    double W[9], W2[9];
    skew(w, W);
    matmul3(W, W, W2);
    for (int i = 0; i < 9; ++i) R[i] = a * W[i] + b * W2[i];
    R[0] += 1.0; R[4] += 1.0; R[8] += 1.0;
}

/* Left Jacobian of SO(3): Exp(w + e) = Exp(Jl(w) e) Exp(w) to first order,
 * Jl = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2. */
void orc_so3_left_jacobian(const double w[3], double J[9])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-4) {
        a = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        b = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        a = (1.0 - cos(th)) / th2;
        b = (th - sin(th)) / (th2 * th);
    }
    double W[9], W2[9];
    skew(w, W);
    matmul3(W, W, W2);
    for (int i = 0; i < 9; ++i) J[i] = a * W[i] + b * W2[i];
    J[0] += 1.0; J[4] += 1.0; J[8] += 1.0;
}

/* ------------------------------------------------------------------------
 * measurement factor (Sec. 4 and Sec. 6)
 * ---------------------------------------------------------------------- */

/* Sec. 6: cost M^2 becomes M^2 (2N/M - N^2/M^2) beyond the threshold, i.e.
 * the information of the factor is scaled by this weight. */
double orc_huber_weight(double M, double nsigma)
{
    if (nsigma <= 0.0 || M <= nsigma) return 1.0;
    return 2.0 * nsigma / M - (nsigma * nsigma) / (M * M);
}

/* Camera-frame point p = R_k (l_m - c_k) in the chart. */
static void camera_point(const double Rref[9], const double cref[3], const double lref[3],
                         const double xk[6], const double xl[3], double R[9], double p[3])
{
    double dR[9];
    orc_so3_exp(xk + 3, dR);
    matmul3(dR, Rref, R);
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = (lref[i] + xl[i]) - (cref[i] + xk[i]);
    for (int i = 0; i < 3; ++i) p[i] = R[i * 3 + 0] * d[0] + R[i * 3 + 1] * d[1] + R[i * 3 + 2] * d[2];
}

double orc_project(const orc_cam* cam, const double Rref[9], const double cref[3], const double lref[3],
                   const double xk[6], const double xl[3], double uv[2])
{
    double R[9], p[3];
    camera_point(Rref, cref, lref, xk, xl, R, p);
    uv[0] = cam->fx * p[0] / p[2] + cam->cx;
    uv[1] = cam->fy * p[1] / p[2] + cam->cy;
    return p[2];
}

int orc_linearise(const orc_cam* cam, const orc_params* prm, const double Rref[9], const double cref[3],
                  const double lref[3], const double xk[6], const double xl[3], const double z[2],
                  double J[18], double r[2], double* k, double A[81], double c[9])
{
    double R[9], p[3];
    camera_point(Rref, cref, lref, xk, xl, R, p);
    memset(J, 0, sizeof(double) * 18);
    memset(A, 0, sizeof(double) * 81);
    memset(c, 0, sizeof(double) * 9);
    r[0] = r[1] = 0.0;
    *k = 1.0;
    if (p[2] < prm->z_min) return 0;

    double h[2] = { cam->fx * p[0] / p[2] + cam->cx, cam->fy * p[1] / p[2] + cam->cy };
    r[0] = z[0] - h[0];
    r[1] = z[1] - h[1];

    /* d pi / d p */
    double Jp[6] = { cam->fx / p[2], 0.0, -cam->fx * p[0] / (p[2] * p[2]),
                     0.0, cam->fy / p[2], -cam->fy * p[1] / (p[2] * p[2]) };
    /* d p / d dc = -R,  d p / d dw = -[p]x Jl(dw),  d p / d dl = R */
    double S[9], Jl[9], SJ[9];
    skew(p, S);
    orc_so3_left_jacobian(xk + 3, Jl);
    matmul3(S, Jl, SJ);
    double dp[27]; /* 3 x 9 */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            dp[i * 9 + j] = -R[i * 3 + j];
            dp[i * 9 + 3 + j] = -SJ[i * 3 + j];
            dp[i * 9 + 6 + j] = R[i * 3 + j];
        }
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s += Jp[a * 3 + i] * dp[i * 9 + j];
            J[a * 9 + j] = s;
        }

    /* Sec. 6: Mahalanobis distance and Huber weight */
    double sigma = prm->sigma_px;
    double M = sqrt(r[0] * r[0] + r[1] * r[1]) / sigma;
    *k = orc_huber_weight(M, prm->huber_nsigma);
    double w = *k / (sigma * sigma);

    /* Sec. 4: Lambda = J^T W J,  eta = J^T W (J x0 + r) */
    double x0[9];
    for (int i = 0; i < 6; ++i) x0[i] = xk[i];
    for (int i = 0; i < 3; ++i) x0[6 + i] = xl[i];
    double y[2];
    for (int a = 0; a < 2; ++a) {
        double s = r[a];
        for (int j = 0; j < 9; ++j) s += J[a * 9 + j] * x0[j];
        y[a] = s;
    }
    for (int i = 0; i < 9; ++i) {
        for (int j = 0; j < 9; ++j) A[i * 9 + j] = w * (J[i] * J[j] + J[9 + i] * J[9 + j]);
        c[i] = w * (J[i] * y[0] + J[9 + i] * y[1]);
    }
    return 1;
}

/* Sec. 5, message equations: the message to variable block a takes the
 * product of the factor with the incoming message on block b and
 * marginalises b:
 *   eta_out = c_a - A_ab (A_bb + lam_in)^-1 (c_b + eta_in)
 *   lam_out = A_aa - A_ab (A_bb + lam_in)^-1 A_ba                          */
int orc_factor_message(const double A[81], const double c[9], int target,
                       const double* lam_in, const double* eta_in, double* lam_out, double* eta_out)
{
    int a0 = target == 0 ? 0 : 6, na = target == 0 ? 6 : 3;
    int b0 = target == 0 ? 6 : 0, nb = target == 0 ? 3 : 6;
    double S[36], L[36], e[6];
    for (int i = 0; i < nb; ++i) {
        for (int j = 0; j < nb; ++j) S[i * nb + j] = A[(b0 + i) * 9 + b0 + j] + lam_in[i * nb + j];
        e[i] = c[b0 + i] + eta_in[i];
    }
    if (cholesky(nb, S, L) != 0) return -1;
    /* X = S^-1 A_ba (nb x na), y = S^-1 e */
    double X[54], col[6], sol[6], y[6];
    for (int j = 0; j < na; ++j) {
        for (int i = 0; i < nb; ++i) col[i] = A[(b0 + i) * 9 + a0 + j];
        cholesky_solve(nb, L, col, sol);
        for (int i = 0; i < nb; ++i) X[i * na + j] = sol[i];
    }
    cholesky_solve(nb, L, e, y);
    for (int i = 0; i < na; ++i) {
        for (int j = 0; j < na; ++j) {
            double s = A[(a0 + i) * 9 + a0 + j];
            for (int p = 0; p < nb; ++p) s -= A[(a0 + i) * 9 + b0 + p] * X[p * na + j];
            lam_out[i * na + j] = s;
        }
        double s = c[a0 + i];
        for (int p = 0; p < nb; ++p) s -= A[(a0 + i) * 9 + b0 + p] * y[p];
        eta_out[i] = s;
    }
    return 0;
}

/* Sec. 8: priors start at the measurement scale and weaken geometrically to
 * prior_final_scale over prior_anneal_iters iterations. */
double orc_prior_scale(const orc_params* prm, int t)
{
    int T = prm->prior_anneal_iters;
    if (T <= 0) return prm->prior_final_scale;
    int tt = t < T ? t : T;
    return pow(prm->prior_final_scale, (double)tt / (double)T);
}

/* ------------------------------------------------------------------------
 * graph
 * ---------------------------------------------------------------------- */

struct orc_graph {
    orc_cam cam;
    orc_params prm;
    int n_kf, n_lm, n_f, t;
    double *Rref, *cref, *lref;          /* references (initial values)          */
    int *fk, *fm;
    double *z;
    unsigned char *anchored;
    int *kf_birth, *lm_birth;            /* iteration at which each variable was added */
    double *Dk, *Dl;                     /* prior diagonals                      */
    double *kf_lam, *kf_eta, *lm_lam, *lm_eta;   /* beliefs b^t              */
    double *kf_mu, *lm_mu;                       /* means of b^t             */
    double *mk_lam, *mk_eta, *ml_lam, *ml_eta;   /* messages m^t             */
    double *nk_lam, *nk_eta, *nl_lam, *nl_eta;   /* messages m^{t+1}         */
    double *linA, *linc;                 /* current linearisation of each factor */
    double *x0;                          /* its linearisation point [xk; xl]     */
    int *tlin;                           /* iteration at which it was taken      */
    long n_relin;                        /* relinearisations since creation      */
    long n_held;                         /* messages held at their previous value */
    double *lin_r2, *lin_k;              /* |r|^2 and Huber weight at the linearisation (0, 0 if inactive) */
    /* learned damping (no counterpart in the paper) */
    double *hist;                        /* per factor (ORC_HIST): relative message changes at t-1 and t-2,
                                            keyframe side [0..1], landmark side [2..3]; the landmark
                                            message eta of t-1 [4..6]; kept while features are computed */
    double *pk_eta;                      /* per factor: eta of the message to the keyframe at t-1        */
    double *net;                         /* damping network parameters (ORC_NET_NPARAM) or NULL         */
    double *eta_ref;                     /* per factor: reference eta (keyframe 6, landmark 3) or NULL   */
    /* the factors of every variable in increasing factor order (rebuilt
     * when the graph grows): each belief sums its messages in that order */
    int *kf_off, *kf_fac, *lm_off, *lm_fac;
    int csr_nf, csr_nk, csr_nl;
    /* a part of the graph (orc_set_part): the factors whose messages and the
     * variables whose beliefs this graph computes (NULL = all) */
    unsigned char *fac_mask, *var_mask;
};

static void* zalloc(size_t n) { return calloc(n ? n : 1, 1); }

static unsigned char* dup_bytes(const unsigned char* src, size_t n)
{
    unsigned char* d = zalloc(n);
    memcpy(d, src, n);
    return d;
}

enum { ORC_HIST = 8 };

static void build_csr(orc_graph* g)
{
    if (g->kf_off && g->csr_nf == g->n_f && g->csr_nk == g->n_kf && g->csr_nl == g->n_lm) return;
    free(g->kf_off); free(g->kf_fac); free(g->lm_off); free(g->lm_fac);
    g->kf_off = zalloc(sizeof(int) * (size_t)(g->n_kf + 1));
    g->lm_off = zalloc(sizeof(int) * (size_t)(g->n_lm + 1));
    g->kf_fac = zalloc(sizeof(int) * (size_t)g->n_f);
    g->lm_fac = zalloc(sizeof(int) * (size_t)g->n_f);
    for (int f = 0; f < g->n_f; ++f) { g->kf_off[g->fk[f] + 1]++; g->lm_off[g->fm[f] + 1]++; }
    for (int v = 0; v < g->n_kf; ++v) g->kf_off[v + 1] += g->kf_off[v];
    for (int v = 0; v < g->n_lm; ++v) g->lm_off[v + 1] += g->lm_off[v];
    int* fill = zalloc(sizeof(int) * (size_t)(g->n_kf > g->n_lm ? g->n_kf + 1 : g->n_lm + 1));
    for (int v = 0; v < g->n_kf; ++v) fill[v] = g->kf_off[v];
    for (int f = 0; f < g->n_f; ++f) g->kf_fac[fill[g->fk[f]]++] = f;
    for (int v = 0; v < g->n_lm; ++v) fill[v] = g->lm_off[v];
    for (int f = 0; f < g->n_f; ++f) g->lm_fac[fill[g->fm[f]]++] = f;
    free(fill);
    g->csr_nf = g->n_f;
    g->csr_nk = g->n_kf;
    g->csr_nl = g->n_lm;
}

/* Belief b^t of every variable: prior(t) + sum of the current messages
 * (Sec. 5, belief equations), the messages added in increasing factor
 * order; then its mean by a Cholesky solve.  Variables are independent (an
 * OpenMP build runs them in parallel with the same arithmetic). */
static int update_beliefs(orc_graph* g, double* max_dmu)
{
    build_csr(g);
    double dmu = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : dmu) reduction(| : bad)
    for (int v = 0; v < g->n_kf; ++v) {
        if (g->var_mask && !g->var_mask[v]) continue;
        double s = orc_prior_scale(&g->prm, g->t - g->kf_birth[v]);
        double* L = g->kf_lam + 36 * v;
        double* e = g->kf_eta + 6 * v;
        memset(L, 0, sizeof(double) * 36);
        memset(e, 0, sizeof(double) * 6);
        for (int i = 0; i < 6; ++i) {
            L[i * 6 + i] = s * g->Dk[6 * v + i];
            if (g->anchored[v]) L[i * 6 + i] += g->prm.anchor_scale * g->Dk[6 * v + i];
        }
        for (int j = g->kf_off[v]; j < g->kf_off[v + 1]; ++j) {
            int f = g->kf_fac[j];
            for (int i = 0; i < 36; ++i) L[i] += g->mk_lam[36 * f + i];
            for (int i = 0; i < 6; ++i) e[i] += g->mk_eta[6 * f + i];
        }
        double Lf[36], mu[6];
        if (cholesky(6, L, Lf) != 0) { bad = 1; continue; }
        cholesky_solve(6, Lf, e, mu);
        for (int i = 0; i < 6; ++i) {
            double d = fabs(mu[i] - g->kf_mu[6 * v + i]);
            if (d > dmu) dmu = d;
            g->kf_mu[6 * v + i] = mu[i];
        }
    }
#pragma omp parallel for schedule(static) reduction(max : dmu) reduction(| : bad)
    for (int v = 0; v < g->n_lm; ++v) {
        if (g->var_mask && !g->var_mask[g->n_kf + v]) continue;
        double s = orc_prior_scale(&g->prm, g->t - g->lm_birth[v]);
        double* L = g->lm_lam + 9 * v;
        double* e = g->lm_eta + 3 * v;
        memset(L, 0, sizeof(double) * 9);
        memset(e, 0, sizeof(double) * 3);
        for (int i = 0; i < 3; ++i) L[i * 3 + i] = s * g->Dl[3 * v + i];
        for (int j = g->lm_off[v]; j < g->lm_off[v + 1]; ++j) {
            int f = g->lm_fac[j];
            for (int i = 0; i < 9; ++i) L[i] += g->ml_lam[9 * f + i];
            for (int i = 0; i < 3; ++i) e[i] += g->ml_eta[3 * f + i];
        }
        double Lf[9], mu[3];
        if (cholesky(3, L, Lf) != 0) { bad = 1; continue; }
        cholesky_solve(3, Lf, e, mu);
        for (int i = 0; i < 3; ++i) {
            double d = fabs(mu[i] - g->lm_mu[3 * v + i]);
            if (d > dmu) dmu = d;
            g->lm_mu[3 * v + i] = mu[i];
        }
    }
    if (bad) return -1;
    if (max_dmu) *max_dmu = dmu;
    return 0;
}

orc_graph* orc_create(const orc_cam* cam, const orc_params* prm,
                      int n_kf, const double* kf_Rt, int n_lm, const double* lm_xyz,
                      int n_obs, const int* obs_kf, const int* obs_lm, const double* obs_uv,
                      int n_anchor, const int* anchor_kf)
{
    if (!cam || !prm || n_kf < 0 || n_lm < 0 || n_obs < 0 || n_anchor < 0) return NULL;
    for (int f = 0; f < n_obs; ++f)
        if (obs_kf[f] < 0 || obs_kf[f] >= n_kf || obs_lm[f] < 0 || obs_lm[f] >= n_lm) return NULL;
    for (int a = 0; a < n_anchor; ++a)
        if (anchor_kf[a] < 0 || anchor_kf[a] >= n_kf) return NULL;

    orc_graph* g = (orc_graph*)zalloc(sizeof(orc_graph));
    g->cam = *cam;
    g->prm = *prm;
    g->n_kf = n_kf; g->n_lm = n_lm; g->n_f = n_obs; g->t = 0;
    size_t F = (size_t)n_obs;
    g->Rref = zalloc(sizeof(double) * 9 * n_kf);
    g->cref = zalloc(sizeof(double) * 3 * n_kf);
    g->lref = zalloc(sizeof(double) * 3 * n_lm);
    g->fk = zalloc(sizeof(int) * F);
    g->fm = zalloc(sizeof(int) * F);
    g->z = zalloc(sizeof(double) * 2 * F);
    g->anchored = zalloc((size_t)n_kf);
    g->kf_birth = zalloc(sizeof(int) * (n_kf ? n_kf : 1));
    g->lm_birth = zalloc(sizeof(int) * (n_lm ? n_lm : 1));
    g->Dk = zalloc(sizeof(double) * 6 * n_kf);
    g->Dl = zalloc(sizeof(double) * 3 * n_lm);
    g->kf_lam = zalloc(sizeof(double) * 36 * n_kf);
    g->kf_eta = zalloc(sizeof(double) * 6 * n_kf);
    g->lm_lam = zalloc(sizeof(double) * 9 * n_lm);
    g->lm_eta = zalloc(sizeof(double) * 3 * n_lm);
    g->kf_mu = zalloc(sizeof(double) * 6 * n_kf);
    g->lm_mu = zalloc(sizeof(double) * 3 * n_lm);
    g->mk_lam = zalloc(sizeof(double) * 36 * F);
    g->mk_eta = zalloc(sizeof(double) * 6 * F);
    g->ml_lam = zalloc(sizeof(double) * 9 * F);
    g->ml_eta = zalloc(sizeof(double) * 3 * F);
    g->nk_lam = zalloc(sizeof(double) * 36 * F);
    g->nk_eta = zalloc(sizeof(double) * 6 * F);
    g->nl_lam = zalloc(sizeof(double) * 9 * F);
    g->nl_eta = zalloc(sizeof(double) * 3 * F);

    /* references: R, and camera centre c = -R^T t */
    for (int v = 0; v < n_kf; ++v) {
        const double* Rt = kf_Rt + 12 * v;
        for (int i = 0; i < 9; ++i) g->Rref[9 * v + i] = Rt[i];
        for (int i = 0; i < 3; ++i)
            g->cref[3 * v + i] = -(Rt[0 * 3 + i] * Rt[9] + Rt[1 * 3 + i] * Rt[10] + Rt[2 * 3 + i] * Rt[11]);
    }
    memcpy(g->lref, lm_xyz, sizeof(double) * 3 * n_lm);
    for (int f = 0; f < n_obs; ++f) {
        g->fk[f] = obs_kf[f];
        g->fm[f] = obs_lm[f];
        g->z[2 * f] = obs_uv[2 * f];
        g->z[2 * f + 1] = obs_uv[2 * f + 1];
    }
    for (int a = 0; a < n_anchor; ++a) g->anchored[anchor_kf[a]] = 1;

    /* Sec. 4 and Sec. 8: priors generated from the Jacobians at the initial
     * point, at "the same scale as the measurement constraints": a variable's
     * prior precision is the diagonal of the information one of its
     * measurement factors gives it (Huber weight 1), averaged over its
     * factors. */
    orc_params p1 = *prm;
    p1.huber_nsigma = 0.0;
    double zero6[6] = { 0 }, J[18], r[2], k, A[81], c[9];
    for (int f = 0; f < n_obs; ++f) {
        int kk = g->fk[f], m = g->fm[f];
        orc_linearise(cam, &p1, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m, zero6, zero6,
                      g->z + 2 * f, J, r, &k, A, c);
        for (int i = 0; i < 6; ++i) g->Dk[6 * kk + i] += A[i * 9 + i];
        for (int i = 0; i < 3; ++i) g->Dl[3 * m + i] += A[(6 + i) * 9 + 6 + i];
    }
    {
        int* deg_k = zalloc(sizeof(int) * (n_kf ? n_kf : 1));
        int* deg_l = zalloc(sizeof(int) * (n_lm ? n_lm : 1));
        for (int f = 0; f < n_obs; ++f) { deg_k[g->fk[f]]++; deg_l[g->fm[f]]++; }
        for (int v = 0; v < n_kf; ++v)
            if (deg_k[v]) for (int i = 0; i < 6; ++i) g->Dk[6 * v + i] /= deg_k[v];
        for (int v = 0; v < n_lm; ++v)
            if (deg_l[v]) for (int i = 0; i < 3; ++i) g->Dl[3 * v + i] /= deg_l[v];
        free(deg_k);
        free(deg_l);
    }
    /* floor: a zero diagonal entry would leave the prior singular */
    for (int v = 0; v < n_kf; ++v) {
        double mx = 0.0;
        for (int i = 0; i < 6; ++i) if (g->Dk[6 * v + i] > mx) mx = g->Dk[6 * v + i];
        for (int i = 0; i < 6; ++i) {
            if (mx <= 0.0) g->Dk[6 * v + i] = 1.0;
            else if (g->Dk[6 * v + i] < 1e-9 * mx) g->Dk[6 * v + i] = 1e-9 * mx;
        }
    }
    for (int v = 0; v < n_lm; ++v) {
        double mx = 0.0;
        for (int i = 0; i < 3; ++i) if (g->Dl[3 * v + i] > mx) mx = g->Dl[3 * v + i];
        for (int i = 0; i < 3; ++i) {
            if (mx <= 0.0) g->Dl[3 * v + i] = 1.0;
            else if (g->Dl[3 * v + i] < 1e-9 * mx) g->Dl[3 * v + i] = 1e-9 * mx;
        }
    }

    /* every factor is first linearised at the initial point (x0 = 0) */
    g->linA = zalloc(sizeof(double) * 81 * F);
    g->linc = zalloc(sizeof(double) * 9 * F);
    g->x0 = zalloc(sizeof(double) * 9 * F);
    g->tlin = zalloc(sizeof(int) * F);
    g->lin_r2 = zalloc(sizeof(double) * F);
    g->lin_k = zalloc(sizeof(double) * F);
    g->hist = zalloc(sizeof(double) * ORC_HIST * F);
    g->pk_eta = zalloc(sizeof(double) * 6 * F);
    for (int f = 0; f < n_obs; ++f) {
        int kk = g->fk[f], m = g->fm[f];
        int active = orc_linearise(cam, prm, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m, zero6, zero6,
                                   g->z + 2 * f, J, r, &k, g->linA + 81 * f, g->linc + 9 * f);
        g->lin_r2[f] = active ? r[0] * r[0] + r[1] * r[1] : 0.0;
        g->lin_k[f] = active ? k : 0.0;
    }
    /* b^0 = prior(0), messages zero */
    if (update_beliefs(g, NULL) != 0) {
        orc_destroy(g);
        return NULL;
    }
    return g;
}

void orc_destroy(orc_graph* g)
{
    if (!g) return;
    void* ptrs[] = { g->Rref, g->cref, g->lref, g->fk, g->fm, g->z, g->anchored, g->kf_birth, g->lm_birth,
                     g->Dk, g->Dl,
                     g->kf_lam, g->kf_eta, g->lm_lam, g->lm_eta, g->kf_mu, g->lm_mu,
                     g->mk_lam, g->mk_eta, g->ml_lam, g->ml_eta, g->nk_lam, g->nk_eta, g->nl_lam, g->nl_eta,
                     g->linA, g->linc, g->x0, g->tlin, g->lin_r2, g->lin_k, g->hist, g->pk_eta, g->net,
                     g->eta_ref, g->kf_off, g->kf_fac, g->lm_off, g->lm_fac, g->fac_mask, g->var_mask };
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); ++i) free(ptrs[i]);
    free(g);
}

/* ------------------------------------------------------------------------
 * learned damping (no counterpart in the paper: it replaces the fixed d of
 * Sec. 5 / Sec. 8 by a per-factor prediction)
 * ---------------------------------------------------------------------- */

double orc_net_forward(const double* P, const double x[ORC_NET_NFEAT])
{
    const double *W1 = P, *b1 = P + 1024, *W2 = P + 1088, *b2 = P + 5184, *W3 = P + 5248, b3 = P[5312];
    double h1[64], h2[64];
    for (int j = 0; j < 64; ++j) {
        double s = b1[j];
        for (int i = 0; i < ORC_NET_NFEAT; ++i) s += x[i] * W1[i * 64 + j];
        h1[j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < 64; ++j) {
        double s = b2[j];
        for (int i = 0; i < 64; ++i) s += h1[i] * W2[i * 64 + j];
        h2[j] = s > 0.0 ? s : 0.0;
    }
    double z = b3;
    for (int j = 0; j < 64; ++j) z += h2[j] * W3[j];
    return 0.9 / (1.0 + exp(-z));
}

static double norm_n(const double* a, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * a[i];
    return sqrt(s);
}

/* |new - old| / (|new| + |old|): 0 for an unchanged message, 1 for a new one */
static double rel_change(const double* nw, const double* old, int n)
{
    double d[6];
    for (int i = 0; i < n; ++i) d[i] = nw[i] - old[i];
    return norm_n(d, n) / (norm_n(nw, n) + norm_n(old, n) + 1e-30);
}

/* |(1 - d) new + d old - ref|^2 is a parabola in d; returns its vertex
 * <old - new, ref - new> / |old - new|^2.  *valid = 0 when old = new (up to
 * 1e-10 of their squared norms), where every d is equally good. */
static double damping_vertex(const double* nw, const double* old, const double* ref, int n, int* valid)
{
    double uu = 0.0, uv = 0.0, nn = 0.0;
    for (int i = 0; i < n; ++i) {
        double u = old[i] - nw[i];
        uu += u * u;
        uv += u * (ref[i] - nw[i]);
        nn += nw[i] * nw[i] + old[i] * old[i];
    }
    *valid = uu > 1e-10 * nn && uu > 0.0;
    return *valid ? uv / uu : 0.0;
}

/* cosine between the proposed step new - old and the previous step old - prev */
static double step_cosine(const double* nw, const double* old, const double* prev, int n)
{
    double a[6], b[6], ab = 0.0;
    for (int i = 0; i < n; ++i) {
        a[i] = nw[i] - old[i];
        b[i] = old[i] - prev[i];
        ab += a[i] * b[i];
    }
    return ab / (norm_n(a, n) * norm_n(b, n) + 1e-30);
}

static double trace_n(const double* A, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += A[i * n + i];
    return s;
}

/* The 16 features of factor f, from this iteration's undamped new messages
 * (nk_*, nl_*), the messages m^t (mk_*, ml_*) and m^{t-1} (pk_eta, stored
 * landmark eta), the beliefs b^t and the stored history; then the history
 * moves one step. */
static void factor_features(orc_graph* g, int f, const int* deg_k, const int* deg_l, double* x)
{
    int kk = g->fk[f], m = g->fm[f];
    double Pk[36], Pm[9];
    for (int i = 0; i < 36; ++i) Pk[i] = g->kf_lam[36 * kk + i] - g->mk_lam[36 * f + i];
    for (int i = 0; i < 9; ++i) Pm[i] = g->lm_lam[9 * m + i] - g->ml_lam[9 * f + i];
    double tlk = trace_n(g->nk_lam + 36 * f, 6), tlm = trace_n(g->nl_lam + 9 * f, 3);
    double M = sqrt(g->lin_r2[f]) / g->prm.sigma_px;
    double ck = rel_change(g->nk_eta + 6 * f, g->mk_eta + 6 * f, 6);
    double cm = rel_change(g->nl_eta + 3 * f, g->ml_eta + 3 * f, 3);
    double* h = g->hist + ORC_HIST * f;
    int dt_lin = g->t - g->tlin[f], dt_birth = g->t - g->lm_birth[m];
    x[0] = log1p(M) / 3.0;
    x[1] = g->lin_k[f];
    x[2] = tlk / (tlk + trace_n(Pk, 6) + 1e-30);
    x[3] = tlm / (tlm + trace_n(Pm, 3) + 1e-30);
    x[4] = ck;
    x[5] = h[0];
    x[6] = h[1];
    /* the keyframe-side step cosine compares the steps of the last two
     * iterations only when the three messages share one linearisation
     * (none in this iteration or the previous one); 0 otherwise */
    x[7] = dt_lin >= 2 ? step_cosine(g->nk_eta + 6 * f, g->mk_eta + 6 * f, g->pk_eta + 6 * f, 6) : 0.0;
    x[8] = cm;
    x[9] = h[2];
    x[10] = h[3];
    x[11] = step_cosine(g->nl_eta + 3 * f, g->ml_eta + 3 * f, h + 4, 3);
    x[12] = log1p((double)deg_k[kk]) / 5.0;
    x[13] = log1p((double)deg_l[m]) / 3.0;
    x[14] = (dt_lin < 50 ? dt_lin : 50) / 50.0;
    x[15] = (dt_birth < 50 ? dt_birth : 50) / 50.0;
    h[1] = h[0]; h[0] = ck;
    h[3] = h[2]; h[2] = cm;
    for (int i = 0; i < 3; ++i) h[4 + i] = g->ml_eta[3 * f + i];
}

int orc_set_damping_net(orc_graph* g, const double* params)
{
    free(g->net);
    g->net = NULL;
    if (!params) return 0;
    for (int i = 0; i < ORC_NET_NPARAM; ++i)
        if (!isfinite(params[i])) return -1;
    g->net = malloc(sizeof(double) * ORC_NET_NPARAM);
    memcpy(g->net, params, sizeof(double) * ORC_NET_NPARAM);
    return 0;
}

void orc_set_reference_messages(orc_graph* g, const double* eta_ref)
{
    free(g->eta_ref);
    g->eta_ref = NULL;
    if (!eta_ref) return;
    g->eta_ref = zalloc(sizeof(double) * 9 * (size_t)g->n_f);
    memcpy(g->eta_ref, eta_ref, sizeof(double) * 9 * (size_t)g->n_f);
}

/* mode 0: the fixed schedule; 1: learned d_f (needs a network); 2: fixed
 * schedule, recording features into X (n x n_f x 16) and damping targets
 * toward eta_ref into T (n x n_f; -1 where the schedule does not damp or
 * neither message changed).  Both schedules damp only after the undamped
 * hold of Sec. 8; the learned one with d_f in place of d. */
/* One synchronous iteration t in two phases (Sec. 5).  The factor phase
 * forms m^{t+1} of every factor from b^t and m^t (relinearisation, both
 * messages, damping); mode 0: the fixed schedule, 1: learned d_f, 2: fixed
 * schedule recording features and targets into row block `it` of X / T.
 * deg_k / deg_l: variable degrees (modes 1 and 2). */
static void factor_phase(orc_graph* g, int mode, double* X, double* T, int it, const int* deg_k, const int* deg_l)
{
    long relin_add = 0, held_add = 0;
    /* factors are independent within an iteration: they read b^t and m^t
     * only (an OpenMP build runs them in parallel) */
#pragma omp parallel for schedule(static) reduction(+ : relin_add, held_add)
    for (int f = 0; f < g->n_f; ++f) {
        if (g->fac_mask && !g->fac_mask[f]) continue;
        double J[18], r[2], k;
        int kk = g->fk[f], m = g->fm[f];
        double* x0 = g->x0 + 9 * f;
        /* the variable-to-factor messages: each variable's belief divided
         * by this factor's previous message to it (Sec. 5); they do not
         * depend on this iteration's linearisation */
        double lam_inl[9], eta_inl[3], lam_ink[36], eta_ink[6], Ltmp[36];
        for (int i = 0; i < 9; ++i) lam_inl[i] = g->lm_lam[9 * m + i] - g->ml_lam[9 * f + i];
        for (int i = 0; i < 3; ++i) eta_inl[i] = g->lm_eta[3 * m + i] - g->ml_eta[3 * f + i];
        for (int i = 0; i < 36; ++i) lam_ink[i] = g->kf_lam[36 * kk + i] - g->mk_lam[36 * f + i];
        for (int i = 0; i < 6; ++i) eta_ink[i] = g->kf_eta[6 * kk + i] - g->mk_eta[6 * f + i];
        /* a message whose incoming precision is not positive definite
         * cannot be formed and keeps its previous value; a factor with
         * such a message keeps its linearisation point for the iteration
         * (a relinearisation that is due waits), so that a kept message
         * and its factor's linearisation stay the same */
        const int ok_l = cholesky(3, lam_inl, Ltmp) == 0;
        const int ok_k = cholesky(6, lam_ink, Ltmp) == 0;
        if (!g->prm.linear && ok_l && ok_k && g->t - g->tlin[f] >= g->prm.relin_interval) {
            /* Sec. 5 / Sec. 8: relinearise when the adjacent beliefs moved
             * more than beta from the factor's linearisation point, at
             * most once every relin_interval iterations */
            double dist2 = 0.0;
            for (int i = 0; i < 6; ++i) dist2 += (g->kf_mu[6 * kk + i] - x0[i]) * (g->kf_mu[6 * kk + i] - x0[i]);
            for (int i = 0; i < 3; ++i) dist2 += (g->lm_mu[3 * m + i] - x0[6 + i]) * (g->lm_mu[3 * m + i] - x0[6 + i]);
            if (sqrt(dist2) > g->prm.relin_beta) {
                int active = orc_linearise(&g->cam, &g->prm, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m,
                                           g->kf_mu + 6 * kk, g->lm_mu + 3 * m, g->z + 2 * f, J, r, &k,
                                           g->linA + 81 * f, g->linc + 9 * f);
                g->lin_r2[f] = active ? r[0] * r[0] + r[1] * r[1] : 0.0;
                g->lin_k[f] = active ? k : 0.0;
                for (int i = 0; i < 6; ++i) x0[i] = g->kf_mu[6 * kk + i];
                for (int i = 0; i < 3; ++i) x0[6 + i] = g->lm_mu[3 * m + i];
                g->tlin[f] = g->t;
                relin_add += 1;
            }
        }
        const double* A = g->linA + 81 * f;
        const double* c = g->linc + 9 * f;
        /* to the keyframe, marginalising the landmark */
        if (!ok_l || orc_factor_message(A, c, 0, lam_inl, eta_inl, g->nk_lam + 36 * f, g->nk_eta + 6 * f) != 0) {
            memcpy(g->nk_lam + 36 * f, g->mk_lam + 36 * f, sizeof(double) * 36);
            memcpy(g->nk_eta + 6 * f, g->mk_eta + 6 * f, sizeof(double) * 6);
            held_add += 1;
        }
        /* to the landmark, marginalising the keyframe */
        if (!ok_k || orc_factor_message(A, c, 1, lam_ink, eta_ink, g->nl_lam + 9 * f, g->nl_eta + 3 * f) != 0) {
            memcpy(g->nl_lam + 9 * f, g->ml_lam + 9 * f, sizeof(double) * 9);
            memcpy(g->nl_eta + 3 * f, g->ml_eta + 3 * f, sizeof(double) * 3);
            held_add += 1;
        }
        /* damping of the eta update (Sec. 5): messages stay undamped for
         * undamped_iters iterations after a (re)linearisation (Sec. 8); the
         * message sent in the iteration of a (re)linearisation -- including
         * a factor's first message -- is never damped.  Then d, or the
         * network's d_f in the learned schedule. */
        const int hold = g->prm.undamped_iters > 1 ? g->prm.undamped_iters : 1;
        double feat[ORC_NET_NFEAT];
        if (mode != 0) factor_features(g, f, deg_k, deg_l, feat);
        if (mode == 2) {
            double* xo = X + ((size_t)it * g->n_f + f) * ORC_NET_NFEAT;
            for (int j = 0; j < ORC_NET_NFEAT; ++j) xo[j] = feat[j];
            /* the d in [0, 0.9] minimising the sum over the changed sides of
             * |(1 - d) new + d old - ref|^2 / |old - new|^2: each term is a
             * unit-curvature parabola around its vertex, so the minimiser
             * is the clipped mean of the vertices */
            int vk, vm;
            double dk = damping_vertex(g->nk_eta + 6 * f, g->mk_eta + 6 * f, g->eta_ref + 9 * f, 6, &vk);
            double dm = damping_vertex(g->nl_eta + 3 * f, g->ml_eta + 3 * f, g->eta_ref + 9 * f + 6, 3, &vm);
            double target = -1.0;
            if (vk || vm) {
                target = (vk * dk + vm * dm) / (vk + vm);
                target = target < 0.0 ? 0.0 : (target > 0.9 ? 0.9 : target);
            }
            if (g->t - g->tlin[f] < hold || !(g->lin_k[f] > 0.0)) target = -1.0;
            T[(size_t)it * g->n_f + f] = target;
        }
        double d = -1.0;
        if (g->t - g->tlin[f] >= hold) d = mode == 1 ? orc_net_forward(g->net, feat) : g->prm.damping;
        if (d >= 0.0) {
            for (int i = 0; i < 6; ++i) g->nk_eta[6 * f + i] = (1.0 - d) * g->nk_eta[6 * f + i] + d * g->mk_eta[6 * f + i];
            for (int i = 0; i < 3; ++i) g->nl_eta[3 * f + i] = (1.0 - d) * g->nl_eta[3 * f + i] + d * g->ml_eta[3 * f + i];
        }
    }
    g->n_relin += relin_add;
    g->n_held += held_add;
}

/* The belief phase: m^{t+1} replaces m^t, t advances, and every belief
 * b^{t+1} = prior(t+1) + sum of messages is formed with its mean. */
static int belief_phase(orc_graph* g, double* max_dmu)
{
    /* synchronous schedule: every factor used m^t; now m^{t+1} replaces it */
    memcpy(g->pk_eta, g->mk_eta, sizeof(double) * 6 * (size_t)g->n_f);
    double* tmp;
    tmp = g->mk_lam; g->mk_lam = g->nk_lam; g->nk_lam = tmp;
    tmp = g->mk_eta; g->mk_eta = g->nk_eta; g->nk_eta = tmp;
    tmp = g->ml_lam; g->ml_lam = g->nl_lam; g->nl_lam = tmp;
    tmp = g->ml_eta; g->ml_eta = g->nl_eta; g->nl_eta = tmp;
    g->t += 1;
    return update_beliefs(g, max_dmu);
}

static int iterate_impl(orc_graph* g, int n, double* max_dmu, int mode, double* X, double* T)
{
    int *deg_k = NULL, *deg_l = NULL;
    if (mode != 0) {
        deg_k = zalloc(sizeof(int) * (size_t)g->n_kf);
        deg_l = zalloc(sizeof(int) * (size_t)g->n_lm);
        for (int f = 0; f < g->n_f; ++f) { deg_k[g->fk[f]]++; deg_l[g->fm[f]]++; }
    }
    int status = 0;
    for (int it = 0; it < n && status == 0; ++it) {
        factor_phase(g, mode, X, T, it, deg_k, deg_l);
        if (belief_phase(g, max_dmu) != 0) status = -1;
    }
    free(deg_k);
    free(deg_l);
    return status;
}

int orc_factor_phase(orc_graph* g)
{
    if (g->net) return -1;
    factor_phase(g, 0, NULL, NULL, 0, NULL, NULL);
    return 0;
}

int orc_belief_phase(orc_graph* g, double* max_dmu) { return belief_phase(g, max_dmu); }

int orc_set_part(orc_graph* g, const unsigned char* fac_mask, const unsigned char* var_mask)
{
    free(g->fac_mask);
    free(g->var_mask);
    g->fac_mask = g->var_mask = NULL;
    if (fac_mask) g->fac_mask = dup_bytes(fac_mask, (size_t)g->n_f);
    if (var_mask) g->var_mask = dup_bytes(var_mask, (size_t)(g->n_kf + g->n_lm));
    return 0;
}

void orc_get_new_kf_messages(const orc_graph* g, int n, const int* f, double* lam, double* eta)
{
    for (int i = 0; i < n; ++i) {
        memcpy(lam + 36 * (size_t)i, g->nk_lam + 36 * (size_t)f[i], sizeof(double) * 36);
        memcpy(eta + 6 * (size_t)i, g->nk_eta + 6 * (size_t)f[i], sizeof(double) * 6);
    }
}

void orc_put_new_kf_messages(orc_graph* g, int n, const int* f, const double* lam, const double* eta)
{
    for (int i = 0; i < n; ++i) {
        memcpy(g->nk_lam + 36 * (size_t)f[i], lam + 36 * (size_t)i, sizeof(double) * 36);
        memcpy(g->nk_eta + 6 * (size_t)f[i], eta + 6 * (size_t)i, sizeof(double) * 6);
    }
}

void orc_get_kf_beliefs(const orc_graph* g, int n, const int* k, double* rec)
{
    for (int i = 0; i < n; ++i) {
        double* o = rec + 48 * (size_t)i;
        memcpy(o, g->kf_lam + 36 * (size_t)k[i], sizeof(double) * 36);
        memcpy(o + 36, g->kf_eta + 6 * (size_t)k[i], sizeof(double) * 6);
        memcpy(o + 42, g->kf_mu + 6 * (size_t)k[i], sizeof(double) * 6);
    }
}

void orc_put_kf_beliefs(orc_graph* g, int n, const int* k, const double* rec)
{
    for (int i = 0; i < n; ++i) {
        const double* o = rec + 48 * (size_t)i;
        memcpy(g->kf_lam + 36 * (size_t)k[i], o, sizeof(double) * 36);
        memcpy(g->kf_eta + 6 * (size_t)k[i], o + 36, sizeof(double) * 6);
        memcpy(g->kf_mu + 6 * (size_t)k[i], o + 42, sizeof(double) * 6);
    }
}

int orc_iterate(orc_graph* g, int n, double* max_dmu)
{
    if (g->net) return iterate_impl(g, n, max_dmu, 1, NULL, NULL);
    return iterate_impl(g, n, max_dmu, 0, NULL, NULL);
}

int orc_iterate_record(orc_graph* g, int n, double* X, double* T)
{
    if (!g->eta_ref || !X || !T) return -2;
    return iterate_impl(g, n, NULL, 2, X, T);
}

int orc_iterations_done(const orc_graph* g) { return g->t; }

void orc_get_means(const orc_graph* g, double* kf_mu, double* lm_mu)
{
    memcpy(kf_mu, g->kf_mu, sizeof(double) * 6 * g->n_kf);
    memcpy(lm_mu, g->lm_mu, sizeof(double) * 3 * g->n_lm);
}

void orc_get_world(const orc_graph* g, double* kf_Rt, double* lm_xyz)
{
    for (int v = 0; v < g->n_kf; ++v) {
        double dR[9], R[9], c[3];
        orc_so3_exp(g->kf_mu + 6 * v + 3, dR);
        matmul3(dR, g->Rref + 9 * v, R);
        for (int i = 0; i < 3; ++i) c[i] = g->cref[3 * v + i] + g->kf_mu[6 * v + i];
        for (int i = 0; i < 9; ++i) kf_Rt[12 * v + i] = R[i];
        for (int i = 0; i < 3; ++i) kf_Rt[12 * v + 9 + i] = -(R[i * 3] * c[0] + R[i * 3 + 1] * c[1] + R[i * 3 + 2] * c[2]);
    }
    for (int v = 0; v < g->n_lm; ++v)
        for (int i = 0; i < 3; ++i) lm_xyz[3 * v + i] = g->lref[3 * v + i] + g->lm_mu[3 * v + i];
}

void orc_get_beliefs(const orc_graph* g, double* kf_lam, double* kf_eta, double* lm_lam, double* lm_eta)
{
    memcpy(kf_lam, g->kf_lam, sizeof(double) * 36 * g->n_kf);
    memcpy(kf_eta, g->kf_eta, sizeof(double) * 6 * g->n_kf);
    memcpy(lm_lam, g->lm_lam, sizeof(double) * 9 * g->n_lm);
    memcpy(lm_eta, g->lm_eta, sizeof(double) * 3 * g->n_lm);
}

void orc_get_prior_diag(const orc_graph* g, double* kf_d, double* lm_d)
{
    memcpy(kf_d, g->Dk, sizeof(double) * 6 * g->n_kf);
    memcpy(lm_d, g->Dl, sizeof(double) * 3 * g->n_lm);
}

void orc_get_messages(const orc_graph* g, double* mk_lam, double* mk_eta, double* ml_lam, double* ml_eta)
{
    memcpy(mk_lam, g->mk_lam, sizeof(double) * 36 * g->n_f);
    memcpy(mk_eta, g->mk_eta, sizeof(double) * 6 * g->n_f);
    memcpy(ml_lam, g->ml_lam, sizeof(double) * 9 * g->n_f);
    memcpy(ml_eta, g->ml_eta, sizeof(double) * 3 * g->n_f);
}

/* Sec. 9.1: average reprojection error over the measurements. */
void orc_get_relin_iters(const orc_graph* g, int* tlin)
{
    memcpy(tlin, g->tlin, sizeof(int) * (size_t)g->n_f);
}

int orc_set_messages(orc_graph* g, const double* mk_lam, const double* mk_eta, const double* ml_lam,
                     const double* ml_eta)
{
    size_t F = (size_t)g->n_f;
    memcpy(g->mk_lam, mk_lam, sizeof(double) * 36 * F);
    memcpy(g->mk_eta, mk_eta, sizeof(double) * 6 * F);
    memcpy(g->ml_lam, ml_lam, sizeof(double) * 9 * F);
    memcpy(g->ml_eta, ml_eta, sizeof(double) * 3 * F);
    return update_beliefs(g, NULL);
}

double orc_are(const orc_graph* g, const unsigned char* mask, int* count)
{
    double sum = 0.0;
    int n = 0;
    for (int f = 0; f < g->n_f; ++f) {
        if (mask && !mask[f]) continue;
        int kk = g->fk[f], m = g->fm[f];
        double uv[2];
        double depth = orc_project(&g->cam, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m,
                                   g->kf_mu + 6 * kk, g->lm_mu + 3 * m, uv);
        if (depth < g->prm.z_min) continue;
        double du = g->z[2 * f] - uv[0], dv = g->z[2 * f + 1] - uv[1];
        sum += sqrt(du * du + dv * dv);
        ++n;
    }
    if (count) *count = n;
    return n ? sum / n : 0.0;
}

double orc_are_vs(const orc_graph* g, const double* ref_kf_Rt, const double* ref_lm, int* count)
{
    double sum = 0.0;
    int n = 0;
    for (int f = 0; f < g->n_f; ++f) {
        int kk = g->fk[f], m = g->fm[f];
        double uv[2];
        double depth = orc_project(&g->cam, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m,
                                   g->kf_mu + 6 * kk, g->lm_mu + 3 * m, uv);
        const double* Rt = ref_kf_Rt + 12 * kk;
        const double* X = ref_lm + 3 * m;
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = Rt[i * 3] * X[0] + Rt[i * 3 + 1] * X[1] + Rt[i * 3 + 2] * X[2] + Rt[9 + i];
        if (depth < g->prm.z_min || p[2] < g->prm.z_min) continue;
        double du = g->cam.fx * p[0] / p[2] + g->cam.cx - uv[0];
        double dv = g->cam.fy * p[1] / p[2] + g->cam.cy - uv[1];
        sum += sqrt(du * du + dv * dv);
        ++n;
    }
    if (count) *count = n;
    return n ? sum / n : 0.0;
}

int orc_huber_count(const orc_graph* g)
{
    int n = 0;
    if (g->prm.huber_nsigma <= 0.0) return 0;
    for (int f = 0; f < g->n_f; ++f) {
        int kk = g->fk[f], m = g->fm[f];
        double uv[2];
        double depth = orc_project(&g->cam, g->Rref + 9 * kk, g->cref + 3 * kk, g->lref + 3 * m,
                                   g->kf_mu + 6 * kk, g->lm_mu + 3 * m, uv);
        if (depth < g->prm.z_min) continue;
        double du = g->z[2 * f] - uv[0], dv = g->z[2 * f + 1] - uv[1];
        if (sqrt(du * du + dv * dv) / g->prm.sigma_px > g->prm.huber_nsigma) ++n;
    }
    return n;
}

long orc_relinearisations(const orc_graph* g) { return g->n_relin; }

long orc_held_messages(const orc_graph* g) { return g->n_held; }

/* ------------------------------------------------------------------------
 * incremental SLAM (Sec. 9.2)
 * ---------------------------------------------------------------------- */

static void* grow(void* p, size_t old_bytes, size_t new_bytes)
{
    void* q = realloc(p, new_bytes ? new_bytes : 1);
    if (q && new_bytes > old_bytes) memset((char*)q + old_bytes, 0, new_bytes - old_bytes);
    return q;
}

int orc_sizes(const orc_graph* g, int* n_kf, int* n_lm, int* n_obs)
{
    if (n_kf) *n_kf = g->n_kf;
    if (n_lm) *n_lm = g->n_lm;
    if (n_obs) *n_obs = g->n_f;
    return 0;
}

int orc_add_keyframe(orc_graph* g, const double* kf_Rt_init, int n_new_lm, const double* new_lm_xyz,
                     int n_obs, const int* obs_lm, const double* obs_uv)
{
    const int K0 = g->n_kf, L0 = g->n_lm, F0 = g->n_f;
    const int K1 = K0 + 1, L1 = L0 + n_new_lm, F1 = F0 + n_obs;
    if (n_new_lm < 0 || n_obs < 0) return -1;
    if (!kf_Rt_init && K0 == 0) return -1;
    for (int i = 0; i < n_obs; ++i)
        if (obs_lm[i] < 0 || obs_lm[i] >= L1) return -1;
    for (int j = L0; j < L1; ++j) {
        int seen = 0;
        for (int i = 0; i < n_obs && !seen; ++i) seen = obs_lm[i] == j;
        if (!seen && !new_lm_xyz) return -1;
    }

    /* pose of the new keyframe: given, or the latest keyframe's current estimate */
    double Rt[12];
    if (kf_Rt_init) {
        memcpy(Rt, kf_Rt_init, sizeof Rt);
    } else {
        double dR[9], R[9], c[3];
        orc_so3_exp(g->kf_mu + 6 * (K0 - 1) + 3, dR);
        matmul3(dR, g->Rref + 9 * (K0 - 1), R);
        for (int i = 0; i < 3; ++i) c[i] = g->cref[3 * (K0 - 1) + i] + g->kf_mu[6 * (K0 - 1) + i];
        for (int i = 0; i < 9; ++i) Rt[i] = R[i];
        for (int i = 0; i < 3; ++i) Rt[9 + i] = -(R[i * 3] * c[0] + R[i * 3 + 1] * c[1] + R[i * 3 + 2] * c[2]);
    }

    size_t d = sizeof(double);
#define GROW(ptr, per, oldn, newn) ptr = grow(ptr, (size_t)(per) * (oldn), (size_t)(per) * (newn))
    GROW(g->Rref, 9 * d, K0, K1); GROW(g->cref, 3 * d, K0, K1); GROW(g->anchored, 1, K0, K1);
    GROW(g->kf_birth, sizeof(int), K0, K1); GROW(g->Dk, 6 * d, K0, K1); GROW(g->kf_lam, 36 * d, K0, K1);
    GROW(g->kf_eta, 6 * d, K0, K1); GROW(g->kf_mu, 6 * d, K0, K1);
    GROW(g->lref, 3 * d, L0, L1); GROW(g->lm_birth, sizeof(int), L0, L1); GROW(g->Dl, 3 * d, L0, L1);
    GROW(g->lm_lam, 9 * d, L0, L1); GROW(g->lm_eta, 3 * d, L0, L1); GROW(g->lm_mu, 3 * d, L0, L1);
    GROW(g->fk, sizeof(int), F0, F1); GROW(g->fm, sizeof(int), F0, F1); GROW(g->z, 2 * d, F0, F1);
    GROW(g->mk_lam, 36 * d, F0, F1); GROW(g->mk_eta, 6 * d, F0, F1); GROW(g->ml_lam, 9 * d, F0, F1);
    GROW(g->ml_eta, 3 * d, F0, F1); GROW(g->nk_lam, 36 * d, F0, F1); GROW(g->nk_eta, 6 * d, F0, F1);
    GROW(g->nl_lam, 9 * d, F0, F1); GROW(g->nl_eta, 3 * d, F0, F1); GROW(g->linA, 81 * d, F0, F1);
    GROW(g->linc, 9 * d, F0, F1); GROW(g->x0, 9 * d, F0, F1); GROW(g->tlin, sizeof(int), F0, F1);
    GROW(g->lin_r2, d, F0, F1); GROW(g->lin_k, d, F0, F1); GROW(g->hist, ORC_HIST * d, F0, F1);
    GROW(g->pk_eta, 6 * d, F0, F1);
#undef GROW
    free(g->eta_ref);   /* the reference covered the old factors only */
    g->eta_ref = NULL;

    /* references of the new variables = their initial values */
    for (int i = 0; i < 9; ++i) g->Rref[9 * K0 + i] = Rt[i];
    for (int i = 0; i < 3; ++i)
        g->cref[3 * K0 + i] = -(Rt[0 * 3 + i] * Rt[9] + Rt[1 * 3 + i] * Rt[10] + Rt[2 * 3 + i] * Rt[11]);
    g->kf_birth[K0] = g->t;
    for (int j = L0; j < L1; ++j) {
        g->lm_birth[j] = g->t;
        if (new_lm_xyz) {
            for (int i = 0; i < 3; ++i) g->lref[3 * j + i] = new_lm_xyz[3 * (j - L0) + i];
        } else {
            /* Sec. 9.2: 1 m depth along the first ray that observes it */
            int o = 0;
            while (obs_lm[o] != j) ++o;
            double pc[3] = { (obs_uv[2 * o] - g->cam.cx) / g->cam.fx, (obs_uv[2 * o + 1] - g->cam.cy) / g->cam.fy, 1.0 };
            for (int i = 0; i < 3; ++i)
                g->lref[3 * j + i] = g->cref[3 * K0 + i] + Rt[0 * 3 + i] * pc[0] + Rt[1 * 3 + i] * pc[1] + Rt[2 * 3 + i] * pc[2];
        }
    }
    g->n_kf = K1;
    g->n_lm = L1;
    g->n_f = F1;

    /* new factors: linearised at the current means (new variables at their
     * chart origin), zero messages, (re)linearised now */
    orc_params p1 = g->prm;
    p1.huber_nsigma = 0.0;
    double J[18], r[2], k, A[81], c[9];
    int* deg_l = zalloc(sizeof(int) * (n_new_lm ? n_new_lm : 1));
    int deg_k = 0;
    for (int i = 0; i < n_obs; ++i) {
        int f = F0 + i, m = obs_lm[i];
        g->fk[f] = K0;
        g->fm[f] = m;
        g->z[2 * f] = obs_uv[2 * i];
        g->z[2 * f + 1] = obs_uv[2 * i + 1];
        double* x0 = g->x0 + 9 * f;
        for (int q = 0; q < 6; ++q) x0[q] = g->kf_mu[6 * K0 + q];
        for (int q = 0; q < 3; ++q) x0[6 + q] = g->lm_mu[3 * m + q];
        g->tlin[f] = g->t;
        int active = orc_linearise(&g->cam, &g->prm, g->Rref + 9 * K0, g->cref + 3 * K0, g->lref + 3 * m, x0,
                                   x0 + 6, g->z + 2 * f, J, r, &k, g->linA + 81 * f, g->linc + 9 * f);
        g->lin_r2[f] = active ? r[0] * r[0] + r[1] * r[1] : 0.0;
        g->lin_k[f] = active ? k : 0.0;
        /* prior of the new variables (Sec. 4 / Sec. 8), from these factors
         * at this point with Huber weight 1 */
        orc_linearise(&g->cam, &p1, g->Rref + 9 * K0, g->cref + 3 * K0, g->lref + 3 * m, x0, x0 + 6,
                      g->z + 2 * f, J, r, &k, A, c);
        for (int q = 0; q < 6; ++q) g->Dk[6 * K0 + q] += A[q * 9 + q];
        deg_k++;
        if (m >= L0) {
            for (int q = 0; q < 3; ++q) g->Dl[3 * m + q] += A[(6 + q) * 9 + 6 + q];
            deg_l[m - L0]++;
        }
    }
    {
        double mx = 0.0;
        for (int q = 0; q < 6; ++q) {
            if (deg_k) g->Dk[6 * K0 + q] /= deg_k;
            if (g->Dk[6 * K0 + q] > mx) mx = g->Dk[6 * K0 + q];
        }
        for (int q = 0; q < 6; ++q) {
            if (mx <= 0.0) g->Dk[6 * K0 + q] = 1.0;
            else if (g->Dk[6 * K0 + q] < 1e-9 * mx) g->Dk[6 * K0 + q] = 1e-9 * mx;
        }
    }
    for (int j = L0; j < L1; ++j) {
        double mx = 0.0;
        for (int q = 0; q < 3; ++q) {
            if (deg_l[j - L0]) g->Dl[3 * j + q] /= deg_l[j - L0];
            if (g->Dl[3 * j + q] > mx) mx = g->Dl[3 * j + q];
        }
        for (int q = 0; q < 3; ++q) {
            if (mx <= 0.0) g->Dl[3 * j + q] = 1.0;
            else if (g->Dl[3 * j + q] < 1e-9 * mx) g->Dl[3 * j + q] = 1e-9 * mx;
        }
    }
    free(deg_l);

    /* beliefs of the new variables: their prior at scale s(0), mean 0 */
    double s0 = orc_prior_scale(&g->prm, 0);
    for (int i = 0; i < 6; ++i) g->kf_lam[36 * K0 + i * 6 + i] = s0 * g->Dk[6 * K0 + i];
    for (int j = L0; j < L1; ++j)
        for (int i = 0; i < 3; ++i) g->lm_lam[9 * j + i * 3 + i] = s0 * g->Dl[3 * j + i];
    return K0;
}
