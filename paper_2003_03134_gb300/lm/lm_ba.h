/*
 * lm_ba.h -- Levenberg-Marquardt bundle adjustment with a dense Schur
 * complement (CPU comparison baseline), the objective GBP settles on:
 * reprojection errors under the Huber loss (Sec. 6) plus the weak priors of
 * Sec. 4 at their final strength (Sec. 8) and the anchor.
 */
#ifndef LM_BA_H
#define LM_BA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_kf, n_lm, n_obs, n_anchor;
    const double* Rref;      /* n_kf x 9, reference rotations (world to camera), the chart origins */
    const double* cref;      /* n_kf x 3, reference camera centres */
    const double* lref;      /* n_lm x 3, reference points */
    const int* obs_kf;
    const int* obs_lm;
    const double* obs_uv;    /* n_obs x 2 pixels */
    const int* anchor_kf;
    double fx, fy, cx, cy, sigma, huber_n, z_min, prior_scale, anchor_scale;
} lm_problem;

typedef struct lm_ctx lm_ctx;

/* Copies the problem; state = the references (chart origin). */
lm_ctx* lm_create(const lm_problem* P);
void lm_destroy(lm_ctx* c);
/* Up to n LM iterations (each: linearise, then damped steps until one
 * lowers the objective); stops early once a step is below tol (max |dx|)
 * or the objective stops decreasing.  Returns the iterations run. */
int lm_iterate(lm_ctx* c, int n, double tol);
double lm_cost(const lm_ctx* c);
int lm_converged(const lm_ctx* c);
/* World-frame estimate: kf_Rt n_kf x 12 (R row-major, t), lm_xyz n_lm x 3. */
void lm_state(const lm_ctx* c, double* kf_Rt, double* lm_xyz);

#ifdef __cplusplus
}
#endif
#endif
