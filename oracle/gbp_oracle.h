/*
 * gbp_oracle.h -- plain FP64 Gaussian Belief Propagation for bundle adjustment.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct CPU oracle
 * that the CUDA path is checked against.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * Model (Sec. 4): keyframe poses x_k and landmark points l_m, measurement
 * h(x_k, l_m) = pi(R_k l_m + t_k) with a pinhole pi, Gaussian pixel noise
 * sigma^2 I, weak Gaussian priors on every variable, optional Huber
 * rescaling of each measurement factor (Sec. 6).
 *
 * Chart (the paper only says R_k, t_k are "derived from" x_k): every variable
 * is a perturbation of a fixed reference equal to its initial value.
 *   keyframe  x_k = [dc (3), dw (3)]:  R_k = Exp(dw) Rref_k,  c_k = cref_k + dc,
 *             t_k = -R_k c_k  (c_k is the camera centre in the world frame)
 *   landmark  x_m = [dl (3)]:          l_m = lref_m + dl
 * so h = pi(R_k (l_m - c_k)).
 *
 * Schedule (Sec. 5): synchronous.  Iteration t reads beliefs b^t and the
 * previous factor-to-variable messages m^t, writes m^{t+1} for every factor,
 * then forms b^{t+1} = prior(t+1) + sum of m^{t+1}.
 */
#ifndef GBP_ORACLE_H
#define GBP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double fx, fy, cx, cy;
} orc_cam;

typedef struct {
    double damping;            /* d in the damping rule of Sec. 5 (0.4 in Sec. 8)             */
    double huber_nsigma;       /* N_sigma of Sec. 6 in Mahalanobis units; <= 0 disables      */
    double sigma_px;           /* measurement noise std, Sigma_M = sigma^2 I                  */
    double prior_final_scale;  /* priors end this factor of the measurement scale (Sec. 4, 8) */
    int    prior_anneal_iters; /* iterations over which priors weaken (Sec. 8); 0 = fixed      */
    double anchor_scale;       /* strength of the anchor prior on anchored keyframes          */
    double z_min;              /* a factor whose point has depth < z_min sends zero information*/
    int    linear;             /* 1: linearise once at the initial point and never again      */
    double relin_beta;         /* relinearise when |mu - x0| > beta (Sec. 5, 8: 0.01)          */
    int    relin_interval;     /* ... but at most every this many iterations (Sec. 8: 10)      */
    int    undamped_iters;     /* messages undamped this many iterations after (Sec. 8: 8)     */
} orc_params;

typedef struct orc_graph orc_graph;

/* kf_Rt: n_kf x 12 (R row-major, t), world->camera.  lm_xyz: n_lm x 3.
 * obs_*: n_obs observations (keyframe index, landmark index, pixel).
 * Returns NULL on invalid input. */
orc_graph* orc_create(const orc_cam* cam, const orc_params* prm,
                      int n_kf, const double* kf_Rt, int n_lm, const double* lm_xyz,
                      int n_obs, const int* obs_kf, const int* obs_lm, const double* obs_uv,
                      int n_anchor, const int* anchor_kf);
void orc_destroy(orc_graph* g);

/* Incremental SLAM (Sec. 9.2): add one keyframe observing n_obs points.
 * kf_Rt_init (12) or NULL: the latest keyframe's current world pose.
 * New points get indices n_lm .. n_lm + n_new_lm - 1; new_lm_xyz (n_new_lm x
 * 3) or NULL: 1 m depth along the first observation of each in this call.
 * New variables take their initial value as chart origin and a prior built
 * like the others' (from their factors' Jacobians there), annealed from
 * this iteration on; new factors are linearised at the current means and
 * start with zero messages.  Returns the new keyframe's index, or -1. */
int orc_add_keyframe(orc_graph* g, const double* kf_Rt_init, int n_new_lm, const double* new_lm_xyz,
                     int n_obs, const int* obs_lm, const double* obs_uv);
int orc_sizes(const orc_graph* g, int* n_kf, int* n_lm, int* n_obs);

/* Run n synchronous iterations.  Returns 0, or -1 if a belief stopped being
 * positive definite.  A message whose incoming precision is not positive
 * definite keeps its previous value instead, and its factor does not
 * relinearise in that iteration.  *max_dmu (nullable) = max_v |mu_v^{t+1} -
 * mu_v^t|_inf of the last iteration. */
int orc_iterate(orc_graph* g, int n, double* max_dmu);
int orc_iterations_done(const orc_graph* g);

/* Chart means of the current beliefs. */
void orc_get_means(const orc_graph* g, double* kf_mu /* n_kf x 6 */, double* lm_mu /* n_lm x 3 */);
/* World-frame estimates of the current beliefs. */
void orc_get_world(const orc_graph* g, double* kf_Rt /* n_kf x 12 */, double* lm_xyz /* n_lm x 3 */);
/* Current beliefs in information form (full symmetric matrices). */
void orc_get_beliefs(const orc_graph* g, double* kf_lam /* n_kf x 36 */, double* kf_eta /* n_kf x 6 */,
                     double* lm_lam /* n_lm x 9 */, double* lm_eta /* n_lm x 3 */);
/* Prior diagonals generated at creation (before annealing). */
void orc_get_prior_diag(const orc_graph* g, double* kf_d /* n_kf x 6 */, double* lm_d /* n_lm x 3 */);
/* Current factor-to-variable messages (full symmetric matrices). */
void orc_get_messages(const orc_graph* g, double* mk_lam /* n_f x 36 */, double* mk_eta /* n_f x 6 */,
                      double* ml_lam /* n_f x 9 */, double* ml_eta /* n_f x 3 */);

/* Iteration at which each factor (caller order) was last (re)linearised:
 * t_lin of the schedule of Sec. 5 / Sec. 8 (0 = still at its first
 * linearisation). */
void orc_get_relin_iters(const orc_graph* g, int* tlin /* n_f */);
/* Test hook: replace the current messages m^t (full symmetric matrices, the
 * layout of orc_get_messages) and recompute every belief b^t = prior(t) +
 * sum of messages and its mean.  Returns 0, or -1 if a belief is not
 * positive definite (the graph is then unusable). */
int orc_set_messages(orc_graph* g, const double* mk_lam, const double* mk_eta, const double* ml_lam,
                     const double* ml_eta);

/* Average reprojection error over measurements whose point lies in front of
 * the camera (depth >= z_min).  mask (nullable) selects measurements.
 * *count (nullable) receives the number averaged. */
double orc_are(const orc_graph* g, const unsigned char* mask, int* count);
/* Average distance between the projections at the current means and at a
 * reference world solution (ref_kf_Rt n_kf x 12, ref_lm n_lm x 3). */
double orc_are_vs(const orc_graph* g, const double* ref_kf_Rt, const double* ref_lm, int* count);
/* Number of factors currently in the Huber (linear-loss) regime. */
int orc_huber_count(const orc_graph* g);
/* Relinearisations performed since creation (all factors). */
long orc_relinearisations(const orc_graph* g);
/* Messages left at their previous value because their incoming precision
 * (the marginalised variable's belief divided by the previous message) was
 * not positive definite, so the Schur complement of Sec. 5 does not exist. */
long orc_held_messages(const orc_graph* g);

/* ---- one graph solved in parts (the multi-rank split of the iteration) ----
 * orc_set_part restricts which factors form messages (fac_mask, n_f bytes)
 * and which variables form beliefs (var_mask: keyframes then landmarks);
 * NULL = all.  orc_iterate is orc_factor_phase then orc_belief_phase.
 * Between the two, the new messages to keyframes (m^{t+1}, full 6x6 and 6)
 * of chosen factors can be read and written; after the belief phase, chosen
 * keyframe beliefs (Lambda 36, eta 6, mean 6 per keyframe) likewise.  Fixed
 * damping schedule only (orc_factor_phase returns -1 with a network set). */
int orc_set_part(orc_graph* g, const unsigned char* fac_mask, const unsigned char* var_mask);
int orc_factor_phase(orc_graph* g);
int orc_belief_phase(orc_graph* g, double* max_dmu);
void orc_get_new_kf_messages(const orc_graph* g, int n, const int* f, double* lam, double* eta);
void orc_put_new_kf_messages(orc_graph* g, int n, const int* f, const double* lam, const double* eta);
void orc_get_kf_beliefs(const orc_graph* g, int n, const int* k, double* rec /* n x 48 */);
void orc_put_kf_beliefs(orc_graph* g, int n, const int* k, const double* rec);

/* ---- learned damping (no counterpart in the paper: a per-factor d in place
 * of the fixed d of Sec. 5 / Sec. 8) ----
 * Network: 16 features -> 64 -> 64 -> 1, ReLU hidden layers, output
 * 0.9 * sigmoid; ORC_NET_NPARAM parameters in the order W1 (16 x 64, row =
 * input), b1, W2 (64 x 64), b2, W3 (64), b3.  Features of factor f at
 * iteration t, with eta_new this iteration's undamped message, eta_old =
 * m^t and eta_prev = m^{t-1} on each side:
 *   0  log(1 + M) / 3 with M = |r| / sigma at the factor's linearisation
 *   1  its Huber weight (0 if the point is behind z_min)
 *   2  tr Lambda_new(f->k) / (tr Lambda_new(f->k) + tr P_k), P_k = the
 *      keyframe belief's precision minus the factor's previous message
 *   3  the same for the landmark
 *   4  |eta_new - eta_old| / (|eta_new| + |eta_old|) of the message to the
 *      keyframe; 5, 6 its values at t-1 and t-2
 *   7  cosine between eta_new - eta_old and eta_old - eta_prev (keyframe side);
 *      0 unless t - t_lin >= 2 (the three messages share one linearisation)
 *   8-11 the same four for the message to the landmark (its eta_prev is
 *      remembered only while features are computed: learned or record runs)
 *   12 log(1 + deg k) / 5;  13 log(1 + deg m) / 3
 *   14 min(t - t_lin, 50) / 50;  15 min(t - t_birth(m), 50) / 50
 * Learned schedule: with a network set, orc_iterate damps both eta messages
 * of factor f by d_f = net(features) wherever the fixed schedule damps
 * (after the undamped hold of Sec. 8). */
#define ORC_NET_NFEAT 16
#define ORC_NET_NPARAM 5313
double orc_net_forward(const double* params, const double x[ORC_NET_NFEAT]);
/* params (copied) or NULL to return to the fixed schedule; -1 if not finite. */
int orc_set_damping_net(orc_graph* g, const double* params);
/* Reference eta of the damping targets, per factor (caller order): the
 * message to the keyframe (6) then to the landmark (3); copied.  NULL
 * clears it. */
void orc_set_reference_messages(orc_graph* g, const double* eta_ref /* n_f x 9 */);
/* n iterations of the fixed schedule writing, for iteration i and factor f
 * (caller order), X[(i n_f + f) 16 + j] = feature j and T[i n_f + f] = the
 * damping target: the d in [0, 0.9] minimising the sum over the message
 * sides where eta_old != eta_new of
 * |(1 - d) eta_new + d eta_old - eta_ref|^2 / |eta_old - eta_new|^2;
 * -1 where neither side changed, where the schedule does not damp (the
 * undamped hold after a (re)linearisation), or for a factor behind z_min.  Returns 0, -1 (belief not positive definite) or -2 (no
 * reference set). */
int orc_iterate_record(orc_graph* g, int n, double* X, double* T);

/* ---- pieces exposed for unit pins ---- */
void orc_so3_exp(const double w[3], double R[9]);
void orc_so3_left_jacobian(const double w[3], double J[9]);
double orc_huber_weight(double M, double nsigma);
double orc_prior_scale(const orc_params* prm, int t);
/* Projection in the chart; returns the depth p_z. */
double orc_project(const orc_cam* cam, const double Rref[9], const double cref[3], const double lref[3],
                   const double xk[6], const double xl[3], double uv[2]);
/* Linearised factor at (xk, xl): J (2x9 row-major), residual r = z - h,
 * Huber weight k, information matrix A (9x9) and vector c (9).
 * Returns 1 if active, 0 if the point is closer than z_min (A = c = 0). */
int orc_linearise(const orc_cam* cam, const orc_params* prm, const double Rref[9], const double cref[3],
                  const double lref[3], const double xk[6], const double xl[3], const double z[2],
                  double J[18], double r[2], double* k, double A[81], double c[9]);
/* Factor-to-variable message from a 9x9 factor (A, c).  target 0: to the
 * keyframe block (0..5), marginalising the landmark block; target 1: to the
 * landmark block (6..8), marginalising the keyframe block.  lam_in/eta_in is
 * the message arriving from the marginalised variable.  Returns 0, or -1 if
 * the matrix to invert is not positive definite. */
int orc_factor_message(const double A[81], const double c[9], int target,
                       const double* lam_in, const double* eta_in, double* lam_out, double* eta_out);

#ifdef __cplusplus
}
#endif
#endif
