/*
 * gbp.h -- C ABI of libgbp: synchronous Gaussian Belief Propagation for
 * bundle adjustment on a GB300 (sm_103a) GPU.
 *
 * Method: Ortiz, Pupilli, Leutenegger, Davison, "Bundle Adjustment on a
 * Graph Processor" (CVPR 2020, arXiv 2003.03134).
 *   Sec. 4  the factor graph: keyframe poses, landmark points, weak priors,
 *           reprojection factors h = pi(R l + t) linearised in information
 *           form (eta = J^T S^-1 (J x0 + z - h(x0)), Lambda = J^T S^-1 J).
 *   Sec. 5  factor-to-variable messages by Schur complement (eqs.
 *           messageeta / messagelambda), beliefs as prior + sum of
 *           messages (eqs. beliefeta / belieflambda), synchronous
 *           schedule, lazy relinearisation, damping of eta.
 *   Sec. 6  Huber rescale of a factor's information.
 *   Sec. 8  constants: beta = 0.01, relinearise at most every 10
 *           iterations, d = 0.4, undamped 8 iterations after
 *           relinearisation, priors annealed to 1/100 over 10 iterations.
 *   Sec. 9  average reprojection error (ARE); Sec. 9.2 incremental SLAM
 *           (new keyframe at the latest pose, new points at 1 m depth).
 *
 * Conventions
 *   - Every call returns a gbp_status and never aborts.  A per-graph detail
 *     string is available from gbp_last_error().
 *   - Host pointers are caller-owned; inputs are copied before the call
 *     returns, outputs are caller-allocated (sizes from gbp_get_sizes()).
 *   - All device memory is allocated and owned by the library and released
 *     by gbp_destroy_graph().  All device work is issued on the CUDA stream
 *     given at creation (NULL = the legacy default stream); calls that
 *     return host data synchronise that stream.
 *   - Poses at the boundary: kf_Rt is n x 12 doubles, R row-major then t,
 *     mapping world points into the camera frame (x_c = R x_w + t), camera
 *     x right, y down, z forward.  Points are n x 3 doubles (world).
 *   - One graph must not be used from two host threads at once.
 */
#ifndef GBP_H
#define GBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbp_graph gbp_graph;

typedef enum {
    GBP_OK = 0,
    GBP_EINVAL = 1,     /* invalid argument (index out of range, non-finite value, bad size)   */
    GBP_ENOMEM = 2,     /* host or device allocation failed                                    */
    GBP_ECUDA = 3,      /* a CUDA call failed (no device, launch error, ...)                   */
    GBP_EDIVERGED = 4,  /* a belief stopped being positive definite or its mean became non-finite */
    GBP_ETIMEOUT = 5,   /* a bounded device-side wait gave up                                   */
    GBP_ESTATE = 6      /* call not valid in the graph's current state                          */
} gbp_status;

typedef struct {
    double fx, fy, cx, cy;      /* pinhole intrinsics, pixels */
    int32_t width, height;      /* image size, pixels (informational) */
} gbp_intrinsics;

typedef struct {
    float   damping;            /* d of Sec. 5; default 0.4 (Sec. 8)                                */
    float   huber_nsigma;       /* N_sigma of Sec. 6 in units of sigma_px; <= 0 disables; default 0 */
    float   sigma_px;           /* measurement noise std, pixels; default 1                         */
    int32_t iterations;         /* iterations per gbp_iterate() call when n_iters <= 0; default 200 */
    float   conv_tol;           /* stop once max |mu^{t+1} - mu^t|_inf < conv_tol; 0 = fixed count   */
    int32_t check_every;        /* iterations between convergence checks; default 16.  With
                                   per-phase launches, check blocks of up to 64 iterations run in
                                   one launch of a device-side graph loop that makes the check on
                                   the GPU (no host round trip per block); the same checks, the
                                   same results.                                                   */
    float   prior_final_scale;  /* priors end this fraction of one measurement's strength; 0.01   */
    int32_t prior_anneal_iters; /* geometric anneal from scale 1 over this many iterations; 10     */
    float   anchor_scale;       /* anchor prior = anchor_scale x the keyframe's prior; 1000        */
    float   z_min;              /* depth below which a factor sends no information, m; 0.05       */
    float   relin_beta;         /* relinearise when |mu - x0|_2 > beta (Sec. 5); 0.01 (Sec. 8)     */
    int32_t relin_interval;     /* ... at most every this many iterations; 10 (Sec. 8)             */
    int32_t undamped_iters;     /* messages undamped this many iterations after (re)linearisation; 8 */
    float   fp64_pivot_ratio;   /* FP32 Cholesky with min/max pivot below this is redone in FP64; 1e-6 */
    int32_t precision_mode;     /* 0: FP32 + FP64 fallback, 1: FP32 only, 2: FP64 throughout        */
    int32_t linear;             /* 1: never relinearise (linear GBP at the initial point)          */
    int32_t launch_mode;        /* 0: auto (gbp_autotune on first use; a graph whose device, storage,
                                   precision and damping modes and sizes match one already tuned in
                                   this process takes that graph's choice), 1: one persistent launch per
                                   gbp_iterate call with a grid barrier between phases, 2: one launch
                                   per phase (factor kernel, belief kernel) replayed as a CUDA graph.
                                   All modes give bitwise identical results.                        */
    int32_t damping_mode;       /* 0: the fixed d above (Sec. 5, Sec. 8); 1: per-factor d predicted by
                                   the damping network given to gbp_set_damping_model (see below)   */
    int32_t factor_shape;       /* FP32 fixed schedule, per-phase launches: launch shape of the factor
                                   kernel, -1 = the autotuner's choice (default; before tuning: 1 for
                                   large graphs, else 0); 0: 128 threads per block, no register
                                   budget; 1: 128 threads, >= 3 blocks per SM; 2: 128 threads, >= 4
                                   blocks per SM; 3: 64 threads, no budget; 4 and 5: 128 threads, >= 4
                                   or >= 3 blocks per SM, the rare tiles that need the FP64 redo left
                                   to a second kernel (so the first holds no registers for it).
                                   Every shape gives bitwise identical results.                     */
    int32_t persistent_shape;   /* persistent launches: -1 (default) or 0, the one shape (no
                                   register budget); kept for the autotuner's report.               */
    int32_t fp64_exact_cavity;  /* FP32 + FP64 fallback: 1 = every keyframe incoming precision
                                   b^t - m^t (Sec. 5) that takes the FP64 redo is summed exactly
                                   from its parts (the keyframe's prior plus every other factor's
                                   message), not formed as belief minus message; 0 (default) = only
                                   where belief minus message is not positive definite.  Slower;
                                   the results differ from 0 by rounding only.                       */
} gbp_params;

typedef struct {
    int32_t iterations;         /* iterations run since creation / reset                          */
    float   max_dmu;            /* max |mu^{t+1} - mu^t|_inf of the last iteration (chart units)  */
    double  are;                /* average reprojection error over measurements in front of the camera, px */
    double  are_ref;            /* average |h(mu) - h(reference)| (gbp_set_reference), px; -1 if unset */
    int32_t n_are;              /* measurements counted in are                                    */
    int32_t huber_count;        /* measurements currently beyond the Huber threshold              */
    int32_t fp64_fallbacks;     /* FP32 Cholesky factorisations redone in FP64 since creation     */
    int32_t relinearisations;   /* factor relinearisations since creation                         */
    int32_t launch_mode;        /* launch mode gbp_iterate() used last (1 persistent, 2 per phase) */
    int64_t kernel_launches;    /* kernels this graph has launched since creation (graph replays
                                   count each kernel they contain)                                 */
    int32_t held_messages;      /* messages left at their previous value since creation / reset:
                                   the incoming precision (belief / previous message of the
                                   marginalised variable) was not positive definite even after the
                                   FP64 redo -- in FP32 mode, rounding of the stored messages in a
                                   direction that only the weak prior constrains                    */
    int32_t fp64_resums;        /* keyframe incoming precisions b^t - m^t (Sec. 5) that the FP64 redo
                                   had to sum again exactly from their parts (prior plus the other
                                   factors' messages) because the FP32 belief's rounding left the
                                   difference indefinite; counted with fp64_fallbacks              */
} gbp_stats;

/* Fill *out with the defaults listed above. */
void gbp_default_params(gbp_params* out);

/* Build a graph (Sec. 4): n_kf keyframes with initial poses kf_Rt (n_kf x 12),
 * n_lm landmarks with initial positions lm_xyz (n_lm x 3), n_obs
 * reprojection factors (keyframe obs_kf[i] sees landmark obs_lm[i] at pixel
 * obs_uv[2i..2i+1]), n_anchor keyframes held by a strong prior at their
 * initial pose.  Every variable's reference (chart origin) is its initial
 * value; priors are generated from the measurement Jacobians there.  The
 * graph starts at iteration 0 with beliefs equal to the priors.
 * GBP_EINVAL: negative counts, an index out of range, a non-finite value, or
 * an observation whose point is not in front of its camera (depth < z_min)
 * at the initial values.  cuda_stream: a cudaStream_t or NULL. */
gbp_status gbp_create_graph(const gbp_intrinsics* intr,
                            int32_t n_kf, const double* kf_Rt,
                            int32_t n_lm, const double* lm_xyz,
                            int32_t n_obs, const int32_t* obs_kf, const int32_t* obs_lm,
                            const double* obs_uv,
                            int32_t n_anchor, const int32_t* anchor_kf,
                            void* cuda_stream, gbp_graph** out);

/* One problem of a batch (all host pointers, indices local to the problem). */
typedef struct {
    int32_t n_kf;
    const double* kf_Rt;        /* n_kf x 12 */
    int32_t n_lm;
    const double* lm_xyz;       /* n_lm x 3  */
    int32_t n_obs;
    const int32_t* obs_kf;
    const int32_t* obs_lm;
    const double* obs_uv;       /* n_obs x 2 */
    int32_t n_anchor;
    const int32_t* anchor_kf;
} gbp_problem_desc;

/* Batching: n_problems independent problems (same intrinsics) as one
 * disconnected graph, so that one launch iterates all of them.  Variables
 * are numbered problem by problem (gbp_get_batch_info gives the offsets);
 * every other call treats the batch as one graph.  No warp tile spans two
 * problems, so each problem's results are bitwise identical to solving it
 * alone with the same parameters and iteration count.  The convergence test
 * (conv_tol) uses the largest mean change over all problems.  Errors as for
 * gbp_create_graph. */
gbp_status gbp_create_batch(const gbp_intrinsics* intr, int32_t n_problems, const gbp_problem_desc* problems,
                            void* cuda_stream, gbp_graph** out);

/* Problem table of a graph (a single graph is one problem): *n_problems;
 * kf_offsets / lm_offsets (nullable, n_problems + 1 entries) the first
 * keyframe / landmark of each problem and the totals; obs_counts (nullable,
 * n_problems) the observations of each. */
gbp_status gbp_get_batch_info(const gbp_graph* g, int32_t* n_problems, int32_t* kf_offsets, int32_t* lm_offsets,
                              int32_t* obs_counts);

/* Average reprojection error (Sec. 9.1) of each problem at the current
 * means: are[n_problems]; n_are / huber (nullable) the measurements counted
 * and those beyond the Huber threshold.  One fixed-order reduction per
 * problem on the device.  Synchronises the stream. */
gbp_status gbp_get_problem_are(const gbp_graph* g, double* are, int32_t* n_are, int32_t* huber);

/* Replace the solver parameters (values are checked: GBP_EINVAL on a
 * non-positive sigma_px, damping outside [0,1), ...).  Takes effect at the
 * next gbp_iterate(). */
gbp_status gbp_set_params(gbp_graph* g, const gbp_params* params);
gbp_status gbp_get_params(const gbp_graph* g, gbp_params* out);

/* Run synchronous GBP iterations (Sec. 5): every factor (re)linearises as
 * its schedule allows, sends both messages, then every variable updates its
 * belief and mean.  n_iters <= 0 uses params.iterations.  With conv_tol > 0
 * it stops early once the largest mean change falls below conv_tol (checked
 * every check_every iterations).  *iters_done (nullable) receives the count
 * run.  Asynchronous unless a convergence check is needed; errors from the
 * device (GBP_EDIVERGED) are reported by the next synchronising call. */
gbp_status gbp_iterate(gbp_graph* g, int32_t n_iters, int32_t* iters_done);

/* Return the graph to iteration 0 (beliefs = priors, messages = 0, every
 * factor linearised at its reference), keeping parameters and sizes. */
gbp_status gbp_reset(gbp_graph* g);

/* World-frame means of the current beliefs: kf_Rt (n_kf x 12), lm_xyz
 * (n_lm x 3).  kf_cov / lm_cov (nullable) receive the belief covariances
 * in the chart (n_kf x 36: [dc, dw] with c the camera centre and R =
 * Exp(dw) R_ref; n_lm x 9).  Synchronises the stream. */
gbp_status gbp_get_beliefs(const gbp_graph* g, double* kf_Rt, double* lm_xyz,
                           double* kf_cov, double* lm_cov);

/* Chart means of the current beliefs: kf_mu (n_kf x 6, [dc, dw]), lm_mu
 * (n_lm x 3, dl).  Synchronises the stream. */
gbp_status gbp_get_means(const gbp_graph* g, double* kf_mu, double* lm_mu);

/* Give a reference world solution (e.g. a converged solution from another
 * solver); gbp_get_stats() then reports are_ref against it. */
gbp_status gbp_set_reference(gbp_graph* g, const double* ref_kf_Rt, const double* ref_lm_xyz);

/* Incremental SLAM (Sec. 9.2): add one keyframe and its observations.
 * kf_Rt_init (12 doubles) or NULL = the latest keyframe's current pose.
 * n_new_lm new landmarks get indices n_lm .. n_lm+n_new_lm-1; new_lm_xyz
 * (n_new_lm x 3) or NULL = 1 m depth along the first ray that observes
 * each.  obs_lm[i] (n_obs) may name old or new landmarks; every new
 * landmark must be observed.  New variables start with their prior, new
 * factors with zero messages, linearised at the current means.
 * *new_kf_index (nullable) receives the keyframe's index. */
gbp_status gbp_add_keyframe(gbp_graph* g, const double* kf_Rt_init,
                            int32_t n_new_lm, const double* new_lm_xyz,
                            int32_t n_obs, const int32_t* obs_lm, const double* obs_uv,
                            int32_t* new_kf_index);

/* Metrics of the current means (Sec. 9.1 ARE and friends), computed on the
 * device with a fixed-order reduction.  Synchronises the stream. */
gbp_status gbp_get_stats(const gbp_graph* g, gbp_stats* out);

gbp_status gbp_get_sizes(const gbp_graph* g, int32_t* n_kf, int32_t* n_lm, int32_t* n_obs);

/* Reprojection error of every observation at the current means (Sec. 9.1):
 * err[i] = |z_i - pi(R l + t)| in pixels, caller's observation order (host,
 * n_obs doubles), or -1 where the point lies closer than z_min to its
 * camera.  With huber_nsigma N, an observation with err > N sigma_px is in
 * the linear (outlier) regime of the Huber loss (Sec. 6).  Synchronises the
 * stream. */
gbp_status gbp_get_residuals(const gbp_graph* g, double* err);

/* Iteration at which each observation's factor was last (re)linearised
 * (t_lin of the lazy schedule of Sec. 5 / Sec. 8; 0 = still at its first
 * linearisation), n_obs int32 in the caller's observation order (host).
 * Synchronises the stream. */
gbp_status gbp_get_relin_iters(const gbp_graph* g, int32_t* tlin);

/* Kernel timing.  ms_out[0]: mean device time per iteration in the current
 * launch mode (n_iters iterations from reset, CUDA events on the graph's
 * stream).  ms_out[1]: mean device time of one factor-kernel launch (phase
 * A alone), replayed n_iters times as a CUDA graph with its outputs sent to
 * scratch buffers so that every launch does the same work.  The graph is
 * reset to iteration 0 afterwards (as gbp_reset()).  Synchronises. */
gbp_status gbp_profile_iterations(gbp_graph* g, int32_t n_iters, double* ms_out);

/* Autotuner: run n_trial iterations from the current state in every
 * candidate launch configuration, timing each with CUDA events after one
 * untimed run, restoring the state after each, and remember the fastest for
 * launch_mode = 0 and shapes = -1.  The candidates change no summation
 * order, so every one gives bitwise identical results: the launch mode
 * (persistent or per phase) and, for the FP32 fixed schedule, the factor
 * kernel's threads per block and register budget and the persistent
 * kernel's register budget.  The warp tile (up to 32 factors, whole
 * landmarks) is not tuned: it decides which landmarks are summed across
 * tiles, and so the arithmetic.  *chosen (nullable) receives the chosen
 * mode; ms_out (nullable, 2 doubles) the best mean time per iteration of
 * modes 1 and 2 (-1: no candidate of that mode could launch, e.g. a
 * persistent grid that does not fit).  gbp_get_tuning reports every
 * candidate.  Synchronises the stream. */
gbp_status gbp_autotune(gbp_graph* g, int32_t n_trial, int32_t* chosen, double* ms_out);

#define GBP_MAX_TUNING_CANDIDATES 12
typedef struct {
    int32_t launch_mode;            /* chosen: 1 persistent, 2 per phase (0: not tuned yet)        */
    int32_t factor_shape;           /* chosen factor-kernel shape (see gbp_params)                 */
    int32_t persistent_shape;       /* chosen persistent-kernel shape                              */
    int32_t factor_threads;         /* threads per block of the chosen factor-kernel shape         */
    int32_t factor_min_blocks;      /* its blocks-per-SM register budget (1 = none)                */
    int32_t persistent_min_blocks;  /* the persistent kernel's (1 = none)                          */
    int32_t tile_factors;           /* factors per warp tile (fixed, see gbp_autotune)             */
    int32_t n_candidates;           /* candidates timed by the last gbp_autotune                   */
    int32_t cand_mode[GBP_MAX_TUNING_CANDIDATES];
    int32_t cand_shape[GBP_MAX_TUNING_CANDIDATES];
    double  cand_ms[GBP_MAX_TUNING_CANDIDATES];   /* mean ms per iteration, -1: could not launch  */
} gbp_tuning;

/* The launch configuration in use and the candidates of the last
 * gbp_autotune (n_candidates = 0 before the first). */
gbp_status gbp_get_tuning(const gbp_graph* g, gbp_tuning* out);

/* ------------------------------------------------------------------------
 * One graph split across ranks (GPUs).  The paper runs one graph on one
 * IPU and points to multi-chip scaling as the way forward (Sec. 10); here
 * each rank holds the whole graph's layout but forms the messages of the
 * factors of its landmarks and the beliefs of its keyframes and landmarks,
 * and per iteration exchanges, host-staged, the boundary records:
 *   1. gbp_split_phase(g, 0)  -- the factor phase of iteration t (Sec. 5) on
 *      this rank's factors;
 *   2. message records (kind 0) of this rank's factors whose keyframe
 *      another rank owns go to that owner (gbp_get_split_records there,
 *      gbp_put_split_records on the owner);
 *   3. gbp_split_phase(g, 1)  -- the belief phase for this rank's keyframes
 *      and landmarks (closes iteration t);
 *   4. keyframe records (kind 1) of this rank's keyframes that other ranks'
 *      factors observe go to those ranks.
 * Every keyframe then sums exactly the messages the whole graph would, in
 * the same order, so the split run gives the whole graph's bits (FP32 path,
 * fixed damping schedule).  Landmarks must be numbered so that each rank's
 * are contiguous.  ------------------------------------------------------- */
#define GBP_SPLIT_MSG_FLOATS 20   /* kind 0: a factor's compact message to its keyframe (8) and Jacobian block (12) */
#define GBP_SPLIT_KF_FLOATS 56    /* kind 1: a keyframe's belief record                                          */

/* Keyframes [kf_begin, kf_end) and landmarks [lm_begin, lm_end) are this
 * graph's part (lm_end < 0: the whole graph again).  Rebuilds the layout (its
 * tiles break at the landmark range) and resets to iteration 0; gbp_iterate
 * then refuses (GBP_ESTATE) until the partition is removed.  GBP_ESTATE for
 * a batch or the FP64 mode; GBP_EINVAL for ranges out of bounds. */
gbp_status gbp_set_partition(gbp_graph* g, int32_t kf_begin, int32_t kf_end, int32_t lm_begin, int32_t lm_end);
/* phase 0: the factor phase of the current iteration on this part's
 * factors; phase 1: the belief phase of this part's variables, which closes
 * the iteration.  Asynchronous on the graph's stream. */
gbp_status gbp_split_phase(gbp_graph* g, int32_t phase);
/* Read (get) or write (put) n records, host float arrays of n x
 * GBP_SPLIT_MSG_FLOATS (kind 0, index = caller observation indices; valid
 * between phase 0 and phase 1) or n x GBP_SPLIT_KF_FLOATS (kind 1, index =
 * keyframes; after phase 1).  Synchronise the stream. */
gbp_status gbp_get_split_records(const gbp_graph* g, int32_t kind, int32_t n, const int32_t* index, float* out);
gbp_status gbp_put_split_records(gbp_graph* g, int32_t kind, int32_t n, const int32_t* index, const float* in);

void gbp_destroy_graph(gbp_graph* g);

/* Largest n_obs that gbp_reprojection_error_noalloc() accepts. */
#define GBP_NOALLOC_MAX_OBS (1 << 20)

/* Average reprojection error of caller-owned DEVICE arrays, computed without
 * allocating any memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need the
 * number -- for example a real-time loop that reserves all device memory at
 * start-up and must not pay cudaMalloc's device-wide synchronisation later,
 * or an application whose own allocator owns all device memory.
 *   intr      pinhole intrinsics (host pointer)
 *   z_min     observations whose point lies closer than z_min to the camera
 *             are left out of the average
 *   n_kf, kf_Rt   device, n_kf x 12 doubles (R row-major, t; world to camera)
 *   n_lm, lm_xyz  device, n_lm x 3 doubles
 *   obs_kf, obs_lm  device, n_obs int32 indices; an observation whose
 *             keyframe or landmark index is out of range is left out of the
 *             average (its arrays are never read through it)
 *   obs_uv    device, n_obs x 2 doubles (pixels)
 *   out       device, 2 doubles: out[0] = mean |z - pi(R l + t)| in pixels,
 *             out[1] = number of observations averaged
 *   cuda_stream  stream to run on (NULL = legacy default stream); the call
 *             is asynchronous on it.
 * Scratch: a fixed 64 KiB array in the library's device memory, present on
 * every GPU that loads the library until the process exits; no cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on a
 * device looks up that array's device address and caches it for the rest of
 * the process (make that first call before any stream capture; after a
 * cudaDeviceReset of that device the cached address is stale, so do not
 * call this entry point on it again in the same process).  All calls share
 * the array and it keeps the last call's partial sums, so calls whose
 * kernels overlap on the GPU (different streams, or several host threads)
 * race and must be serialised by the caller.
 * GBP_EINVAL: a negative count, n_obs > GBP_NOALLOC_MAX_OBS (the scratch
 * array's capacity), or a required pointer is NULL.  GBP_ECUDA: no device or
 * a launch failed. */
gbp_status gbp_reprojection_error_noalloc(const gbp_intrinsics* intr, double z_min, int32_t n_kf, const double* kf_Rt,
                                          int32_t n_lm, const double* lm_xyz, int32_t n_obs, const int32_t* obs_kf,
                                          const int32_t* obs_lm, const double* obs_uv, double* out,
                                          void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned damping network.  The paper damps every message with one fixed d
 * (Sec. 5, d = 0.4 in Sec. 8); this extension predicts a per-factor d in
 * (0, 0.9) from 16 features of the factor's recent messages with a small
 * MLP (16 -> 64 -> 64 -> 1, ReLU hidden layers, output 0.9 * sigmoid), and
 * trains it on targets recorded from GBP runs.  It has no counterpart in the
 * paper.  Damping never changes GBP's fixed point, so the learned path ends
 * at the same beliefs as fixed damping.
 *
 * Parameters: one flat float32 vector of GBP_MLP_NPARAM values, in order
 * W1 [16][64] (row = input feature), b1 [64], W2 [64][64] (row = input
 * unit), b2 [64], W3 [64], b3 [1]; layer l computes h_l = relu(h_{l-1} W_l +
 * b_l).  Arithmetic: weights and activations rounded to BF16, products on
 * tensor cores (mma.sync m16n8k16) accumulated in FP32; master weights, Adam
 * moments and gradients in FP32.
 * ------------------------------------------------------------------------ */
#define GBP_MLP_NFEAT 16
#define GBP_MLP_NPARAM 5313

typedef struct gbp_mlp gbp_mlp;

/* Create a network with the given host parameters (GBP_MLP_NPARAM floats,
 * all finite, else GBP_EINVAL); Adam moments start at zero.  All device
 * memory is owned by the network; work goes on cuda_stream (NULL = legacy
 * default stream). */
gbp_status gbp_mlp_create(const float* params, void* cuda_stream, gbp_mlp** out);
/* Replace the parameters (host, GBP_MLP_NPARAM floats) and zero the Adam
 * state and step count. */
gbp_status gbp_mlp_set_params(gbp_mlp* net, const float* params);
/* Copy the FP32 master parameters to the host.  Synchronises the stream. */
gbp_status gbp_mlp_get_params(const gbp_mlp* net, float* params);
/* Predictions for count rows of DEVICE features X (count x 16 floats,
 * row-major) into DEVICE y (count floats).  Asynchronous on the stream. */
gbp_status gbp_mlp_forward(gbp_mlp* net, const float* X, int32_t count, float* y);
/* Mean-squared-error loss over count rows of DEVICE X (count x 16) against
 * DEVICE targets (count floats), and its gradient with respect to the flat
 * parameters, written to HOST grad (GBP_MLP_NPARAM floats) and *loss
 * (nullable).  Partial sums are added in a fixed order, so the result is
 * reproducible.  Synchronises the stream. */
gbp_status gbp_mlp_gradient(gbp_mlp* net, const float* X, const float* target, int32_t count, float* grad,
                            double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; Kingma
 * and Ba 2015) at learning rate lr on the mean-squared-error loss of a
 * minibatch: rows idx[0..count) (DEVICE int32, nullable = rows 0..count) of
 * DEVICE X and target.  *loss_out (nullable, host) receives the minibatch
 * loss before the step and then the call synchronises; with loss_out NULL
 * the call is asynchronous. */
gbp_status gbp_mlp_train_step(gbp_mlp* net, const float* X, const float* target, const int32_t* idx,
                              int32_t count, float lr, float* loss_out);
void gbp_mlp_destroy(gbp_mlp* net);

/* Give graph g its own copy of the network's current weights (later
 * training of net does not affect g until the next call); NULL removes it.
 * With damping_mode = 1 each factor's eta messages are damped by the
 * network's prediction d_f in place of d:
 *   eta_{f->v} = (1 - d_f) eta_new + d_f eta_old,  Lambda undamped (Sec. 5),
 * wherever the fixed schedule damps (after the undamped_iters hold that
 * follows a (re)linearisation, Sec. 8).  d_f comes from 16 features of the
 * factor: its Mahalanobis residual and Huber weight (Sec. 6), how much of
 * each variable's incoming precision it supplies, for each of its two
 * messages the relative change over the last 3 iterations and the cosine
 * between the proposed and the previous step (oscillation or steady
 * progress), the two variables' degrees, and the iterations since its
 * linearisation and since its landmark appeared.  The per-factor history
 * behind these features is kept only while damping_mode = 1 or while
 * recording, and restarts from zero on gbp_reset.  Iterating with
 * damping_mode = 1 and no network gives GBP_ESTATE. */
gbp_status gbp_set_damping_model(gbp_graph* g, const gbp_mlp* net);

/* Training data for the network.  gbp_capture_messages stores the graph's
 * current messages as the reference (normally after running to
 * convergence); gbp_record_iterations then runs n_iters iterations from the
 * current state with the fixed damping schedule and writes, per iteration i
 * and factor f (the library's internal factor order, row i * n_obs + f):
 *   X[row * 16 + j]  the 16 features above (DEVICE, 16-byte aligned,
 *                    n_iters * n_obs * 16 floats)
 *   target[row]      the d in [0, 0.9] minimising, over the message sides
 *                    s whose eta changed,
 *                    sum_s |(1 - d) eta_new,s + d eta_old,s - eta_ref,s|^2
 *                          / |eta_old,s - eta_new,s|^2
 *                    (eta_new undamped, eta_old the previous message,
 *                    eta_ref the captured reference); -1 where the schedule
 *                    does not damp (the hold after a relinearisation), for
 *                    a factor behind the camera, or where neither message
 *                    changed (DEVICE, n_iters * n_obs floats).
 * GBP_ESTATE without a captured reference (also after gbp_add_keyframe,
 * which drops it).  Synchronises the stream. */
gbp_status gbp_capture_messages(gbp_graph* g);
/* The caller's observation index of each of the library's internal factors
 * (n_obs int32, host): the row order of gbp_record_iterations. */
gbp_status gbp_get_factor_order(const gbp_graph* g, int32_t* obs_index);
gbp_status gbp_record_iterations(gbp_graph* g, int32_t n_iters, float* X, float* target);

const char* gbp_status_string(gbp_status s);
const char* gbp_last_error(const gbp_graph* g);

#ifdef __cplusplus
}
#endif
#endif
