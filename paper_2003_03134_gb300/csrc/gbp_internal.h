// gbp_internal.h -- device-side data layout shared by the kernels and the
// host side of libgbp (not part of the public ABI).
//
// A reprojection factor's information is rank 2 (Sec. 4: Lambda_f = W J^T J,
// eta_f = W J^T y), and so is each of its two messages: every message is
// stored in the exact compact form Lambda = J_v^T M J_v, eta = J_v^T g with
// M a symmetric 2 x 2 and g a 2-vector, J_v the factor's Jacobian block of
// the receiving variable at the factor's current linearisation point.
//
// Layout in HBM (n_f factors sorted by landmark then keyframe):
//   per factor, static:   z (2 Real), fk, fm, kpos (int32)
//   per factor, dynamic:  x0  -- linearisation point [dc dw | dl], 9 Real, SoA (9 x n_f)
//                         tlin -- iteration of the last (re)linearisation, int32
//                         lin -- that linearisation: y = J x0 + r (2), Huber-
//                                weighted W (Sec. 6), |r|^2; SoA (NLIN x n_f)
//                         ml  -- message to the landmark, compact, SoA (NML x n_f):
//                                M00 M01 M11 g0 g1
//                         mlx -- the same expanded (Lambda 6, eta 3), SoA 9 x n_f,
//                                written only for factors of landmarks split
//                                across tiles (read by the belief phase)
//   per factor, in keyframe CSR order (slot kpos[f], so that a keyframe's
//   records are contiguous):
//                         mk  -- message to the keyframe, compact record of KREC
//                                Real: M00 M01 M11 g0 g1, t_lin of the
//                                linearisation it was formed at (int bits),
//                                pad; two buffers, alternating by iteration
//                                parity
//                         kj  -- the keyframe Jacobian block (2 x 6) of the
//                                factor's current linearisation, which both
//                                of its messages are expressed in
//                         kjs -- staging: the new block of factors
//                                (re)linearised in this iteration (the
//                                belief phase moves it into kj)
//   per keyframe:         Rref (9 double), cref (3 double), prior diagonal D (6),
//                         anchor diagonal (6), belief record KBEL Real:
//                                Cholesky factor of Lambda (packed lower, 1/L_ii
//                                on the diagonal) 21, mu 6, tr Lambda 1 -- the
//                                part the factor phase reads -- then
//                                Lambda 21, eta 6, pad
//   per landmark:         lref (3 double), prior diagonal (3), belief record
//                         LBEL Real: Lambda (6), eta (3), mu (3)
//   per factor, learned damping: hist -- relative message changes of the
//                                last 2 iterations and the previous landmark
//                                message eta, float SoA (HIST x n_f)
//   CSR keyframe -> factor list (kf_off, kf_list); landmark -> contiguous
//   factor range (lm_off), since factors are sorted by landmark; warp tiles
//   of whole landmarks (tile_start); per-variable arrival counters.
// Packed symmetric storage: element (i, j), j <= i, at i*(i+1)/2 + j.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct gbp_mlp;

namespace gbp {

constexpr int KREC = 8;    // compact keyframe message record (Real elements)
constexpr int KREC_TL = 5; // its slot holding t_lin of the record's linearisation (int bits)
constexpr int KJ = 12;     // keyframe Jacobian block record: row 0 (6), row 1 (6)
constexpr int NML = 5;     // compact landmark message (SoA rows)
constexpr int NLIN = 4;    // per-factor linearisation record (SoA rows): y0, y1, W, |r|^2
// keyframe belief record
constexpr int KB_L = 0;    // Cholesky factor of Lambda, packed lower, 1/L_ii on the diagonal (21)
constexpr int KB_MU = 21;  // mean (6)
constexpr int KB_TR = 27;  // trace of Lambda
constexpr int KB_A = 28;   // the factor phase reads [0, KB_A)
constexpr int KB_LAM = 28; // Lambda, packed lower (21)
constexpr int KB_ETA = 49; // eta (6)
constexpr int KBEL = 56;
constexpr int LBEL = 12;   // landmark belief record

// Solver parameters as the kernels see them, in the kernel's own precision
// (no double-to-float conversions in the hot loop).
template <typename R>
struct KParams {
    R fx, fy, cx, cy;
    R inv_sigma2;             // 1 / sigma^2
    R inv_sigma;              // 1 / sigma
    R huber_n;                // <= 0 disables
    R damping;
    R z_min;
    R relin_beta;
    R anchor_scale;
    R pivot_ratio;
    R cav_ratio;              // FP32 path: a keyframe cavity keeping less than this share of its belief's
                              // precision volume (det(I - M G)) is formed again in FP64
    const R* prior_s;         // device table: prior scale at iteration t is prior_s[min(t, prior_T)]
    int32_t prior_T;
    int32_t relin_interval;
    int32_t damp_hold;        // damping applies when t - tlin >= damp_hold (>= 1)
    int32_t linear;
    int32_t fallback;         // FP32 path: redo ill-conditioned factorisations in FP64
    int32_t exact_cavity;     // FP32 path: FP64 keyframe cavities always summed from their parts
    // learned damping (network weights packed by gbp_mlp.cu)
    const uint32_t* mlp_frag; // BF16 B-operand fragments of layers 1-3
    const float* mlp_bias;    // b1 (64), b2 (64), b3, pad, W3 (64)
};

// Damping schedules (kernel template argument).
enum DampMode : int {
    DAMP_FIXED = 0,    // d of Sec. 5 after the undamped hold of Sec. 8
    DAMP_LEARNED = 1,  // per-factor d from the network, from the second iteration after a (re)linearisation
    DAMP_RECORD = 2    // fixed schedule; features and damping targets written to rec_X / rec_T
};
constexpr int N_FEAT = 16;
constexpr int HIST = 8;   // per-factor history floats: |d eta| at t-1, t-2 (kf, lm), landmark eta of t-1, pad

template <typename R>
struct DevGraph {
    int32_t n_kf, n_lm, n_f;
    // static
    const R* z;               // 2 x n_f interleaved (u, v)
    const int32_t* fk;
    const int32_t* fm;
    const double* kf_R;       // n_kf x 9
    const double* kf_c;       // n_kf x 3
    const double* lm_ref;     // n_lm x 3
    const R* kf_Rr;           // n_kf x 9: kf_R rounded to R (the linearisation's reference rotation)
    const R* f_dlc;           // 3 x n_f: lm_ref[m] - kf_c[k] of each factor, subtracted in double and
                              // rounded to R (the large world coordinates cancel there)
    const int32_t* kf_off;    // n_kf + 1
    const int32_t* kf_list;   // n_f
    const int32_t* kpos;      // n_f: slot of factor f's keyframe message = its position in kf_list
    const int32_t* lm_off;    // n_lm + 1
    const int32_t* tile_start;// n_tiles + 1: warp tiles of whole landmarks (<= 32 factors each)
    const int32_t* big_lm;    // landmarks split across tiles (more than 32 factors)
    int32_t* deferred;        // n_tiles: tiles left to factor_deferred_kernel in this iteration
    const int32_t* orphan;    // variables without factors: keyframe v, or n_kf + landmark
    int32_t n_tiles, n_big, n_orphan;
    // the part of the graph a launch covers (the whole graph unless it is
    // split across ranks): tiles [tile_off, tile_off + n_tiles) -- n_tiles
    // counts them -- and belief items: keyframes [kf_item_off, + kf_item_n),
    // split landmarks big_lm[big_item_off, + big_item_n), every orphan
    int32_t tile_off, kf_item_off, kf_item_n, big_item_off, big_item_n;
    int32_t b_warps;          // warps per belief-phase item: 4 (a block) for small graphs, else 1
    const int32_t* kf_birth;  // n_kf: iteration at which the keyframe was added (prior anneal start)
    const int32_t* lm_birth;  // n_lm
    const R* kf_D;            // n_kf x 6, prior diagonal at sigma = 1
    const R* kf_A;            // n_kf x 6, anchor diagonal at sigma = 1 (0 = not anchored)
    const R* lm_D;            // n_lm x 3
    const R* uv_ref;          // 2 x n_f reference projections or nullptr
    // dynamic
    R* x0;                    // 9 x n_f
    int32_t* tlin;            // n_f
    R* mk;                    // n_f x KREC, messages of even iterations (slot order)
    R* mk2;                   // n_f x KREC, messages of odd iterations
    R* mk_redirect;           // if set, receives the keyframe-message writes (kernel timing)
    R* kj;                    // n_f x KJ, Jacobian blocks of the current keyframe messages (slot order)
    R* lin;                   // NLIN x n_f: y0, y1, W, |r|^2 of each factor's current linearisation
    R* kjs;                   // n_f x KJ, staging for factors (re)linearised in this iteration
    R* ml;                    // NML x n_f    (read by the factor kernel)
    R* ml_out;                // where the factor kernel writes m^{t+1} (normally == ml)
    R* mlx;                   // 9 x n_f expanded landmark messages of split landmarks' factors
    R* kf_bel;                // n_kf x KBEL  (read as b^t)
    R* lm_bel;                // n_lm x LBEL  (read as b^t)
    R* kf_bel_out;            // where b^{t+1} is written (normally == kf_bel)
    R* lm_bel_out;            // (normally == lm_bel)
    // learned damping
    float* hist;              // HIST x n_f: message-change history of the learned schedule
    const R* eta_inf;         // record: 9 x n_f reference messages eta (kf side 6, lm side 3)
    float* rec_X;             // record: n_f x 16 features of the current iteration
    float* rec_T;             // record: n_f damping targets (-1: a sample the learned schedule never uses)
    // control block
    int32_t* ctl;             // see Ctl
};

// int32 slots of the device control block
enum Ctl : int {
    CTL_ITER = 0,          // completed iterations
    CTL_DONE = 1,          // (unused)
    CTL_DMU_ACC = 2,       // running max |dmu| (float bits) of even iterations
    CTL_DMU_LAST = 3,      // persistent kernel: max |dmu| of the last iteration it ran (float bits)
    CTL_FALLBACKS = 4,     // FP64 redo count
    CTL_RELINS = 5,        // relinearisation count
    CTL_ERR = 6,           // 1: a belief lost positive definiteness / became non-finite; 2: barrier timeout
    CTL_ERR_WHERE = 7,     // first variable / factor index that raised CTL_ERR = 1
    CTL_DMU_ACC1 = 8,      // running max |dmu| of odd iterations
    CTL_BAR_COUNT = 9,     // grid barrier arrivals
    CTL_BAR_GEN = 10,      // grid barrier generation
    CTL_ITERS_RUN = 11,    // iterations run by the last persistent launch
    CTL_HELD = 12,         // messages left at their previous value (incoming precision not positive definite)
    CTL_ITER_B = 13,       // per-phase launches: the iteration the belief kernel closes (set by the factor kernel)
    CTL_DEFER_N0 = 14,     // tiles listed for factor_deferred_kernel in even iterations
    CTL_DEFER_N1 = 15,     // in odd iterations
    CTL_DEFER_DONE = 16,   // blocks of factor_deferred_kernel done (its last block clears the list)
    CTL_RESUMS = 17,       // keyframe incoming precisions summed again exactly from their parts (FP64)
    CTL_N = 20
};

// metrics reduction output (double slots)
enum Met : int { MET_ARE = 0, MET_ARE_REF = 1, MET_N_ARE = 2, MET_HUBER = 3, MET_N = 4 };

constexpr int FACTOR_BLOCK = 128;   // 4 warps per block (every kernel of the iteration)
constexpr int METRIC_BLOCK = 256;

// kernel launchers (gbp_kernels.cu)
// pdl: programmatic dependent launch (the kernel may start while the
// previous kernel in the stream finishes; it waits for that kernel's writes)
// shape: the FP32 fixed schedule's factor-kernel launch shape (autotuned):
// 0 128 threads, no register budget; 1 128 threads, >= 3 blocks per SM;
// 2 128 threads, >= 4 blocks per SM; 3 64 threads, no budget; 4 and 5: 128
// threads, >= 4 or >= 3 blocks per SM, with tiles that need the FP64 redo
// deferred to factor_deferred_kernel (launched right after)
constexpr int N_FACTOR_SHAPES = 6;
constexpr int N_PERSISTENT_SHAPES = 1;   // no register budget
template <typename R> cudaError_t launch_factor(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s,
                                                int mode = DAMP_FIXED, bool pdl = false, int shape = 0);
// The previous layout's per-factor state, for relayout_kernel (incremental
// SLAM): src_f maps the new layout's factors to the previous internal
// indices (-1: a factor of the new keyframe).
template <typename R>
struct RelayoutSrc {
    const int32_t* src_f;
    int32_t n_f, n_lm, t;
    const R* x0;
    const int32_t* tlin;
    const R* ml;
    const R* lin;
    const float* hist;
    const int32_t* kpos;
    const R* kj;
    const R* mk_cur;          // m^t, slot order
    const R* mk_oth;          // m^{t-1}
    const R* lm_bel;
};
template <typename R> cudaError_t launch_relayout(const DevGraph<R>& nw, const RelayoutSrc<R>& o, int phase,
                                                  cudaStream_t s);
template <typename R> cudaError_t launch_init(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s);
template <typename R> cudaError_t launch_belief(const DevGraph<R>& g, const KParams<R>& p, cudaStream_t s,
                                                bool pdl = false);
template <typename R> int persistent_grid(const DevGraph<R>& g, int mode, int shape);   // co-resident blocks; 0 on error
template <typename R> cudaError_t launch_persistent(const DevGraph<R>& g, const KParams<R>& p, int n_iters,
                                                    float conv_tol, int check_every, int grid, cudaStream_t s,
                                                    int mode, int shape);
template <typename R> cudaError_t launch_capture_messages(const DevGraph<R>& g, int t, R* eta_inf, cudaStream_t s);
template <typename R> cudaError_t launch_prior(const DevGraph<R>& g, const KParams<R>& p, R* tmp_k, R* tmp_l,
                                               R* kf_D, R* lm_D, cudaStream_t s);
template <typename R> cudaError_t launch_metrics(const DevGraph<R>& g, const KParams<R>& p, double* partials,
                                                 int n_partials, double* out, cudaStream_t s);
template <typename R> cudaError_t launch_problem_metrics(const DevGraph<R>& g, const KParams<R>& p,
                                                         const int32_t* prob_f0, int n_problems, double* out,
                                                         cudaStream_t s);
template <typename R> cudaError_t launch_residuals(const DevGraph<R>& g, const KParams<R>& p, double* out,
                                                   cudaStream_t s);
template <typename R> cudaError_t launch_split_records(const DevGraph<R>& g, int kind, int put, int n,
                                                       const int32_t* idx, float* io, cudaStream_t s);
int metrics_blocks(int n_f);

// damping network (gbp_mlp.cu): device-to-device copy of a network's packed
// forward weights (FWD_FRAG_WORDS words, MLP_BIAS_WORDS floats), ordered
// after the network's pending work
cudaError_t mlp_copy_packed(const gbp_mlp* net, uint32_t* frag, float* bias, cudaStream_t s);

}  // namespace gbp
