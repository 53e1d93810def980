// gbp_internal.h -- device-side data layout shared by the kernels and the
// host side of libgbp (not part of the public ABI).
//
// Layout in HBM (n_f factors sorted by landmark then keyframe):
//   per factor, static:   z (2 Real), fk, fm (int32)
//   per factor, dynamic:  x0  -- linearisation point [dc dw | dl], 9 Real, SoA (9 x n_f)
//                         tlin -- iteration of the last (re)linearisation, int32
//                         mk  -- message to the keyframe, AoS record of KREC Real:
//                                Lambda packed lower 6x6 (21), eta (6), pad
//                         ml  -- message to the landmark, SoA (9 x n_f):
//                                Lambda packed lower 3x3 (6), eta (3)
//   per keyframe:         Rref (9 double), cref (3 double), prior diagonal D (6),
//                         anchor diagonal (6), belief record KBEL Real:
//                                Lambda (21), eta (6), mu (6), pad
//   per landmark:         lref (3 double), prior diagonal (3), belief record
//                         LBEL Real: Lambda (6), eta (3), mu (3)
//   CSR keyframe -> factor list (kf_off, kf_list); landmark -> contiguous
//   factor range (lm_off), since factors are sorted by landmark.
// Packed symmetric storage: element (i, j), j <= i, at i*(i+1)/2 + j.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbp {

constexpr int KREC = 28;   // keyframe message record (Real elements)
constexpr int KBEL = 36;   // keyframe belief record
constexpr int LBEL = 12;   // landmark belief record

struct KParams {
    double fx, fy, cx, cy;
    double inv_sigma2;        // 1 / sigma^2
    double inv_sigma;         // 1 / sigma
    double huber_n;           // <= 0 disables
    double damping;
    double z_min;
    double relin_beta;
    double anchor_scale;
    double pivot_ratio;
    double prior_final;       // final prior scale
    int32_t relin_interval;
    int32_t damp_hold;        // damping applies when t - tlin >= damp_hold (>= 1)
    int32_t prior_anneal;
    int32_t linear;
    int32_t fallback;         // FP32 path: redo ill-conditioned factorisations in FP64
};

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
    const int32_t* kf_off;    // n_kf + 1
    const int32_t* kf_list;   // n_f
    const int32_t* lm_off;    // n_lm + 1
    const R* kf_D;            // n_kf x 6, prior diagonal at sigma = 1
    const R* kf_A;            // n_kf x 6, anchor diagonal at sigma = 1 (0 = not anchored)
    const R* lm_D;            // n_lm x 3
    const R* uv_ref;          // 2 x n_f reference projections or nullptr
    // dynamic
    R* x0;                    // 9 x n_f
    int32_t* tlin;            // n_f
    R* mk;                    // n_f x KREC   (read by the factor kernel)
    R* ml;                    // 9 x n_f      (read by the factor kernel)
    R* mk_out;                // where the factor kernel writes m^{t+1} (normally == mk)
    R* ml_out;                // (normally == ml)
    R* kf_bel;                // n_kf x KBEL
    R* lm_bel;                // n_lm x LBEL
    // control block
    int32_t* ctl;             // see Ctl
};

// int32 slots of the device control block
enum Ctl : int {
    CTL_ITER = 0,          // completed iterations
    CTL_DONE = 1,          // blocks finished in the current belief launch
    CTL_DMU_ACC = 2,       // running max |dmu| (float bits), current iteration
    CTL_DMU_LAST = 3,      // max |dmu| of the last completed iteration (float bits)
    CTL_FALLBACKS = 4,     // FP64 redo count
    CTL_RELINS = 5,        // relinearisation count
    CTL_ERR = 6,           // nonzero: a belief lost positive definiteness / became non-finite
    CTL_ERR_WHERE = 7,     // first variable / factor index that raised CTL_ERR
    CTL_N = 16
};

// metrics reduction output (double slots)
enum Met : int { MET_ARE = 0, MET_ARE_REF = 1, MET_N_ARE = 2, MET_HUBER = 3, MET_N = 4 };

constexpr int FACTOR_BLOCK = 128;
constexpr int BELIEF_BLOCK = 128;
constexpr int METRIC_BLOCK = 256;

// kernel launchers (gbp_kernels.cu)
template <typename R> cudaError_t launch_factor(const DevGraph<R>& g, const KParams& p, cudaStream_t s);
template <typename R> cudaError_t launch_belief(const DevGraph<R>& g, const KParams& p, cudaStream_t s);
template <typename R> cudaError_t launch_prior(const DevGraph<R>& g, const KParams& p, R* tmp_k, R* tmp_l,
                                               R* kf_D, R* lm_D, cudaStream_t s);
template <typename R> cudaError_t launch_metrics(const DevGraph<R>& g, const KParams& p, double* partials,
                                                 int n_partials, double* out, cudaStream_t s);
int metrics_blocks(int n_f);

}  // namespace gbp
