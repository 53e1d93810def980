// gbp_noalloc.cu -- average reprojection error of caller-owned device arrays
// without any device allocation.
//
// This is a variant of the library's metrics reduction (per-observation
// reprojection error, per-block partial sums, one fixed-order final sum) for
// callers that cannot allocate device memory at the point where they need
// the number: for example a real-time tracking loop that reserves all of its
// device memory at start-up and must never hit cudaMalloc's device-wide
// synchronisation and unbounded latency afterwards, or a host application
// whose own allocator owns every byte of device memory.  Such callers pass
// their inputs and an output slot; the per-block partials live in the
// fixed-size device array below, which every GPU that loads the library keeps
// until the process exits.
#include "../../include/gbp.h"

#include <cuda_runtime.h>

#include <atomic>

namespace {

constexpr int NOALLOC_BLOCK = 256;
constexpr int NOALLOC_MAX_BLOCKS = GBP_NOALLOC_MAX_OBS / NOALLOC_BLOCK;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Partial sums: slot b holds block b's error sum, slot NOALLOC_MAX_BLOCKS + b
// its count.  Shared by every call on a device; each call overwrites exactly
// the slots it later reads.
static __device__ __align__(256) double g_are_scratch[2 * NOALLOC_MAX_BLOCKS];

// Device address of g_are_scratch per device, looked up once per device.
// Several host threads may make their first call on a device at once: each
// looks the address up and stores the same value, so relaxed atomics suffice.
static std::atomic<double*> g_scratch_addr[NOALLOC_MAX_DEVICES];

__global__ void __launch_bounds__(NOALLOC_BLOCK)
are_partials_kernel(double fx, double fy, double cx, double cy, double z_min, int32_t n_kf,
                    const double* __restrict__ kf_Rt, int32_t n_lm, const double* __restrict__ lm_xyz, int32_t n_obs,
                    const int32_t* __restrict__ obs_kf, const int32_t* __restrict__ obs_lm,
                    const double* __restrict__ obs_uv, double* scratch) {
    __shared__ double red[2][NOALLOC_BLOCK];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * NOALLOC_BLOCK + tid;
    double e = 0.0, c = 0.0;
    // an observation whose indices are out of range is left out, never read through
    const int k = i < n_obs ? obs_kf[i] : -1;
    const int m = i < n_obs ? obs_lm[i] : -1;
    if (k >= 0 && k < n_kf && m >= 0 && m < n_lm) {
        const double* Rt = kf_Rt + 12 * (size_t)k;
        const double* X = lm_xyz + 3 * (size_t)m;
        double p0 = Rt[0] * X[0] + Rt[1] * X[1] + Rt[2] * X[2] + Rt[9];
        double p1 = Rt[3] * X[0] + Rt[4] * X[1] + Rt[5] * X[2] + Rt[10];
        double p2 = Rt[6] * X[0] + Rt[7] * X[1] + Rt[8] * X[2] + Rt[11];
        if (p2 >= z_min) {
            double du = obs_uv[2 * (size_t)i] - (fx * p0 / p2 + cx);
            double dv = obs_uv[2 * (size_t)i + 1] - (fy * p1 / p2 + cy);
            e = sqrt(du * du + dv * dv);
            c = 1.0;
        }
    }
    red[0][tid] = e;
    red[1][tid] = c;
    __syncthreads();
    for (int st = NOALLOC_BLOCK / 2; st > 0; st >>= 1) {
        if (tid < st) {
            red[0][tid] += red[0][tid + st];
            red[1][tid] += red[1][tid + st];
        }
        __syncthreads();
    }
    if (tid == 0) {
        scratch[blockIdx.x] = red[0][0];
        scratch[NOALLOC_MAX_BLOCKS + blockIdx.x] = red[1][0];
    }
}

__global__ void __launch_bounds__(NOALLOC_BLOCK) are_finish_kernel(const double* scratch, int nb, double* out) {
    __shared__ double red[2][NOALLOC_BLOCK];
    const int tid = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int b = tid; b < nb; b += NOALLOC_BLOCK) {
        s += scratch[b];
        c += scratch[NOALLOC_MAX_BLOCKS + b];
    }
    red[0][tid] = s;
    red[1][tid] = c;
    __syncthreads();
    for (int st = NOALLOC_BLOCK / 2; st > 0; st >>= 1) {
        if (tid < st) {
            red[0][tid] += red[0][tid + st];
            red[1][tid] += red[1][tid + st];
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[0] = red[1][0] > 0.0 ? red[0][0] / red[1][0] : 0.0;
        out[1] = red[1][0];
    }
}

}  // namespace

extern "C" gbp_status gbp_reprojection_error_noalloc(const gbp_intrinsics* intr, double z_min, int32_t n_kf,
                                                     const double* kf_Rt, int32_t n_lm, const double* lm_xyz,
                                                     int32_t n_obs, const int32_t* obs_kf, const int32_t* obs_lm,
                                                     const double* obs_uv, double* out, void* cuda_stream) {
    if (!intr || !out || n_obs < 0 || n_kf < 0 || n_lm < 0) return GBP_EINVAL;
    if (n_obs > GBP_NOALLOC_MAX_OBS) return GBP_EINVAL;   // more observations than the scratch array holds
    if (n_obs > 0 && (!kf_Rt || !lm_xyz || !obs_kf || !obs_lm || !obs_uv)) return GBP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return GBP_ECUDA;
    // one-time set-up on this device: host code needs the scratch array's
    // device address (its name in host code is only a host-side stand-in)
    double* scratch = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (!scratch) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_are_scratch) != cudaSuccess || !p) return GBP_ECUDA;
        scratch = static_cast<double*>(p);
        g_scratch_addr[dev].store(scratch, std::memory_order_relaxed);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    (void)cudaGetLastError();   // an error left by an unrelated earlier call is not this call's to report
    const int nb = (n_obs + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK;
    if (nb > 0)
        are_partials_kernel<<<nb, NOALLOC_BLOCK, 0, s>>>(intr->fx, intr->fy, intr->cx, intr->cy, z_min, n_kf, kf_Rt,
                                                         n_lm, lm_xyz, n_obs, obs_kf, obs_lm, obs_uv, scratch);
    are_finish_kernel<<<1, NOALLOC_BLOCK, 0, s>>>(scratch, nb, out);
    return cudaGetLastError() == cudaSuccess ? GBP_OK : GBP_ECUDA;
}
