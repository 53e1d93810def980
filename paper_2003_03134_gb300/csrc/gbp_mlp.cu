// gbp_mlp.cu -- training of the per-factor damping network on BF16 tensor
// cores (forward and backward GEMMs with mma.sync m16n8k16, FP32
// accumulation), FP32 master weights and Adam (Kingma and Ba 2015), and the
// C ABI of the gbp_mlp object.
//
// One training step over a batch of B samples:
//   mlp_grad_kernel    one block per 128 samples (4 warps x 32): forward,
//                      backward, this block's partial gradient (warp
//                      partials added in fixed warp order) and loss;
//   mlp_reduce_kernel  one thread per parameter: sum of the block partials in
//                      block order (deterministic), then optionally Adam;
//   mlp_pack_kernel    BF16 B-operand fragments and FP32 biases from the
//                      master weights.
#include "gbp_mlp.cuh"
#include "gbp_internal.h"
#include "../../include/gbp.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace gbp {

static_assert(MLP_NPARAM == GBP_MLP_NPARAM && MLP_IN == GBP_MLP_NFEAT, "parameter layout");

constexpr int MLP_BLOCK = 128;               // samples per block
constexpr int MLP_WARPS = MLP_BLOCK / 32;

// ------------------------------------------------------------------------
// packing: fragment tile t, lane l holds B[2q..2q+1][g] and B[2q+8..2q+9][g]
// of the tile's 16 x 8 sub-matrix of B (K x N).

__device__ __forceinline__ float mlp_b_elem(const float* W, int t, int k, int n) {
    if (t < FT_L2) return W[MLP_OFF_W1 + k * MLP_H + 8 * t + n];                 // W1[k][n]
    if (t < FT_L3) {
        const int ks = (t - FT_L2) / 8, nt = (t - FT_L2) % 8;
        return W[MLP_OFF_W2 + (16 * ks + k) * MLP_H + 8 * nt + n];               // W2[k][n]
    }
    if (t < FT_W2T) {
        const int ks = t - FT_L3;
        return n == 0 ? W[MLP_OFF_W3 + 16 * ks + k] : 0.0f;                      // W3 in column 0
    }
    const int ks = (t - FT_W2T) / 8, nt = (t - FT_W2T) % 8;
    return W[MLP_OFF_W2 + (8 * nt + n) * MLP_H + 16 * ks + k];                   // W2^T[k][n]
}

__global__ void mlp_pack_kernel(const float* __restrict__ W, uint32_t* __restrict__ frag, float* __restrict__ bias) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < FT_N * 32) {
        const int t = i / 32, lane = i % 32, g = lane >> 2, q = lane & 3;
        frag[2 * i] = pack_bf16(mlp_b_elem(W, t, 2 * q, g), mlp_b_elem(W, t, 2 * q + 1, g));
        frag[2 * i + 1] = pack_bf16(mlp_b_elem(W, t, 2 * q + 8, g), mlp_b_elem(W, t, 2 * q + 9, g));
    }
    if (i < MLP_H) {
        bias[i] = W[MLP_OFF_B1 + i];
        bias[MLP_H + i] = W[MLP_OFF_B2 + i];
        bias[2 * MLP_H + 2 + i] = W[MLP_OFF_W3 + i];   // W3 in FP32 for the backward pass
    }
    if (i == 0) bias[2 * MLP_H] = W[MLP_OFF_B3];
}


// ------------------------------------------------------------------------
// forward over samples (inference)

__global__ void __launch_bounds__(MLP_BLOCK) mlp_forward_kernel(const uint32_t* __restrict__ frag_g,
                                                                const float* __restrict__ bias_g,
                                                                const float* __restrict__ X, int n,
                                                                float* __restrict__ y) {
    __shared__ __align__(16) uint32_t frag[FWD_FRAG_WORDS];
    __shared__ float bias[MLP_BIAS_WORDS];
    __shared__ __align__(16) __nv_bfloat16 xs[MLP_WARPS][32 * XS];
    __shared__ __align__(16) __nv_bfloat16 hs[MLP_WARPS][32 * HS];
    for (int i = threadIdx.x; i < FWD_FRAG_WORDS; i += MLP_BLOCK) frag[i] = frag_g[i];
    for (int i = threadIdx.x; i < MLP_BIAS_WORDS; i += MLP_BLOCK) bias[i] = bias_g[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * MLP_BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < MLP_IN; ++j) xs[warp][lane * XS + j] = __float2bfloat16_rn(s < n ? X[(size_t)s * MLP_IN + j] : 0.f);
    __syncthreads();
    const float z3 = mlp_forward_warp(frag, bias, xs[warp], hs[warp], nullptr, lane);
    if (s < n) y[s] = mlp_output(z3);
}

// ------------------------------------------------------------------------
// forward + backward of one block of samples

struct GradSmem {
    uint32_t frag[FRAG_WORDS];
    float bias[MLP_BIAS_WORDS];
    alignas(16) __nv_bfloat16 x[MLP_WARPS][32 * XS];
    alignas(16) __nv_bfloat16 h1[MLP_WARPS][32 * HS];
    alignas(16) __nv_bfloat16 h2[MLP_WARPS][32 * HS];   // h2, later dz1
    alignas(16) __nv_bfloat16 dz[MLP_WARPS][32 * HS];   // dz2
    float dz3[MLP_WARPS][32];
    float gW2[MLP_H * MLP_H];
    float gW1[MLP_IN * MLP_H];
    float gvec[MLP_H * 3 + 1];              // b1, b2, W3, b3 partials
    float loss;
};

__global__ void __launch_bounds__(MLP_BLOCK) mlp_grad_kernel(const uint32_t* __restrict__ frag_g,
                                                             const float* __restrict__ bias_g,
                                                             const float* __restrict__ X, const float* __restrict__ T,
                                                             const int32_t* __restrict__ idx, int n, float inv_batch,
                                                             float* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    for (int i = tid; i < FRAG_WORDS; i += MLP_BLOCK) S.frag[i] = frag_g[i];
    for (int i = tid; i < MLP_BIAS_WORDS; i += MLP_BLOCK) S.bias[i] = bias_g[i];
    for (int i = tid; i < MLP_H * MLP_H; i += MLP_BLOCK) S.gW2[i] = 0.f;
    for (int i = tid; i < MLP_IN * MLP_H; i += MLP_BLOCK) S.gW1[i] = 0.f;
    for (int i = tid; i < MLP_H * 3 + 1; i += MLP_BLOCK) S.gvec[i] = 0.f;
    if (tid == 0) S.loss = 0.f;
    const int si = blockIdx.x * MLP_BLOCK + tid;      // this lane's sample slot
    const bool valid = si < n;
    const int sample = valid ? (idx ? idx[si] : si) : 0;
#pragma unroll
    for (int j = 0; j < MLP_IN; ++j)
        S.x[warp][lane * XS + j] = __float2bfloat16_rn(valid ? X[(size_t)sample * MLP_IN + j] : 0.f);
    __syncthreads();

    // forward, keeping h1 and h2
    const float z3 = mlp_forward_warp(S.frag, S.bias, S.x[warp], S.h2[warp], S.h1[warp], lane);
    // the forward pass reused the input tile: restore it for dW1
#pragma unroll
    for (int j = 0; j < MLP_IN; ++j)
        S.x[warp][lane * XS + j] = __float2bfloat16_rn(valid ? X[(size_t)sample * MLP_IN + j] : 0.f);
    const float sg = 1.0f / (1.0f + __expf(-z3));
    const float y = MLP_DMAX * sg;
    const float r = valid ? y - T[sample] : 0.f;
    // loss = mean r^2 ; dL/dz3 = 2 r / B * 0.9 s (1 - s)
    const float dz3 = 2.0f * r * inv_batch * MLP_DMAX * sg * (1.0f - sg);
    S.dz3[warp][lane] = dz3;
    __syncwarp();
    float r2 = r * r * inv_batch;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);

    // dz2[s][j] = dz3[s] W3[j] [h2 > 0]  (row s = this lane), as BF16
    const float* W3 = S.bias + 2 * MLP_H + 2;
#pragma unroll 8
    for (int j = 0; j < MLP_H; j += 2) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(S.h2[warp] + lane * HS + j);
        const float v0 = __bfloat162float(h.x) > 0.f ? dz3 * W3[j] : 0.f;
        const float v1 = __bfloat162float(h.y) > 0.f ? dz3 * W3[j + 1] : 0.f;
        *reinterpret_cast<uint32_t*>(S.dz[warp] + lane * HS + j) = pack_bf16(v0, v1);
    }
    __syncwarp();
    // vector partials of this warp: dW3[j] = sum_s h2[s][j] dz3[s], db2[j] =
    // sum_s dz2[s][j], db3 = sum_s dz3[s] (lane takes j = lane, lane + 32)
    float pW3[2] = {0.f, 0.f}, pb2[2] = {0.f, 0.f};
    for (int s = 0; s < 32; ++s) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = lane + 32 * h;
            pW3[h] += __bfloat162float(S.h2[warp][s * HS + j]) * S.dz3[warp][s];
            pb2[h] += __bfloat162float(S.dz[warp][s * HS + j]);
        }
    }
    float pb3 = dz3;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pb3 += __shfl_down_sync(0xffffffffu, pb3, o);
    __syncwarp();

    // dh1 = dz2 W2^T ; dz1 = dh1 [h1 > 0]  -> BF16 into the h2 tile
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) load_a(S.dz[warp], HS, 16 * mt, 16 * ks, lane, a[ks][0], a[ks][1], a[ks][2], a[ks][3]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t b0, b1;
                load_b(S.frag, FT_W2T + ks * 8 + nt, lane, b0, b1);
                mma_bf16(d, a[ks][0], a[ks][1], a[ks][2], a[ks][3], b0, b1);
            }
            // apply the ReLU mask of layer 1 and store dz1 as BF16
            const __nv_bfloat16* H1 = S.h1[warp];
            const int r0 = 16 * mt + g, c0 = 8 * nt + 2 * q;
            const __nv_bfloat162 m0 = *reinterpret_cast<const __nv_bfloat162*>(H1 + r0 * HS + c0);
            const __nv_bfloat162 m1 = *reinterpret_cast<const __nv_bfloat162*>(H1 + (r0 + 8) * HS + c0);
            *reinterpret_cast<uint32_t*>(S.h2[warp] + r0 * HS + c0) =
                pack_bf16(__bfloat162float(m0.x) > 0.f ? d[0] : 0.f, __bfloat162float(m0.y) > 0.f ? d[1] : 0.f);
            *reinterpret_cast<uint32_t*>(S.h2[warp] + (r0 + 8) * HS + c0) =
                pack_bf16(__bfloat162float(m1.x) > 0.f ? d[2] : 0.f, __bfloat162float(m1.y) > 0.f ? d[3] : 0.f);
        }
    }
    __syncwarp();
    float pb1[2] = {0.f, 0.f};
    for (int s = 0; s < 32; ++s) {
#pragma unroll
        for (int h = 0; h < 2; ++h) pb1[h] += __bfloat162float(S.h2[warp][s * HS + lane + 32 * h]);
    }

    // weight-gradient GEMMs over this warp's 32 samples (K = samples):
    // dW2 = h1^T dz2 (64 x 64), dW1 = x^T dz1 (16 x 64)
    float dW2[4][8][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) dW2[mt][nt][0] = dW2[mt][nt][1] = dW2[mt][nt][2] = dW2[mt][nt][3] = 0.f;
    float dW1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) dW1[nt][0] = dW1[nt][1] = dW1[nt][2] = dW1[nt][3] = 0.f;
    const unsigned short* H1u = reinterpret_cast<const unsigned short*>(S.h1[warp]);
    const unsigned short* DZu = reinterpret_cast<const unsigned short*>(S.dz[warp]);
    const unsigned short* D1u = reinterpret_cast<const unsigned short*>(S.h2[warp]);
    const unsigned short* Xu = reinterpret_cast<const unsigned short*>(S.x[warp]);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        const int s0 = 16 * ks + 2 * q;   // samples of this lane's A columns / B rows
        uint32_t bz[8][2], b1f[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + g;
            bz[nt][0] = uint32_t(DZu[s0 * HS + col]) | (uint32_t(DZu[(s0 + 1) * HS + col]) << 16);
            bz[nt][1] = uint32_t(DZu[(s0 + 8) * HS + col]) | (uint32_t(DZu[(s0 + 9) * HS + col]) << 16);
            b1f[nt][0] = uint32_t(D1u[s0 * HS + col]) | (uint32_t(D1u[(s0 + 1) * HS + col]) << 16);
            b1f[nt][1] = uint32_t(D1u[(s0 + 8) * HS + col]) | (uint32_t(D1u[(s0 + 9) * HS + col]) << 16);
        }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int ra = 16 * mt + g;    // rows of A = h1 units
            const uint32_t a0 = uint32_t(H1u[s0 * HS + ra]) | (uint32_t(H1u[(s0 + 1) * HS + ra]) << 16);
            const uint32_t a1 = uint32_t(H1u[s0 * HS + ra + 8]) | (uint32_t(H1u[(s0 + 1) * HS + ra + 8]) << 16);
            const uint32_t a2 = uint32_t(H1u[(s0 + 8) * HS + ra]) | (uint32_t(H1u[(s0 + 9) * HS + ra]) << 16);
            const uint32_t a3 = uint32_t(H1u[(s0 + 8) * HS + ra + 8]) | (uint32_t(H1u[(s0 + 9) * HS + ra + 8]) << 16);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(dW2[mt][nt], a0, a1, a2, a3, bz[nt][0], bz[nt][1]);
        }
        {
            const int ra = g;              // rows of A = input features
            const uint32_t a0 = uint32_t(Xu[s0 * XS + ra]) | (uint32_t(Xu[(s0 + 1) * XS + ra]) << 16);
            const uint32_t a1 = uint32_t(Xu[s0 * XS + ra + 8]) | (uint32_t(Xu[(s0 + 1) * XS + ra + 8]) << 16);
            const uint32_t a2 = uint32_t(Xu[(s0 + 8) * XS + ra]) | (uint32_t(Xu[(s0 + 9) * XS + ra]) << 16);
            const uint32_t a3 = uint32_t(Xu[(s0 + 8) * XS + ra + 8]) | (uint32_t(Xu[(s0 + 9) * XS + ra + 8]) << 16);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(dW1[nt], a0, a1, a2, a3, b1f[nt][0], b1f[nt][1]);
        }
    }
    // add the warp partials into the block accumulators in warp order
    for (int w = 0; w < MLP_WARPS; ++w) {
        if (warp == w) {
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int r = 16 * mt + g, c = 8 * nt + 2 * q;
                    S.gW2[r * MLP_H + c] += dW2[mt][nt][0];
                    S.gW2[r * MLP_H + c + 1] += dW2[mt][nt][1];
                    S.gW2[(r + 8) * MLP_H + c] += dW2[mt][nt][2];
                    S.gW2[(r + 8) * MLP_H + c + 1] += dW2[mt][nt][3];
                }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int c = 8 * nt + 2 * q;
                S.gW1[g * MLP_H + c] += dW1[nt][0];
                S.gW1[g * MLP_H + c + 1] += dW1[nt][1];
                S.gW1[(g + 8) * MLP_H + c] += dW1[nt][2];
                S.gW1[(g + 8) * MLP_H + c + 1] += dW1[nt][3];
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                S.gvec[lane + 32 * h] += pb1[h];
                S.gvec[MLP_H + lane + 32 * h] += pb2[h];
                S.gvec[2 * MLP_H + lane + 32 * h] += pW3[h];
            }
            if (lane == 0) {
                S.gvec[3 * MLP_H] += pb3;
                S.loss += r2;
            }
        }
        __syncthreads();
    }
    // write this block's partial gradient in the flat parameter layout
    float* out = partials + (size_t)blockIdx.x * (MLP_NPARAM + 1);
    for (int i = tid; i < MLP_IN * MLP_H; i += MLP_BLOCK) out[MLP_OFF_W1 + i] = S.gW1[i];
    for (int i = tid; i < MLP_H * MLP_H; i += MLP_BLOCK) out[MLP_OFF_W2 + i] = S.gW2[i];
    for (int i = tid; i < MLP_H; i += MLP_BLOCK) {
        out[MLP_OFF_B1 + i] = S.gvec[i];
        out[MLP_OFF_B2 + i] = S.gvec[MLP_H + i];
        out[MLP_OFF_W3 + i] = S.gvec[2 * MLP_H + i];
    }
    if (tid == 0) {
        out[MLP_OFF_B3] = S.gvec[3 * MLP_H];
        out[MLP_NPARAM] = S.loss;
    }
}

// Sum of the block partials in block order; optionally an Adam step
// (step >= 1).  grad_out (nullable) receives the gradient, loss_out the loss.
__global__ void mlp_reduce_kernel(const float* __restrict__ partials, int n_blocks, float* __restrict__ W,
                                  float* __restrict__ m, float* __restrict__ v, int step, float lr,
                                  float* __restrict__ grad_out, float* __restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > MLP_NPARAM) return;
    float gsum = 0.f;
    for (int b = 0; b < n_blocks; ++b) gsum += partials[(size_t)b * (MLP_NPARAM + 1) + p];
    if (p == MLP_NPARAM) {
        if (loss_out) *loss_out = gsum;
        return;
    }
    if (grad_out) grad_out[p] = gsum;
    if (step > 0) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float mm = b1 * m[p] + (1.f - b1) * gsum;
        const float vv = b2 * v[p] + (1.f - b2) * gsum * gsum;
        m[p] = mm;
        v[p] = vv;
        const float mh = mm / (1.f - powf(b1, float(step)));
        const float vh = vv / (1.f - powf(b2, float(step)));
        W[p] -= lr * mh / (sqrtf(vh) + eps);
    }
}

}  // namespace gbp

// ==========================================================================
// C ABI

using namespace gbp;

struct gbp_mlp {
    cudaStream_t stream = nullptr;
    float* W = nullptr;         // master weights (FP32)
    float* m = nullptr;         // Adam moments
    float* v = nullptr;
    uint32_t* frag = nullptr;   // packed BF16 fragments
    float* bias = nullptr;      // b1, b2, b3, pad, W3 (FP32)
    float* partials = nullptr;
    int cap_blocks = 0;
    float* d_loss = nullptr;
    float* d_grad = nullptr;
    int step = 0;
};

namespace {

gbp_status mlp_pack(gbp_mlp* n) {
    mlp_pack_kernel<<<(FT_N * 32 + 127) / 128, 128, 0, n->stream>>>(n->W, n->frag, n->bias);
    return cudaGetLastError() == cudaSuccess ? GBP_OK : GBP_ECUDA;
}

gbp_status mlp_grad(gbp_mlp* n, const float* X, const float* T, const int32_t* idx, int count, int step, float lr,
                    float* grad_out) {
    if (count <= 0) return GBP_EINVAL;
    const int nb = (count + MLP_BLOCK - 1) / MLP_BLOCK;
    if (nb > n->cap_blocks) {
        if (n->partials) cudaFree(n->partials);
        n->partials = nullptr;
        if (cudaMalloc(reinterpret_cast<void**>(&n->partials), sizeof(float) * (size_t)nb * (MLP_NPARAM + 1)) != cudaSuccess)
            return GBP_ENOMEM;
        n->cap_blocks = nb;
    }
    const size_t smem = sizeof(GradSmem);
    if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GBP_ECUDA;
    mlp_grad_kernel<<<nb, MLP_BLOCK, smem, n->stream>>>(n->frag, n->bias, X, T, idx, count, 1.0f / count, n->partials);
    mlp_reduce_kernel<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, n->stream>>>(n->partials, nb, n->W, n->m, n->v, step, lr,
                                                                           grad_out, n->d_loss);
    if (cudaGetLastError() != cudaSuccess) return GBP_ECUDA;
    if (step > 0) return mlp_pack(n);
    return GBP_OK;
}

}  // namespace

extern "C" {

gbp_status gbp_mlp_create(const float* params, void* cuda_stream, gbp_mlp** out) {
    if (!out || !params) return GBP_EINVAL;
    *out = nullptr;
    for (int i = 0; i < MLP_NPARAM; ++i)
        if (!std::isfinite(params[i])) return GBP_EINVAL;
    gbp_mlp* n = new (std::nothrow) gbp_mlp();
    if (!n) return GBP_ENOMEM;
    n->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&n->W), sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->m), sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->v), sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->frag), sizeof(uint32_t) * FRAG_WORDS);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->bias), sizeof(float) * MLP_BIAS_WORDS);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->d_loss), sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&n->d_grad), sizeof(float) * MLP_NPARAM);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->W, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * MLP_NPARAM, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * MLP_NPARAM, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);   // params is the caller's
    if (e != cudaSuccess || mlp_pack(n) != GBP_OK) {
        gbp_mlp_destroy(n);
        return GBP_ECUDA;
    }
    *out = n;
    return GBP_OK;
}

void gbp_mlp_destroy(gbp_mlp* n) {
    if (!n) return;
    void* ptrs[] = {n->W, n->m, n->v, n->frag, n->bias, n->partials, n->d_loss, n->d_grad};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete n;
}

gbp_status gbp_mlp_set_params(gbp_mlp* n, const float* params) {
    if (!n || !params) return GBP_EINVAL;
    for (int i = 0; i < MLP_NPARAM; ++i)
        if (!std::isfinite(params[i])) return GBP_EINVAL;
    if (cudaMemcpyAsync(n->W, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->m, 0, sizeof(float) * MLP_NPARAM, n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->v, 0, sizeof(float) * MLP_NPARAM, n->stream) != cudaSuccess)
        return GBP_ECUDA;
    n->step = 0;
    // the host buffer may be reused by the caller as soon as we return
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) return GBP_ECUDA;
    return mlp_pack(n);
}

gbp_status gbp_mlp_get_params(const gbp_mlp* n, float* params) {
    if (!n || !params) return GBP_EINVAL;
    if (cudaMemcpyAsync(params, n->W, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return GBP_ECUDA;
    return GBP_OK;
}

gbp_status gbp_mlp_forward(gbp_mlp* n, const float* X, int32_t count, float* y) {
    if (!n || count < 0 || (count && (!X || !y))) return GBP_EINVAL;
    if (count == 0) return GBP_OK;
    mlp_forward_kernel<<<(count + MLP_BLOCK - 1) / MLP_BLOCK, MLP_BLOCK, 0, n->stream>>>(n->frag, n->bias, X, count, y);
    return cudaGetLastError() == cudaSuccess ? GBP_OK : GBP_ECUDA;
}

gbp_status gbp_mlp_gradient(gbp_mlp* n, const float* X, const float* target, int32_t count, float* grad,
                            double* loss) {
    if (!n || !X || !target || !grad || count <= 0) return GBP_EINVAL;
    gbp_status st = mlp_grad(n, X, target, nullptr, count, 0, 0.f, n->d_grad);
    if (st != GBP_OK) return st;
    float l = 0.f;
    if (cudaMemcpyAsync(grad, n->d_grad, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(&l, n->d_loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return GBP_ECUDA;
    if (loss) *loss = l;
    return GBP_OK;
}

gbp_status gbp_mlp_train_step(gbp_mlp* n, const float* X, const float* target, const int32_t* idx, int32_t count,
                              float lr, float* loss_out) {
    if (!n || !X || !target || count <= 0 || !(lr > 0.f)) return GBP_EINVAL;
    n->step += 1;
    gbp_status st = mlp_grad(n, X, target, idx, count, n->step, lr, nullptr);
    if (st != GBP_OK) return st;
    if (loss_out) {
        if (cudaMemcpyAsync(loss_out, n->d_loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
            cudaStreamSynchronize(n->stream) != cudaSuccess)
            return GBP_ECUDA;
    }
    return GBP_OK;
}

}  // extern "C"

namespace gbp {
cudaError_t mlp_copy_packed(const gbp_mlp* n, uint32_t* frag, float* bias, cudaStream_t s) {
    // the network's own stream may still be packing its latest weights
    cudaError_t e = cudaStreamSynchronize(n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(frag, n->frag, sizeof(uint32_t) * FWD_FRAG_WORDS, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bias, n->bias, sizeof(float) * MLP_BIAS_WORDS, cudaMemcpyDeviceToDevice, s);
    return e;
}
}  // namespace gbp
