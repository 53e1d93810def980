// gbp_mlp.cuh -- device building blocks of the per-factor damping network
// (16 -> 64 -> 64 -> 1, ReLU, output 0.9 * sigmoid) on BF16 tensor cores
// (mma.sync m16n8k16, FP32 accumulation).  Shared by the training kernels
// (gbp_mlp.cu) and the learned-damping iteration kernel (gbp_kernels.cu).
//
// A warp evaluates 32 rows (factors or training samples) at once: rows live
// in a shared-memory BF16 tile, weights are pre-packed per lane into the
// B-operand fragment layout, so every operand load is one 32-bit shared-
// memory access.
//
// Flat parameter layout (float32, same as the CPU reference):
//   W1 [16][64] (row = input), b1 [64], W2 [64][64], b2 [64], W3 [64], b3.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace gbp {

constexpr int MLP_IN = 16;
constexpr int MLP_H = 64;
constexpr int MLP_NPARAM = 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1;   // 5313
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 1024, MLP_OFF_W2 = 1088, MLP_OFF_B2 = 5184, MLP_OFF_W3 = 5248,
              MLP_OFF_B3 = 5312;
constexpr float MLP_DMAX = 0.9f;

// B-fragment tiles: layer 1 (8 n-tiles), layer 2 (4 k-steps x 8 n-tiles),
// layer 3 (4 k-steps, output column 0), then W2^T for the backward pass.
constexpr int FT_L1 = 0, FT_L2 = 8, FT_L3 = 40, FT_W2T = 44, FT_N = 76;
constexpr int FRAG_WORDS = FT_N * 32 * 2;        // uint32 words
constexpr int FWD_FRAG_WORDS = FT_W2T * 32 * 2;  // words the forward pass needs
// FP32 side buffer: b1 [64], b2 [64], b3, pad, W3 [64] (W3 for the backward
// pass), pad to a multiple of 16 bytes (copied in 16-byte pieces)
constexpr int MLP_BIAS_WORDS = 2 * MLP_H + 2 + MLP_H + 2;

// shared-memory row strides (BF16 elements), chosen so that the 8 rows a
// fragment load touches fall in distinct banks
constexpr int XS = 24;   // 16-wide input tile
constexpr int HS = 72;   // 64-wide hidden tile

// two FP32 values -> a BF16 pair (lo in bits 0-15), round to nearest even,
// one conversion instruction; the _relu form also clamps negatives to 0
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// A fragment (16 x 16, rows r0.., cols c0..) of a row-major BF16 tile.
__device__ __forceinline__ void load_a(const __nv_bfloat16* T, int stride, int r0, int c0, int lane, uint32_t& a0,
                                       uint32_t& a1, uint32_t& a2, uint32_t& a3) {
    const int g = lane >> 2, q = lane & 3;
    a0 = *reinterpret_cast<const uint32_t*>(T + (r0 + g) * stride + c0 + 2 * q);
    a1 = *reinterpret_cast<const uint32_t*>(T + (r0 + g + 8) * stride + c0 + 2 * q);
    a2 = *reinterpret_cast<const uint32_t*>(T + (r0 + g) * stride + c0 + 2 * q + 8);
    a3 = *reinterpret_cast<const uint32_t*>(T + (r0 + g + 8) * stride + c0 + 2 * q + 8);
}

// Store a 16 x 8 D fragment (after f) as BF16 pairs into a row-major tile.
template <typename F>
__device__ __forceinline__ void store_d_bf16(__nv_bfloat16* T, int stride, int r0, int c0, int lane,
                                             const float (&d)[4], F f) {
    const int g = lane >> 2, q = lane & 3;
    *reinterpret_cast<uint32_t*>(T + (r0 + g) * stride + c0 + 2 * q) = pack_bf16(f(d[0], c0 + 2 * q), f(d[1], c0 + 2 * q + 1));
    *reinterpret_cast<uint32_t*>(T + (r0 + g + 8) * stride + c0 + 2 * q) =
        pack_bf16(f(d[2], c0 + 2 * q), f(d[3], c0 + 2 * q + 1));
}

// B fragment of tile `tile` for this lane.
__device__ __forceinline__ void load_b(const uint32_t* frag, int tile, int lane, uint32_t& b0, uint32_t& b1) {
    const uint2 v = *reinterpret_cast<const uint2*>(frag + (tile * 32 + lane) * 2);
    b0 = v.x;
    b1 = v.y;
}

// Forward pass of one warp over 32 rows.  X: the 32 x 16 input tile (BF16,
// stride XS); H: a 32 x 64 scratch tile (stride HS; on return it holds h2).
// When H1 is given, h1 is also kept there (training).  Returns the output
// pre-activation z3 of row `lane`.  frag/bias in shared memory; bias =
// b1 (64), b2 (64), b3 (1).
__device__ __forceinline__ float mlp_forward_warp(const uint32_t* frag, const float* bias, __nv_bfloat16* X,
                                                  __nv_bfloat16* H, __nv_bfloat16* H1, int lane) {
    const int g = lane >> 2, q = lane & 3;
    (void)g;
    __nv_bfloat16* L1out = H1 ? H1 : H;
    // layer 1: h1 = relu(X W1 + b1)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a0, a1, a2, a3;
        load_a(X, XS, 16 * mt, 0, lane, a0, a1, a2, a3);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t b0, b1;
            load_b(frag, FT_L1 + nt, lane, b0, b1);
            mma_bf16(d, a0, a1, a2, a3, b0, b1);
            store_d_bf16(L1out, HS, 16 * mt, 8 * nt, lane, d, [&](float v, int c) { return fmaxf(v + bias[c], 0.f); });
        }
    }
    __syncwarp();
    // layer 2: h2 = relu(h1 W2 + b2), one 16-row block at a time so that it
    // can overwrite h1 in place when no separate h1 tile is kept
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) load_a(L1out, HS, 16 * mt, 16 * ks, lane, a[ks][0], a[ks][1], a[ks][2], a[ks][3]);
        float d[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t b0, b1;
                load_b(frag, FT_L2 + ks * 8 + nt, lane, b0, b1);
                mma_bf16(d[nt], a[ks][0], a[ks][1], a[ks][2], a[ks][3], b0, b1);
            }
        }
        __syncwarp();
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
            store_d_bf16(H, HS, 16 * mt, 8 * nt, lane, d[nt],
                         [&](float v, int c) { return fmaxf(v + bias[MLP_H + c], 0.f); });
    }
    __syncwarp();
    // layer 3: z3 = h2 W3 + b3 (W3 in output column 0 of the tile)
    float* out = reinterpret_cast<float*>(X);   // the input tile is free now
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a0, a1, a2, a3, b0, b1;
            load_a(H, HS, 16 * mt, 16 * ks, lane, a0, a1, a2, a3);
            load_b(frag, FT_L3 + ks, lane, b0, b1);
            mma_bf16(d, a0, a1, a2, a3, b0, b1);
        }
        __syncwarp();
        if (q == 0) {
            out[16 * mt + (lane >> 2)] = d[0];
            out[16 * mt + (lane >> 2) + 8] = d[2];
        }
    }
    __syncwarp();
    const float z3 = out[lane] + bias[2 * MLP_H];
    __syncwarp();
    return z3;
}

__device__ __forceinline__ float mlp_output(float z3) { return MLP_DMAX / (1.0f + __expf(-z3)); }

// Register-resident forward pass for inference: the D fragments of one
// layer (16 x 8 tiles, FP32) are exactly the A fragments of the next layer
// (16 x 16, BF16 pairs) once packed -- tile 2j supplies columns 0-7 and tile
// 2j+1 columns 8-15 of k-step j -- so activations never leave registers.
// Bitwise equal to mlp_forward_warp (same roundings, same mma order).
// X: the warp's 32 x 16 input tile (BF16, stride XS) in shared memory;
// frag/bias as for mlp_forward_warp.  Returns z3 of row `lane`.
__device__ __forceinline__ float mlp_forward_regs(const uint32_t* frag, const float* bias, const __nv_bfloat16* X,
                                                  int lane) {
    const int g = lane >> 2, q = lane & 3;
    float z[2][2];   // [m-tile][row g / g + 8] of output column 0 (lanes with q == 0)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        // layer 1: h1 = relu(X W1 + b1) -> A fragments of layer 2
        uint32_t x0, x1, x2, x3;
        load_a(X, XS, 16 * mt, 0, lane, x0, x1, x2, x3);
        uint32_t a1[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t b0, b1;
            load_b(frag, FT_L1 + nt, lane, b0, b1);
            mma_bf16(d, x0, x1, x2, x3, b0, b1);
            const int c = 8 * nt + 2 * q;
            const float bc0 = bias[c], bc1 = bias[c + 1];
            const uint32_t lo = pack_bf16_relu(d[0] + bc0, d[1] + bc1);
            const uint32_t hi = pack_bf16_relu(d[2] + bc0, d[3] + bc1);
            a1[nt >> 1][(nt & 1) ? 2 : 0] = lo;
            a1[nt >> 1][(nt & 1) ? 3 : 1] = hi;
        }
        // layer 2: h2 = relu(h1 W2 + b2) -> A fragments of layer 3
        uint32_t a2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                uint32_t b0, b1;
                load_b(frag, FT_L2 + ks * 8 + nt, lane, b0, b1);
                mma_bf16(d, a1[ks][0], a1[ks][1], a1[ks][2], a1[ks][3], b0, b1);
            }
            const int c = 8 * nt + 2 * q;
            const float bc0 = bias[MLP_H + c], bc1 = bias[MLP_H + c + 1];
            const uint32_t lo = pack_bf16_relu(d[0] + bc0, d[1] + bc1);
            const uint32_t hi = pack_bf16_relu(d[2] + bc0, d[3] + bc1);
            a2[nt >> 1][(nt & 1) ? 2 : 0] = lo;
            a2[nt >> 1][(nt & 1) ? 3 : 1] = hi;
        }
        // layer 3: z3 = h2 W3 (column 0 of the output tile)
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t b0, b1;
            load_b(frag, FT_L3 + ks, lane, b0, b1);
            mma_bf16(d, a2[ks][0], a2[ks][1], a2[ks][2], a2[ks][3], b0, b1);
        }
        z[mt][0] = d[0];
        z[mt][1] = d[2];
    }
    // row r = lane: m-tile r / 16, held by lane 4 (r % 8) as row g (r % 16 < 8) or g + 8
    const int src = (lane & 7) << 2;
    const float v00 = __shfl_sync(0xffffffffu, z[0][0], src);
    const float v01 = __shfl_sync(0xffffffffu, z[0][1], src);
    const float v10 = __shfl_sync(0xffffffffu, z[1][0], src);
    const float v11 = __shfl_sync(0xffffffffu, z[1][1], src);
    const float v = (lane < 16) ? ((lane & 8) ? v01 : v00) : ((lane & 8) ? v11 : v10);
    (void)g;
    return v + bias[2 * MLP_H];
}

}  // namespace gbp
