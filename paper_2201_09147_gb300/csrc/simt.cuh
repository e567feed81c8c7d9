// Building blocks of the FP32 SIMT kernels (inference and training): a
// 128-row activation tile held transposed in shared memory and a
// register-tiled GEMM against a weight matrix streamed from global memory.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace sdfnn {
namespace simt {

constexpr int kSimtThreads = 256;
constexpr int kChunkK = 16;  // rows of W^T staged per step

// Activation tile X^T[k][r] (k = feature, r = row) with 4-float groups of r
// permuted by (k / 4) % 8 to keep the epilogue's column stores conflict free.
__device__ __forceinline__ int xt_index(int k, int r) { return k * 128 + ((((r >> 2) ^ ((k >> 2) & 7))) << 2) + (r & 3); }


// acc[i][j] = sum_k X[r0 + i][k] * W[n_j][k] for the thread's 8 rows and its
// features n_j = (j / 4) * 64 + fg * 4 + j % 4.  W^T is streamed from global
// memory (L2 resident) through a double-buffered shared-memory stage.
// Starts and ends with the block synchronised.
template <int W>
__device__ __forceinline__ void simt_gemm(const float* __restrict__ xt, const float* __restrict__ wt_g,
                                          float* __restrict__ ws, float (&acc)[8][W / 16], int r0, int fg) {
    constexpr int G = W / 64;
    constexpr int NCH = W / kChunkK;
    constexpr int F4_PER_CHUNK = kChunkK * W / 4;
    constexpr int PER_T = F4_PER_CHUNK / kSimtThreads;
    static_assert(PER_T >= 1, "chunk too small");
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < W / 16; ++j) acc[i][j] = 0.0f;

    const float4* src = reinterpret_cast<const float4*>(wt_g);
    float4 pre[PER_T];
#pragma unroll
    for (int u = 0; u < PER_T; ++u) pre[u] = __ldg(src + tid + u * kSimtThreads);
#pragma unroll
    for (int u = 0; u < PER_T; ++u) reinterpret_cast<float4*>(ws)[tid + u * kSimtThreads] = pre[u];
    __syncthreads();

    for (int c = 0; c < NCH; ++c) {
        const float* wsc = ws + (c & 1) * kChunkK * W;
        if (c + 1 < NCH) {
#pragma unroll
            for (int u = 0; u < PER_T; ++u) pre[u] = __ldg(src + (c + 1) * F4_PER_CHUNK + tid + u * kSimtThreads);
        }
#pragma unroll 4
        for (int kk = 0; kk < kChunkK; ++kk) {
            const int k = c * kChunkK + kk;
            const int sw = (k >> 2) & 7;
            const float4 xa = *reinterpret_cast<const float4*>(xt + k * 128 + ((((r0 >> 2)) ^ sw) << 2));
            const float4 xb = *reinterpret_cast<const float4*>(xt + k * 128 + ((((r0 >> 2) + 1) ^ sw) << 2));
            const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const float4 wv = *reinterpret_cast<const float4*>(wsc + kk * W + g * 64 + fg * 4);
                const float w4[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[i][g * 4 + e] = fmaf(x[i], w4[e], acc[i][g * 4 + e]);
            }
        }
        if (c + 1 < NCH) {
            float4* dst = reinterpret_cast<float4*>(ws + ((c + 1) & 1) * kChunkK * W);
#pragma unroll
            for (int u = 0; u < PER_T; ++u) dst[tid + u * kSimtThreads] = pre[u];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int feat_of(int j, int fg) { return (j >> 2) * 64 + fg * 4 + (j & 3); }

// Sum over the 16 lanes that share a row group (lanes l and l ^ 1, 2, 4, 8).
__device__ __forceinline__ float reduce16(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

}  // namespace simt
}  // namespace sdfnn
