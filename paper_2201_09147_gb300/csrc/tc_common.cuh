// Pieces shared by the tensor-core kernels of the inference and training
// paths: operand types, layer-0 staging and the persistent launcher.
#pragma once

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "launch_cache.h"

namespace sdfnn {
namespace {

// Operand types of the tensor-core contractions: bfloat16 or IEEE half
// (kind::f16), or E4M3 (kind::f8f6f4; sine activations stored as 256 sin).
enum : int { kOpBF16 = 0, kOpF16 = 1, kOpE4M3 = 2 };
constexpr float kFp8ActScale = 256.0f;

// Layer-0 parameters in shared memory: (w_x, w_y, w_z, b) per unit as a
// float4, and the time column w_t apart.  With per-ray times (TIMED) b is
// the plain bias and each ray adds w_t * t_ray; otherwise the launch's
// constant time is folded into b.  (Gradient kernels.)
__device__ __forceinline__ void stage_layer0(const NetView& net, float time, bool timed, int i, float* w0s,
                                             float* wts) {
#pragma unroll
    for (int c = 0; c < 3; ++c) w0s[i * 4 + c] = net.w0[i * net.in_dim + c];
    float bb = net.b0[i];
    const float wt = net.in_dim == 4 ? net.w0[i * 4 + 3] : 0.0f;
    if (!timed) bb = fmaf(wt, time, bb);
    w0s[i * 4 + 3] = bb;
    wts[i] = timed ? wt : 0.0f;
}

// CTAs of `k` that fit on one SM, from its registers, shared memory, threads
// and TMEM columns (the runtime's occupancy query reports 1 for kernels that
// use tcgen05, whatever their footprint).
template <class Kernel>
cudaError_t resident_ctas(Kernel k, int threads, size_t smem, int tmem_cols, int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return e;
    cudaFuncAttributes at;
    if ((e = cudaFuncGetAttributes(&at, k)) != cudaSuccess) return e;
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((at.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
    int n = 32;
    n = std::min(n, static_cast<int>(smem_sm / (smem + at.sharedSizeBytes + reserved)));
    n = std::min(n, regs_sm / std::max(1, regs_warp * warps));
    n = std::min(n, threads_sm / threads);
    n = std::min(n, 512 / tmem_cols);
    *out = n;
    return n >= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <class Kernel>
cudaError_t launch_tc(Kernel k, int threads, size_t smem, int tmem_cols, int num_sms, cudaStream_t s,
                      const void* arg) {
    cudaError_t e = ensure_smem_attributes(k);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = launch_cached(reinterpret_cast<const void*>(k), smem,
                      (static_cast<uint64_t>(threads) << 32) | static_cast<uint32_t>(tmem_cols), &per_sm,
                      [&](int* v) { return resident_ctas(k, threads, smem, tmem_cols, v); });
    if (e != cudaSuccess) return e;
    void* args[] = {const_cast<void*>(arg)};
    return cudaLaunchKernel(reinterpret_cast<const void*>(k), dim3(num_sms * per_sm), dim3(threads), args, smem, s);
}

}  // namespace
}  // namespace sdfnn
