// FP32 SIMT kernels: the plain FP32 path (SDF_FP32) and its building blocks.
//
// Both kernels evaluate the sine MLP of Eq. 2 on tiles of 128 rows held in
// shared memory, one layer at a time, as a register-tiled FP32 GEMM
// (256 threads; each thread owns 8 rows x width/16 output features), with the
// sine (or sine/cosine) epilogue fused after each layer.
//
//   trace_level_simt : one level of multiscale sphere tracing (Alg. 1).  The
//                      128 rows are persistent ray slots; a slot whose ray
//                      finishes is refilled from the level's work list with a
//                      warp-aggregated atomic (ballot + popc), so tiles stay
//                      dense until the work runs out.
//   grad_simt        : analytic gradients (Alg. 2, Eqs. 3-4).  The 128 rows
//                      are 32 points x 4 streams: the forward activations and
//                      the three forward tangents G^x, G^y, G^z, which share
//                      every weight load.
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "launch_cache.h"
#include "rays.cuh"
#include "simt.cuh"

namespace sdfnn {
namespace {

using namespace simt;

template <int W>
struct SimtSmem {
    float xt[W * 128];
    float ws[2 * kChunkK * W];
    float f[128];
    float px[128], py[128], pz[128];  // ray positions (trace) / points (grad)
    float pt[128];                    // per-row time (4-input networks with per-ray / per-point times)
    int idx[128];
    long long tile;
};

// ---------------------------------------------------------------------------
// trace kernel
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kSimtThreads) trace_level_simt_kernel(const LevelArgs a) {
    extern __shared__ float4 smem_f4[];
    SimtSmem<W>& S = *reinterpret_cast<SimtSmem<W>*>(smem_f4);
    constexpr int FPT = W / 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * 2 + (lane >> 4), fg = lane & 15, r0 = rg * 8;
    const NetView& net = a.net;
    const long long n_work = a.in_list ? static_cast<long long>(*a.in_count) : a.n;
    Ray ray;  // threads 0..127 own ray slot tid

    while (true) {
        if (tid < 128) {
            refill_ray(a, ray, n_work);
            S.px[tid] = ray.px;
            S.py[tid] = ray.py;
            S.pz[tid] = ray.pz;
            S.pt[tid] = (a.ray_time && ray.state == kSlotActive) ? a.ray_time[ray.idx] : 0.0f;
        }
        if (!__syncthreads_or(tid < 128 && ray.state == kSlotActive)) break;
        if (a.cap <= 0) {
            if (tid < 128) pass_ray(a, ray);
            continue;
        }

        // layer 0 (FP32): X[r][n] = sin(W_0[n] . (p_r, time_r) + b_0[n])
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int n = feat_of(j, fg);
            const float wx = __ldg(net.w0 + n * net.in_dim + 0), wy = __ldg(net.w0 + n * net.in_dim + 1),
                        wz = __ldg(net.w0 + n * net.in_dim + 2);
            float bb = __ldg(net.b0 + n), wt = 0.0f;
            if (net.in_dim == 4) {
                if (a.ray_time)
                    wt = __ldg(net.w0 + n * 4 + 3);
                else
                    bb = fmaf(__ldg(net.w0 + n * 4 + 3), a.time, bb);
            }
            float o[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = r0 + i;
                const float z = fmaf(wx, S.px[r], fmaf(wy, S.py[r], fmaf(wz, S.pz[r], fmaf(wt, S.pt[r], bb))));
                o[i] = sin_r(z);
            }
            *reinterpret_cast<float4*>(S.xt + xt_index(n, r0)) = make_float4(o[0], o[1], o[2], o[3]);
            *reinterpret_cast<float4*>(S.xt + xt_index(n, r0 + 4)) = make_float4(o[4], o[5], o[6], o[7]);
        }
        __syncthreads();

        float acc[8][FPT];
        for (int l = 0; l < net.n_hidden; ++l) {
            simt_gemm<W>(S.xt, net.wt[l], S.ws, acc, r0, fg);
            if (l + 1 < net.n_hidden) {
#pragma unroll
                for (int j = 0; j < FPT; ++j) {
                    const int n = feat_of(j, fg);
                    const float bb = __ldg(net.bh[l] + n);
                    float o[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) o[i] = sin_r(acc[i][j] + bb);
                    *reinterpret_cast<float4*>(S.xt + xt_index(n, r0)) = make_float4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<float4*>(S.xt + xt_index(n, r0 + 4)) = make_float4(o[4], o[5], o[6], o[7]);
                }
                __syncthreads();
            } else {
                // output layer: f = W_n P_{n-1} + b_n
                float dot[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) dot[i] = 0.0f;
#pragma unroll
                for (int j = 0; j < FPT; ++j) {
                    const int n = feat_of(j, fg);
                    const float bb = __ldg(net.bh[l] + n), wo = __ldg(net.wout + n);
#pragma unroll
                    for (int i = 0; i < 8; ++i) dot[i] = fmaf(wo, sin_r(acc[i][j] + bb), dot[i]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float s = reduce16(dot[i]);
                    if (fg == 0) S.f[r0 + i] = s + net.bout;
                }
            }
        }
        __syncthreads();
        if (tid < 128) step_ray(a, ray, S.f[tid]);
    }
}

// ---------------------------------------------------------------------------
// gradient kernel (Alg. 2 with the three tangents sharing the forward pass)
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kSimtThreads) grad_simt_kernel(const GradArgs a) {
    extern __shared__ float4 smem_f4[];
    SimtSmem<W>& S = *reinterpret_cast<SimtSmem<W>*>(smem_f4);
    constexpr int FPT = W / 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * 2 + (lane >> 4), fg = lane & 15, r0 = rg * 8;
    const int p0 = r0 >> 2;  // this thread's rows are points p0, p0 + 1, four streams each
    const NetView& net = a.net;
    const long long n_work = a.list ? static_cast<long long>(*a.count) : a.n;

    while (true) {
        if (tid == 0) S.tile = static_cast<long long>(atomicAdd(a.grab, 1ull));
        __syncthreads();
        const long long base = S.tile * 32;
        if (base >= n_work) break;
        if (tid < 32) {
            const long long k = base + tid;
            int i = -1;
            if (k < n_work) i = a.list ? a.list[k] : static_cast<int>(k);
            S.idx[tid] = i;
            S.px[tid] = i >= 0 ? a.pts[i] : 0.0f;
            S.py[tid] = i >= 0 ? a.pts[a.n + i] : 0.0f;
            S.pz[tid] = i >= 0 ? a.pts[2 * a.n + i] : 0.0f;
            S.pt[tid] = (i >= 0 && a.pt_time) ? a.pt_time[i] : 0.0f;
        }
        __syncthreads();

        // input layer: A_0 = W_0 p + b_0;  P_0 = sin(A_0);  G_0^c = W_0[:, c] (.) cos(A_0)
#pragma unroll
        for (int j = 0; j < FPT; ++j) {
            const int n = feat_of(j, fg);
            const float wx = __ldg(net.w0 + n * net.in_dim + 0), wy = __ldg(net.w0 + n * net.in_dim + 1),
                        wz = __ldg(net.w0 + n * net.in_dim + 2);
            float bb = __ldg(net.b0 + n), wt = 0.0f;
            if (net.in_dim == 4) {
                if (a.pt_time)
                    wt = __ldg(net.w0 + n * 4 + 3);
                else
                    bb = fmaf(__ldg(net.w0 + n * 4 + 3), a.time, bb);
            }
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int p = p0 + pp;
                const float z = fmaf(wx, S.px[p], fmaf(wy, S.py[p], fmaf(wz, S.pz[p], fmaf(wt, S.pt[p], bb))));
                float s, c;
                sincos_r(z, &s, &c);
                *reinterpret_cast<float4*>(S.xt + xt_index(n, r0 + pp * 4)) = make_float4(s, wx * c, wy * c, wz * c);
            }
        }
        __syncthreads();

        float acc[8][FPT];
        for (int l = 0; l < net.n_hidden; ++l) {
            simt_gemm<W>(S.xt, net.wt[l], S.ws, acc, r0, fg);
            const bool last = (l + 1 == net.n_hidden);
            float dot[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) dot[i] = 0.0f;
#pragma unroll
            for (int j = 0; j < FPT; ++j) {
                const int n = feat_of(j, fg);
                const float bb = __ldg(net.bh[l] + n);
                const float wo = last ? __ldg(net.wout + n) : 0.0f;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    // hidden layer: P_i = sin(A_i);  G_i = (W_i G_{i-1}) (.) cos(A_i)
                    float s, c;
                    sincos_r(acc[pp * 4][j] + bb, &s, &c);
                    const float g0 = c * acc[pp * 4 + 1][j], g1 = c * acc[pp * 4 + 2][j], g2 = c * acc[pp * 4 + 3][j];
                    if (!last) {
                        *reinterpret_cast<float4*>(S.xt + xt_index(n, r0 + pp * 4)) = make_float4(s, g0, g1, g2);
                    } else {
                        dot[pp * 4 + 0] = fmaf(wo, s, dot[pp * 4 + 0]);
                        dot[pp * 4 + 1] = fmaf(wo, g0, dot[pp * 4 + 1]);
                        dot[pp * 4 + 2] = fmaf(wo, g1, dot[pp * 4 + 2]);
                        dot[pp * 4 + 3] = fmaf(wo, g2, dot[pp * 4 + 3]);
                    }
                }
            }
            if (!last) {
                __syncthreads();
            } else {
                // output layer: grad_c = W_n G^c_{n-1}
#pragma unroll
                for (int i = 0; i < 8; ++i) dot[i] = reduce16(dot[i]);
                if (fg == 0) {
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int i = S.idx[p0 + pp];
                        if (i >= 0) {
                            float gx = dot[pp * 4 + 1], gy = dot[pp * 4 + 2], gz = dot[pp * 4 + 3];
                            if (a.normalize) {
                                const float len = sqrtf(gx * gx + gy * gy + gz * gz);
                                const float inv = len >= 1e-12f ? 1.0f / len : 0.0f;
                                gx *= inv;
                                gy *= inv;
                                gz *= inv;
                            }
                            a.out[i] = gx;
                            a.out[a.n + i] = gy;
                            a.out[2 * a.n + i] = gz;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Compaction of the masked points for the gradient kernels: list[0 .. *count)
// receives every i with mask[i] != 0 (in order within a block's 4096 points;
// the blocks' slices in the order their atomics land), and, when out is given,
// out[c * n + i] = 0 for every point (the gradient kernel then writes the
// masked-in ones).  Each thread takes 16 consecutive mask bytes; the block
// places its points with a warp scan and a scan over its 8 warps, and takes
// its slice of the list with one atomic (one per 4096 points instead of one
// per 32, which serialised on the counter).
constexpr int kCompactPer = 16;
constexpr int kCompactThreads = 256;

__global__ void __launch_bounds__(kCompactThreads) mask_compact_kernel(const uint8_t* __restrict__ mask, int64_t n,
                                                                      int32_t* __restrict__ list,
                                                                      unsigned long long* count,
                                                                      float* __restrict__ out) {
    __shared__ uint32_t warp_off[kCompactThreads / 32];
    __shared__ unsigned long long block_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int64_t kBlockPts = static_cast<int64_t>(kCompactThreads) * kCompactPer;
    // 16-byte vector stores of the zeros need every component row 16-byte aligned
    const bool vec_out = out != nullptr && (n % 4) == 0 && (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
    for (int64_t b0 = static_cast<int64_t>(blockIdx.x) * kBlockPts; b0 < n;
         b0 += static_cast<int64_t>(gridDim.x) * kBlockPts) {
        const int64_t i0 = b0 + static_cast<int64_t>(tid) * kCompactPer;
        const bool full = i0 + kCompactPer <= n;
        uint32_t bits = 0;  // bit j: point i0 + j is masked in
        if (full && (reinterpret_cast<uintptr_t>(mask + i0) & 15u) == 0) {
            const uint4 v = *reinterpret_cast<const uint4*>(mask + i0);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < kCompactPer; ++j) bits |= (((w[j >> 2] >> (8 * (j & 3))) & 0xFFu) != 0u ? 1u : 0u) << j;
        } else {
            for (int j = 0; j < kCompactPer; ++j)
                if (i0 + j < n && mask[i0 + j] != 0) bits |= 1u << j;
        }
        const uint32_t c = static_cast<uint32_t>(__popc(bits));
        uint32_t x = c;  // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_off[warp] = x;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kCompactThreads / 32; ++w) {
                const uint32_t v = warp_off[w];
                warp_off[w] = t;
                t += v;
            }
            block_base = t ? atomicAdd(count, static_cast<unsigned long long>(t)) : 0ull;
        }
        __syncthreads();
        unsigned long long k = block_base + warp_off[warp] + (x - c);
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1u;
            list[k++] = static_cast<int32_t>(i0 + j);
        }
        if (out) {
            if (vec_out && full) {
                const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int comp = 0; comp < 3; ++comp)
#pragma unroll
                    for (int q = 0; q < kCompactPer / 4; ++q)
                        reinterpret_cast<float4*>(out + comp * n + i0)[q] = z;
            } else {
                for (int j = 0; j < kCompactPer && i0 + j < n; ++j) {
                    out[i0 + j] = 0.0f;
                    out[n + i0 + j] = 0.0f;
                    out[2 * n + i0 + j] = 0.0f;
                }
            }
        }
        __syncthreads();  // warp_off and block_base are rewritten by the next round
    }
}

// One thread waits, with the library's bounded-wait loop but a budget of
// `budget_ns`, on an mbarrier that nothing ever arrives on; on expiry it
// latches kStatusTimeout in *status and the kernel returns normally.
__global__ void wait_timeout_selftest_kernel(int* status, unsigned long long budget_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    fence_mbar_init();
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait(b, 0u)) {
        if (globaltimer_ns() - t0 > budget_ns) {
            raise_status(status, kStatusTimeout);
            return;
        }
    }
}

template <class Kernel>
cudaError_t launch_persistent(Kernel k, size_t smem, int num_sms, cudaStream_t s, const void* arg) {
    // the attributes are set and the occupancy counted once per kernel and device; the
    // largest shared-memory carveout lets the occupancy query (and the launch) place as
    // many CTAs per SM as shared memory allows
    cudaError_t e = ensure_smem_attributes(k);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = launch_cached(reinterpret_cast<const void*>(k), smem, kSimtThreads, &per_sm, [&](int* v) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, k, kSimtThreads, smem);
    });
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    void* args[] = {const_cast<void*>(arg)};
    return cudaLaunchKernel(reinterpret_cast<const void*>(k), dim3(num_sms * per_sm), dim3(kSimtThreads), args, smem,
                            s);
}

}  // namespace

cudaError_t launch_trace_level_simt(const LevelArgs& a, int num_sms, cudaStream_t s) {
    switch (a.net.width) {
    case 64:
        return launch_persistent(trace_level_simt_kernel<64>, sizeof(SimtSmem<64>), num_sms, s, &a);
    case 128:
        return launch_persistent(trace_level_simt_kernel<128>, sizeof(SimtSmem<128>), num_sms, s, &a);
    case 256:
        return launch_persistent(trace_level_simt_kernel<256>, sizeof(SimtSmem<256>), num_sms, s, &a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_grad_simt(const GradArgs& a, int num_sms, cudaStream_t s) {
    switch (a.net.width) {
    case 64:
        return launch_persistent(grad_simt_kernel<64>, sizeof(SimtSmem<64>), num_sms, s, &a);
    case 128:
        return launch_persistent(grad_simt_kernel<128>, sizeof(SimtSmem<128>), num_sms, s, &a);
    case 256:
        return launch_persistent(grad_simt_kernel<256>, sizeof(SimtSmem<256>), num_sms, s, &a);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_wait_timeout_selftest(int* status, unsigned long long budget_ns, cudaStream_t s) {
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(status, budget_ns);
    return cudaGetLastError();
}

cudaError_t launch_mask_compact(const uint8_t* mask, int64_t n, int32_t* list, unsigned long long* count, float* out,
                                int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t per_block = static_cast<int64_t>(kCompactThreads) * kCompactPer;
    int64_t blocks = (n + per_block - 1) / per_block;
    if (blocks > static_cast<int64_t>(num_sms) * 8) blocks = static_cast<int64_t>(num_sms) * 8;
    mask_compact_kernel<<<static_cast<int>(blocks), kCompactThreads, 0, s>>>(mask, n, list, count, out);
    return cudaGetLastError();
}

}  // namespace sdfnn
