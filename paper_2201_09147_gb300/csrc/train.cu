// Training path of the sine MLPs (FP32 SIMT).
//
// The fitting objective (values, gradient directions near the surface and
// the Eikonal term) depends on f and on grad f, so its parameter gradient
// runs backwards through Eq. 2 and through the tangent recursion of Alg. 2:
//
//   forward (per layer i):  A_i = W_i P_{i-1} + b_i,  H_i^c = W_i G_{i-1}^c,
//                           P_i = sin A_i,  G_i^c = cos A_i (.) H_i^c,
//                           f = w . P_k + b,  (grad f)_c = w . G_k^c
//   backward:               dA_i  = dP_i (.) cos A_i - sin A_i (.) sum_c dG_i^c (.) H_i^c
//                           dH_i^c = dG_i^c (.) cos A_i
//                           dP_{i-1} = W_i^T dA_i,  dG_{i-1}^c = W_i^T dH_i^c
//                           dW_i = dA_i P_{i-1}^T + sum_c dH_i^c (G_{i-1}^c)^T,  db_i = dA_i
//
// with layer 0 fed by the point (G_0^c = cos A_0 (.) W_0[:, c]).  Tiles of 32
// points x 4 streams (value, three tangents) run through the same
// register-tiled GEMM as the FP32 inference kernels; the forward saves A_i
// and H_i for every layer, the backward writes (dA_i, dH_i) and the weight
// gradients dW_i are separate GEMMs over all points.  Biases, W_0 and w_out
// are reduced per CTA in shared memory and added once at the end.
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "launch_cache.h"
#include "simt.cuh"

namespace sdfnn {

TrainShape train_shape(int in_dim, int width, int n_hidden) {
    TrainShape s{};
    s.in_dim = in_dim;
    s.width = width;
    s.n_hidden = n_hidden;
    int64_t o = 0;
    s.off_w0 = o;
    o += static_cast<int64_t>(width) * in_dim;
    s.off_b0 = o;
    o += width;
    for (int l = 0; l < n_hidden; ++l) {
        s.off_w[l] = o;
        o += static_cast<int64_t>(width) * width;
        s.off_b[l] = o;
        o += width;
    }
    s.off_wout = o;
    o += width;
    s.off_bout = o;
    o += 1;
    s.count = o;
    return s;
}

namespace {
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
}  // namespace

size_t train_workspace_bytes(const TrainShape& sh, int64_t n) {
    const size_t W = sh.width, k = sh.n_hidden, N = static_cast<size_t>(n);
    return align256(k * W * W * 4) + align256(N * W * 4) + 2 * align256(k * N * 4 * W * 4) + 256;
}

TrainWork train_work(const TrainShape& sh, int64_t n, void* ws) {
    const size_t W = sh.width, k = sh.n_hidden, N = static_cast<size_t>(n);
    uint8_t* p = static_cast<uint8_t*>(ws);
    TrainWork w{};
    w.wt = reinterpret_cast<float*>(p);
    p += align256(k * W * W * 4);
    w.z0 = reinterpret_cast<float*>(p);
    p += align256(N * W * 4);
    w.z = reinterpret_cast<float*>(p);
    p += align256(k * N * 4 * W * 4);
    w.d = reinterpret_cast<float*>(p);
    p += align256(k * N * 4 * W * 4);
    w.counters = reinterpret_cast<unsigned long long*>(p);
    return w;
}

namespace {

using namespace simt;

constexpr int kTilePts = 32;  // 32 points x 4 streams = the 128 rows of a tile

// W^T of every hidden layer (the forward GEMM streams W^T).
__global__ void transpose_hidden_kernel(const float* __restrict__ theta, TrainShape sh, float* __restrict__ wt) {
    __shared__ float t[32][33];
    const int W = sh.width, l = blockIdx.z;
    const float* src = theta + sh.off_w[l];
    float* dst = wt + static_cast<size_t>(l) * W * W;
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) t[y][threadIdx.x] = src[(by + y) * W + bx + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) dst[(bx + y) * W + by + threadIdx.x] = t[threadIdx.x][y];
}

// ---------------------------------------------------------------------------
// forward with saved pre-activations
// ---------------------------------------------------------------------------
template <int W>
struct FwdSmem {
    float xt[W * 128];
    float ws[2 * kChunkK * W];
    float px[kTilePts], py[kTilePts], pz[kTilePts], pt[kTilePts];
    long long tile;
};

template <int W>
__global__ void __launch_bounds__(kSimtThreads) train_fwd_kernel(const TrainArgs a) {
    extern __shared__ float4 smem_f4[];
    FwdSmem<W>& S = *reinterpret_cast<FwdSmem<W>*>(smem_f4);
    constexpr int FPT = W / 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * 2 + (lane >> 4), fg = lane & 15, r0 = rg * 8, p0 = r0 >> 2;
    const TrainShape& sh = a.sh;
    const int IN = sh.in_dim, KH = sh.n_hidden;
    const float* W0 = a.theta + sh.off_w0;
    const float* B0 = a.theta + sh.off_b0;
    const float* WO = a.theta + sh.off_wout;
    const float bout = a.theta[sh.off_bout];
    const int64_t n = a.n;

    while (true) {
        if (tid == 0) S.tile = static_cast<long long>(atomicAdd(&a.w.counters[0], 1ull));
        __syncthreads();
        const int64_t base = S.tile * kTilePts;
        if (base >= n) break;
        if (tid < kTilePts) {
            const int64_t i = base + tid;
            const bool v = i < n;
            S.px[tid] = v ? a.pts[i] : 0.0f;
            S.py[tid] = v ? a.pts[n + i] : 0.0f;
            S.pz[tid] = v ? a.pts[2 * n + i] : 0.0f;
            S.pt[tid] = (v && a.pt_time) ? a.pt_time[i] : 0.0f;
        }
        __syncthreads();

        // layer 0: A_0 = W_0 (p, t) + b_0;  P_0 = sin A_0;  G_0^c = W_0[:, c] cos A_0
#pragma unroll
        for (int jg = 0; jg < FPT / 4; ++jg) {
            float za[2][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int nn = feat_of(jg * 4 + e, fg);
                const float wx = W0[nn * IN], wy = W0[nn * IN + 1], wz = W0[nn * IN + 2];
                const float wt = IN == 4 ? W0[nn * IN + 3] : 0.0f;
                const float bb = B0[nn];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int p = p0 + pp;
                    const float z = fmaf(wx, S.px[p], fmaf(wy, S.py[p], fmaf(wz, S.pz[p], fmaf(wt, S.pt[p], bb))));
                    za[pp][e] = z;
                    float sn, cs;
                    sincos_r(z, &sn, &cs);
                    *reinterpret_cast<float4*>(S.xt + xt_index(nn, r0 + pp * 4)) =
                        make_float4(sn, wx * cs, wy * cs, wz * cs);
                }
            }
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int64_t i = base + p0 + pp;
                if (i < n)
                    *reinterpret_cast<float4*>(a.w.z0 + i * W + feat_of(jg * 4, fg)) =
                        make_float4(za[pp][0], za[pp][1], za[pp][2], za[pp][3]);
            }
        }
        __syncthreads();

        float acc[8][FPT];
        for (int l = 0; l < KH; ++l) {
            simt_gemm<W>(S.xt, a.w.wt + static_cast<size_t>(l) * W * W, S.ws, acc, r0, fg);
            const float* bl = a.theta + sh.off_b[l];
            float* zl = a.w.z + static_cast<size_t>(l) * n * 4 * W;
            const bool last = l + 1 == KH;
            float dot[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) dot[i] = 0.0f;
#pragma unroll
            for (int jg = 0; jg < FPT / 4; ++jg) {
                float zs[2][4][4];  // [point][stream][feature]
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = jg * 4 + e, nn = feat_of(j, fg);
                    const float bb = bl[nn];
                    const float wo = last ? WO[nn] : 0.0f;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const float A = acc[pp * 4][j] + bb;
                        const float h0 = acc[pp * 4 + 1][j], h1 = acc[pp * 4 + 2][j], h2 = acc[pp * 4 + 3][j];
                        zs[pp][0][e] = A;
                        zs[pp][1][e] = h0;
                        zs[pp][2][e] = h1;
                        zs[pp][3][e] = h2;
                        float sn, cs;
                        sincos_r(A, &sn, &cs);
                        if (!last) {
                            *reinterpret_cast<float4*>(S.xt + xt_index(nn, r0 + pp * 4)) =
                                make_float4(sn, cs * h0, cs * h1, cs * h2);
                        } else {
                            dot[pp * 4 + 0] = fmaf(wo, sn, dot[pp * 4 + 0]);
                            dot[pp * 4 + 1] = fmaf(wo, cs * h0, dot[pp * 4 + 1]);
                            dot[pp * 4 + 2] = fmaf(wo, cs * h1, dot[pp * 4 + 2]);
                            dot[pp * 4 + 3] = fmaf(wo, cs * h2, dot[pp * 4 + 3]);
                        }
                    }
                }
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int64_t i = base + p0 + pp;
                    if (i < n) {
#pragma unroll
                        for (int st = 0; st < 4; ++st)
                            *reinterpret_cast<float4*>(zl + (i * 4 + st) * W + feat_of(jg * 4, fg)) =
                                make_float4(zs[pp][st][0], zs[pp][st][1], zs[pp][st][2], zs[pp][st][3]);
                    }
                }
            }
            if (!last) {
                __syncthreads();
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) dot[i] = reduce16(dot[i]);
                if (fg == 0) {
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int64_t i = base + p0 + pp;
                        if (i < n) {
                            a.out_f[i] = dot[pp * 4] + bout;
                            a.out_grad[i] = dot[pp * 4 + 1];
                            a.out_grad[n + i] = dot[pp * 4 + 2];
                            a.out_grad[2 * n + i] = dot[pp * 4 + 3];
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// backward through the forward and tangent passes
// ---------------------------------------------------------------------------
template <int W>
struct BwdSmem {
    float xt[W * 128];
    float ws[2 * kChunkK * W];
    float px[kTilePts], py[kTilePts], pz[kTilePts], pt[kTilePts];
    float df[kTilePts], dg[3][kTilePts];
    float gb[(kMaxHidden + 1) * W];  // db_0 .. db_k
    float gw0[4 * W];                // dW_0 [unit][input]
    float gwo[W];                    // dw_out
    float gbo;                       // db_out
    long long tile;
};

template <int W>
__global__ void __launch_bounds__(kSimtThreads) train_bwd_kernel(const TrainArgs a) {
    extern __shared__ float4 smem_f4[];
    BwdSmem<W>& S = *reinterpret_cast<BwdSmem<W>*>(smem_f4);
    constexpr int FPT = W / 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rg = warp * 2 + (lane >> 4), fg = lane & 15, r0 = rg * 8, p0 = r0 >> 2;
    const TrainShape& sh = a.sh;
    const int IN = sh.in_dim, KH = sh.n_hidden;
    const float* W0 = a.theta + sh.off_w0;
    const float* WO = a.theta + sh.off_wout;
    const int64_t n = a.n;

    for (int i = tid; i < (KH + 1) * W; i += kSimtThreads) S.gb[i] = 0.0f;
    for (int i = tid; i < 4 * W; i += kSimtThreads) S.gw0[i] = 0.0f;
    for (int i = tid; i < W; i += kSimtThreads) S.gwo[i] = 0.0f;
    if (tid == 0) S.gbo = 0.0f;

    while (true) {
        __syncthreads();
        if (tid == 0) S.tile = static_cast<long long>(atomicAdd(&a.w.counters[1], 1ull));
        __syncthreads();
        const int64_t base = S.tile * kTilePts;
        if (base >= n) break;
        if (tid < kTilePts) {
            const int64_t i = base + tid;
            const bool v = i < n;
            S.px[tid] = v ? a.pts[i] : 0.0f;
            S.py[tid] = v ? a.pts[n + i] : 0.0f;
            S.pz[tid] = v ? a.pts[2 * n + i] : 0.0f;
            S.pt[tid] = (v && a.pt_time) ? a.pt_time[i] : 0.0f;
            const float dfi = v ? a.d_f[i] : 0.0f;
            S.df[tid] = dfi;
            S.dg[0][tid] = v ? a.d_grad[i] : 0.0f;
            S.dg[1][tid] = v ? a.d_grad[n + i] : 0.0f;
            S.dg[2][tid] = v ? a.d_grad[2 * n + i] : 0.0f;
            float sdf = dfi;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sdf += __shfl_xor_sync(0xffffffffu, sdf, o);
            if (tid == 0) S.gbo += sdf;
        }
        __syncthreads();

        // adjoints of the last layer's outputs: dP_k = df w_out, dG_k^c = dg_c w_out,
        // and dw_out = sum_p (df P_k + sum_c dg_c G_k^c)
        float Y[8][FPT];
        {
            const float* zl = a.w.z + static_cast<size_t>(KH - 1) * n * 4 * W;
#pragma unroll
            for (int jg = 0; jg < FPT / 4; ++jg) {
                float4 z[2][4];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int64_t i = base + p0 + pp;
#pragma unroll
                    for (int st = 0; st < 4; ++st)
                        z[pp][st] = i < n ? *reinterpret_cast<const float4*>(zl + (i * 4 + st) * W + feat_of(jg * 4, fg))
                                          : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = jg * 4 + e, nn = feat_of(j, fg);
                    const float wo = WO[nn];
                    float gsum = 0.0f;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int p = p0 + pp;
                        const float A = reinterpret_cast<const float*>(&z[pp][0])[e];
                        float sn, cs;
                        sincos_r(A, &sn, &cs);
                        const float h0 = reinterpret_cast<const float*>(&z[pp][1])[e];
                        const float h1 = reinterpret_cast<const float*>(&z[pp][2])[e];
                        const float h2 = reinterpret_cast<const float*>(&z[pp][3])[e];
                        gsum += S.df[p] * sn + cs * (S.dg[0][p] * h0 + S.dg[1][p] * h1 + S.dg[2][p] * h2);
                        Y[pp * 4 + 0][j] = S.df[p] * wo;
                        Y[pp * 4 + 1][j] = S.dg[0][p] * wo;
                        Y[pp * 4 + 2][j] = S.dg[1][p] * wo;
                        Y[pp * 4 + 3][j] = S.dg[2][p] * wo;
                    }
                    atomicAdd(&S.gwo[nn], gsum);
                }
            }
        }

        // hidden layers, last to first: (dA_l, dH_l) from (dP_l, dG_l), then dP_{l-1}, dG_{l-1}
        for (int l = KH - 1; l >= 0; --l) {
            const float* zl = a.w.z + static_cast<size_t>(l) * n * 4 * W;
            float* dl = a.w.d + static_cast<size_t>(l) * n * 4 * W;
#pragma unroll
            for (int jg = 0; jg < FPT / 4; ++jg) {
                float4 z[2][4];
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int64_t i = base + p0 + pp;
#pragma unroll
                    for (int st = 0; st < 4; ++st)
                        z[pp][st] = i < n ? *reinterpret_cast<const float4*>(zl + (i * 4 + st) * W + feat_of(jg * 4, fg))
                                          : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
                float dv[2][4][4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = jg * 4 + e, nn = feat_of(j, fg);
                    float bsum = 0.0f;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const float A = reinterpret_cast<const float*>(&z[pp][0])[e];
                        const float h0 = reinterpret_cast<const float*>(&z[pp][1])[e];
                        const float h1 = reinterpret_cast<const float*>(&z[pp][2])[e];
                        const float h2 = reinterpret_cast<const float*>(&z[pp][3])[e];
                        float sn, cs;
                        sincos_r(A, &sn, &cs);
                        const float dA = Y[pp * 4][j] * cs -
                                         sn * (Y[pp * 4 + 1][j] * h0 + Y[pp * 4 + 2][j] * h1 + Y[pp * 4 + 3][j] * h2);
                        const float d0 = Y[pp * 4 + 1][j] * cs, d1 = Y[pp * 4 + 2][j] * cs, d2 = Y[pp * 4 + 3][j] * cs;
                        dv[pp][0][e] = dA;
                        dv[pp][1][e] = d0;
                        dv[pp][2][e] = d1;
                        dv[pp][3][e] = d2;
                        bsum += dA;
                        *reinterpret_cast<float4*>(S.xt + xt_index(nn, r0 + pp * 4)) = make_float4(dA, d0, d1, d2);
                    }
                    atomicAdd(&S.gb[(l + 1) * W + nn], bsum);
                }
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int64_t i = base + p0 + pp;
                    if (i < n) {
#pragma unroll
                        for (int st = 0; st < 4; ++st)
                            *reinterpret_cast<float4*>(dl + (i * 4 + st) * W + feat_of(jg * 4, fg)) =
                                make_float4(dv[pp][st][0], dv[pp][st][1], dv[pp][st][2], dv[pp][st][3]);
                    }
                }
            }
            __syncthreads();
            // rows x W_l (row-major [unit][input]): dP_{l-1} = W_l^T dA_l, dG_{l-1}^c = W_l^T dH_l^c
            simt_gemm<W>(S.xt, a.theta + sh.off_w[l], S.ws, Y, r0, fg);
        }

        // layer 0: dA_0 = dP_0 cos A_0 - sin A_0 sum_c dG_0^c W_0[:, c];
        // dW_0[:, c] = dA_0 x_c + dG_0^c cos A_0 (c < 3), dA_0 t (c = 3);  db_0 = dA_0
#pragma unroll
        for (int jg = 0; jg < FPT / 4; ++jg) {
            float4 z[2];
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int64_t i = base + p0 + pp;
                z[pp] = i < n ? *reinterpret_cast<const float4*>(a.w.z0 + i * W + feat_of(jg * 4, fg))
                              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jg * 4 + e, nn = feat_of(j, fg);
                const float wx = W0[nn * IN], wy = W0[nn * IN + 1], wz = W0[nn * IN + 2];
                float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, g3 = 0.0f, gbs = 0.0f;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int p = p0 + pp;
                    const float A = reinterpret_cast<const float*>(&z[pp])[e];
                    float sn, cs;
                    sincos_r(A, &sn, &cs);
                    const float y1 = Y[pp * 4 + 1][j], y2 = Y[pp * 4 + 2][j], y3 = Y[pp * 4 + 3][j];
                    const float dA = Y[pp * 4][j] * cs - sn * (y1 * wx + y2 * wy + y3 * wz);
                    g0 += dA * S.px[p] + y1 * cs;
                    g1 += dA * S.py[p] + y2 * cs;
                    g2 += dA * S.pz[p] + y3 * cs;
                    g3 += dA * S.pt[p];
                    gbs += dA;
                }
                atomicAdd(&S.gw0[nn * 4 + 0], g0);
                atomicAdd(&S.gw0[nn * 4 + 1], g1);
                atomicAdd(&S.gw0[nn * 4 + 2], g2);
                atomicAdd(&S.gw0[nn * 4 + 3], g3);
                atomicAdd(&S.gb[nn], gbs);
            }
        }
    }

    // per-CTA partial sums into dL/dtheta
    __syncthreads();
    for (int i = tid; i < W; i += kSimtThreads) {
        atomicAdd(a.d_theta + sh.off_b0 + i, S.gb[i]);
        for (int l = 0; l < KH; ++l) atomicAdd(a.d_theta + sh.off_b[l] + i, S.gb[(l + 1) * W + i]);
        for (int c = 0; c < IN; ++c) atomicAdd(a.d_theta + sh.off_w0 + i * IN + c, S.gw0[i * 4 + c]);
        atomicAdd(a.d_theta + sh.off_wout + i, S.gwo[i]);
    }
    if (tid == 0) atomicAdd(a.d_theta + sh.off_bout, S.gbo);
}

// ---------------------------------------------------------------------------
// dW_l = sum over rows (point, stream) of (dA_l, dH_l)[row] x (P_{l-1}, G_{l-1})[row]
// ---------------------------------------------------------------------------
// Block: all W units x 64 inputs of dW_l, over a contiguous range of rows
// (split-K over blockIdx.y); the input activations are recomputed from the
// saved pre-activations of the layer below (or layer 0).
constexpr int kWgRows = 32;

template <int W>
__global__ void __launch_bounds__(256) wgrad_kernel(const TrainArgs a, int l, int64_t rows_per_split) {
    constexpr int TM = W / 32;  // units per thread
    __shared__ float Ds[kWgRows][W];
    __shared__ float Xs[kWgRows][64 + 4];
    const int tid = threadIdx.x, tm = tid >> 3, tn = tid & 7;
    const int kb = blockIdx.x * 64;
    const TrainShape& sh = a.sh;
    const int IN = sh.in_dim;
    const int64_t n = a.n, rows = 4 * n;
    const int64_t r_begin = static_cast<int64_t>(blockIdx.y) * rows_per_split;
    const int64_t r_end = r_begin + rows_per_split < rows ? r_begin + rows_per_split : rows;
    const float* dl = a.w.d + static_cast<size_t>(l) * n * 4 * W;
    const float* zb = l > 0 ? a.w.z + static_cast<size_t>(l - 1) * n * 4 * W : nullptr;
    const float* W0 = a.theta + sh.off_w0;
    float acc[TM][8];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[i][b] = 0.0f;

    for (int64_t r0 = r_begin; r0 < r_end; r0 += kWgRows) {
        // adjoint rows (all W units)
        for (int q = tid; q < kWgRows * W / 4; q += 256) {
            const int rr = q / (W / 4), c4 = q % (W / 4);
            const int64_t r = r0 + rr;
            const float4 v = r < r_end ? *reinterpret_cast<const float4*>(dl + r * W + c4 * 4)
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            *reinterpret_cast<float4*>(&Ds[rr][c4 * 4]) = v;
        }
        // input activations of this block's 64 inputs: row tid / 8, inputs (tid % 8) * 8 .. + 7
        {
            const int rr = tid >> 3, c0 = (tid & 7) * 8;
            const int64_t r = r0 + rr;
            const int64_t p = r >> 2;
            const int st = static_cast<int>(r & 3);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int k = kb + c0 + b;
                float x = 0.0f;
                if (r < r_end) {
                    float sn, cs;
                    if (l > 0) {
                        sincos_r(zb[(p * 4) * W + k], &sn, &cs);
                        x = st == 0 ? sn : cs * zb[(p * 4 + st) * W + k];
                    } else {
                        sincos_r(a.w.z0[p * W + k], &sn, &cs);
                        x = st == 0 ? sn : cs * W0[k * IN + st - 1];
                    }
                }
                Xs[rr][c0 + b] = x;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kWgRows; ++rr) {
            float dv[TM], xv[8];
#pragma unroll
            for (int i = 0; i < TM; ++i) dv[i] = Ds[rr][tm * TM + i];
#pragma unroll
            for (int b = 0; b < 8; ++b) xv[b] = Xs[rr][tn * 8 + b];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[i][b] = fmaf(dv[i], xv[b], acc[i][b]);
        }
        __syncthreads();
    }
    float* gw = a.d_theta + sh.off_w[l];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int b = 0; b < 8; ++b) atomicAdd(gw + (tm * TM + i) * W + kb + tn * 8 + b, acc[i][b]);
}

// ---------------------------------------------------------------------------
// fitting objective and its adjoints
// ---------------------------------------------------------------------------
__global__ void count_near_kernel(const uint8_t* __restrict__ near, int64_t n, unsigned long long* cnt) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned c = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) c += near[i] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, static_cast<unsigned long long>(c));
}

__device__ __forceinline__ float sign_of(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

// Per point: the three terms of the objective and dL/df, dL/d(grad f):
//   value:      |f - g|                       -> sign(f - g) / n
//   direction:  1 - <a, b> / (|a| |b|)  (near) -> -(b / (|a| |b|) - cos a / |a|^2) * lam_n / n_near
//   Eikonal:    | |a| - 1 |                    -> sign(|a| - 1) a / |a| * lam_e / n
// (a = grad f, b = the target gradient).  Sums of the terms go to sums[0..2].
__global__ void fit_loss_kernel(const float* __restrict__ f, const float* __restrict__ grad,
                                const float* __restrict__ tf, const float* __restrict__ tgrad,
                                const uint8_t* __restrict__ near, int64_t n, float lam_n, float lam_e,
                                const unsigned long long* n_near, float* __restrict__ df, float* __restrict__ dgrad,
                                double* sums) {
    __shared__ double red[3][8];
    const unsigned long long nn = *n_near;
    const float inv_n = 1.0f / static_cast<float>(n);
    const float dir_w = nn ? lam_n / static_cast<float>(nn) : 0.0f;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float e = f[i] - tf[i];
        df[i] = sign_of(e) * inv_n;
        s0 += fabs(static_cast<double>(e));
        const float ax = grad[i], ay = grad[n + i], az = grad[2 * n + i];
        const float bx = tgrad[i], by = tgrad[n + i], bz = tgrad[2 * n + i];
        const float na = sqrtf(ax * ax + ay * ay + az * az), nb = sqrtf(bx * bx + by * by + bz * bz);
        float gx = 0.0f, gy = 0.0f, gz = 0.0f;
        if (na > 0.0f) {
            const float ek = sign_of(na - 1.0f) * lam_e * inv_n / na;
            gx = ek * ax;
            gy = ek * ay;
            gz = ek * az;
        }
        s2 += fabs(static_cast<double>(na) - 1.0);
        if (near[i] && na > 0.0f && nb > 0.0f) {
            const float inv_ab = 1.0f / (na * nb);
            const float cs = (ax * bx + ay * by + az * bz) * inv_ab;
            s1 += 1.0 - static_cast<double>(cs);
            const float ca = cs / (na * na);
            gx -= dir_w * (bx * inv_ab - ca * ax);
            gy -= dir_w * (by * inv_ab - ca * ay);
            gz -= dir_w * (bz * inv_ab - ca * az);
        }
        dgrad[i] = gx;
        dgrad[n + i] = gy;
        dgrad[2 * n + i] = gz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = s0;
        red[1][w] = s1;
        red[2][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < (blockDim.x >> 5); ++k) t += red[threadIdx.x][k];
        atomicAdd(&sums[threadIdx.x], t);
    }
}

// out = (mean |f - g|, mean over near points of (1 - cos), mean | |grad f| - 1 |, total)
__global__ void fit_loss_finalize_kernel(const double* sums, int64_t n, const unsigned long long* n_near, float lam_n,
                                         float lam_e, double* out) {
    const double lv = sums[0] / static_cast<double>(n);
    const double ld = *n_near ? sums[1] / static_cast<double>(*n_near) : 0.0;
    const double le = sums[2] / static_cast<double>(n);
    out[0] = lv;
    out[1] = ld;
    out[2] = le;
    out[3] = lv + static_cast<double>(lam_n) * ld + static_cast<double>(lam_e) * le;
}

// Adam (Kingma and Ba): m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
// theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float beta1, float beta2, float eps,
                            float c1, float c2) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
        const float g = grad[i];
        const float mi = fmaf(beta1, m[i], (1.0f - beta1) * g);
        const float vi = fmaf(beta2, v[i], (1.0f - beta2) * g * g);
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

template <class Kernel>
cudaError_t launch_simt_persistent(Kernel k, size_t smem, int num_sms, cudaStream_t s, const void* arg) {
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

template <int W>
cudaError_t forward_w(const TrainArgs& a, int num_sms, cudaStream_t s) {
    if (a.sh.n_hidden > 0) {
        dim3 grid(W / 32, W / 32, a.sh.n_hidden);
        transpose_hidden_kernel<<<grid, dim3(32, 8), 0, s>>>(a.theta, a.sh, a.w.wt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemsetAsync(a.w.counters, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    return launch_simt_persistent(train_fwd_kernel<W>, sizeof(FwdSmem<W>), num_sms, s, &a);
}

template <int W>
cudaError_t backward_w(const TrainArgs& a, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.w.counters, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = launch_simt_persistent(train_bwd_kernel<W>, sizeof(BwdSmem<W>), num_sms, s, &a);
    if (e != cudaSuccess) return e;
    // split the rows of each weight-gradient GEMM over about two CTAs per SM
    const int64_t rows = 4 * a.n;
    const int kblocks = W / 64;
    int64_t splits = (2 * num_sms + kblocks - 1) / kblocks;
    int64_t per = (rows + splits - 1) / splits;
    per = (per + kWgRows - 1) / kWgRows * kWgRows;
    splits = (rows + per - 1) / per;
    for (int l = 0; l < a.sh.n_hidden; ++l) {
        wgrad_kernel<W><<<dim3(kblocks, static_cast<unsigned>(splits)), 256, 0, s>>>(a, l, per);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_train_forward(const TrainArgs& a, int num_sms, cudaStream_t s) {
    switch (a.sh.width) {
    case 64:
        return forward_w<64>(a, num_sms, s);
    case 128:
        return forward_w<128>(a, num_sms, s);
    case 256:
        return forward_w<256>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_train_backward(const TrainArgs& a, int num_sms, cudaStream_t s) {
    switch (a.sh.width) {
    case 64:
        return backward_w<64>(a, num_sms, s);
    case 128:
        return backward_w<128>(a, num_sms, s);
    case 256:
        return backward_w<256>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fit_loss(const float* f, const float* grad, const float* tf, const float* tgrad,
                            const uint8_t* near, int64_t n, float lam_n, float lam_e, float* d_f, float* d_grad,
                            double* sums, unsigned long long* n_near, double* out, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sums, 0, 3 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_near, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int blocks = static_cast<int>((n + 255) / 256);
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    if (blocks < 1) blocks = 1;
    count_near_kernel<<<blocks, 256, 0, s>>>(near, n, n_near);
    fit_loss_kernel<<<blocks, 256, 0, s>>>(f, grad, tf, tgrad, near, n, lam_n, lam_e, n_near, d_f, d_grad, sums);
    fit_loss_finalize_kernel<<<1, 1, 0, s>>>(sums, n, n_near, lam_n, lam_e, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                        float beta2, float eps, int step, int num_sms, cudaStream_t s) {
    const double c1 = 1.0 / (1.0 - std::pow(static_cast<double>(beta1), step));
    const double c2 = 1.0 / (1.0 - std::pow(static_cast<double>(beta2), step));
    int blocks = static_cast<int>((count + 255) / 256);
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    if (blocks < 1) blocks = 1;
    adam_kernel<<<blocks, 256, 0, s>>>(theta, grad, m, v, count, lr, beta1, beta2, eps, static_cast<float>(c1),
                                       static_cast<float>(c2));
    return cudaGetLastError();
}

}  // namespace sdfnn
