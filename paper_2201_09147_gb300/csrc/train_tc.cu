// Training path on the tensor cores (SDF_BF16 / SDF_FP16 operands, FP32
// accumulation in TMEM).
//
// The fitting objective depends on f and grad f, so its parameter gradient runs
// backwards through Eq. 2 and the tangent recursion of Alg. 2 (Sec. 5.1).  Per
// hidden layer l, with X_l = (P_l, G_l^x, G_l^y, G_l^z) the four point-streams:
//
//   forward:   A_l = W_l P_{l-1} + b_l,  H_l^c = W_l G_{l-1}^c          (one MMA over X_{l-1})
//              P_l = sin A_l,  G_l^c = cos A_l (.) H_l^c
//   backward:  Y_l = (dP_l, dG_l^c);  D_l = (dA_l, dH_l^c) with
//              dA_l = dP_l (.) cos A_l - sin A_l (.) sum_c dG_l^c (.) H_l^c,  dH_l^c = dG_l^c (.) cos A_l
//              Y_{l-1} = W_l^T D_l                                        (one MMA over D_l)
//              dW_l = sum over point-streams of D_l X_{l-1}^T,  db_l = sum dA_l   (split over the batch)
//
// Three kernels:
//   - the training forward is the analytic-gradient kernel's TRAIN variant
//     (grad_tc.cuh): it saves A_0 and (A_l, H_l) in FP32 and writes f, grad f;
//   - train_bwd_tc_kernel walks a tile of 64 points from the top layer down:
//     the epilogue threads (one per feature) form D_l from Y_l and the saved
//     (A_l, H_l), store it in the MN-major 16-bit layout as the B operand of
//     the MMA Y_{l-1} = W_l^T D_l (W_l^T streamed from L2 by bulk copies), and
//     copy the same 16-byte chunks to a global tile image; the input layer
//     ends in FP32 reductions for W_0, b_0 (and w_out, b_out at the top);
//   - train_wgrad_tc_kernel splits every layer's point-streams over the CTAs:
//     per K block of 64 point-streams it bulk-copies the D tile (a K-major A
//     operand: rows = output units), rebuilds X_{l-1} from the saved
//     pre-activations (K-major B operand: rows = input units) and accumulates
//     dW_l in TMEM, then adds its partial sum to dL/dtheta.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "grad_tc.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace sdfnn {

namespace {

// Half-tiles of 32 points the backward writes D tiles for: it walks pairs of
// halves, so the count is even (the last pair's second half may hold no point).
size_t tile_halves(size_t N) { return 2 * ((N + 63) / 64); }
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
int rows_pad_of(int W) { return W < 128 ? 128 : W; }

}  // namespace


size_t train_tc_workspace_bytes(const TrainShape& sh, int64_t n) {
    const size_t W = sh.width, k = sh.n_hidden, N = static_cast<size_t>(n);
    const size_t halves = tile_halves(N);
    const size_t wimg = static_cast<size_t>(rows_pad_of(sh.width)) * W * 2 * k;
    const size_t NP = static_cast<size_t>(rec_points(n));
    return 2 * align256(wimg) + align256(N * W * 4) + align256(k * NP * W * 4) + align256(k * NP * W * 8) +
           align256(k * halves * W * 256) + 256;
}

TrainWork train_tc_work(const TrainShape& sh, int64_t n, void* ws) {
    const size_t W = sh.width, k = sh.n_hidden, N = static_cast<size_t>(n);
    const size_t halves = tile_halves(N);
    const size_t wimg = static_cast<size_t>(rows_pad_of(sh.width)) * W * 2 * k;
    uint8_t* p = static_cast<uint8_t*>(ws);
    TrainWork w{};
    w.wbf = p;
    p += align256(wimg);
    w.wbft = p;
    p += align256(wimg);
    w.z0 = reinterpret_cast<float*>(p);
    p += align256(N * W * 4);
    const size_t NP = static_cast<size_t>(rec_points(n));
    w.qa = reinterpret_cast<float*>(p);
    p += align256(k * NP * W * 4);
    w.qh = reinterpret_cast<uint2*>(p);
    p += align256(k * NP * W * 8);
    w.dtile = p;
    p += align256(k * halves * W * 256);
    w.counters = reinterpret_cast<unsigned long long*>(p);
    w.n_halves = static_cast<int64_t>(halves);
    return w;
}

namespace {

// Hidden weights of theta as 16-bit tensor-core operands, K-major with the
// 128-byte swizzle and rows padded to max(W, 128): wbf[l] = W_l (rows = output
// units, K = inputs: the forward's A operand) and wbft[l] = W_l^T (rows =
// inputs, K = output units: the backward's A operand).
template <bool F16>
__global__ void pack_hidden_kernel(const float* __restrict__ theta, TrainShape sh, int rows_pad, uint8_t* wbf,
                                   uint8_t* wbft) {
    const int W = sh.width;
    const int64_t per = static_cast<int64_t>(rows_pad) * W, total = per * sh.n_hidden;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int l = static_cast<int>(i / per);
        const int r = static_cast<int>((i % per) / W), k = static_cast<int>(i % W);
        const float* Wl = theta + sh.off_w[l];
        const size_t off = static_cast<size_t>(l) * per * 2 + sw128_offset(r, k, rows_pad);
        uint16_t a = 0, b = 0;
        if (r < W) {
            a = bits16<F16>(Wl[r * W + k]);
            b = bits16<F16>(Wl[k * W + r]);
        }
        *reinterpret_cast<uint16_t*>(wbf + off) = a;
        *reinterpret_cast<uint16_t*>(wbft + off) = b;
    }
}

struct TrainTcArgs {
    NetView net;                 // wbf = the W_l^T images; the FP32 pointers into theta
    TrainShape sh;
    const float* theta;
    const float* pts;            // SoA (3, n)
    const float* pt_time;        // (n) or NULL
    int64_t n;
    const float* d_f;            // (n)
    const float* d_grad;         // SoA (3, n)
    const float* a0;             // [n][W] A_0 (training forward)
    const float* qa;             // A_l records (rec_a layout)
    const uint2* qh;             // H_l records, 16-bit operand type (x, y | z, 0) (rec_h layout)
    int64_t np;                  // points of the record layout (n rounded up to 64)
    uint8_t* dtile;              // [k][n_halves][W * 256]: D_l tiles, 16-bit, the swizzled operand image
    int64_t n_halves;
    float* d_theta;
    int* status;
    const uint32_t* amax_bits;   // bits of max |d_f|, |d_grad| (a non-negative float)
};

// A saved (A_l, H_l) from its A and its 16-bit H image (x, y | z, 0).  The
// kernels load the records of a chunk of consecutive points as 16-byte
// vectors (4 points' A, 2 points' H per load), all in flight at once, and
// decode each one where it is used.
template <bool F16>
__device__ __forceinline__ float4 decode_q(float a, uint32_t hxy, uint32_t hz) {
    return make_float4(a, from16<F16>(static_cast<uint16_t>(hxy & 0xFFFFu)), from16<F16>(static_cast<uint16_t>(hxy >> 16)),
                       from16<F16>(static_cast<uint16_t>(hz & 0xFFFFu)));
}
__device__ __forceinline__ float pick4(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// Hint: bring the line holding p into L2 (no register, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Largest |d_f|, |d_grad| of the batch, as the bits of a non-negative float
// (their order is the floats' order, so an integer maximum serves).
__global__ void adjoint_max_kernel(const float* __restrict__ d_f, const float* __restrict__ d_grad, int64_t n,
                                   uint32_t* amax_bits) {
    uint32_t m = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < 4 * n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float v = i < n ? d_f[i] : d_grad[i - n];
        const uint32_t b = __float_as_uint(fabsf(v));
        if (b < 0x7F800000u && b > m) m = b;  // finite values only
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(amax_bits, m);
}

// ---------------------------------------------------------------------------
// backward through the hidden layers and the input layer
// ---------------------------------------------------------------------------
// The warp roles, weight ring and MMA schedule of the analytic-gradient kernel:
// two epilogue groups (halves of 32 points), a bulk-copy producer streaming the
// W_l^T K blocks of the layers in the order k .. 1, and an MMA warp.  Per pair
// and half: top epilogue (Y_k from the adjoints of the outputs) -> D_k -> MMA
// -> Y_{k-1} -> ... -> D_1 -> MMA -> Y_0 -> input-layer epilogue.
template <int W, bool F16>
__global__ void __launch_bounds__(GradCfg<W, kOpBF16>::THREADS) train_bwd_tc_kernel(const TrainTcArgs a) {
    using C = GradCfg<W, kOpBF16>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const TrainShape& sh = a.sh;
    const int KH = sh.n_hidden, IN = sh.in_dim;
    const GradLayout L = grad_layout<W, kOpBF16>(KH);
    float* w0s = reinterpret_cast<float*>(base + L.w0);
    float* wts = reinterpret_cast<float*>(base + L.wt);
    float4* pts = reinterpret_cast<float4*>(base + L.pts);    // (x, y, z, t) per point
    float4* adj = reinterpret_cast<float4*>(base + L.woutb);  // (df, dg_x, dg_y, dg_z) per point
    int* idxs = reinterpret_cast<int*>(base + L.idx);
    // per-CTA sums (shared, flushed at the end): rows 0..k-1 db_l, k db_0, k+1 dw_out, k+2.. dW_0[:, c]
    float* acc = reinterpret_cast<float*>(base + L.total);
    const int acc_rows = KH + 6;
    const uint32_t bar_full = base_s + L.bars, bar_empty = bar_full + 8u * C::NS;
    const uint32_t bar_xready = bar_empty + 8u * C::NS, bar_dfull = bar_xready + 16u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L.misc + 4);
    float* dbout_s = reinterpret_cast<float*>(base + L.misc + 8);
    const uint32_t x_s = base_s + L.x, ring_s = base_s + L.ring;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < C::NS; ++s) {
            mbar_init(bar_full + 8u * s, 1);
            mbar_init(bar_empty + 8u * s, 1);
        }
        for (int h = 0; h < 2; ++h) {
            mbar_init(bar_xready + 8u * h, C::GROUP_THREADS);
            mbar_init(bar_dfull + 8u * h, 1);
        }
        *abort_flag = 0;
        *dbout_s = 0.0f;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    for (int i = tid; i < W; i += C::THREADS) stage_layer0(a.net, 0.0f, true, i, w0s, wts);
    for (int i = tid; i < acc_rows * W; i += C::THREADS) acc[i] = 0.0f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // S = 2^(126 - e) for the largest |adjoint| 2^(e - 127) * 1.m: S max|adjoint| in [0.5, 1)
    const uint32_t amax_bits = *a.amax_bits;
    const uint32_t e_bits = (amax_bits >> 23) & 0xFFu;
    const float S = (e_bits == 0u) ? 1.0f : __uint_as_float(static_cast<uint32_t>(min(max(253 - static_cast<int>(e_bits), 1), 254)) << 23);
    const float invS = 1.0f / S;  // exact: a power of two

    const long long n_pairs = (a.n + 2 * C::HPTS - 1) / (2 * C::HPTS);
    const long long G = gridDim.x;
    const long long my_pairs = n_pairs > blockIdx.x ? (n_pairs - blockIdx.x + G - 1) / G : 0;
    constexpr int LAG = 1;
    const int n_groups = static_cast<int>(my_pairs) * KH;
    bool ok = true;

    if (warp == C::PRODUCER_WARP) {
        if (lane == 0) {
            uint32_t g = 0;
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    const int l = KH - 1 - grp % KH;  // layers from the top
                    for (int sg = 0; sg < C::STAGES_PER_LAYER && ok; ++sg, ++g) {
                        const uint32_t stage = g % C::NS, use = g / C::NS;
                        if (use > 0) ok = mbar_wait_bounded(bar_empty + 8u * stage, (use - 1) & 1u, a.status, abort_flag);
                        if (!ok) break;
                        mbar_arrive_expect_tx(bar_full + 8u * stage, C::STAGE_BYTES);
                        bulk_g2s(ring_s + stage * C::STAGE_BYTES,
                                 a.net.wbf + static_cast<size_t>(l) * a.net.wbf_layer_bytes +
                                     static_cast<size_t>(sg) * C::STAGE_BYTES,
                                 C::STAGE_BYTES, bar_full + 8u * stage);
                    }
                }
            for (uint32_t gg = g > C::NS ? g - C::NS : 0; gg < g; ++gg)
                mbar_drain(bar_full + 8u * (gg % C::NS), (gg / C::NS) & 1u);
        }
    } else if (warp == C::MMA_WARP) {
        if (lane == 0) {
            constexpr uint32_t idesc_h = idesc_f32acc(128, C::HROWS, F16) | kIdescMajorMnB;
            uint32_t g = 0, xr_phase[2] = {0u, 0u};
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2 && ok; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    ok = mbar_wait_bounded(bar_xready + 8u * h, xr_phase[h], a.status, abort_flag);
                    xr_phase[h] ^= 1u;
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t xh = x_s + h * (W * 256u);
                    for (int sg = 0; sg < C::STAGES_PER_LAYER && ok; ++sg, ++g) {
                        const uint32_t stage = g % C::NS, use = g / C::NS;
                        ok = mbar_wait_bounded(bar_full + 8u * stage, use & 1u, a.status, abort_flag);
                        if (!ok) break;
                        tc_fence_after();
#pragma unroll
                        for (int kr = 0; kr < C::SKB; ++kr) {
                            const int kb = sg * C::SKB + kr;
#pragma unroll
                            for (int mt = 0; mt < C::MT; ++mt)
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    const uint64_t xd = desc_mnmajor_sw128(xh + (kb * 8 + kk * 2) * 1024u, W * 128u);
                                    const uint32_t wa =
                                        ring_s + stage * C::STAGE_BYTES + (kr * C::MT + mt) * 16384u + kk * 32u;
                                    mma_f16kind(tmem + mt * 256u + h * 128u, desc_kmajor_sw128(wa), xd, idesc_h,
                                                (kb | kk) != 0);
                                }
                        }
                        mma_commit(bar_empty + 8u * stage);
                    }
                    if (ok) mma_commit(bar_dfull + 8u * h);
                }
        }
    } else {
        // epilogue group h: thread <-> feature row m (of the layer below the MMA), points 32h .. 32h+31
        const int h = warp / C::GROUP_WARPS, ge = warp % C::GROUP_WARPS;
        const int mt = ge >> 2, quad = ge & 3;
        const int m = mt * 128 + quad * 32 + lane;
        const bool live = m < W;
        const int gt = ge * 32 + lane;
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quad * 32) << 16) + mt * 256u + h * 128u;
        const int p0 = h * C::HPTS;
        const float wo = live ? __ldg(a.theta + sh.off_wout + m) : 0.0f;
        const float4 w0m = live ? reinterpret_cast<const float4*>(w0s)[m] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool timed = a.pt_time != nullptr && IN == 4;
        uint32_t df_phase = 0;
        for (long long i = 0; i < my_pairs; ++i) {
            const long long T = (i * G + blockIdx.x) * 2 + h;  // half-tile of the batch
            if (gt < C::HPTS) {
                const long long k = T * C::HPTS + gt;
                const int idx = k < a.n ? static_cast<int>(k) : -1;
                idxs[p0 + gt] = idx;
                pts[p0 + gt] = idx >= 0 ? make_float4(a.pts[idx], a.pts[a.n + idx], a.pts[2 * a.n + idx],
                                                      timed ? a.pt_time[idx] : 0.0f)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                adj[p0 + gt] = idx >= 0 ? make_float4(a.d_f[idx], a.d_grad[idx], a.d_grad[a.n + idx],
                                                      a.d_grad[2 * a.n + idx])
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            bar_named(1 + h, C::GROUP_THREADS);

            // hidden layers from the top: D_l from Y_l and the saved (A_l, H_l)
            for (int l = KH - 1; l >= -1 && ok; --l) {
                const bool top = l == KH - 1;
                if (!top) {
                    // Y_l (Y_0 of the input layer for l = -1) from the MMA over D_{l+1}
                    ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_dfull + 8u * h, df_phase, a.status, abort_flag));
                    df_phase ^= 1u;
                    if (!ok) break;
                    tc_fence_after();
                }
                uint8_t* dt = l >= 0 ? a.dtile + (static_cast<size_t>(l) * a.n_halves + T) * (W * 256u) : nullptr;
                float s_b = 0.0f, s_o = 0.0f, s_w[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                for (int q = 0; q < C::HROWS / 32; ++q) {
                    // 32 accumulator columns (8 points x 4 streams) of Y; single-buffered: the
                    // global loads below dominate the latency, and registers are scarce at width 256
                    float v[32];
                    if (!top) {
                        tmem_ld32(lane_addr + q * 32u, v);
                        tmem_wait_ld();
                    }
                    if (live && l >= 0) {
                        // the chunk's 8 saved (A, H): independent read-only loads, all in flight at once
                        // the chunk's 8 points are consecutive, the first a multiple of 8
                        float4 a4[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
                        uint4 h4[4] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u),
                                       make_uint4(0u, 0u, 0u, 0u)};
                        const int idx8 = idxs[p0 + q * 8];
                        if (idx8 >= 0) {
#pragma unroll
                            for (int u = 0; u < 2; ++u)
                                a4[u] = __ldg(reinterpret_cast<const float4*>(a.qa + rec_a(l, a.np, W, idx8 + 4 * u, m)));
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                h4[u] = __ldg(reinterpret_cast<const uint4*>(a.qh + rec_h(l, a.np, W, idx8 + 2 * u, m)));
                        }
                        // the next chunk's records (this layer's next chunk, or the first chunk of the
                        // layer below) towards L2 while this one is processed
                        {
                            const int ln = q + 1 < C::HROWS / 32 ? l : l - 1;
                            const int in8 = idxs[p0 + ((q + 1) % (C::HROWS / 32)) * 8];
                            if (ln >= 0 && in8 >= 0) {
#pragma unroll
                                for (int u = 0; u < 2; ++u) prefetch_l2(a.qa + rec_a(ln, a.np, W, in8 + 4 * u, m));
#pragma unroll
                                for (int u = 0; u < 4; ++u) prefetch_l2(a.qh + rec_h(ln, a.np, W, in8 + 2 * u, m));
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            uint32_t w[4];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int p = p0 + q * 8 + 2 * c + e, j = (2 * c + e) * 4;
                                const int ee = 2 * c + e;  // point of the chunk
                                const uint4& hp = h4[ee >> 1];
                                const float4 Q = idxs[p] >= 0 ? decode_q<F16>(pick4(a4[ee >> 2], ee & 3),
                                                                              (ee & 1) ? hp.z : hp.x, (ee & 1) ? hp.w : hp.y)
                                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                                float y0, y1, y2, y3;
                                if (top) {
                                    // the adjoints enter scaled by S (a power of two): 16-bit operands
                                    // then stay in their normal range whatever the loss normalisation
                                    const float4 ad = adj[p];
                                    const float ws = wo * S;
                                    y0 = ad.x * ws;
                                    y1 = ad.y * ws;
                                    y2 = ad.z * ws;
                                    y3 = ad.w * ws;
                                } else {
                                    y0 = v[j];
                                    y1 = v[j + 1];
                                    y2 = v[j + 2];
                                    y3 = v[j + 3];
                                }
                                float sn, cs;
                                sincos_fast(Q.x, &sn, &cs);
                                const float dA = y0 * cs - sn * (y1 * Q.y + y2 * Q.z + y3 * Q.w);
                                s_b += dA;
                                if (top) {
                                    const float4 ad = adj[p];
                                    s_o += ad.x * sn + cs * (ad.y * Q.y + ad.z * Q.z + ad.w * Q.w);
                                }
                                w[2 * e] = pack16x2<F16>(dA, y1 * cs);
                                w[2 * e + 1] = pack16x2<F16>(y2 * cs, y3 * cs);
                            }
                            st_shared_v4(x_s + xoff16<W>(h, m, q * 4 + c), w[0], w[1], w[2], w[3]);
                            *reinterpret_cast<uint4*>(dt + xoff16<W>(0, m, q * 4 + c)) = make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                    if (live && l < 0) {
                        // input layer: dA_0 = dP_0 cos A_0 - sin A_0 sum_c dG_0^c W_0[:, c];
                        // dW_0[:, c] += dA_0 x_c + dG_0^c cos A_0 (c < 3), dA_0 t (c = 3); db_0 += dA_0
                        float A0c[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int idx = idxs[p0 + q * 8 + e];
                            A0c[e] = idx >= 0 ? __ldg(a.a0 + static_cast<size_t>(idx) * W + m) : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int p = p0 + q * 8 + e, j = e * 4;
                            const float A0 = A0c[e];
                            float sn, cs;
                            sincos_fast(A0, &sn, &cs);
                            const float dA = v[j] * cs - sn * (v[j + 1] * w0m.x + v[j + 2] * w0m.y + v[j + 3] * w0m.z);
                            const float4 x = pts[p];
                            s_b += dA;
                            s_w[0] += dA * x.x + v[j + 1] * cs;
                            s_w[1] += dA * x.y + v[j + 2] * cs;
                            s_w[2] += dA * x.z + v[j + 3] * cs;
                            s_w[3] += dA * x.w;
                        }
                    }
                }
                if (live) {
                    atomicAdd(&acc[(l >= 0 ? l : KH) * W + m], s_b);
                    if (top) atomicAdd(&acc[(KH + 1) * W + m], s_o);
                    if (l < 0)
#pragma unroll
                        for (int c = 0; c < 4; ++c) atomicAdd(&acc[(KH + 2 + c) * W + m], s_w[c]);
                }
                if (l >= 0) {
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(bar_xready + 8u * h);
                }
            }
            if (gt == 0) {
                float s = 0.0f;
                for (int p = 0; p < C::HPTS; ++p) s += adj[p0 + p].x;
                atomicAdd(dbout_s, s);
            }
            tc_fence_before();
            // the next pair's point data overwrites this half's; one stop decision for the group
            if (bar_or(1 + h, C::GROUP_THREADS, !ok || *abort_flag != 0)) break;
        }
    }

    tc_fence_before();
    __syncthreads();
    // the CTA's sums into dL/dtheta
    // every sum but dw_out (formed from the unscaled adjoints) carries the factor S
    for (int i = tid; i < W; i += C::THREADS) {
        for (int l = 0; l < KH; ++l) atomicAdd(a.d_theta + sh.off_b[l] + i, acc[l * W + i] * invS);
        atomicAdd(a.d_theta + sh.off_b0 + i, acc[KH * W + i] * invS);
        atomicAdd(a.d_theta + sh.off_wout + i, acc[(KH + 1) * W + i]);
        for (int c = 0; c < IN; ++c)
            atomicAdd(a.d_theta + sh.off_w0 + i * IN + c, acc[(KH + 2 + c) * W + i] * invS);
    }
    if (tid == 0) atomicAdd(a.d_theta + sh.off_bout, *dbout_s);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int W>
size_t bwd_smem_bytes(int KH) {
    return grad_layout<W, kOpBF16>(KH).total + static_cast<size_t>(KH + 6) * W * 4 + 1024;
}

// ---------------------------------------------------------------------------
// weight gradients dW_l = sum over point-streams of D_l X_{l-1}^T
// ---------------------------------------------------------------------------
template <int W>
struct WgCfg {
    static constexpr int MT = W >= 128 ? W / 128 : 1;    // TMEM slabs of 128 output units
    static constexpr uint32_t A_BYTES = MT * 16384u;     // D rows of one K block, padded to 128 rows
    static constexpr uint32_t X_BYTES = W * 128u;        // X rows of one K block
    static constexpr uint32_t STAGE = A_BYTES + X_BYTES;
    static constexpr int NS_FIT = static_cast<int>((200u * 1024u) / STAGE);
    static constexpr int NS = NS_FIT > 6 ? 6 : NS_FIT;
    static constexpr int XW = W / 32;                    // builder warps: one thread per input unit
    static constexpr int PRODUCER_WARP = XW, MMA_WARP = XW + 1;
    static constexpr int THREADS = (XW + 2) * 32;
    static constexpr int TMEM_COLS = MT * W;
    static_assert(NS >= 2, "stages");
};

template <int W>
constexpr size_t wgrad_smem_bytes() {
    using C = WgCfg<W>;
    return C::NS * C::STAGE + W * 16u + (3 * C::NS + 2) * 8u + 32u + 1024u;
}

template <int W, bool F16>
__global__ void __launch_bounds__(WgCfg<W>::THREADS) train_wgrad_tc_kernel(const TrainTcArgs a) {
    using C = WgCfg<W>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const TrainShape& sh = a.sh;
    const int KH = sh.n_hidden;
    const uint32_t st_s = base_s;                               // NS stages: [A | X]
    float* w0s = reinterpret_cast<float*>(base + C::NS * C::STAGE);  // W_0[:, 0..2] per unit (float4)
    const uint32_t bars = base_s + C::NS * C::STAGE + W * 16u;
    const uint32_t bar_full = bars, bar_xfull = bars + 8u * C::NS, bar_empty = bars + 16u * C::NS;
    const uint32_t bar_done = bars + 24u * C::NS, bar_flushed = bar_done + 8u;
    uint8_t* misc = base + C::NS * C::STAGE + W * 16u + (3 * C::NS + 2) * 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < C::NS; ++s) {
            mbar_init(bar_full + 8u * s, 1);
            mbar_init(bar_xfull + 8u * s, C::XW * 32);
            mbar_init(bar_empty + 8u * s, 1);
        }
        mbar_init(bar_done, 1);
        mbar_init(bar_flushed, C::XW * 32);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    // widths below 128: the A operand's rows W .. 127 stay zero (copies write rows 0 .. W-1)
    if (W < 128)
        for (int s = 0; s < C::NS; ++s)
            for (uint32_t i = W * 128u + tid * 16u; i < C::A_BYTES; i += C::THREADS * 16u)
                st_shared_v4(st_s + s * C::STAGE + i, 0u, 0u, 0u, 0u);
    for (int i = tid; i < W; i += C::THREADS)
        for (int c = 0; c < 4; ++c) w0s[i * 4 + c] = c < 3 ? a.net.w0[i * sh.in_dim + c] : 0.0f;
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the D tiles carry the backward's adjoint scale S (a power of two)
    const uint32_t e_bits = (*a.amax_bits >> 23) & 0xFFu;
    const float invS = (e_bits == 0u)
                           ? 1.0f
                           : 1.0f / __uint_as_float(static_cast<uint32_t>(min(max(253 - static_cast<int>(e_bits), 1), 254)) << 23);

    // K blocks (64 point-streams = 16 points) of every layer, split over the CTAs
    const int64_t total = 2 * a.n_halves;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t kb_lo = static_cast<int64_t>(blockIdx.x) * per;
    const int64_t kb_hi = std::min<int64_t>(total, kb_lo + per);
    bool ok = true;

    if (kb_hi > kb_lo) {
        if (warp == C::PRODUCER_WARP) {
            if (lane == 0) {
                uint32_t g = 0;
                for (int l = 0; l < KH && ok; ++l)
                    for (int64_t kb = kb_lo; kb < kb_hi && ok; ++kb, ++g) {
                        const uint32_t stage = static_cast<uint32_t>(g % C::NS), use = static_cast<uint32_t>(g / C::NS);
                        if (use > 0) ok = mbar_wait_bounded(bar_empty + 8u * stage, (use - 1) & 1u, a.status, abort_flag);
                        if (!ok) break;
                        mbar_arrive_expect_tx(bar_full + 8u * stage, W * 128u);
                        bulk_g2s(st_s + stage * C::STAGE,
                                 a.dtile + (static_cast<size_t>(l) * a.n_halves + kb / 2) * (W * 256u) +
                                     static_cast<size_t>(kb & 1) * (W * 128u),
                                 W * 128u, bar_full + 8u * stage);
                    }
                for (uint32_t gg = g > C::NS ? g - C::NS : 0; gg < g; ++gg)
                    mbar_drain(bar_full + 8u * (gg % C::NS), (gg / C::NS) & 1u);
            }
        } else if (warp == C::MMA_WARP) {
            if (lane == 0) {
                constexpr uint32_t idesc = idesc_f32acc(128, W, F16);
                uint32_t g = 0;
                for (int l = 0; l < KH && ok; ++l) {
                    if (l > 0) ok = mbar_wait_bounded(bar_flushed, (l - 1) & 1u, a.status, abort_flag);
                    for (int64_t kb = kb_lo; kb < kb_hi && ok; ++kb, ++g) {
                        const uint32_t stage = static_cast<uint32_t>(g % C::NS), use = static_cast<uint32_t>(g / C::NS);
                        ok = mbar_wait_bounded(bar_full + 8u * stage, use & 1u, a.status, abort_flag) &&
                             mbar_wait_bounded(bar_xfull + 8u * stage, use & 1u, a.status, abort_flag);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t sa = st_s + stage * C::STAGE, sx = sa + C::A_BYTES;
#pragma unroll
                        for (int mt = 0; mt < C::MT; ++mt)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_f16kind(tmem + mt * W, desc_kmajor_sw128(sa + mt * 16384u + kk * 32u),
                                            desc_kmajor_sw128(sx + kk * 32u), idesc, (kb != kb_lo || kk != 0) ? 1u : 0u);
                        mma_commit(bar_empty + 8u * stage);
                    }
                    if (ok) mma_commit(bar_done);
                }
            }
        } else {
            // builders: thread k = input unit of X_{l-1}; then the TMEM rows of dW_l
            const int k = tid;
            const int mt = warp >> 2, quad = warp & 3;
            const int nrow = mt * 128 + quad * 32 + lane;  // output unit of the TMEM lane read below
            const float4 w0k = reinterpret_cast<const float4*>(w0s)[k];
            uint32_t g = 0;
            for (int l = 0; l < KH && ok; ++l) {
                for (int64_t kb = kb_lo; kb < kb_hi && ok; ++kb, ++g) {
                    const uint32_t stage = static_cast<uint32_t>(g % C::NS), use = static_cast<uint32_t>(g / C::NS);
                    if (use > 0)
                        ok = __all_sync(0xffffffffu,
                                        mbar_wait_bounded(bar_empty + 8u * stage, (use - 1) & 1u, a.status, abort_flag));
                    if (!ok) break;
                    const uint32_t sx = st_s + stage * C::STAGE + C::A_BYTES;
                    const int64_t pbase = (kb >> 1) * 32 + (kb & 1) * 16;
                    // the K block's 16 saved (A, H) (or A_0): independent read-only loads first
                    // the K block's 16 consecutive points (pbase a multiple of 16): layer l - 1's records
                    // as 4 + 8 16-byte loads, or A_0 (layer 0, whose tangents are W_0's columns)
                    float4 a4[4];
                    uint4 h4[8];
#pragma unroll
                    for (int u = 0; u < 4; ++u) a4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 8; ++u) h4[u] = make_uint4(0u, 0u, 0u, 0u);
                    if (pbase < a.n) {
                        if (l > 0) {
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                a4[u] = __ldg(reinterpret_cast<const float4*>(a.qa + rec_a(l - 1, a.np, W, pbase + 4 * u, k)));
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                h4[u] = __ldg(reinterpret_cast<const uint4*>(a.qh + rec_h(l - 1, a.np, W, pbase + 2 * u, k)));
                        } else {
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float v0 = pbase + u < a.n ? __ldg(a.a0 + static_cast<size_t>(pbase + u) * W + k) : 0.0f;
                                if ((u & 3) == 0) a4[u >> 2].x = v0;
                                else if ((u & 3) == 1) a4[u >> 2].y = v0;
                                else if ((u & 3) == 2) a4[u >> 2].z = v0;
                                else a4[u >> 2].w = v0;
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        uint32_t w[4];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int64_t p = pbase + 2 * c + e;
                            const int ee = 2 * c + e;
                            const uint4& hp = h4[ee >> 1];
                            const float A = pick4(a4[ee >> 2], ee & 3);
                            // layer 0's tangents are W_0's columns (FP32); above, the saved H_l;
                            // points past the batch (the padding is never written) are zero
                            float4 Q = l > 0 ? decode_q<F16>(A, (ee & 1) ? hp.z : hp.x, (ee & 1) ? hp.w : hp.y)
                                             : make_float4(A, w0k.x, w0k.y, w0k.z);
                            if (p >= a.n) Q = make_float4(0.f, 0.f, 0.f, 0.f);
                            float sn = 0.0f, cs = 0.0f;
                            if (p < a.n) sincos_fast(Q.x, &sn, &cs);
                            w[2 * e] = pack16x2<F16>(sn, cs * Q.y);
                            w[2 * e + 1] = pack16x2<F16>(cs * Q.z, cs * Q.w);
                        }
                        st_shared_v4(sx + (k >> 3) * 1024u + (k & 7) * 128u + ((c ^ (k & 7)) << 4), w[0], w[1], w[2],
                                     w[3]);
                    }
                    fence_proxy_async_smem();
                    mbar_arrive(bar_xfull + 8u * stage);
                }
                if (!ok) break;
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_done, l & 1u, a.status, abort_flag));
                if (!ok) break;
                tc_fence_after();
                float* gw = a.d_theta + sh.off_w[l];
                for (int cc = 0; cc < W / 32; ++cc) {
                    float v[32];
                    tmem_ld32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + mt * W + cc * 32u, v);
                    tmem_wait_ld();
                    if (nrow < W) {
                        // 16-byte vector reductions: a quarter of the atomic operations of scalar ones
                        float4* row = reinterpret_cast<float4*>(gw + static_cast<size_t>(nrow) * W + cc * 32);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            atomicAdd(row + i, make_float4(v[4 * i] * invS, v[4 * i + 1] * invS, v[4 * i + 2] * invS,
                                                           v[4 * i + 3] * invS));
                    }
                }
                tc_fence_before();
                mbar_arrive(bar_flushed);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int W, bool F16>
cudaError_t forward_tc_w(const TrainArgs& a, int num_sms, cudaStream_t s) {
    const TrainShape& sh = a.sh;
    const int rows_pad = rows_pad_of(W);
    const int64_t cells = static_cast<int64_t>(rows_pad) * W * sh.n_hidden;
    int blocks = static_cast<int>(std::min<int64_t>((cells + 255) / 256, 8 * num_sms));
    pack_hidden_kernel<F16><<<blocks, 256, 0, s>>>(a.theta, sh, rows_pad, a.w.wbf, a.w.wbft);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    NetView v{};
    v.in_dim = sh.in_dim;
    v.width = W;
    v.n_hidden = sh.n_hidden;
    v.w0 = a.theta + sh.off_w0;
    v.b0 = a.theta + sh.off_b0;
    for (int l = 0; l < sh.n_hidden; ++l) v.bh[l] = a.theta + sh.off_b[l];
    v.wout = a.theta + sh.off_wout;
    v.wbf = a.w.wbf;
    v.wbf_layer_bytes = static_cast<uint32_t>(rows_pad) * W * 2u;
    v.rows_pad = rows_pad;
    v.op_f16 = F16 ? 1 : 0;
    GradArgs ga{};
    ga.net = v;
    ga.pt_time = a.pt_time;
    ga.pts = a.pts;
    ga.n = a.n;
    ga.out = a.out_grad;
    ga.grab = a.w.counters;
    ga.status = a.status;
    ga.save_a0 = a.w.z0;
    ga.save_a = a.w.qa;
    ga.save_h = a.w.qh;
    ga.save_np = rec_points(a.n);
    ga.out_f = a.out_f;
    ga.out_bias = a.theta + sh.off_bout;
    using C = GradCfg<W, F16 ? kOpF16 : kOpBF16>;
    const size_t smem = grad_layout<W, F16 ? kOpF16 : kOpBF16, true>(sh.n_hidden).total + 1024;
    return launch_tc(grad_tc_kernel<W, F16 ? kOpF16 : kOpBF16, true>, C::THREADS, smem, C::TMEM_COLS, num_sms, s,
                     &ga);
}

template <int W, bool F16>
cudaError_t backward_tc_w(const TrainArgs& a, int num_sms, cudaStream_t s) {
    const TrainShape& sh = a.sh;
    const int rows_pad = rows_pad_of(W);
    TrainTcArgs t{};
    t.net.in_dim = sh.in_dim;
    t.net.width = W;
    t.net.n_hidden = sh.n_hidden;
    t.net.w0 = a.theta + sh.off_w0;
    t.net.b0 = a.theta + sh.off_b0;
    t.net.wbf = a.w.wbft;
    t.net.wbf_layer_bytes = static_cast<uint32_t>(rows_pad) * W * 2u;
    t.net.rows_pad = rows_pad;
    t.sh = sh;
    t.theta = a.theta;
    t.pts = a.pts;
    t.pt_time = a.pt_time;
    t.n = a.n;
    t.d_f = a.d_f;
    t.d_grad = a.d_grad;
    t.a0 = a.w.z0;
    t.qa = a.w.qa;
    t.qh = a.w.qh;
    t.np = rec_points(a.n);
    t.dtile = a.w.dtile;
    t.n_halves = a.w.n_halves;
    t.d_theta = a.d_theta;
    t.status = a.status;
    uint32_t* amax = reinterpret_cast<uint32_t*>(a.w.counters);
    t.amax_bits = amax;
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    adjoint_max_kernel<<<num_sms * 4, 256, 0, s>>>(a.d_f, a.d_grad, a.n, amax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    using C = GradCfg<W, kOpBF16>;
    e = launch_tc(train_bwd_tc_kernel<W, F16>, C::THREADS, bwd_smem_bytes<W>(sh.n_hidden), C::TMEM_COLS,
                              num_sms, s, &t);
    if (e != cudaSuccess) return e;
    using D = WgCfg<W>;
    return launch_tc(train_wgrad_tc_kernel<W, F16>, D::THREADS, wgrad_smem_bytes<W>(), D::TMEM_COLS, num_sms, s, &t);
}

}  // namespace

cudaError_t launch_train_forward_tc(const TrainArgs& a, bool f16, int num_sms, cudaStream_t s) {
    switch (a.sh.width) {
    case 64:
        return f16 ? forward_tc_w<64, true>(a, num_sms, s) : forward_tc_w<64, false>(a, num_sms, s);
    case 128:
        return f16 ? forward_tc_w<128, true>(a, num_sms, s) : forward_tc_w<128, false>(a, num_sms, s);
    case 256:
        return f16 ? forward_tc_w<256, true>(a, num_sms, s) : forward_tc_w<256, false>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_train_backward_tc(const TrainArgs& a, bool f16, int num_sms, cudaStream_t s) {
    switch (a.sh.width) {
    case 64:
        return f16 ? backward_tc_w<64, true>(a, num_sms, s) : backward_tc_w<64, false>(a, num_sms, s);
    case 128:
        return f16 ? backward_tc_w<128, true>(a, num_sms, s) : backward_tc_w<128, false>(a, num_sms, s);
    case 256:
        return f16 ? backward_tc_w<256, true>(a, num_sms, s) : backward_tc_w<256, false>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sdfnn
