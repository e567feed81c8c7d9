// Tensor-core (tcgen05) kernels of the 16-bit and 8-bit paths (SDF_BF16,
// SDF_FP16, SDF_FP8), FP32 accumulation in TMEM; the operand type is a
// template parameter (tcgen05.mma.kind::f16 for bfloat16 / half,
// kind::f8f6f4 for E4M3).
//
// trace_level_tc : one level of multiscale sphere tracing (Alg. 1).  A CTA
//   holds up to six independent tiles of 128 persistent ray slots, one per
//   thread and per TMEM lane, sharing one copy of the weights.  Each
//   evaluation of f (Eq. 2) runs layer 0 in FP32 on the CUDA cores, writes
//   sin(A_0) in 16 bits (head and remainder) into the A operand (128 rays x
//   width, K-major, 128-byte swizzle), then for every hidden layer one thread
//   of the tile issues tcgen05.mma (M = 128 rays, N = width, K = width)
//   against the resident 16-bit weights; each thread reads its own row back
//   with tcgen05.ld, adds the bias and applies the sine in registers.  The
//   output layer is an FP32 dot product of the last sine layer straight from
//   TMEM, so the step t = f - d is never rounded to 16 bits.  Once the work
//   list is empty the CTA regroups its remaining rays into its first tiles
//   every few iterations.  Width 256 (trace_level_tc_stream): two tiles share
//   hidden weights streamed through a ring of bulk-copied stages.
//
// grad_tc : analytic gradients (Alg. 2).  Tiles of 64 points in two halves;
//   the MMA runs with the features as rows (M = 128 per TMEM tile,
//   width/128 tiles) and N = 128 columns = 32 points x {forward, G^x, G^y,
//   G^z} per half, so one weight tile feeds the forward pass and the three
//   tangents at once and the thread that owns feature m finds A_i[m] and the
//   three G_i[m] of a point in its own TMEM lane: the epilogue
//   P_i = sin(A_i), G_i = cos(A_i) (.) (W_i G_{i-1}) needs no data exchange.
//   Hidden weights stream from L2 through a ring of shared-memory stages
//   filled by bulk copies (TMA); the output layer W_n G_{n-1} is one more
//   small MMA (rows = the 128 point-streams of a half, N = 16, w_out as a
//   head row plus a remainder row).
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "grad_tc.cuh"
#include "internal.h"
#include "launch_cache.h"
#include "rays.cuh"
#include "tc_common.cuh"

namespace sdfnn {
namespace {


// ---------------------------------------------------------------------------
// trace kernel
// ---------------------------------------------------------------------------

struct TraceLayout {
    uint32_t x, xlo, w, wlo, w0, wt, bh, wout, bars, misc, total;
};

// Shared-memory layout of the resident-weight trace kernel with T ray tiles
// (128 rays each) sharing one copy of the weights.  With `split` the
// activations and weights are each held as a 16-bit head plus the 16-bit
// rounding of the remainder (two operand copies).
__host__ __device__ inline TraceLayout trace_layout(int W, int KH, bool split, int T) {
    TraceLayout L;
    uint32_t o = 0;
    const uint32_t xbytes = 128u * W * 2u, wbytes = static_cast<uint32_t>(KH) * W * W * 2u;
    L.x = o;
    o += xbytes * T;
    L.xlo = o;
    o += split ? xbytes * T : 0u;
    L.w = o;
    o += wbytes;
    L.wlo = o;
    o += split ? wbytes : 0u;
    L.w0 = o;
    o += W * 4u * 4u;
    L.wt = o;
    o += W * 4u;
    L.bh = o;
    o += static_cast<uint32_t>(KH) * W * 4u;
    L.wout = o;
    o += W * 4u;
    L.bars = o;
    o += 8u * (1 + 8);
    o = (o + 15u) & ~15u;
    L.misc = o;
    o += 64u;
    L.total = o;
    return L;
}

constexpr uint32_t kSplitSmemLimit = 200u * 1024u;
constexpr int kTailRound = 4;  // trace iterations between two regroupings of the tail's rays
constexpr int kMaxTraceTiles = 6;
constexpr int kTraceMaxThreads = 128 * kMaxTraceTiles;

// The trace kernel's tensor pipe is mostly idle (its time goes to the sines),
// so whenever the doubled operands fit it computes each hidden layer as
// hi(W) hi(X) + lo(W) hi(X) + hi(W) lo(X) with hi/lo the 16-bit head and
// remainder: the contraction then carries ~16 (BF16) or ~22 (FP16)
// significant bits instead of 8 or 11.
inline bool trace_split(int W, int KH) { return trace_layout(W, KH, true, 1).total + 1024 <= kSplitSmemLimit; }

__host__ __device__ inline uint32_t tmem_cols_for(int cols) {
    uint32_t n = 32;
    while (n < static_cast<uint32_t>(cols)) n <<= 1;
    return n;
}

// 16-bit head and remainder of two floats, packed as pairs (the two
// remainders in one packed FP32 operation: a - head(a) by an FMA with -1,
// which is exact in the product, so each lane is the rounded difference).
template <bool F16>
__device__ __forceinline__ void pack_split(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pack16x2<F16>(a, b);
    const float2 h = make_float2(from16<F16>(static_cast<uint16_t>(hi & 0xFFFFu)),
                                 from16<F16>(static_cast<uint16_t>(hi >> 16)));
    const float2 r = __ffma2_rn(h, make_float2(-1.0f, -1.0f), make_float2(a, b));
    lo = pack16x2<F16>(r.x, r.y);
}


// The same parameters laid out for packed FP32 arithmetic on unit pairs
// (trace kernels): pair p = units 2p, 2p+1 as two float4s,
// (w_x0, w_x1, w_y0, w_y1) and (w_z0, w_z1, b0, b1); w_t per unit as before.
__device__ __forceinline__ void stage_layer0_pairs(const NetView& net, float time, bool timed, int i, float* w0s,
                                                   float* wts) {
    const int p = i >> 1, e = i & 1;
    float bb = net.b0[i];
    const float wt = net.in_dim == 4 ? net.w0[i * 4 + 3] : 0.0f;
    if (!timed) bb = fmaf(wt, time, bb);
    w0s[p * 8 + e] = net.w0[i * net.in_dim + 0];
    w0s[p * 8 + 2 + e] = net.w0[i * net.in_dim + 1];
    w0s[p * 8 + 4 + e] = net.w0[i * net.in_dim + 2];
    w0s[p * 8 + 6 + e] = bb;
    wts[i] = timed ? wt : 0.0f;
}

// Layer 0 (FP32) of one ray row: X[row] = 16-bit sin(W_0 (p, t) + b_0),
// as a head and (SPLIT) the rounding of the remainder.  Two units per packed
// FP32 FMA chain, in the same order as the scalar form
// w_x p_x + (w_y p_y + (w_z p_z + b)), so each lane rounds as a scalar FMA
// would.  With TIMED the ray's time is read here (it is not kept in a
// register between steps).
// w0p: the pairs in shared memory, or (width 64) in the launch parameters.
template <int W, bool F16, bool SPLIT, bool TIMED>
__device__ __forceinline__ void trace_layer0(const LevelArgs& a, const float4* w0p, const float* wts, const Ray& ray,
                                             int row, uint32_t x_s, uint32_t xlo_s) {
    const float tm = (TIMED && ray.state == kSlotActive) ? __ldg(a.ray_time + ray.idx) : 0.0f;
    const float2 px = make_float2(ray.px, ray.px), py = make_float2(ray.py, ray.py), pz = make_float2(ray.pz, ray.pz);
    const float2 t2 = make_float2(tm, tm);
    for (int k8 = 0; k8 < W / 8; ++k8) {
        uint32_t pk[4], pl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int pr = k8 * 4 + q;
            const float4 A = w0p[2 * pr];
            const float4 B = w0p[2 * pr + 1];
            float2 c = make_float2(B.z, B.w);
            if (TIMED) c = __ffma2_rn(reinterpret_cast<const float2*>(wts)[pr], t2, c);
            const float2 z = __ffma2_rn(make_float2(A.x, A.y), px,
                                        __ffma2_rn(make_float2(A.z, A.w), py, __ffma2_rn(make_float2(B.x, B.y), pz, c)));
            if (SPLIT)
                pack_split<F16>(sin_fast(z.x), sin_fast(z.y), pk[q], pl[q]);
            else
                pk[q] = pack16x2<F16>(sin_fast(z.x), sin_fast(z.y));
        }
        const uint32_t off = sw128_chunk_offset(row, k8, 128);
        st_shared_v4(x_s + off, pk[0], pk[1], pk[2], pk[3]);
        if (SPLIT) st_shared_v4(xlo_s + off, pl[0], pl[1], pl[2], pl[3]);
    }
}

// Output layer of one ray row from N of its TMEM accumulator columns:
// acc += w_out . sin(D + b), the bias additions and the products on unit
// pairs (two packed accumulators, for units 4j, 4j+1 and 4j+2, 4j+3).
template <int N, bool SCALED = false>
__device__ __forceinline__ void output_dot(const float (&v)[N], const float* bl, const float* wo, float2& acc01,
                                           float2& acc23, float sc = 1.0f) {
    const float2 sc2 = make_float2(sc, sc);
#pragma unroll
    for (int j4 = 0; j4 < N / 4; ++j4) {
        const float4 b4 = reinterpret_cast<const float4*>(bl)[j4];
        const float4 w4 = reinterpret_cast<const float4*>(wo)[j4];
        const float2 v01 = make_float2(v[4 * j4 + 0], v[4 * j4 + 1]), v23 = make_float2(v[4 * j4 + 2], v[4 * j4 + 3]);
        // SCALED (E4M3 operands): the accumulator times the inverse of the operand scales
        const float2 x01 = SCALED ? __ffma2_rn(v01, sc2, make_float2(b4.x, b4.y)) : __fadd2_rn(v01, make_float2(b4.x, b4.y));
        const float2 x23 = SCALED ? __ffma2_rn(v23, sc2, make_float2(b4.z, b4.w)) : __fadd2_rn(v23, make_float2(b4.z, b4.w));
        acc01 = __ffma2_rn(make_float2(w4.x, w4.y), make_float2(sin_fast(x01.x), sin_fast(x01.y)), acc01);
        acc23 = __ffma2_rn(make_float2(w4.z, w4.w), make_float2(sin_fast(x23.x), sin_fast(x23.y)), acc23);
    }
}

template <bool SCALED = false>
__device__ __forceinline__ void output_dot32(const float (&v)[32], const float* bl, const float* wo, float2& acc01,
                                             float2& acc23, float sc = 1.0f) {
    output_dot<32, SCALED>(v, bl, wo, acc01, acc23, sc);
}

// Hidden epilogue of one ray row for N columns from c0 (N a multiple of 8):
// X row chunks = 16-bit sin(D + b) (head, and with SPLIT the remainder),
// bias additions on unit pairs.
template <int N, bool F16, bool SPLIT>
__device__ __forceinline__ void hidden_epilogue(const float (&v)[N], const float* bl, int row, int c0, uint32_t x_s,
                                                uint32_t xlo_s) {
#pragma unroll
    for (int q = 0; q < N / 8; ++q) {
        uint32_t pk[4], pl[4];
        const float4 ba = reinterpret_cast<const float4*>(bl + c0)[2 * q];
        const float4 bb = reinterpret_cast<const float4*>(bl + c0)[2 * q + 1];
        const float2 b2[4] = {make_float2(ba.x, ba.y), make_float2(ba.z, ba.w), make_float2(bb.x, bb.y),
                              make_float2(bb.z, bb.w)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = q * 8 + 2 * e;
            const float2 x = __fadd2_rn(make_float2(v[j], v[j + 1]), b2[e]);
            const float s0 = sin_fast(x.x), s1 = sin_fast(x.y);
            if (SPLIT)
                pack_split<F16>(s0, s1, pk[e], pl[e]);
            else
                pk[e] = pack16x2<F16>(s0, s1);
        }
        const uint32_t off = sw128_chunk_offset(row, (c0 >> 3) + q, 128);
        st_shared_v4(x_s + off, pk[0], pk[1], pk[2], pk[3]);
        if (SPLIT) st_shared_v4(xlo_s + off, pl[0], pl[1], pl[2], pl[3]);
    }
}

template <bool F16, bool SPLIT>
__device__ __forceinline__ void hidden_epilogue32(const float (&v)[32], const float* bl, int row, int c0,
                                                  uint32_t x_s, uint32_t xlo_s) {
    hidden_epilogue<32, F16, SPLIT>(v, bl, row, c0, x_s, xlo_s);
}

// T = blockDim.x / 128 independent ray tiles per CTA.  Tile t owns warps
// 4t..4t+3 (so its threads read TMEM lanes 0..127), TMEM columns
// [t*W, (t+1)*W), its own activation buffers, MMA mbarrier and named barrier
// 1 + t; the weights and layer parameters are shared.
template <int W, bool F16, bool SPLIT>
__global__ void __launch_bounds__(kTraceMaxThreads, 1) trace_level_tc_kernel(const LevelArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const NetView& net = a.net;
    const int KH = net.n_hidden;
    const int T = blockDim.x >> 7;
    const TraceLayout L = trace_layout(W, KH, SPLIT, T);
    float* w0s = reinterpret_cast<float*>(base + L.w0);
    float* wts = reinterpret_cast<float*>(base + L.wt);
    float* bhs = reinterpret_cast<float*>(base + L.bh);
    float* wos = reinterpret_cast<float*>(base + L.wout);
    // layer 0, the last hidden bias and the output weights: launch parameters at width 64
    constexpr bool kc = W == kConstWidth;
    const float4* w0p = kc ? a.k.w0 : reinterpret_cast<const float4*>(w0s);
    const float* blast = kc ? reinterpret_cast<const float*>(a.k.bl) : bhs + (KH - 1) * W;
    const float* wop = kc ? reinterpret_cast<const float*>(a.k.wo) : wos;
    const uint32_t bar_w = base_s + L.bars;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L.misc + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = tid >> 7, ttid = tid & 127, twarp = ttid >> 5;
    const int issuer = 32 * (tile & 3);  // lane 0 of the tile's warp (tile mod 4)
    constexpr uint32_t xbytes = 128u * W * 2u;
    const uint32_t bar_mma = base_s + L.bars + 8u * (1 + tile);
    const uint32_t x_s = base_s + L.x + tile * xbytes, xlo_s = base_s + L.xlo + tile * xbytes;
    const uint32_t w_s = base_s + L.w, wlo_s = base_s + L.wlo;
    const uint32_t tcols = tmem_cols_for(T * W);

    if (tid == 0) {
        mbar_init(bar_w, 1);
        for (int t = 0; t < T; ++t) mbar_init(base_s + L.bars + 8u * (1 + t), 1);
        *abort_flag = 0;
        *reinterpret_cast<uint32_t*>(base + L.misc + 16) = 0u;  // tail round counter
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), tcols);
        tmem_relinquish();
    }
    const bool timed = a.ray_time != nullptr && net.in_dim == 4;
    for (int i = tid; i < W; i += blockDim.x) {
        stage_layer0_pairs(net, a.time, timed, i, w0s, wts);
        wos[i] = net.wout[i];
        for (int l = 0; l < KH; ++l) bhs[l * W + i] = net.bh[l][i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot + static_cast<uint32_t>(tile * W);

    if (tid == 0) {
        mbar_arrive_expect_tx(bar_w, static_cast<uint32_t>(KH) * W * W * 2u * (SPLIT ? 2u : 1u));
        for (int l = 0; l < KH; ++l)
            for (int kb = 0; kb < W / 64; ++kb) {
                const size_t src = static_cast<size_t>(l) * net.wbf_layer_bytes + static_cast<size_t>(kb) * net.rows_pad * 128u;
                bulk_g2s(w_s + l * W * W * 2u + kb * W * 128u, net.wbf + src, W * 128u, bar_w);
                if (SPLIT) bulk_g2s(wlo_s + l * W * W * 2u + kb * W * 128u, net.wbf_lo + src, W * 128u, bar_w);
            }
    }
    // the weights are in, or the whole block gives up (one decision for all threads)
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar_w, 0, a.status, abort_flag) ? 1 : 0) != 0;

    const long long n_work = a.in_list ? static_cast<long long>(*a.in_count) : a.n;
    const uint32_t lane_base = static_cast<uint32_t>(twarp * 32) << 16;
    constexpr uint32_t idesc = idesc_f32acc(128, W, F16);
    uint32_t mma_phase = 0;
    const int bar_id = 1 + tile;
    Ray ray;

    if (ok && a.cap <= 0) {
        // a level with no iterations passes its rays on unchanged
        while (true) {
            refill_ray(a, ray, n_work);
            if (!bar_or(bar_id, 128, ray.state == kSlotActive)) break;
            pass_ray(a, ray);
        }
    } else if (ok) {
        // Two phases.  While the work list lasts, each tile refills its slots
        // and runs on its own; the first time a refill comes back empty the
        // tile enters the tail.  In the tail the block works in rounds of
        // kTailRound iterations: at each round boundary (all tiles at a block
        // barrier) the active rays of all tiles are gathered and dealt out
        // again to the first tiles, so the long rays that remain run in as few
        // tiles as possible instead of keeping every tile alive for a few rays.
        // A thread that sees a timeout drops its ray; every stop decision goes
        // through a barrier that all threads of the tile (or block) reach.
        uint32_t* tail_count = reinterpret_cast<uint32_t*>(base + L.misc + 16);
        uint32_t* rec = reinterpret_cast<uint32_t*>(base + L.x);  // round records, 12 words per ray
        bool tail = false, live = true;
        int it = 0;
        while (true) {
            if (!tail) {
                refill_ray(a, ray, n_work);
            } else if (it >= kTailRound || !live) {
                __syncthreads();  // every tile is at the boundary: X, TMEM and the records are free
                if (ray.state == kSlotActive) {
                    const uint32_t r = atomicAdd(tail_count, 1u) * 12u;
                    st_shared_v4(smem_u32(rec + r), static_cast<uint32_t>(ray.idx), static_cast<uint32_t>(ray.nlev),
                                 static_cast<uint32_t>(ray.ntot), __float_as_uint(ray.tau));
                    st_shared_v4(smem_u32(rec + r + 4), __float_as_uint(ray.px), __float_as_uint(ray.py),
                                 __float_as_uint(ray.pz), __float_as_uint(ray.vx));
                    st_shared_v4(smem_u32(rec + r + 8), __float_as_uint(ray.vy), __float_as_uint(ray.vz), 0u, 0u);
                }
                __syncthreads();
                const int count = static_cast<int>(*tail_count);
                const bool stop = count == 0 || *abort_flag != 0;
                if (!stop && tid < count) {
                    const uint32_t* q = rec + tid * 12;
                    ray.idx = static_cast<int>(q[0]);
                    ray.nlev = static_cast<int>(q[1]);
                    ray.ntot = static_cast<int>(q[2]);
                    ray.tau = __uint_as_float(q[3]);
                    ray.px = __uint_as_float(q[4]);
                    ray.py = __uint_as_float(q[5]);
                    ray.pz = __uint_as_float(q[6]);
                    ray.vx = __uint_as_float(q[7]);
                    ray.vy = __uint_as_float(q[8]);
                    ray.vz = __uint_as_float(q[9]);
                    ray.state = kSlotActive;
                } else {
                    ray.state = kSlotDone;
                }
                __syncthreads();  // records read before layer 0 overwrites X
                if (stop) break;
                if (tid == 0) *tail_count = 0u;  // next written after the next boundary's first barrier
                live = count > tile * 128;       // the same for all threads of a tile
                it = 0;
                if (!live) continue;
            }
            // layer 0 (FP32): row ttid of X = 16-bit sin(W_0 (p, t) + b_0).  A warp
            // with no active slot skips its rows and their epilogues: its 32 rows of
            // X keep stale values, and an MMA row depends on its own A row only.
            const bool wact = __any_sync(0xffffffffu, ray.state == kSlotActive);
            if (wact) {
                if (timed)
                    trace_layer0<W, F16, SPLIT, true>(a, w0p, wts, ray, ttid, x_s, xlo_s);
                else
                    trace_layer0<W, F16, SPLIT, false>(a, w0p, wts, ray, ttid, x_s, xlo_s);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            // one barrier: X is complete, and the tile's decision.  Before the tail:
            // an empty refill anywhere in the tile starts the tail (this layer 0 is
            // dropped; the rays keep their state).  In the tail: no active ray left
            // ends the tile's round.
            if (!tail) {
                if (bar_or(bar_id, 128, ray.state == kSlotDone)) {
                    tail = true;
                    it = kTailRound;
                    continue;
                }
            } else if (!bar_or(bar_id, 128, ray.state == kSlotActive)) {
                it = kTailRound;
                continue;
            }

            float f = 0.0f;
            bool good = true;
            for (int l = 0; l < KH; ++l) {
                // the tile's MMAs are issued from its warp (tile mod 4), so that the issue work of
                // the CTA's tiles is spread over the four schedulers of the SM (warp w of every
                // tile runs on scheduler w)
                if (ttid == issuer) {
                    tc_fence_after();
                    const uint64_t xd0 = desc_kmajor_sw128(x_s), xld0 = desc_kmajor_sw128(xlo_s);
                    const uint64_t wd0 = desc_kmajor_sw128(w_s + l * W * W * 2u);
                    const uint64_t wld0 = desc_kmajor_sw128(wlo_s + l * W * W * 2u);
#pragma unroll
                    for (int kb = 0; kb < W / 64; ++kb)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t xo = kb * 128u * 128u + kk * 32u, wo = kb * W * 128u + kk * 32u;
                            mma_f16kind(tmem, desc_add(xd0, xo), desc_add(wd0, wo), idesc, (kb | kk) != 0);
                            if (SPLIT) {
                                mma_f16kind(tmem, desc_add(xd0, xo), desc_add(wld0, wo), idesc, 1u);
                                mma_f16kind(tmem, desc_add(xld0, xo), desc_add(wd0, wo), idesc, 1u);
                            }
                        }
                    mma_commit(bar_mma);
                }
                // a warp either reads the accumulator whole or not at all
                good = __all_sync(0xffffffffu, mbar_wait_bounded(bar_mma, mma_phase, a.status, abort_flag) && good);
                mma_phase ^= 1u;
                tc_fence_after();
                const float* bl = bhs + l * W;
                const bool rd = good && wact;
                // the accumulator row in 16-column chunks, the next chunk loading from
                // TMEM while the current one is processed
                float va[16], vb[16];
                if (rd) {
                    tmem_ld16(tmem + lane_base, va);
                    tmem_wait_ld();
                }
                if (l + 1 < KH) {
                    // hidden epilogue: X row = 16-bit sin(D + b)
                    if (rd) {
#pragma unroll
                        for (int q = 0; q < W / 16; ++q) {
                            float(&v)[16] = (q & 1) ? vb : va;
                            float(&vn)[16] = (q & 1) ? va : vb;
                            if (q + 1 < W / 16) tmem_ld16(tmem + lane_base + (q + 1) * 16u, vn);
                            hidden_epilogue<16, F16, SPLIT>(v, bl, ttid, q * 16, x_s, xlo_s);
                            tmem_wait_ld();
                        }
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    bar_named(bar_id, 128);
                } else {
                    // output layer in FP32: f = w_out . sin(D + b) + b_out
                    float2 acc01 = make_float2(0.0f, 0.0f), acc23 = make_float2(0.0f, 0.0f);
                    if (rd) {
#pragma unroll
                        for (int q = 0; q < W / 16; ++q) {
                            float(&v)[16] = (q & 1) ? vb : va;
                            float(&vn)[16] = (q & 1) ? va : vb;
                            if (q + 1 < W / 16) tmem_ld16(tmem + lane_base + (q + 1) * 16u, vn);
                            output_dot<16>(v, blast + q * 16, wop + q * 16, acc01, acc23);
                            tmem_wait_ld();
                        }
                    }
                    f = ((acc01.x + acc01.y) + (acc23.x + acc23.y)) + net.bout;
                }
            }
            tc_fence_before();
            if (good)
                step_ray(a, ray, f);
            else
                ray.state = kSlotDone;  // timed out (the status word says so): the ray is dropped
            ++it;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(*tmem_slot, tcols);
    }
}

// Layer 0 of one ray row as E4M3 bytes of 256 sin(W_0 (p, t) + b_0): K-major
// rows of 128-element blocks with the 128-byte swizzle, one 16-byte chunk
// (16 units) per vector store; the units in pairs as in trace_layer0.
template <int W, bool TIMED>
__device__ __forceinline__ void trace_layer0_e4m3(const LevelArgs& a, const float* w0s, const float* wts,
                                                  const Ray& ray, int row, uint32_t x_s) {
    const float tm = (TIMED && ray.state == kSlotActive) ? __ldg(a.ray_time + ray.idx) : 0.0f;
    const float2 px = make_float2(ray.px, ray.px), py = make_float2(ray.py, ray.py), pz = make_float2(ray.pz, ray.pz);
    const float2 t2 = make_float2(tm, tm);
    for (int j16 = 0; j16 < W / 16; ++j16) {
        float sv[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int pr = j16 * 8 + q;
            const float4 A = reinterpret_cast<const float4*>(w0s)[2 * pr];
            const float4 B = reinterpret_cast<const float4*>(w0s)[2 * pr + 1];
            float2 c = make_float2(B.z, B.w);
            if (TIMED) c = __ffma2_rn(reinterpret_cast<const float2*>(wts)[pr], t2, c);
            const float2 z = __ffma2_rn(make_float2(A.x, A.y), px,
                                        __ffma2_rn(make_float2(A.z, A.w), py, __ffma2_rn(make_float2(B.x, B.y), pz, c)));
            sv[2 * q] = kFp8ActScale * sin_fast(z.x);
            sv[2 * q + 1] = kFp8ActScale * sin_fast(z.y);
        }
        st_shared_v4(x_s + sw128_chunk_offset(row, j16, 128), pack_e4m3x4(sv[0], sv[1], sv[2], sv[3]),
                     pack_e4m3x4(sv[4], sv[5], sv[6], sv[7]), pack_e4m3x4(sv[8], sv[9], sv[10], sv[11]),
                     pack_e4m3x4(sv[12], sv[13], sv[14], sv[15]));
    }
}

// Hidden epilogue of one ray row for accumulator columns c0 .. c0+31 with
// E4M3 operands: X = E4M3(256 sin(D * mf + b)), two 16-byte chunks.
__device__ __forceinline__ void hidden_epilogue32_e4m3(const float (&v)[32], const float* bl, float mf, int row,
                                                       int c0, uint32_t x_s) {
    const float2 mf2 = make_float2(mf, mf);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float sv[16];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = h * 16 + 2 * e;
            const float2 x = __ffma2_rn(make_float2(v[j], v[j + 1]), mf2, make_float2(bl[c0 + j], bl[c0 + j + 1]));
            sv[2 * e] = kFp8ActScale * sin_fast(x.x);
            sv[2 * e + 1] = kFp8ActScale * sin_fast(x.y);
        }
        st_shared_v4(x_s + sw128_chunk_offset(row, (c0 >> 4) + h, 128), pack_e4m3x4(sv[0], sv[1], sv[2], sv[3]),
                     pack_e4m3x4(sv[4], sv[5], sv[6], sv[7]), pack_e4m3x4(sv[8], sv[9], sv[10], sv[11]),
                     pack_e4m3x4(sv[12], sv[13], sv[14], sv[15]));
    }
}

// ---------------------------------------------------------------------------
// trace kernel, width 256 with streamed weights
// ---------------------------------------------------------------------------
// Same per-ray structure as trace_level_tc_kernel, for width 256, whose
// hidden weights (128 KB per layer) leave no room for a second tile of
// activations when held in shared memory.  A producer warp streams the 64-wide K blocks of every
// hidden layer (256 rows x 128 bytes = 32 KB) from L2 through a ring in the
// order the MMAs consume them, cycling over the layers for as long as rays
// remain; thread 0 issues the MMAs as stages arrive.  ST ray tiles of 128
// (TMEM columns [t*256, (t+1)*256), 64 KB of activations each) share every
// weight stage: with two tiles each streamed byte serves twice the rays and
// eight warps instead of four overlap their layer-0 and epilogue work.
constexpr int kStreamW = 256;
constexpr uint32_t kStreamStageBytes = kStreamW * 128u;
__host__ __device__ constexpr int stream_stages(int ST) { return ST == 1 ? 3 : 2; }
__host__ __device__ constexpr int stream_threads(int ST) { return 128 * ST + 32; }  // ray threads + producer warp

struct StreamLayout {
    uint32_t x, ring, w0, wt, bh, wout, bars, misc, total;
};

__host__ __device__ inline StreamLayout stream_layout(int KH, int ST, int EB) {
    StreamLayout L;
    uint32_t o = 0;
    L.x = o;
    o += static_cast<uint32_t>(ST) * 128u * kStreamW * static_cast<uint32_t>(EB);
    L.ring = o;
    o += stream_stages(ST) * kStreamStageBytes;
    L.w0 = o;
    o += kStreamW * 4u * 4u;
    L.wt = o;
    o += kStreamW * 4u;
    L.bh = o;
    o += static_cast<uint32_t>(KH) * kStreamW * 4u;
    L.wout = o;
    o += kStreamW * 4u;
    L.bars = o;
    o += (2 * stream_stages(ST) + 1) * 8u;
    o = (o + 15u) & ~15u;
    L.misc = o;
    o += 32u;
    L.total = o;
    return L;
}

template <int OP, int ST>
__global__ void __launch_bounds__(stream_threads(ST)) trace_level_tc_stream_kernel(const LevelArgs a) {
    constexpr bool F16 = OP == kOpF16, FP8 = OP == kOpE4M3;
    constexpr int EB = FP8 ? 1 : 2;  // operand bytes per element
    // 128-byte K blocks per layer; a stage is one K block of all 256 rows (32 KB)
    constexpr int W = kStreamW, KB = W * EB / 128, NS = stream_stages(ST), NRAY = 128 * ST;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const NetView& net = a.net;
    const int KH = net.n_hidden;
    const StreamLayout L = stream_layout(KH, ST, EB);
    float* w0s = reinterpret_cast<float*>(base + L.w0);
    float* wts = reinterpret_cast<float*>(base + L.wt);
    float* bhs = reinterpret_cast<float*>(base + L.bh);
    float* wos = reinterpret_cast<float*>(base + L.wout);
    const uint32_t bar_full = base_s + L.bars, bar_empty = bar_full + 8u * NS, bar_mma = bar_empty + 8u * NS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L.misc + 4);
    volatile int* done_flag = reinterpret_cast<volatile int*>(base + L.misc + 8);
    volatile uint32_t* consumed = reinterpret_cast<volatile uint32_t*>(base + L.misc + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = tid >> 7, ttid = tid & 127;
    constexpr uint32_t xbytes = 128u * W * EB;
    const uint32_t x_s = base_s + L.x + static_cast<uint32_t>(tile < ST ? tile : 0) * xbytes;
    const uint32_t ring_s = base_s + L.ring;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(bar_full + 8u * s, 1);
            mbar_init(bar_empty + 8u * s, 1);
        }
        mbar_init(bar_mma, 1);
        *abort_flag = 0;
        *done_flag = 0;
        *consumed = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), W * ST);
        tmem_relinquish();
    }
    const bool timed = a.ray_time != nullptr && net.in_dim == 4;
    for (int i = tid; i < W; i += stream_threads(ST)) {
        stage_layer0_pairs(net, a.time, timed, i, w0s, wts);
        wos[i] = net.wout[i];
        for (int l = 0; l < KH; ++l) bhs[l * W + i] = net.bh[l][i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem0 = *tmem_slot;

    if (warp == 4 * ST) {
        // producer: K blocks of layer 0..KH-1 in consumption order, cyclically
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            while (ok) {
                const uint32_t stage = g % NS, use = g / NS;
                if (use > 0) {
                    const uint32_t bar = bar_empty + 8u * stage, par = (use - 1) & 1u;
                    const uint64_t t0 = globaltimer_ns();
                    bool got = false;
                    while (!(got = mbar_try_wait(bar, par))) {
                        if (*done_flag || *abort_flag) break;
                        if (globaltimer_ns() - t0 > kWaitBudgetNs) {
                            raise_status(a.status, kStatusTimeout);
                            *abort_flag = 1;
                            break;
                        }
                    }
                    if (!got) break;
                }
                const uint32_t l = (g / KB) % KH, kb = g % KB;
                mbar_arrive_expect_tx(bar_full + 8u * stage, kStreamStageBytes);
                bulk_g2s(ring_s + stage * kStreamStageBytes,
                         net.wbf + static_cast<size_t>(l) * net.wbf_layer_bytes +
                             static_cast<size_t>(kb) * net.rows_pad * 128u,
                         kStreamStageBytes, bar_full + 8u * stage);
                ++g;
            }
            // every copy issued must land before the block exits
            for (uint32_t gg = *consumed; gg < g; ++gg) mbar_drain(bar_full + 8u * (gg % NS), (gg / NS) & 1u);
        }
    } else {
        const long long n_work = a.in_list ? static_cast<long long>(*a.in_count) : a.n;
        const uint32_t lane_base = static_cast<uint32_t>((ttid >> 5) * 32) << 16;
        const uint32_t tmem = tmem0 + static_cast<uint32_t>(tile * W);
        // E4M3: the format fields 0 of this descriptor select E4M3 under kind::f8f6f4
        constexpr uint32_t idesc = idesc_f32acc(128, W, F16 || FP8);
        const uint64_t rd0 = desc_kmajor_sw128(ring_s);
        uint32_t mma_phase = 0, g = 0;
        bool issue_ok = true;  // thread 0: every weight stage so far arrived in time
        Ray ray;
        // Stop decisions go through the ray threads' barrier: a timed-out wait
        // drops the ray (the status word reports it) instead of leaving the loop.
        while (true) {
            refill_ray(a, ray, n_work);
            if (a.cap <= 0) {
                if (!bar_or(1, NRAY, ray.state == kSlotActive)) break;
                pass_ray(a, ray);
                continue;
            }
            // a warp with no active slot skips its rows (as in trace_level_tc_kernel)
            const bool wact = __any_sync(0xffffffffu, ray.state == kSlotActive);
            if (wact) {
                if (FP8) {
                    if (timed)
                        trace_layer0_e4m3<W, true>(a, w0s, wts, ray, ttid, x_s);
                    else
                        trace_layer0_e4m3<W, false>(a, w0s, wts, ray, ttid, x_s);
                } else if (timed) {
                    trace_layer0<W, F16, false, true>(a, reinterpret_cast<const float4*>(w0s), wts, ray, ttid, x_s, x_s);
                } else {
                    trace_layer0<W, F16, false, false>(a, reinterpret_cast<const float4*>(w0s), wts, ray, ttid, x_s, x_s);
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            if (!bar_or(1, NRAY, ray.state == kSlotActive)) break;

            float f = 0.0f;
            bool good = true;
            for (int l = 0; l < KH; ++l) {
                if (tid == 0) {
                    tc_fence_after();
                    for (int kb = 0; kb < KB && issue_ok; ++kb, ++g) {
                        const uint32_t stage = g % NS;
                        issue_ok = mbar_wait_bounded(bar_full + 8u * stage, (g / NS) & 1u, a.status, abort_flag);
                        if (!issue_ok) break;
                        tc_fence_after();
#pragma unroll
                        for (int t = 0; t < ST; ++t) {
                            const uint64_t xd0 = desc_kmajor_sw128(base_s + L.x + t * xbytes);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t xd = desc_add(xd0, kb * 128u * 128u + kk * 32u);
                                const uint64_t wd = desc_add(rd0, stage * kStreamStageBytes + kk * 32u);
                                if (FP8)
                                    mma_f8kind(tmem0 + t * W, xd, wd, idesc, (kb | kk) != 0);
                                else
                                    mma_f16kind(tmem0 + t * W, xd, wd, idesc, (kb | kk) != 0);
                            }
                        }
                        mma_commit(bar_empty + 8u * stage);
                    }
                    if (issue_ok) mma_commit(bar_mma);
                }
                // a warp either reads the accumulator whole or not at all
                good = __all_sync(0xffffffffu, mbar_wait_bounded(bar_mma, mma_phase, a.status, abort_flag) && good);
                mma_phase ^= 1u;
                tc_fence_after();
                const float* bl = bhs + l * W;
                const bool rd = good && wact;
                // E4M3: accumulator -> value (the operand scales q_w and 256 divided out)
                const float mf = FP8 ? 1.0f / (net.q_w[l] * kFp8ActScale) : 1.0f;
                // 32-column chunks, the next one loading from TMEM while the current
                // one is processed
                float va[32], vb[32];
                if (rd) {
                    tmem_ld32(tmem + lane_base, va);
                    tmem_wait_ld();
                }
                if (l + 1 < KH) {
                    if (rd) {
#pragma unroll
                        for (int q = 0; q < W / 32; ++q) {
                            float(&v)[32] = (q & 1) ? vb : va;
                            float(&vn)[32] = (q & 1) ? va : vb;
                            if (q + 1 < W / 32) tmem_ld32(tmem + lane_base + (q + 1) * 32u, vn);
                            if (FP8)
                                hidden_epilogue32_e4m3(v, bl, mf, ttid, q * 32, x_s);
                            else
                                hidden_epilogue32<F16, false>(v, bl, ttid, q * 32, x_s, x_s);
                            tmem_wait_ld();
                        }
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    bar_named(1, NRAY);
                } else {
                    float2 acc01 = make_float2(0.0f, 0.0f), acc23 = make_float2(0.0f, 0.0f);
                    if (rd) {
#pragma unroll
                        for (int q = 0; q < W / 32; ++q) {
                            float(&v)[32] = (q & 1) ? vb : va;
                            float(&vn)[32] = (q & 1) ? va : vb;
                            if (q + 1 < W / 32) tmem_ld32(tmem + lane_base + (q + 1) * 32u, vn);
                            output_dot32<FP8>(v, bl + q * 32, wos + q * 32, acc01, acc23, mf);
                            tmem_wait_ld();
                        }
                    }
                    f = ((acc01.x + acc01.y) + (acc23.x + acc23.y)) + net.bout;
                }
            }
            tc_fence_before();
            if (good)
                step_ray(a, ray, f);
            else
                ray.state = kSlotDone;
        }
        if (tid == 0) *consumed = g;
        bar_named(1, NRAY);
        if (tid == 0) {
            __threadfence_block();
            *done_flag = 1;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem0, W * ST);
    }
}



}  // namespace

bool tc_trace_supported(int width, int n_hidden) {
    return n_hidden >= 1 && n_hidden <= kMaxHidden && (width == 64 || width == 128 || width == 256);
}

bool tc_grad_supported(int width, int n_hidden) {
    return n_hidden >= 1 && n_hidden <= kMaxHidden && (width == 64 || width == 128 || width == 256);
}

// Ray tiles per CTA for the resident trace kernel: as many as shared memory,
// registers, TMEM and the thread limit allow (all tiles share the weights).
template <class Kernel>
static int trace_tiles_uncached(Kernel k, int W, int KH, bool split) {
    int dev = 0, smem_optin = 0, regs_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes at;
    if (cudaFuncGetAttributes(&at, k) != cudaSuccess) return 1;
    const int regs_warp = ((at.numRegs * 32 + 255) / 256) * 256;
    int T = kMaxTraceTiles;
    while (T > 1 && (trace_layout(W, KH, split, T).total + 1024 > static_cast<uint32_t>(smem_optin) ||
                     regs_warp * 4 * T > regs_sm || static_cast<int>(tmem_cols_for(T * W)) > 512))
        --T;
    return T;
}

template <class Kernel>
static int trace_tiles(Kernel k, int W, int KH, bool split) {
    int T = 1;
    if (launch_cached(reinterpret_cast<const void*>(k), static_cast<uint64_t>(W) * 16 + KH, split ? 1 : 0, &T,
                      [&](int* v) {
                          *v = trace_tiles_uncached(k, W, KH, split);
                          return cudaSuccess;
                      }) != cudaSuccess)
        return 1;
    return T;
}

// The launch takes min(a.tiles, maximum) tiles per CTA when a.tiles > 0.
template <int W, bool F16>
static cudaError_t launch_trace_resident(const LevelArgs& a, int num_sms, cudaStream_t s) {
    const int KH = a.net.n_hidden;
    const bool split = a.net.wbf_lo != nullptr && trace_split(W, KH);
    if (split) {
        auto k = trace_level_tc_kernel<W, F16, true>;
        int T = trace_tiles(k, W, KH, true);
        if (a.tiles > 0) T = std::min(T, a.tiles);
        return launch_tc(k, 128 * T, trace_layout(W, KH, true, T).total + 1024, tmem_cols_for(T * W), num_sms, s, &a);
    }
    auto k = trace_level_tc_kernel<W, F16, false>;
    int T = trace_tiles(k, W, KH, false);
    if (a.tiles > 0) T = std::min(T, a.tiles);
    return launch_tc(k, 128 * T, trace_layout(W, KH, false, T).total + 1024, tmem_cols_for(T * W), num_sms, s, &a);
}

template <int W, bool F16>
static int trace_tiles_resident(const NetView& net) {
    const int KH = net.n_hidden;
    if (net.wbf_lo != nullptr && trace_split(W, KH)) return trace_tiles(trace_level_tc_kernel<W, F16, true>, W, KH, true);
    return trace_tiles(trace_level_tc_kernel<W, F16, false>, W, KH, false);
}

int trace_tiles_max(const NetView& net) {
    if (!tc_trace_supported(net.width, net.n_hidden)) return 0;
    const bool f16 = net.op_f16 != 0;
    switch (net.width) {
    case 64:
        return f16 ? trace_tiles_resident<64, true>(net) : trace_tiles_resident<64, false>(net);
    case 128:
        return f16 ? trace_tiles_resident<128, true>(net) : trace_tiles_resident<128, false>(net);
    case 256:
        return 2;  // the streamed-weight kernel: one or two tiles
    }
    return 0;
}

// Streamed-weight trace: two ray tiles per CTA unless a.tiles asks for one.
template <int OP>
static cudaError_t launch_trace_stream(const LevelArgs& a, int num_sms, cudaStream_t s) {
    const int KH = a.net.n_hidden, EB = OP == kOpE4M3 ? 1 : 2;
    if (a.tiles == 1)
        return launch_tc(trace_level_tc_stream_kernel<OP, 1>, stream_threads(1),
                         stream_layout(KH, 1, EB).total + 1024, kStreamW, num_sms, s, &a);
    return launch_tc(trace_level_tc_stream_kernel<OP, 2>, stream_threads(2), stream_layout(KH, 2, EB).total + 1024,
                     2 * kStreamW, num_sms, s, &a);
}

cudaError_t launch_trace_level_tc(const LevelArgs& a, int num_sms, cudaStream_t s) {
    const bool f16 = a.net.op_f16 != 0;
    switch (a.net.width) {
    case 64:
        return f16 ? launch_trace_resident<64, true>(a, num_sms, s) : launch_trace_resident<64, false>(a, num_sms, s);
    case 128:
        return f16 ? launch_trace_resident<128, true>(a, num_sms, s) : launch_trace_resident<128, false>(a, num_sms, s);
    case 256:
        if (a.net.op_fp8) return launch_trace_stream<kOpE4M3>(a, num_sms, s);
        return f16 ? launch_trace_stream<kOpF16>(a, num_sms, s) : launch_trace_stream<kOpBF16>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

bool tc_trace_split(int width, int n_hidden) { return width <= 128 && trace_split(width, n_hidden); }

template <int W, int OP>
static cudaError_t launch_grad_op(const GradArgs& a, int num_sms, cudaStream_t s) {
    using C = GradCfg<W, OP>;
    const size_t smem = grad_layout<W, OP>(a.net.n_hidden).total + 1024;
    return launch_tc(grad_tc_kernel<W, OP>, C::THREADS, smem, C::TMEM_COLS, num_sms, s, &a);
}

template <int W>
static cudaError_t launch_grad_w(const GradArgs& a, int num_sms, cudaStream_t s) {
    if (a.net.op_f16) return launch_grad_op<W, kOpF16>(a, num_sms, s);
    return launch_grad_op<W, kOpBF16>(a, num_sms, s);
}

// Sine throughput of the tensor-core kernels' sine (sin_fast): every thread
// runs 8 independent chains x <- sin_fast(x) * c + d for `iters` steps (the
// multiply-add keeps the chains from settling and costs an FMA-pipe slot, as
// the kernels' own uses do).
__global__ void __launch_bounds__(256) sine_rate_kernel(float* out, int iters) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 0.1f * static_cast<float>(threadIdx.x + i);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(sin_fast(x[i]), 1.7f, 0.3f);
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc += x[i];
    if (acc == 12345.678f) out[0] = acc;  // keeps the chains live
}

cudaError_t measure_sine_rate(int num_sms, cudaStream_t s, double* sines_per_s) {
    float* out = nullptr;
    cudaError_t e = cudaMallocAsync(&out, 16, s);
    if (e != cudaSuccess) return e;
    const int blocks = num_sms * 8, iters = 4096;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        sine_rate_kernel<<<blocks, 256, 0, s>>>(out, iters);  // warm-up
        cudaEventRecord(a, s);
        sine_rate_kernel<<<blocks, 256, 0, s>>>(out, iters);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
    }
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) *sines_per_s = static_cast<double>(blocks) * 256.0 * 8.0 * iters / (ms * 1e-3);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(out, s);
    return e;
}

// The sine/cosine variants of the kernels at given arguments, for accuracy
// checks: variant 0 is the FP32 path's (reduction by 2 pi, then the hardware
// approximation), variant 1 the tensor-core paths' (the hardware
// approximation applied directly).
__global__ void sine_eval_kernel(int variant, const float* __restrict__ x, int64_t n, float* __restrict__ out_sin,
                                 float* __restrict__ out_cos) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float sn, cs;
        if (variant == 0)
            sincos_r(x[i], &sn, &cs);
        else
            sincos_fast(x[i], &sn, &cs);
        out_sin[i] = sn;
        out_cos[i] = cs;
        if (variant == 0 && sn != sin_r(x[i])) out_sin[i] = NAN;     // the trace's sine is the same value
        if (variant == 1 && sn != sin_fast(x[i])) out_sin[i] = NAN;
    }
}

cudaError_t launch_sine_eval(int variant, const float* x, int64_t n, float* out_sin, float* out_cos, int num_sms,
                             cudaStream_t s) {
    sine_eval_kernel<<<num_sms * 4, 256, 0, s>>>(variant, x, n, out_sin, out_cos);
    return cudaGetLastError();
}

cudaError_t launch_grad_tc(const GradArgs& a, int num_sms, cudaStream_t s) {
    if (a.net.op_fp8) {
        if (a.net.width == 128) return launch_grad_op<128, kOpE4M3>(a, num_sms, s);
        if (a.net.width == 256) return launch_grad_op<256, kOpE4M3>(a, num_sms, s);
        return cudaErrorInvalidValue;
    }
    switch (a.net.width) {
    case 64:
        return launch_grad_w<64>(a, num_sms, s);
    case 128:
        return launch_grad_w<128>(a, num_sms, s);
    case 256:
        return launch_grad_w<256>(a, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sdfnn
