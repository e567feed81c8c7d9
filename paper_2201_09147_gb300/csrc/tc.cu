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
#include "internal.h"
#include "launch_cache.h"
#include "rays.cuh"

namespace sdfnn {
namespace {

// Operand types of the tensor-core contractions: bfloat16 or IEEE half
// (kind::f16), or E4M3 (kind::f8f6f4; sine activations stored as 256 sin).
enum : int { kOpBF16 = 0, kOpF16 = 1, kOpE4M3 = 2 };
constexpr float kFp8ActScale = 256.0f;

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
template <int W, bool F16, bool SPLIT, bool TIMED>
__device__ __forceinline__ void trace_layer0(const LevelArgs& a, const float* w0s, const float* wts, const Ray& ray,
                                             int row, uint32_t x_s, uint32_t xlo_s) {
    const float tm = (TIMED && ray.state == kSlotActive) ? __ldg(a.ray_time + ray.idx) : 0.0f;
    const float2 px = make_float2(ray.px, ray.px), py = make_float2(ray.py, ray.py), pz = make_float2(ray.pz, ray.pz);
    const float2 t2 = make_float2(tm, tm);
    for (int k8 = 0; k8 < W / 8; ++k8) {
        uint32_t pk[4], pl[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int pr = k8 * 4 + q;
            const float4 A = reinterpret_cast<const float4*>(w0s)[2 * pr];
            const float4 B = reinterpret_cast<const float4*>(w0s)[2 * pr + 1];
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
    const uint32_t bar_w = base_s + L.bars;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L.misc + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = tid >> 7, ttid = tid & 127, twarp = ttid >> 5;
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
                    trace_layer0<W, F16, SPLIT, true>(a, w0s, wts, ray, ttid, x_s, xlo_s);
                else
                    trace_layer0<W, F16, SPLIT, false>(a, w0s, wts, ray, ttid, x_s, xlo_s);
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
                if (ttid == 0) {
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
                            output_dot<16>(v, bl + q * 16, wos + q * 16, acc01, acc23);
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
                    trace_layer0<W, F16, false, true>(a, w0s, wts, ray, ttid, x_s, x_s);
                } else {
                    trace_layer0<W, F16, false, false>(a, w0s, wts, ray, ttid, x_s, x_s);
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

// ---------------------------------------------------------------------------
// gradient kernel
// ---------------------------------------------------------------------------
// A tile of 64 points is processed as two halves of 32 points (128 X rows =
// 32 points x 4 streams each).  Each half has its own epilogue warp group,
// TMEM columns and barriers; the MMA warp alternates between the halves, so
// the tensor core works on one half while the other half's epilogue
// (sin/cos, tangent scaling, operand stores) runs.  The producer warp streams
// every hidden layer's K blocks once per half.
//
// X layout.  16-bit operands: MN-major (point-streams contiguous) with the
// 128-byte swizzle: per half, 2 atoms of 64 point-streams at stride W * 128
// bytes, 8-feature K groups of 1024 bytes; the thread that owns feature m
// writes two points (8 values, 16 bytes) per vector store, with no exchange
// between lanes.  The hidden MMAs read X as an MN-major B operand, the output
// MMA as an MN-major A operand.  E4M3 operands: K-major (rows =
// point-streams), written through a lane-quad byte transpose.
//
// Operand types (OP): bfloat16 or IEEE half (kind::f16), or E4M3
// (kind::f8f6f4, widths 128 and 256).  With E4M3 every stored operand carries
// a scale: hidden weights W_l * q_w[l] (q_w = 448 / max|W_l|), the sine
// stream 256 * sin, the tangent streams G_l * q_g[l] (q_g from the load-time
// calibration), w_out * q_o as a head row plus a remainder row scaled by a
// further 16; the epilogues divide the accumulators back.

template <int W, int OP>
struct GradCfg {
    static constexpr int EB = OP == kOpE4M3 ? 1 : 2;  // operand bytes per element
    static constexpr int MT = (W + 127) / 128;      // TMEM tiles of 128 feature rows
    static constexpr int KB = W * EB / 128;         // 128-byte K blocks
    static constexpr int NPTS = 64;                 // points per tile
    static constexpr int HPTS = 32;                 // points per half
    static constexpr int NROWS = 4 * NPTS;          // rows of X (point-streams)
    static constexpr int HROWS = 4 * HPTS;          // rows of X per half = MMA N
    // Weight ring.  A stage is SKB consecutive K blocks for all TMEM tiles: one
    // contiguous 32 KB bulk copy where the layer allows it (bulk-copy throughput
    // per SM grows with the copy size: ~20 B/clk with 16 KB copies, ~41 with
    // 32 KB, measured with a copy ring on GB300).  NS fills what the activation
    // tile leaves of the shared memory.
    static constexpr int SKB = (MT * 16384 >= 32768 || KB == 1) ? 1 : 2;
    static constexpr uint32_t STAGE_BYTES = static_cast<uint32_t>(SKB) * MT * 16384u;
    static constexpr int STAGES_PER_LAYER = KB / SKB;
    static constexpr uint32_t X_BYTES = 4u * 64u * 128u * KB;
    static constexpr int NS_FIT = static_cast<int>((200u * 1024u - X_BYTES) / STAGE_BYTES);
    static constexpr int NS = NS_FIT > 8 ? 8 : NS_FIT;
    static constexpr int GROUP_WARPS = 4 * MT;      // epilogue warps per half
    static constexpr int GROUP_THREADS = GROUP_WARPS * 32;
    static constexpr int EPI_WARPS = 2 * GROUP_WARPS;
    static constexpr int PRODUCER_WARP = EPI_WARPS;
    static constexpr int MMA_WARP = EPI_WARPS + 1;
    static constexpr int THREADS = (EPI_WARPS + 2) * 32;
    static constexpr int TMEM_COLS = MT * 256;      // per TMEM tile: half 0 at +0, half 1 at +128
    static_assert(KB >= 1, "E4M3 gradients need width >= 128");
    static_assert(NS >= 2 && KB % SKB == 0, "weight ring");
};

struct GradLayout {
    uint32_t x, ring, woutb, w0, wt, pts, idx, nidx, bars, misc, total;
};

template <int W, int OP>
__host__ __device__ inline GradLayout grad_layout(int KH) {
    using C = GradCfg<W, OP>;
    GradLayout L;
    uint32_t o = 0;
    L.x = o;
    o += C::NROWS * 128u * C::KB;
    L.ring = o;
    o += C::NS * C::STAGE_BYTES;
    L.woutb = o;
    o += C::KB * 16u * 128u;
    L.w0 = o;
    o += W * 4u * 4u;
    L.wt = o;
    o += W * 4u;
    L.pts = o;
    o += C::NPTS * 4u * 4u;
    L.idx = o;
    o += C::NPTS * 4u;
    L.nidx = o;
    o += C::NPTS * 4u;
    L.bars = o;
    o += (2 * C::NS + 4) * 8u;
    o = (o + 15u) & ~15u;
    L.misc = o;
    o += 32u;
    L.total = o;
    return L;
}

// Byte offset in the MN-major 16-bit X of the 16-byte chunk holding points
// 2c, 2c + 1 (all four streams) of half h for feature m.
template <int W>
__device__ __forceinline__ uint32_t xoff16(int h, int m, int c) {
    return static_cast<uint32_t>(h) * (W * 256u) + static_cast<uint32_t>(c >> 3) * (W * 128u) +
           static_cast<uint32_t>(m >> 3) * 1024u + static_cast<uint32_t>(m & 7) * 128u +
           (static_cast<uint32_t>((c & 7) ^ (m & 7)) << 4);
}

// a_i for i in 0..3 with two predicated selects per bit (no branch)
__device__ __forceinline__ uint32_t sel4(uint32_t i, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3) {
    const uint32_t lo = (i & 1u) ? a1 : a0, hi = (i & 1u) ? a3 : a2;
    return (i & 2u) ? hi : lo;
}

// Stores into the 8-bit K-major X the four stream values of four points p0 .. p0+3 (v[q][s]: point
// p0 + q, stream s, already scaled), exchanged within the lane quad of
// features m0 .. m0+3 (m0 = m & ~3): lane j = m & 3 gathers point p0 + j of
// all four features and writes its four rows as 32-bit words of features
// m0 .. m0+3.  At step i it writes stream (i + j) & 3, which puts the quad's
// four rows on four different phases of the 128-byte swizzle, so each of the
// warp's four stores is conflict free.
template <int NROWS>
__device__ __forceinline__ void store_quad8(uint32_t x_s, int m, int lane, int p0, const float (&v)[4][4]) {
    const uint32_t j = static_cast<uint32_t>(lane) & 3u;
    const uint32_t w0 = pack_e4m3x4(v[0][0], v[0][1], v[0][2], v[0][3]);
    const uint32_t w1 = pack_e4m3x4(v[1][0], v[1][1], v[1][2], v[1][3]);
    const uint32_t w2 = pack_e4m3x4(v[2][0], v[2][1], v[2][2], v[2][3]);
    const uint32_t w3 = pack_e4m3x4(v[3][0], v[3][1], v[3][2], v[3][3]);
    // lane j keeps its word of point j and swaps its word of point j ^ x with lane j ^ x
    const uint32_t own = sel4(j, w0, w1, w2, w3);
    const uint32_t g1 = __shfl_xor_sync(0xffffffffu, sel4(j ^ 1u, w0, w1, w2, w3), 1);
    const uint32_t g2 = __shfl_xor_sync(0xffffffffu, sel4(j ^ 2u, w0, w1, w2, w3), 2);
    const uint32_t g3 = __shfl_xor_sync(0xffffffffu, sel4(j ^ 3u, w0, w1, w2, w3), 3);
    // r_i: point p0 + j of feature m0 + i (byte s = stream s)
    const uint32_t r0 = sel4(j, own, g1, g2, g3), r1 = sel4(j ^ 1u, own, g1, g2, g3);
    const uint32_t r2 = sel4(j ^ 2u, own, g1, g2, g3), r3 = sel4(j ^ 3u, own, g1, g2, g3);
    const uint32_t m0 = static_cast<uint32_t>(m) & ~3u;
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t st = (i + j) & 3u;
        const uint32_t sel = st | ((st + 4u) << 4);
        const uint32_t word = prmt(prmt(r0, r1, sel), prmt(r2, r3, sel), 0x5410u);
        st_shared_u32(x_s + sw128_offset8((p0 + j) * 4u + st, m0, NROWS), word);
    }
}

template <int OP>
__device__ __forceinline__ void mma_op(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (OP == kOpE4M3)
        mma_f8kind(d, a, b, idesc, acc);
    else
        mma_f16kind(d, a, b, idesc, acc);
}

// Index of point j (j < 0: none) of half h of pair i of this CTA (-1 past the
// work), and its coordinates (zero for -1).
template <int HPTS>
__device__ __forceinline__ int grad_point_index(const GradArgs& a, long long n_work, int cta, int h, int j,
                                                long long i) {
    const long long k = ((i * gridDim.x + cta) * 2 + h) * HPTS + j;
    if (j < 0 || k >= n_work) return -1;
    return a.list ? a.list[k] : static_cast<int>(k);
}

// The same index written to the int at shared address dst: copied there
// asynchronously when it comes from the list (complete after
// cp_async_wait_all in the same thread).
template <int HPTS>
__device__ __forceinline__ void grad_point_index_async(uint32_t dst, const GradArgs& a, long long n_work, int cta,
                                                       int h, int j, long long i) {
    const long long k = ((i * gridDim.x + cta) * 2 + h) * HPTS + j;
    if (j < 0 || k >= n_work)
        st_shared_u32(dst, 0xFFFFFFFFu);
    else if (a.list)
        cp_async4(dst, a.list + k);
    else
        st_shared_u32(dst, static_cast<uint32_t>(k));
}

// Copies (x, y, z, t) of point idx into the float4 at shared address dst
// with asynchronous 4-byte copies (zeros for idx < 0); complete after
// cp_async_wait_all in the same thread.
__device__ __forceinline__ void grad_point_async(uint32_t dst, const GradArgs& a, bool timed, int idx) {
    if (idx < 0) {
        st_shared_v4(dst, 0u, 0u, 0u, 0u);
        return;
    }
    cp_async4(dst, a.pts + idx);
    cp_async4(dst + 4u, a.pts + a.n + idx);
    cp_async4(dst + 8u, a.pts + 2 * a.n + idx);
    if (timed)
        cp_async4(dst + 12u, a.pt_time + idx);
    else
        st_shared_u32(dst + 12u, 0u);
}

template <int W, int OP>
__global__ void __launch_bounds__(GradCfg<W, OP>::THREADS) grad_tc_kernel(const GradArgs a) {
    using C = GradCfg<W, OP>;
    constexpr bool F16 = OP == kOpF16;
    constexpr bool FP8 = OP == kOpE4M3;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const NetView& net = a.net;
    const int KH = net.n_hidden;
    const GradLayout L = grad_layout<W, OP>(KH);
    float* w0s = reinterpret_cast<float*>(base + L.w0);
    float* wts = reinterpret_cast<float*>(base + L.wt);
    float4* pts = reinterpret_cast<float4*>(base + L.pts);  // (x, y, z, t) per point
    int* idxs = reinterpret_cast<int*>(base + L.idx);
    int* nidxs = reinterpret_cast<int*>(base + L.nidx);  // indices of the next pair's points
    const uint32_t bar_full = base_s + L.bars;             // NS barriers
    const uint32_t bar_empty = bar_full + 8u * C::NS;      // NS barriers
    const uint32_t bar_xready = bar_empty + 8u * C::NS;    // 2 barriers (one per half)
    const uint32_t bar_dfull = bar_xready + 16u;           // 2 barriers (one per half)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + L.misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base + L.misc + 4);
    const uint32_t x_s = base_s + L.x, ring_s = base_s + L.ring, wo_s = base_s + L.woutb;
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
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    const bool timed = a.pt_time != nullptr && net.in_dim == 4;
    for (int i = tid; i < W; i += C::THREADS) stage_layer0(net, a.time, timed, i, w0s, wts);
    // w_out as a head (row 0) and the rounding of its remainder (row 1) of a
    // 16-row K-major operand (rows 2..15 zero): the output MMA then carries
    // w_out to about twice the operand's significand bits.
    for (int i = tid; i < C::KB * 16 * 128 / 4; i += C::THREADS) reinterpret_cast<uint32_t*>(base + L.woutb)[i] = 0u;
    __syncthreads();
    for (int k = tid; k < W; k += C::THREADS) {
        if (FP8) {
            base[L.woutb + sw128_offset8(0, k, 16)] = net.wout_q[k];
            base[L.woutb + sw128_offset8(1, k, 16)] = net.wout_q[W + k];
        } else {
            const float w = net.wout[k];
            const uint16_t hi = bits16<F16>(w);
            *reinterpret_cast<uint16_t*>(base + L.woutb + sw128_offset(0, k, 16)) = hi;
            *reinterpret_cast<uint16_t*>(base + L.woutb + sw128_offset(1, k, 16)) = bits16<F16>(w - from16<F16>(hi));
        }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // Static schedule: half-tiles of 32 points; CTA b takes the pairs b, b + G,
    // b + 2G, ... (G = grid size) and half h of each pair is half-tile
    // 2 * pair + h.  Both halves run the same number of pairs, so the MMA warp
    // and the producer can follow the fixed schedule of grad_slot; a half-tile
    // beyond the work is computed with no valid points.
    const long long n_work = a.list ? static_cast<long long>(*a.count) : a.n;
    const long long n_pairs = (n_work + 2 * C::HPTS - 1) / (2 * C::HPTS);
    const long long G = gridDim.x;
    const long long my_pairs = n_pairs > blockIdx.x ? (n_pairs - blockIdx.x + G - 1) / G : 0;
    // MMA schedule: each half runs n_groups groups in order (per pair: the KH
    // hidden layers, then the output layer).  With 16-bit operands half 1 runs
    // one group behind half 0 (LAG = 1):
    //   h0.G0 | h0.G1 h1.G0 | h0.G2 h1.G1 | ... | h1.G(n-1),
    // so the short output-layer group of one half sits between hidden-layer
    // groups of the other, which cover that half's last epilogue and its next
    // input layer.  E4M3 MMAs take half as long as the epilogues they
    // alternate with, and there the halves run in step (LAG = 0: h0.Gk h1.Gk),
    // which measured faster.  The producer streams the weights in the same order.
    constexpr int LAG = FP8 ? 0 : 1;
    const int n_groups = static_cast<int>(my_pairs) * (KH + 1);
    bool ok = true;

    if (warp == C::PRODUCER_WARP) {
        if (lane == 0) {
            // stages in MMA order: per slot of the schedule, the stages of its layer
            // (K blocks SKB * sg .. of every TMEM tile: contiguous in the weight image)
            uint32_t g = 0;
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    const int l = grp % (KH + 1);
                    for (int sg = 0; sg < C::STAGES_PER_LAYER && l < KH && ok; ++sg, ++g) {
                        const uint32_t stage = g % C::NS, use = g / C::NS;
                        if (use > 0) ok = mbar_wait_bounded(bar_empty + 8u * stage, (use - 1) & 1u, a.status, abort_flag);
                        if (!ok) break;
                        mbar_arrive_expect_tx(bar_full + 8u * stage, C::STAGE_BYTES);
                        bulk_g2s(ring_s + stage * C::STAGE_BYTES,
                                 net.wbf + static_cast<size_t>(l) * net.wbf_layer_bytes +
                                     static_cast<size_t>(sg) * C::STAGE_BYTES,
                                 C::STAGE_BYTES, bar_full + 8u * stage);
                    }
                }
            // every copy issued must land before the block exits (the last use of
            // each stage; earlier uses were waited on before their stage was refilled)
            for (uint32_t gg = g > C::NS ? g - C::NS : 0; gg < g; ++gg)
                mbar_drain(bar_full + 8u * (gg % C::NS), (gg / C::NS) & 1u);
        }
    } else if (warp == C::MMA_WARP) {
        if (lane == 0) {
            // E4M3: the format fields 0 of this descriptor select E4M3 under kind::f8f6f4
            constexpr uint32_t idesc_h = idesc_f32acc(128, C::HROWS, F16 || FP8) | (FP8 ? 0u : kIdescMajorMnB);
            constexpr uint32_t idesc_o = idesc_f32acc(128, 16, F16 || FP8) | (FP8 ? 0u : kIdescMajorMnA);
            uint32_t g = 0, xr_phase[2] = {0u, 0u};
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2 && ok; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    const int l = grp % (KH + 1);
                    ok = mbar_wait_bounded(bar_xready + 8u * h, xr_phase[h], a.status, abort_flag);
                    xr_phase[h] ^= 1u;
                    if (!ok) break;
                    tc_fence_after();
                    // X of this half: K-major rows (E4M3), or the MN-major half block (16-bit)
                    const uint32_t xh = FP8 ? x_s + h * C::HROWS * 128u : x_s + h * (W * 256u);
                    if (l < KH) {
                        // D[mt][h] = W_l[mt rows] . X_h^T over all K blocks
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
                                        const uint64_t xd =
                                            FP8 ? desc_kmajor_sw128(xh + kb * C::NROWS * 128u + kk * 32u)
                                                : desc_mnmajor_sw128(xh + (kb * 8 + kk * 2) * 1024u, W * 128u);
                                        const uint32_t wa =
                                            ring_s + stage * C::STAGE_BYTES + (kr * C::MT + mt) * 16384u + kk * 32u;
                                        mma_op<OP>(tmem + mt * 256u + h * 128u, desc_kmajor_sw128(wa), xd, idesc_h,
                                                   (kb | kk) != 0);
                                    }
                            }
                            mma_commit(bar_empty + 8u * stage);
                        }
                    } else {
                        // output layer of this half: rows = its 128 point-streams, N = 16 (w_out head, remainder)
                        for (int kb = 0; kb < C::KB; ++kb)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t xd =
                                    FP8 ? desc_kmajor_sw128(xh + kb * C::NROWS * 128u + kk * 32u)
                                        : desc_mnmajor_sw128(xh + (kb * 8 + kk * 2) * 1024u, W * 128u);
                                mma_op<OP>(tmem + h * 128u, xd, desc_kmajor_sw128(wo_s + kb * 16u * 128u + kk * 32u),
                                           idesc_o, (kb | kk) != 0);
                            }
                    }
                    if (ok) mma_commit(bar_dfull + 8u * h);
                }
        }
    } else {
        // epilogue group h: thread <-> feature row m of TMEM tile mt, points 32h .. 32h+31 of X
        const int h = warp / C::GROUP_WARPS, ge = warp % C::GROUP_WARPS;
        const int mt = ge >> 2, quad = ge & 3;
        const int m = mt * 128 + quad * 32 + lane;
        const bool live = m < W;  // warp-uniform: W is a multiple of 32
        const int gt = ge * 32 + lane;  // thread index within the group
        const uint32_t lane_addr = tmem + (static_cast<uint32_t>(quad * 32) << 16) + mt * 256u + h * 128u;
        const int p0 = h * C::HPTS;
        // E4M3 scales: sine stream, tangents after layer 0
        const float sf = FP8 ? kFp8ActScale : 1.0f;
        const float g0s = FP8 ? net.q_g[0] : 1.0f;
        uint32_t df_phase = 0;
        // Point gt of this half in pair i (threads gt < HPTS): its index is
        // loaded a pair ahead and its coordinates during the pair before, so
        // neither global load sits between two pairs.
        // Point gt < HPTS of this half: its index is copied into shared memory
        // at the start of the pair before, its coordinates once that pair's
        // input layer has read the current ones, so no global load sits
        // between two pairs.
        if (gt < C::HPTS) {
            const int idx = grad_point_index<C::HPTS>(a, n_work, blockIdx.x, h, my_pairs > 0 ? gt : -1, 0);
            nidxs[p0 + gt] = idx;
            grad_point_async(base_s + L.pts + static_cast<uint32_t>(p0 + gt) * 16u, a, timed, idx);
        }
        for (long long i = 0; i < my_pairs; ++i) {
            if (gt < C::HPTS) {
                cp_async_wait_all();
                idxs[p0 + gt] = nidxs[p0 + gt];
                grad_point_index_async<C::HPTS>(base_s + L.nidx + static_cast<uint32_t>(p0 + gt) * 4u, a, n_work,
                                                blockIdx.x, h, i + 1 < my_pairs ? gt : -1, i + 1);
            }
            bar_named(1 + h, C::GROUP_THREADS);
            // input layer: P_0 = sin(A_0), G_0^c = W_0[:, c] (.) cos(A_0); the time
            // input enters A_0 only (the tangents are spatial)
            if (live) {
                const float4 u = reinterpret_cast<const float4*>(w0s)[m];
                const float ut = wts[m];
                if (FP8) {
                    for (int p = p0; p < p0 + C::HPTS; p += 4) {
                        float o[4][4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 q4 = pts[p + q];
                            const float z = fmaf(u.x, q4.x, fmaf(u.y, q4.y, fmaf(u.z, q4.z, fmaf(ut, q4.w, u.w))));
                            float sn, cs;
                            sincos_fast(z, &sn, &cs);
                            const float cg = cs * g0s;
                            o[q][0] = sn * sf; o[q][1] = u.x * cg; o[q][2] = u.y * cg; o[q][3] = u.z * cg;
                        }
                        store_quad8<C::NROWS>(x_s, m, lane, p, o);
                    }
                } else {
#pragma unroll 4
                    for (int c = 0; c < C::HPTS / 2; ++c) {
                        uint32_t w[4];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float4 q4 = pts[p0 + 2 * c + e];
                            const float z = fmaf(u.x, q4.x, fmaf(u.y, q4.y, fmaf(u.z, q4.z, fmaf(ut, q4.w, u.w))));
                            float sn, cs;
                            sincos_fast(z, &sn, &cs);
                            w[2 * e] = pack16x2<F16>(sn, u.x * cs);
                            w[2 * e + 1] = pack16x2<F16>(u.y * cs, u.z * cs);
                        }
                        st_shared_v4(x_s + xoff16<W>(h, m, c), w[0], w[1], w[2], w[3]);
                    }
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(bar_xready + 8u * h);

            for (int l = 0; l < KH && ok; ++l) {
                // warp-uniform, so that a warp's TMEM loads run whole or not at all
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_dfull + 8u * h, df_phase, a.status, abort_flag));
                df_phase ^= 1u;
                if (!ok) break;
                // every thread of the group has read this pair's points by now (the
                // MMA that produced D waited for all of them)
                if (l == 0 && gt < C::HPTS) {
                    cp_async_wait_all();  // the index copied at the top of the pair
                    grad_point_async(base_s + L.pts + static_cast<uint32_t>(p0 + gt) * 16u, a, timed, nidxs[p0 + gt]);
                }
                tc_fence_after();
                const float bb = live ? __ldg(net.bh[l] + m) : 0.0f;  // one load per layer and half-tile
                // accumulator -> value multipliers of the sine and tangent streams, and the
                // tangent scale of the operand this layer stores (all 1 for 16-bit operands)
                const float mf = FP8 ? 1.0f / (net.q_w[l] * sf) : 1.0f;
                const float mg = FP8 ? net.q_g[l + 1] / (net.q_w[l] * net.q_g[l]) : 1.0f;
                // the next 32 columns (8 points) load from TMEM while these 32 are processed
                float va[32], vb[32];
                tmem_ld32(lane_addr, va);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < C::HROWS / 32; ++q) {
                    float(&v)[32] = (q & 1) ? vb : va;
                    float(&vn)[32] = (q & 1) ? va : vb;
                    if (q + 1 < C::HROWS / 32) tmem_ld32(lane_addr + (q + 1) * 32u, vn);
                    if (live && !FP8) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            // P_i = sin(A_i);  G_i = (W_i G_{i-1}) (.) cos(A_i), points 2c, 2c + 1
                            uint32_t w[4];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int j = (2 * c + e) * 4;
                                float sn, cs;
                                sincos_fast(v[j] + bb, &sn, &cs);
                                w[2 * e] = pack16x2<F16>(sn, cs * v[j + 1]);
                                w[2 * e + 1] = pack16x2<F16>(cs * v[j + 2], cs * v[j + 3]);
                            }
                            st_shared_v4(x_s + xoff16<W>(h, m, q * 4 + c), w[0], w[1], w[2], w[3]);
                        }
                    }
                    if (live && FP8) {
#pragma unroll
                        for (int pq = 0; pq < 8; pq += 4) {
                            // the same, rescaled to the stored E4M3 operands
                            float o[4][4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int j = (pq + e) * 4;
                                float sn, cs;
                                sincos_fast(fmaf(v[j], mf, bb), &sn, &cs);
                                const float cg = cs * mg;
                                o[e][0] = sn * sf; o[e][1] = cg * v[j + 1]; o[e][2] = cg * v[j + 2];
                                o[e][3] = cg * v[j + 3];
                            }
                            store_quad8<C::NROWS>(x_s, m, lane, p0 + q * 8 + pq, o);
                        }
                    }
                    tmem_wait_ld();
                }
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(bar_xready + 8u * h);
            }
            if (ok)
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_dfull + 8u * h, df_phase, a.status, abort_flag));
            df_phase ^= 1u;
            if (ok && mt == 0) {
                tc_fence_after();
                float v[32];
                tmem_ld32(tmem + (static_cast<uint32_t>(quad * 32) << 16) + h * 128u, v);
                tmem_wait_ld();
                // lane row r = 32 quad + lane of this half = 4 * point + stream; head + remainder of w_out
                const float val = FP8 ? fmaf(v[1], 1.0f / 16.0f, v[0]) * (1.0f / (net.q_o * net.q_g[KH])) : v[0] + v[1];
                const int g = lane & ~3;
                const float gx = __shfl_sync(0xffffffffu, val, g + 1);
                const float gy = __shfl_sync(0xffffffffu, val, g + 2);
                const float gz = __shfl_sync(0xffffffffu, val, g + 3);
                const int p = p0 + ((32 * quad + lane) >> 2);
                if ((lane & 3) == 0) {
                    const int idx = idxs[p];
                    if (idx >= 0) {
                        float ox = gx, oy = gy, oz = gz;
                        if (a.normalize) {
                            const float len = sqrtf(gx * gx + gy * gy + gz * gz);
                            const float inv = len >= 1e-12f ? 1.0f / len : 0.0f;
                            ox *= inv;
                            oy *= inv;
                            oz *= inv;
                        }
                        a.out[idx] = ox;
                        a.out[a.n + idx] = oy;
                        a.out[2 * a.n + idx] = oz;
                    }
                }
            }
            tc_fence_before();
            // the next half-tile's point load overwrites idxs/pts of this half;
            // the OR-barrier also makes the stop decision uniform over the group
            if (bar_or(1 + h, C::GROUP_THREADS, !ok || *abort_flag != 0)) break;
        }
        if (gt < C::HPTS) cp_async_wait_all();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
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
