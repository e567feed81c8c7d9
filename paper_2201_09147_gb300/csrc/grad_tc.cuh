// Analytic-gradient kernel (Alg. 2) on the tensor cores, shared by the
// normal-mapping path and the training forward pass.
#pragma once

#include "tc_common.cuh"

namespace sdfnn {
namespace {

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
    uint32_t x, ring, woutb, w0, wt, pts, idx, nidx, red, bars, misc, total;
};

// TRAIN adds the per-half sums of the FP32 output layer (128 floats per half).
template <int W, int OP, bool TRAIN = false>
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
    L.red = o;
    o += TRAIN ? 2u * 128u * 4u : 0u;
    L.bars = o;
    o += (2 * C::NS + 4) * 8u;
    o = (o + 15u) & ~15u;
    L.misc = o;
    o += 32u;
    L.total = o;
    return L;
}

// Saved training records of hidden layer l (training forward -> backward and
// weight gradient); np = the point count rounded up to whole 64-point tiles.
// A_l is [l][np/4][W][4] floats and H_l [l][np/2][W][2] uint2, so that the
// records of 4 (A) or 2 (H) consecutive points of one unit are one 16-byte
// vector for the kernels that read them.
__host__ __device__ inline int64_t rec_points(int64_t n) { return (n + 63) / 64 * 64; }
__host__ __device__ inline size_t rec_a(size_t l, size_t np, int W, size_t p, int m) {
    return ((l * (np / 4) + p / 4) * static_cast<size_t>(W) + static_cast<size_t>(m)) * 4 + (p & 3);
}
__host__ __device__ inline size_t rec_h(size_t l, size_t np, int W, size_t p, int m) {
    return ((l * (np / 2) + p / 2) * static_cast<size_t>(W) + static_cast<size_t>(m)) * 2 + (p & 1);
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

// Sum over the 32 lanes of a warp of each of v[0..31]: afterwards lane L holds,
// in v[0], the sum of entry L (recursive halving, 31 shuffles).
__device__ __forceinline__ void warp_sum32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = upper ? v[i] : v[i + s];
            const float keep = upper ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
}

// TRAIN (16-bit operands only): the training forward.  Besides grad f the
// kernel saves A_0 and, per hidden layer, A_l = W_l P_{l-1} + b_l in FP32 and
// H_l = W_l G_{l-1} in the 16-bit operand type for the backward, and the output layer runs in FP32 on
// the CUDA cores instead of as an MMA: f = w_out . sin(A_k) + b_out and
// grad f = w_out . (cos(A_k) (.) H_k), summed over the features by a warp
// butterfly and shared-memory atomics, so no tangent of the last layer is
// rounded to 16 bits.
//
// One block per SM is stated for the width-64/128 training and E4M3 variants,
// where it lets the compiler use the registers that one block leaves free
// instead of spilling (fitting steps of the (64,2) and (128,2) 3 % and 5 %
// faster).  Without it otherwise: the width-256 variants then allocate 96
// registers (the cap of 18 warps, five of which share one scheduler's 16 K
// registers) and spill, and the width-128 normal map measured 1 % slower.
template <int W, int OP, bool TRAIN = false>
__global__ void __launch_bounds__(GradCfg<W, OP>::THREADS, (W < 256 && (TRAIN || OP == kOpE4M3)) ? 1 : 0)
    grad_tc_kernel(const GradArgs a) {
    using C = GradCfg<W, OP>;
    constexpr bool F16 = OP == kOpF16;
    constexpr bool FP8 = OP == kOpE4M3;
    static_assert(!(TRAIN && FP8), "the training forward runs with 16-bit operands");
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t raw_s = smem_u32(smem_raw);
    const uint32_t base_s = (raw_s + 1023u) & ~1023u;
    uint8_t* base = smem_raw + (base_s - raw_s);
    const NetView& net = a.net;
    const int KH = net.n_hidden;
    const GradLayout L = grad_layout<W, OP, TRAIN>(KH);
    float* w0s = reinterpret_cast<float*>(base + L.w0);
    float* red = reinterpret_cast<float*>(base + L.red);  // TRAIN: [half][point * 4 + stream]
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
    if (TRAIN)
        for (int i = tid; i < 256; i += C::THREADS) red[i] = 0.0f;
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
    // groups per pair: the hidden layers, and the output layer unless TRAIN computes it in FP32
    const int GPP = TRAIN ? KH : KH + 1;
    const int n_groups = static_cast<int>(my_pairs) * GPP;
    bool ok = true;

    if (warp == C::PRODUCER_WARP) {
        if (lane == 0) {
            // stages in MMA order: per slot of the schedule, the stages of its layer
            // (K blocks SKB * sg .. of every TMEM tile: contiguous in the weight image)
            uint32_t g = 0;
            int lh[2] = {0, 0};  // slot of each half within its pair (grp mod GPP, counted)
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    const int l = lh[h];
                    lh[h] = l + 1 == GPP ? 0 : l + 1;
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
            int lh[2] = {0, 0};
            for (int k = 0; k < n_groups + LAG && ok; ++k)
#pragma unroll
                for (int h = 0; h < 2 && ok; ++h) {
                    const int grp = k - h * LAG;
                    if (grp < 0 || grp >= n_groups) continue;
                    const int l = lh[h];
                    lh[h] = l + 1 == GPP ? 0 : l + 1;
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
        const float wo = TRAIN && live ? __ldg(net.wout + m) : 0.0f;  // w_out of this feature (TRAIN)
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
                            if (TRAIN) {
                                const int idx = idxs[p0 + 2 * c + e];
                                if (idx >= 0) a.save_a0[static_cast<size_t>(idx) * W + m] = z;
                            }
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
                    if (TRAIN && live) {
                        // save (A_l, H_l) per point; below the last layer write X as usual,
                        // at the last layer form w_out times (P_k, G_k) in place and sum it
                        // over the warp's features
                        const bool last = l + 1 == KH;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            uint32_t w[4];
                            float sa[2];  // this pair's saved records: A_l, and H_l in 16 bits
                            uint2 sh[2];
#pragma unroll
                            for (int e = 0; e < 2; ++e) {
                                const int j = (2 * c + e) * 4;
                                const float A = v[j] + bb;
                                sa[e] = A;
                                sh[e] = make_uint2(pack16x2<F16>(v[j + 1], v[j + 2]), pack16x2<F16>(v[j + 3], 0.0f));
                                float sn, cs;
                                sincos_fast(A, &sn, &cs);
                                if (last) {
                                    const float wc = wo * cs;
                                    v[j] = wo * sn;
                                    v[j + 1] *= wc;
                                    v[j + 2] *= wc;
                                    v[j + 3] *= wc;
                                } else {
                                    w[2 * e] = pack16x2<F16>(sn, cs * v[j + 1]);
                                    w[2 * e + 1] = pack16x2<F16>(cs * v[j + 2], cs * v[j + 3]);
                                }
                            }
                            if (!last) st_shared_v4(x_s + xoff16<W>(h, m, q * 4 + c), w[0], w[1], w[2], w[3]);
                            // the pair's points are consecutive and the first even (training batches
                            // run without a list); a pair past the batch end stores into the padding
                            const int idx = idxs[p0 + q * 8 + 2 * c];
                            if (idx >= 0) {
                                const size_t np = static_cast<size_t>(a.save_np);
                                *reinterpret_cast<float2*>(a.save_a + rec_a(l, np, W, idx, m)) = make_float2(sa[0], sa[1]);
                                *reinterpret_cast<uint4*>(a.save_h + rec_h(l, np, W, idx, m)) =
                                    make_uint4(sh[0].x, sh[0].y, sh[1].x, sh[1].y);
                            }
                        }
                        if (last) {
                            warp_sum32(v, lane);
                            atomicAdd(&red[h * 128 + q * 32 + lane], v[0]);
                        }
                    }
                    if (!TRAIN && live && !FP8) {
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
                if (!TRAIN || l + 1 < KH) mbar_arrive(bar_xready + 8u * h);
            }
            if (TRAIN) {
                // the group's share of the output sums is in red: f and grad f of its 32 points
                bar_named(1 + h, C::GROUP_THREADS);
                if (gt < C::HPTS) {
                    float* r = red + h * 128 + gt * 4;
                    const int idx = idxs[p0 + gt];
                    if (ok && idx >= 0) {
                        a.out_f[idx] = r[0] + *a.out_bias;
                        a.out[idx] = r[1];
                        a.out[a.n + idx] = r[2];
                        a.out[2 * a.n + idx] = r[3];
                    }
                    r[0] = r[1] = r[2] = r[3] = 0.0f;
                }
            }
            if (!TRAIN && ok)
                ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar_dfull + 8u * h, df_phase, a.status, abort_flag));
            if (!TRAIN) df_phase ^= 1u;
            if (!TRAIN && ok && mt == 0) {
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

}  // namespace
}  // namespace sdfnn
