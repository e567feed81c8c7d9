// Device helpers shared by the sdfnn kernels: bounded waits, mbarriers, bulk
// copies, tcgen05 tensor-core/TMEM instructions (inline PTX for sm_103a) and
// the range-reduced sine/cosine used by every sine-layer epilogue.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sdfnn {

constexpr int kStatusTimeout = -6;            // SDF_ERR_TIMEOUT
constexpr uint64_t kWaitBudgetNs = 2000000000ull;  // 2 s per bounded wait

// ---------------------------------------------------------------------------
// geometry constants of the tiles
// ---------------------------------------------------------------------------
constexpr int kTileRows = 128;  // ray slots / GEMM rows per tile (one TMEM lane each)
constexpr float kBoxSlack = 1e-3f;

// ---------------------------------------------------------------------------
// sine / cosine with Cody-Waite argument reduction
// ---------------------------------------------------------------------------
// The sine layers see arguments of tens of radians (omega0 = 30).  The
// hardware approximation is accurate on [-pi, pi] only, so the argument is
// first reduced by the nearest multiple of 2*pi (Cody & Waite, "Software
// Manual for the Elementary Functions", 1980): 2*pi is split into a float
// head (exactly representable) and the float nearest to the remainder; with
// a fused multiply-add the head product is exact, so r = x - k*2*pi carries
// about one rounding for |k| up to 2^8.
constexpr float kInv2Pi = 0x1.45f306p-3f;     // 1/(2 pi) rounded to float
constexpr float k2PiHi = 0x1.921fb6p+2f;      // 2 pi rounded to float
constexpr float k2PiLo = -0x1.777a5cp-23f;    // 2 pi - k2PiHi rounded to float

__device__ __forceinline__ float reduce_2pi(float x) {
    float k = rintf(x * kInv2Pi);
    float r = fmaf(-k, k2PiHi, x);
    return fmaf(-k, k2PiLo, r);
}

__device__ __forceinline__ float sin_r(float x) { return __sinf(reduce_2pi(x)); }

// Sine/cosine for the 16-bit tensor-core paths: the hardware approximation
// applied directly (it scales its argument by 1/(2 pi) itself).  Measured on
// GB300 against double precision: absolute error <= 8.7e-6 for |x| <= 64 and
// <= 3.5e-5 for |x| <= 256, about twice the FP32 rounding of the argument
// itself and far below a 16-bit operand's rounding.  The FP32 path keeps the
// explicit reduction (error <= 5e-7 over |x| <= 256).
__device__ __forceinline__ float sin_fast(float x) { return __sinf(x); }
__device__ __forceinline__ void sincos_fast(float x, float* s, float* c) {
    *s = __sinf(x);
    *c = __cosf(x);
}

__device__ __forceinline__ void sincos_r(float x, float* s, float* c) {
    float r = reduce_2pi(x);
    *s = __sinf(r);
    *c = __cosf(r);
}

// ---------------------------------------------------------------------------
// timers, status word
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void raise_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// shared-memory addresses, fences
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Make this thread's generic-proxy shared-memory writes visible to the async
// proxy (tensor-core operand reads, bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait that may suspend the thread for up to `hint_ns` while the phase
// is incomplete (the thread resumes when the phase completes): waiting
// threads then stop competing for issue slots with working ones.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

constexpr uint32_t kWaitSleepNs = 20000;  // one suspension; the overall bound is kWaitBudgetNs

// Wait for phase `parity` of the barrier to complete, for at most
// kWaitBudgetNs.  On expiry the device status word receives
// kStatusTimeout, the block-wide abort flag is set and false is returned.
// Also returns false as soon as another thread of the block has aborted.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* status,
                                                  volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > kWaitBudgetNs) {
            raise_status(status, kStatusTimeout);
            *abort_flag = 1;
            return false;
        }
    }
}

// Wait for a bulk copy issued by this block to land before the block exits,
// whatever the abort flag says (a copy from valid global memory always
// completes); bounded by kWaitBudgetNs like every other wait.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return;
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_sleep(bar, parity, kWaitSleepNs))
        if (globaltimer_ns() - t0 > kWaitBudgetNs) return;
}

// ---------------------------------------------------------------------------
// bulk copy (TMA, non-tensor): global -> shared, completes on an mbarrier
// ---------------------------------------------------------------------------
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// ---------------------------------------------------------------------------
// tcgen05: TMEM allocation, MMA, commit, loads, fences
// ---------------------------------------------------------------------------
// Allocation is warp-wide (.sync.aligned): every lane of one warp executes it.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand stored with the
// 128-byte swizzle: rows of 64 bf16 (128 bytes), 8-row atoms of 1024 bytes
// whose 16-byte chunks are permuted by chunk ^= (row % 8).  Consecutive
// 8-row atoms are 1024 bytes apart (stride byte offset); the leading byte
// offset is unused for swizzled K-major layouts.  Bits 46-48 hold the fixed
// descriptor version 0b001, bits 61-63 the layout type (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((smem_addr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>(1u) << 16;              // leading byte offset (unused)
    d |= static_cast<uint64_t>(1024u >> 4) << 32;      // stride byte offset
    d |= static_cast<uint64_t>(1u) << 46;              // version
    d |= static_cast<uint64_t>(2u) << 61;              // 128-byte swizzle
    return d;
}

// Shared-memory descriptor of an MN-major operand with the 128-byte swizzle:
// atoms of 8 K rows x 128 bytes of MN; `lbo` = byte stride between atoms
// along MN, SBO = 1024 (8-row K groups back to back).  The instruction
// descriptor marks the operand as MN-major (bit 15 for A, bit 16 for B).
__device__ __forceinline__ uint64_t desc_mnmajor_sw128(uint32_t smem_addr, uint32_t lbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((smem_addr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>(1024u >> 4) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
}
// The descriptor of an operand `bytes` further on (a multiple of 16): the
// start address field holds address >> 4 in 14 bits and shared memory ends
// below 256 KB, so the field never carries into the next one.
__device__ __forceinline__ uint64_t desc_add(uint64_t desc, uint32_t bytes) {
    return desc + static_cast<uint64_t>(bytes >> 4);
}
constexpr uint32_t kIdescMajorMnA = 1u << 15;
constexpr uint32_t kIdescMajorMnB = 1u << 16;

// Instruction descriptor of tcgen05.mma.kind::f16 with FP32 D and both
// operands K-major: D format at bits 4-5 (1 = F32), A/B formats at bits
// 7-9 / 10-12 (0 = F16, 1 = BF16; A and B always share one type), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f32acc(int M, int N, bool f16) {
    return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) { return idesc_f32acc(M, N, false); }

// D[tmem] (+)= A[smem] * B[smem]^T with 16-bit operands (kind::f16), issued by a single thread.
__device__ __forceinline__ void mma_f16kind(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T with 8-bit operands (kind::f8f6f4).  With
// the instruction descriptor's A/B format fields 0 both operands are E4M3;
// one instruction covers K = 32 (32 bytes of each row).
__device__ __forceinline__ void mma_f8kind(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when all previously issued MMAs of this thread
// have completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32*(w%4) .. 32*(w%4)+31).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// BF16 packing and the swizzled K-major operand layout
// ---------------------------------------------------------------------------
// Round-to-nearest-even float -> bf16 pair packed low|high.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Byte offset of element (row, k) of a K-major bf16 operand with `rows` rows
// (a multiple of 8) in the 128-byte-swizzled layout: K is cut into blocks of
// 64 elements; block kb holds all rows, 128 bytes each.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t k, uint32_t rows) {
    uint32_t kb = k >> 6, kk = k & 63u;
    uint32_t chunk = (kk >> 3) ^ (row & 7u);
    return kb * rows * 128u + row * 128u + chunk * 16u + (kk & 7u) * 2u;
}

// Byte offset of 8-bit element k of `row` in the same layout: 128-element
// K blocks, 16-element chunks.
__host__ __device__ __forceinline__ uint32_t sw128_offset8(uint32_t row, uint32_t k, uint32_t rows) {
    uint32_t kb = k >> 7, kk = k & 127u;
    uint32_t chunk = (kk >> 4) ^ (row & 7u);
    return kb * rows * 128u + row * 128u + chunk * 16u + (kk & 15u);
}

// Byte offset of the 16-byte chunk holding elements k8*8 .. k8*8+7 of `row`.
__host__ __device__ __forceinline__ uint32_t sw128_chunk_offset(uint32_t row, uint32_t k8, uint32_t rows) {
    uint32_t kb = k8 >> 3, c = k8 & 7u;
    return kb * rows * 128u + row * 128u + ((c ^ (row & 7u)) * 16u);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// 4-byte asynchronous copy global -> shared (no register staging), and the
// wait for all of this thread's outstanding ones.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void st_shared_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Byte permute: result byte i = byte sel[i] of the 8-byte pair {b:a}.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__device__ __forceinline__ void st_shared_u16(uint32_t addr, uint16_t v) {
    asm volatile("st.shared.u16 [%0], %1;" ::"r"(addr), "h"(v) : "memory");
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(0.0f), "f"(x));
    return static_cast<uint16_t>(r & 0xFFFFu);
}

// Round-to-nearest-even float -> f16 pair packed low|high.
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ uint16_t f16_bits(float x) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(0.0f), "f"(x));
    return static_cast<uint16_t>(r & 0xFFFFu);
}

// 16-bit tensor-core operand type: F16 = true selects IEEE half, else bfloat16.
template <bool F16>
__device__ __forceinline__ uint32_t pack16x2(float lo, float hi) {
    return F16 ? pack_f16x2(lo, hi) : pack_bf16x2(lo, hi);
}
// Four floats as E4M3 bytes (round to nearest even, saturating to +-448),
// a in the lowest byte.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return static_cast<uint32_t>(lo) | (static_cast<uint32_t>(hi) << 16);
}

template <bool F16>
__device__ __forceinline__ uint16_t bits16(float x) {
    return F16 ? f16_bits(x) : bf16_bits(x);
}
template <bool F16>
__device__ __forceinline__ float from16(uint16_t h) {
    if (F16) {
        float f;
        asm("{\n\t.reg .f16 t;\n\tmov.b16 t, %1;\n\tcvt.f32.f16 %0, t;\n\t}" : "=f"(f) : "h"(h));
        return f;
    }
    return __uint_as_float(static_cast<uint32_t>(h) << 16);
}

// ---------------------------------------------------------------------------
// named barriers over a subset of the block's threads
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bar_named(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// OR-reduction barrier over `nthreads` threads (named barrier `id`): true if
// any participating thread passed pred.
__device__ __forceinline__ bool bar_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(pred)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------
// warp-aggregated work distribution
// ---------------------------------------------------------------------------
// Every lane with `want` set receives a distinct index from *counter (one
// atomicAdd per warp).  Must be called by the full warp.
__device__ __forceinline__ long long warp_grab(unsigned long long* counter, bool want) {
    const unsigned mask = __ballot_sync(0xffffffffu, want);
    if (mask == 0) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, static_cast<unsigned long long>(__popc(mask)));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!want) return -1;
    return static_cast<long long>(base + __popc(mask & ((1u << lane) - 1u)));
}

}  // namespace sdfnn
