// Fifth-generation tensor-core primitives of sm_100-family GPUs (sm_103a), in
// inline PTX: tensor-memory (TMEM) allocation, loads and stores, the tcgen05.mma
// contraction with its instruction and shared-memory matrix descriptors, the
// completion signal through an mbarrier, and the fences between the thread and
// tensor-core views of shared and tensor memory.  Used by the many-right-hand-
// side product (matvec_tc.cu); compiled into a small test harness as well, so the
// descriptor conventions are checked on a single tile against a host GEMM.
//
// Conventions (cta_group::1, M = 128):
//   * the accumulator D (128 x N, FP32) occupies TMEM lanes 0..127 (row m <-> lane m)
//     and N consecutive 32-bit columns;
//   * the A operand may sit in TMEM (row m <-> lane m, K consecutive 32-bit columns,
//     one TF32 element per column) or in shared memory; the B operand (N x K) sits
//     in shared memory;
//   * shared-memory operands are K-major without swizzle: a "core matrix" is 8 rows
//     of 16 contiguous bytes (four 32-bit elements along K); the descriptor's leading
//     byte offset (LBO) is the distance between core matrices adjacent in K and its
//     stride byte offset (SBO) the distance between groups of 8 rows;
//   * a warp reaches only its quadrant of TMEM: lanes 32 (w mod 4) ... + 31.
#pragma once

#include <stdint.h>

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// mbarriers (completion of tensor-core work)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the tensor core's (async proxy's) arrivals
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete, at most max_iter polls;
// false if the limit ran out (the caller records an error and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t max_iter) {
    for (uint32_t i = 0; i < max_iter; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// one arrival that also announces `bytes` of bulk copies completing on this barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// ---------------------------------------------------------------------------
// bulk copies global -> shared (the tensor memory accelerator), completion
// counted in bytes on an mbarrier; addresses 16-byte aligned, size a multiple of 16
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// L2 policy for data read once (evicted first)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// named barrier over `count` threads (a multiple of 32), id 1..15
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// signal arrival at a named barrier without waiting (the barrier completes when
// `count` threads have arrived or synced on it)
__device__ __forceinline__ void named_arrive(uint32_t id, uint32_t count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// the same barrier, returning the OR of `pred` over the participating threads (every
// thread gets the same answer, so a decision taken from it keeps them in step)
__device__ __forceinline__ bool named_sync_or(uint32_t id, uint32_t count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------
// tensor memory
// ---------------------------------------------------------------------------
// whole warp: allocate ncols (power of two, 32..512) columns of all 128 lanes; the
// TMEM address (lane 0, first column) is written to *dst (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// order tensor-core operations before / after a thread synchronisation
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's shared-memory stores visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM address of (lane, column) relative to an allocation base
__device__ __forceinline__ uint32_t taddr(uint32_t base, uint32_t lane, uint32_t col) {
    return base + (lane << 16) + col;
}

// whole warp: thread t writes 8 consecutive 32-bit columns of lane (lane(ta) + t)
__device__ __forceinline__ void tmem_st8(uint32_t ta, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
// whole warp: wait until this thread's TMEM stores have completed
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// whole warp: thread t reads 16 consecutive 32-bit columns of lane (lane(ta) + t);
// the load and its completion wait are one statement, so no use of the values can
// be scheduled before the data have arrived
__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&f)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// descriptors and the contraction
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, K-major, no swizzle: start address, leading
// byte offset (between core matrices adjacent in K), stride byte offset (between
// 8-row groups), descriptor version 1 (bits 46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B
// TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), no negation,
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) (+)= A (TMEM) * B (shared memory)^T, one K step of 8 TF32 elements.
// Issued by a single thread.  acc = 0 overwrites D.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_t, uint32_t a_t, uint64_t b_desc, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_t),
        "r"(a_t), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}
// the same with A in shared memory
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_t, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_t),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}
// one arrival on *bar once every tensor-core operation this thread issued so far has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// ---------------------------------------------------------------------------
// three-term TF32 splitting (FP32-level products on the TF32 tensor path)
// ---------------------------------------------------------------------------
// v ~ hi + lo with hi = v rounded to TF32 (10 explicit mantissa bits, nearest,
// ties away) and lo = (v - hi) rounded to TF32 the same way (v - hi is exact in
// FP32 and at most 2^-11 |v|); the product a b is taken as
// hi_a hi_b + hi_a lo_b + lo_a hi_b, whose dropped term lo_a lo_b and the rounding
// of lo leave a relative error of about 2^-22 per product.
// Round to the nearest TF32 value, ties away from zero, on the bit pattern: add half
// a unit of the 10th mantissa bit to the magnitude and clear the 13 bits below it
// (a carry into the exponent is the correct rounding up; finite inputs only).  Two
// integer operations instead of a conversion instruction.
__device__ __forceinline__ uint32_t tf32_hi(float v) { return (__float_as_uint(v) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void tf32_split(float v, uint32_t& hi, uint32_t& lo) {
    hi = tf32_hi(v);
    lo = tf32_hi(v - __uint_as_float(hi));
}

}  // namespace tc
