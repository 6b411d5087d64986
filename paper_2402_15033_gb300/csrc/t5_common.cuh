// Blackwell (sm_103a) building blocks of the fifth-generation tensor-core
// kernels: mbarriers with bounded waits, bulk asynchronous copies (the TMA
// engine, cp.async.bulk), tensor memory (TMEM) allocation and loads, and
// tcgen05.mma on f16 operands held in shared memory.
//
// Operand layouts.  Without swizzling a core matrix is 8 rows of 16 bytes
// (8 f16) stored as 128 contiguous bytes, the descriptor's leading byte offset
// stepping along K and its stride byte offset along M (or N); the tensor core
// then reads the rows of 8 core matrices from one bank group, so the operands
// of the kernels use the 128-byte swizzle instead (t5_sw128), whose atoms
// spread those rows over all banks.
//
// Every wait is bounded: after kT5WaitNs nanoseconds of global time it gives
// up and returns false, and the kernels then mark their results invalid (NaN)
// and leave after releasing their tensor memory, so a lost arrival can never
// hang the GPU.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gm {

constexpr unsigned long long kT5WaitNs = 2000000000ull;   // 2 s of global time per wait

__device__ __forceinline__ uint32_t t5_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long t5_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- mbarriers
__device__ __forceinline__ void t5_bar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(t5_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void t5_bar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Wait for the phase of parity `parity` to complete; false after kT5WaitNs.
// try_wait blocks for a hardware-chosen interval before reporting an
// incomplete phase; the global timer is read between such reports.
__device__ __forceinline__ bool t5_bar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool t5_bar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = t5_smem(bar);
    if (t5_bar_try(a, parity)) return true;
    const unsigned long long t0 = t5_now_ns();
    while (!t5_bar_try(a, parity))
        if (t5_now_ns() - t0 > kT5WaitNs) return false;
    return true;
}
// One plain arrival.
__device__ __forceinline__ void t5_bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(t5_smem(bar)) : "memory");
}
// One arrival that also expects `bytes` of asynchronous copies in this phase.
__device__ __forceinline__ void t5_bar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(t5_smem(bar)), "r"(bytes) : "memory");
}

// ---- bulk copy global -> shared (TMA engine): 16-byte aligned addresses, bytes % 16 == 0
__device__ __forceinline__ void t5_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     t5_smem(dst)),
                 "l"(src), "r"(bytes), "r"(t5_smem(bar))
                 : "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor cores (async proxy).
__device__ __forceinline__ void t5_fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- tensor memory (called by one whole warp)
__device__ __forceinline__ void t5_tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(t5_smem(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void t5_tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void t5_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void t5_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading byte offset,
// stride byte offset, descriptor version 1, layout (0: no swizzle, 2: 128-byte
// swizzle).
constexpr uint32_t kT5NoSwizzle = 0, kT5Swizzle128 = 2;
__device__ __forceinline__ uint64_t t5_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
// 128-byte swizzle, K-major: a row holds 64 f16 K values (128 bytes); eight
// rows form a 1024-byte atom (1024-aligned) in which the 16-byte chunk q of row
// r sits at chunk q ^ (r % 8).  Consecutive 8-row groups are 1024 bytes apart
// (stride byte offset); a 16-wide k-step s starts 32 s bytes into the rows.
__device__ __forceinline__ uint32_t t5_sw128(int row, int chunk) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}
// Instruction descriptor of kind::f16: f16 A and B, FP32 accumulator, M x N,
// A / B MN-major when a_mn / b_mn (K-major otherwise).
__host__ __device__ constexpr uint32_t t5_idesc_f16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
// D (TMEM) = A B^T (+ D when accum): one elected thread issues.
__device__ __forceinline__ void t5_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
// Arrive on bar once every tcgen05 operation this thread issued has completed.
__device__ __forceinline__ void t5_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(t5_smem(bar))
                 : "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. + 31); complete after t5_ld_wait().
__device__ __forceinline__ void t5_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// 8 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void t5_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void t5_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace gm
