// 5th-generation tensor core (tcgen05, sm_100 family) building blocks: tensor
// memory (TMEM) allocation, the MMA issued by one thread with operands in
// shared memory and the accumulator in TMEM, completion through an mbarrier,
// and the TMEM -> register load of the epilogue.
//
// Conventions used by the kernels here:
//  * cta_group::1, kind::f16 with BF16 A and B, FP32 accumulation;
//  * A (M x K) and B (N x K) K-major, no swizzle: 8-row x 16-byte "core
//    matrices"; the element (row r, k) of a K = 16 operand sits at
//      start + (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2 bytes;
//  * M = 128: row r of D lives in TMEM lane r, column n in column base + n.
#pragma once

#include <cstdint>

namespace sq {
namespace tc {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (K)
// and stride (M/N) byte offsets, each >> 4 in 14-bit fields at bits 0, 16
// and 32; descriptor version 1 at bits 46-47; layout type 0 (no swizzle) at
// bits 61-63; base offset 0.
__device__ __forceinline__ uint64_t sdesc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// TMEM columns (a power of two >= 32) for this CTA, by one whole warp; the
// base address lands in *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(unsigned *dst, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B^T (+ D when accum != 0), issued by one thread.
__device__ __forceinline__ void mma_bf16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         unsigned accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// One arrival on the mbarrier once every tcgen05 operation this thread issued
// before it has completed.
__device__ __forceinline__ void mma_commit(unsigned long long *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// This warp's 32 TMEM lanes (taddr's lane field = 32 x the warp's quarter) x
// 32 consecutive FP32 columns: v[j] = column j of the thread's lane.
__device__ __forceinline__ void tmem_ld_32x32(unsigned taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// As tmem_ld_32x32, 16 consecutive columns.
__device__ __forceinline__ void tmem_ld_32x16(unsigned taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// mbarrier helpers for the MMA completions (count 1: the commit's arrival).
__device__ __forceinline__ void mbar_init(unsigned long long *mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// mbarrier expecting `count` arrivals per phase.
__device__ __forceinline__ void mbar_init_count(unsigned long long *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival of this thread (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(unsigned long long *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(mbar)) : "memory");
}
// Waits, at most max_tries polls, for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, unsigned parity, int max_tries) {
  for (int i = 0; i < max_tries; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// As mbar_wait, and gives up early once *fail is set (by another role of the CTA).
__device__ __forceinline__ bool mbar_wait_or_fail(unsigned long long *mbar, unsigned parity, int max_tries,
                                                  const volatile int *fail) {
  for (int i = 0; i < max_tries; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (*fail) return false;
  }
  return false;
}

}  // namespace tc
}  // namespace sq
