// Fifth-generation tensor-core building blocks for sm_103a (inline PTX): tensor-memory (TMEM)
// allocation, shared-memory operand descriptors, tcgen05.mma of kind tf32 with FP32
// accumulation in TMEM, commit to an mbarrier, and TMEM loads for the epilogue.
//
// Operand layout used everywhere here: K-major, no swizzle. A matrix of R rows (M or N
// dimension) and K columns is stored as core matrices of 8 rows x 16 bytes (8 x 4 fp32
// values, 128 contiguous bytes, row r at byte 16 r); the core matrices of one 8-row group
// follow each other along K every kLbo = 128 bytes (leading-dimension byte offset); 8-row
// groups are `sbo` bytes apart (stride-dimension byte offset). Element (r, k) of a tile with
// kc columns therefore sits at byte (r / 8) * sbo + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4
// with sbo = (kc / 4) * 128. One MMA consumes K = 8 (two core matrices along K); the next K
// step starts 256 bytes further.
//
// FP32 accuracy from TF32 units ("3xTF32"): x = x_hi + x_lo with x_hi = x rounded to TF32
// and x_lo = x - x_hi (exact in FP32); a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, the dropped
// a_lo b_lo and the TF32 truncation of the low parts being ~2^-21 relative.
#pragma once
#include <cstdint>

#include "common.cuh"

namespace nsp {
namespace tc {

constexpr uint32_t kLbo = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ int element_offset(int r, int k, int sbo) {   // bytes
  return (r >> 3) * sbo + (k >> 2) * (int)kLbo + ((r & 7) << 4) + ((k & 3) << 2);
}

// 64-bit shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), version 1,
// base offset 0, relative LBO mode, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// 32-bit instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, no
// negation, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation by one full warp; the allocated address is written to *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem] (+)= A B^T for one K step; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((int)accumulate)
      : "memory");
}

// The mbarrier arrives once every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Wait for the phase with the given parity to complete; gives up after max_spins polls and
// returns false (the caller records the timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int max_spins) {
  const uint32_t a = smem_u32(mbar);
  for (int i = 0; i < max_spins; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Eight consecutive 32-bit TMEM columns of this thread's lane (warp w of a warpgroup reads
// lanes 32 (w % 4) .. + 31; taddr carries the lane in bits 16-31, the column in bits 0-15).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Sixteen consecutive 32-bit TMEM columns of this thread's lane, without waiting: the caller
// issues several and then waits once (tmem_wait_ld) before reading any of them.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// x = hi + lo, hi = x rounded to TF32 (round to nearest, ties away), lo = x - hi exactly.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

}  // namespace tc
}  // namespace nsp
