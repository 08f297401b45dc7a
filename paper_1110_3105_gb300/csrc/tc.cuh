// Fifth-generation tensor cores (tcgen05) on sm_103a: thin inline-PTX
// wrappers used by the block products of the multi-column solve.
//
//   * Operands are staged by the CTA's threads in shared memory in the
//     K-major, 128-byte-swizzled canonical layout: an operand of R rows and
//     32 fp32 (or 64 bf16) K-elements per row occupies R * 128 bytes; row r
//     sits at (r / 8) * 1024 + (r % 8) * 128 and its 16-byte chunk c (K
//     elements 4c..4c+3 for fp32, 8c..8c+7 for bf16) is stored at chunk
//     position c ^ (r % 8).  Atoms of 8 rows are 1024 bytes apart (the
//     stride byte offset); the base must be 1024-byte aligned.  One MMA
//     consumes 32 bytes of K per row (8 tf32 or 16 bf16 elements); the
//     k-th such step starts 32 * k bytes into the rows.
//   * The accumulator D (M = 128 rows x N fp32 columns) lives in tensor
//     memory: row i in lane i, column j in column j of the allocation.
//     Warp w of the CTA may read lanes 32 (w % 4) .. 32 (w % 4) + 31.
//   * One thread issues the MMAs; tcgen05.commit makes an mbarrier track
//     their completion; every waiting thread polls it with an iteration
//     limit (past it the wait reports failure instead of spinning on).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rs {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (64 bits): start address >> 4 in bits
// 0-13, leading byte offset >> 4 in 16-29 (unused by swizzled K-major
// layouts, set to 1), stride byte offset >> 4 in 32-45, the descriptor
// version 1 in 46-47, base offset 0 in 49-51, layout type in 61-63
// (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                 // LBO (ignored for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;       // SBO: 8-row atoms 1024 bytes apart
  d |= (uint64_t)1u << 46;                 // version
  d |= (uint64_t)2u << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor (32 bits) of a dense MMA with fp32 accumulation:
// D format in bits 4-5 (1 = f32), A and B formats in 7-9 and 10-12
// (kind::tf32: 2 = tf32; kind::f16: 0 = f16, 1 = bf16), both operands
// K-major (bits 15, 16 clear), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc(int ab_format, int M, int N) {
  return (1u << 4) | ((uint32_t)ab_format << 7) | ((uint32_t)ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
constexpr int FMT_TF32 = 2;
constexpr int FMT_BF16 = 1;

// Byte offset of element (row, k) in a 128B-swizzled K-major operand of
// `esize`-byte elements (32 fp32 or 64 bf16 per row).
__host__ __device__ __forceinline__ uint32_t sw128_offset(int row, int k, int esize) {
  const int byte = k * esize;            // within the 128-byte row
  const int chunk = byte >> 4, within = byte & 15;
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4) + within);
}

// ---------------------------------------------------------------- TMEM
// Allocate `ncols` (power of two >= 32) columns; the whole warp calls it;
// the address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor cores.
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete: gives up
// after max_polls polls or, if limit_ns > 0, once that much time has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_polls, long long limit_ns = 0) {
  unsigned long long t0 = 0;
  if (limit_ns > 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < max_polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (limit_ns > 0 && (i & 255) == 255) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if ((long long)(t - t0) > limit_ns) return false;
    }
  }
  return false;
}

// --------------------------------------------------------------- MMA
// D[tmem] (+)= A[smem] * B[smem]^T, cta_group::1; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                        bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// The mbarrier receives one arrival once every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// ---------------------------------------------------- TMEM -> registers
// 16 consecutive 32-bit columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// fp32 -> tf32 by rounding to nearest (ties away) on the 13 dropped bits,
// and the remainder a - hi (exact in fp32).  The tensor cores read only the
// top 19 bits of a tf32 operand, so hi is exactly what they see.
__device__ __forceinline__ float tf32_hi(float a) {
  uint32_t u = __float_as_uint(a);
  if ((u & 0x7F800000u) == 0x7F800000u) return a;   // inf / nan unchanged
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}
// a = hi + lo with hi, lo tf32 values: |a - hi - lo| <= 2^-22 |a| (3xTF32
// products hi*hi + hi*lo + lo*hi then carry about fp32 accuracy).
__device__ __forceinline__ void tf32_split(float a, float& hi, float& lo) {
  hi = tf32_hi(a);
  lo = tf32_hi(a - hi);
}

}  // namespace tc
}  // namespace rs
