// Fifth-generation tensor cores of sm_100-family GPUs (tcgen05): TF32
// operands staged in shared memory, FP32 accumulators in tensor memory
// (TMEM), one MMA instruction issued by one thread of the CTA.
//
// Operand layout in shared memory (no swizzle, K-major): the M x K (or N x K)
// operand is cut into core matrices of 8 rows x 4 elements (16 bytes per row,
// 128 contiguous bytes per core matrix). Core matrices that follow each other
// along K are LBO bytes apart, those along M (or N) SBO bytes apart. With the
// K extent of a staged tile fixed at kt elements and core matrices packed
// K-fastest, element (r, k) sits at float offset
//   ((r / 8) * (kt / 4) + k / 4) * 32 + (r % 8) * 4 + k % 4,
// LBO = 128 and SBO = kt * 32 bytes; an MMA step over K = 8 starts 256 bytes
// after the previous one.
//
// Accumulator layout (cta_group::1, M = 128): row i of D is TMEM lane i and
// column j is TMEM column (base + j), one FP32 value each. Warp w of the CTA
// may read lanes 32 (w % 4) .. 32 (w % 4) + 31 only.
//
// Precision: a TF32 MMA reads 10 explicit mantissa bits. An FP32 operand x is
// split into hi = rna_tf32(x) and lo = rna_tf32(x - hi); the product of two
// split operands is taken as hi*hi + hi*lo + lo*hi (three MMAs into one FP32
// accumulator, "3xTF32"), which leaves about 2^-21 relative error per term.
#pragma once
#include <cstdint>

namespace tepai {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Float offset of element (r, k) in a K-major staged tile whose K extent is kt.
__host__ __device__ __forceinline__ int kmajor_off(int r, int k, int kt) {
  return (((r >> 3) * (kt >> 2) + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (K) and
// stride (M/N) byte offsets in 16-byte units, descriptor version 1.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, dense, N / 8 and M / 16 in their fields.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A B^T (+ D when acc != 0); A from descriptor a (M x 8), B from
// descriptor b (N x 8). Issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// Arrive on the mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(saddr(bar)) : "memory");
}

// TMEM allocation (one whole warp, converged; ncols a power of two >= 32).
// The base address is written to *slot in shared memory.
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(saddr(slot)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void relinquish() {
  __syncwarp();
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tcgen05 operations across a CTA barrier.
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Generic-proxy writes to shared memory made visible to the tensor core.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Eight consecutive FP32 columns of this thread's TMEM lane (warp-collective;
// taddr carries the warp's lane base in bits 16..31). Waits for the load. The
// instruction is .sync.aligned: every lane of the warp must execute it
// together, so the warp is reconverged first (callers may branch per lane
// between two loads).
__device__ __forceinline__ void ld8(uint32_t taddr, float v[8]) {
  __syncwarp();
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
      : "r"(taddr)
      : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
  v[4] = __uint_as_float(r4); v[5] = __uint_as_float(r5); v[6] = __uint_as_float(r6); v[7] = __uint_as_float(r7);
}

// FP32 -> TF32 (10 explicit mantissa bits), round to nearest, ties away.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace tepai
