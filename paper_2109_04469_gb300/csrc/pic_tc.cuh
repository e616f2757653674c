// pic_tc.cuh -- 5th-generation tensor cores (tcgen05) for sm_103a, as inline PTX: tensor-memory
// allocation, shared-memory matrix descriptors, the BF16 MMA with FP32 accumulation in tensor
// memory, its completion through an mbarrier, and the accumulator read-back.  Used by the
// surrogate network's GEMMs (pic_mlp.cu); the particle path uses no tensor cores.
#pragma once
#include <cstdint>

#include "pic_tma.cuh"

namespace pic {

// Operand tiles in shared memory use the canonical K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes (8 BF16), each 128 contiguous bytes; the core matrices of a
// row group follow each other along K (stride kTcLbo), row groups follow at stride SBO.
constexpr unsigned kTcLbo = 128;

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets
// in 16-byte units, the fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ unsigned long long tc_smem_desc(const void* smem, unsigned lbo,
                                                           unsigned sbo) {
  const unsigned long long a = smem_u32(smem);
  return ((a >> 4) & 0x3FFFull) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ __forceinline__ unsigned tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
         ((unsigned)(M >> 4) << 24);
}

// Tensor-memory columns (power of two, >= 32), allocated by one whole warp; the base address
// is written to *slot (shared memory).
__device__ __forceinline__ void tc_alloc(unsigned* slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 2-D tiled tensor copy global -> shared (TMA) completing on `bar`: the box of the tensor map
// `map` whose first element is (x, y), x counted in elements along the contiguous dimension
// (x times the element size must be a multiple of 16 bytes); box parts outside the tensor are
// zero-filled.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(unsigned dtmem, unsigned long long adesc,
                                            unsigned long long bdesc, unsigned idesc,
                                            bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
      : "memory");
}

// Arrive on *bar once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace pic
