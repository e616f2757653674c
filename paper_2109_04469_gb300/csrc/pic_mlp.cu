// pic_mlp.cu -- the surrogate network of the parameter scans: a
// 7 -> 256 -> 256 -> 192 MLP with GELU, BF16 weights and activations, FP32 accumulation,
// trained and evaluated by this file's kernels.  Every matrix product runs on the tcgen05
// tensor cores (pic_tc.cuh): operand tiles staged in shared memory in the canonical K-major
// layout, the accumulator in tensor memory, read back for an FP32 epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "pic.h"
#include "pic_dev.cuh"
#include "pic_tc.cuh"

namespace pic {
namespace {

constexpr int kTcM = 128;        // rows of A per CTA (one MMA tile)
constexpr int kKc = 64;          // K staged per shared-memory round (four MMA K-steps)
constexpr int kGemmThreads = 128;

size_t gemm_smem_bytes(int N) { return (size_t)kTcM * kKc * 2 + (size_t)N * kKc * 2; }

// C[M x N] (FP32, row stride ldc) = A[M x K] * B[N x K]^T, A and B BF16 row-major (K
// contiguous).  M % 128 == 0, N % 16 == 0 with 16 <= N <= 256, K % 16 == 0, K >= 16.
// One CTA per 128 rows; thread 0 issues the MMAs; the four warps read back their 32 rows.
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                float* __restrict__ C, int N, int K, int ldc, int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sA = tsm;
  unsigned char* sB = tsm + (size_t)kTcM * kKc * 2;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM;
  const unsigned ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
  if (warp == 0) tc_alloc(&tslot, ncols);
  if (tid == 0) {
    mbar_init(&bar, 1u);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = tslot;
  const unsigned idesc = tc_idesc_bf16(kTcM, N);
  unsigned phase = 0;
  for (int k0 = 0; k0 < K; k0 += kKc) {
    const int kc = min(kKc, K - k0);  // a multiple of 16
    const int pieces = kc / 8;        // 16-byte pieces of a row
    const unsigned sbo = (unsigned)pieces * kTcLbo;
    for (int i = tid; i < kTcM * pieces; i += kGemmThreads) {
      const int r = i / pieces, kb = i - r * pieces;
      const uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * K + k0 + 8 * kb);
      *reinterpret_cast<uint4*>(sA + (r >> 3) * sbo + kb * kTcLbo + (r & 7) * 16) = v;
    }
    for (int i = tid; i < N * pieces; i += kGemmThreads) {
      const int r = i / pieces, kb = i - r * pieces;
      const uint4 v = *reinterpret_cast<const uint4*>(B + (size_t)r * K + k0 + 8 * kb);
      *reinterpret_cast<uint4*>(sB + (r >> 3) * sbo + kb * kTcLbo + (r & 7) * 16) = v;
    }
    fence_proxy_async_smem();  // the tiles just written are read by the tensor core
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int s = 0; s < kc / 16; ++s)  // K-step s covers core matrices 2s, 2s+1 along K
        tc_mma_bf16(taddr, tc_smem_desc(sA + s * 2 * kTcLbo, kTcLbo, sbo),
                    tc_smem_desc(sB + s * 2 * kTcLbo, kTcLbo, sbo), idesc, k0 > 0 || s > 0);
      tc_commit(&bar);
    }
    // the MMAs read the tiles: wait before the next round overwrites them
    if (!mbar_wait(&bar, phase)) {
      if (lane == 0) atomicOr(err, 1);
    }
    phase ^= 1u;
    tc_fence_after();
  }
  const int row = m0 + warp * 32 + lane;
  for (int c = 0; c < N; c += 16) {
    float v[16];
    tc_ld16(taddr + ((unsigned)(warp * 32) << 16) + (unsigned)c, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) C[(size_t)row * ldc + c + j] = v[j];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(taddr, ncols);
}

bool gemm_shape_ok(int M, int N, int K) {
  return M > 0 && M % kTcM == 0 && N >= 16 && N <= 256 && N % 16 == 0 && K >= 16 &&
         K % 16 == 0;
}

cudaError_t launch_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                        int K, int ldc, int* err, cudaStream_t s) {
  // room for the widest B tile whatever N is, so no staging can reach past the allocation
  static const cudaError_t configured = cudaFuncSetAttribute(
      k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem_bytes(256));
  if (configured != cudaSuccess) return configured;
  (void)N;
  k_gemm_bf16<<<M / kTcM, kGemmThreads, gemm_smem_bytes(256), s>>>(A, B, C, N, K, ldc, err);
  return cudaGetLastError();
}

__device__ int g_gemm_err;  // timeout flag of the stand-alone GEMM entry point

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" {

int pic_tc_gemm_bf16(const uint16_t* a, const uint16_t* b, float* c, int32_t m, int32_t n,
                     int32_t k, void* cuda_stream) {
  if (!a || !b || !c || !gemm_shape_ok(m, n, k)) return PIC_ERR_PARAM;
  int* err = nullptr;
  const int zero = 0;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetSymbolAddress((void**)&err, g_gemm_err) != cudaSuccess ||
      cudaMemcpyAsync(err, &zero, sizeof zero, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      launch_gemm(reinterpret_cast<const __nv_bfloat16*>(a),
                  reinterpret_cast<const __nv_bfloat16*>(b), c, m, n, k, n, err, s) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  return h ? PIC_ERR_TIMEOUT : PIC_OK;
}

}  // extern "C"
