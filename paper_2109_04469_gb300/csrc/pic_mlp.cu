// pic_mlp.cu -- the surrogate network of the parameter scans of §3 (the paper has none): a
// 7 -> 256 -> 256 -> 192 MLP with GELU, BF16 weights and activations, FP32 accumulation,
// trained and evaluated by this file's kernels.  Every matrix product runs on the tcgen05
// tensor cores (pic_tc.cuh): operand tiles brought into shared memory by TMA tensor copies in
// the canonical K-major layout through a multi-stage mbarrier ring, the accumulator in tensor
// memory, read back for an FP32 epilogue.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

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
constexpr int kKc = 64;          // K per pipeline stage (four MMA K-steps of 16)
constexpr int kGemmStages = 4;   // stages of the TMA -> MMA ring
constexpr int kGemmThreads = 128;
constexpr int kGemmMaxBn = 256;

// GELU, tanh form: g(z) = z/2 (1 + tanh(c (z + 0.044715 z^3))), c = sqrt(2/pi)
__device__ __forceinline__ float gelu(float z) {
  const float c = 0.7978845608028654f;
  return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float c = 0.7978845608028654f;
  const float t = tanhf(c * (z + 0.044715f * z * z * z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

// What the GEMM does with its FP32 accumulator a = (A B^T)[row, col] (row-major arrays use the
// GEMM's row stride ldc; transposed arrays Ht use ldt):
//   kEpiStore     C[row, col] = a
//   kEpiBias      C[row, col] = a + bias[col], rows < `rows` only (the linear output layer)
//   kEpiBiasGelu  z = a + bias[col]; Z[row, col] = z; H[row, col] = Ht[col, row] = BF16(GELU(z))
//   kEpiGeluGrad  g = a GELU'(Zin[row, col]); C[row, col] = g; H[row, col] (if H) and
//                 Ht[col, row] = BF16(g)
enum { kEpiStore = 0, kEpiBias = 1, kEpiBiasGelu = 2, kEpiGeluGrad = 3 };
struct GemmEpi {
  int mode = kEpiStore;
  int rows = 0;
  int ldt = 0;
  const float* bias = nullptr;
  const float* Zin = nullptr;
  float* Z = nullptr;
  __nv_bfloat16* H = nullptr;
  __nv_bfloat16* Ht = nullptr;
};

// Shared memory of one CTA with B tiles of bn rows: kGemmStages x (A tile + B tile), each tile
// K-major without swizzle as the TMA boxes write it, plus alignment slack.
size_t gemm_smem_bytes(int bn) {
  return (size_t)kGemmStages * (size_t)(kTcM + bn) * kKc * 2 + 1024;
}

// C[M x N] (FP32, row stride ldc) = A[M x K] * B[N x K]^T, A and B BF16 row-major (K
// contiguous), read through the tensor maps ta (box 8 x 128) and tb (box 8 x bn).
// CTA (x, y) owns rows [128 x, 128 x + 128) and columns [bn y, bn y + bn).
//
// Each stage holds K = 64 of both operands as eight TMA boxes of 8 elements (16 bytes) per
// row: box kb lands at kb x rows x 16 bytes, row r at r x 16, so the 8-row x 16-byte core
// matrices are contiguous, row groups 128 bytes apart (SBO) and K-neighbours rows x 16 bytes
// apart (LBO).  Thread 0 fills the stages, thread 32 issues the MMAs and frees each stage by a
// commit to its `empty` barrier; after the last K-step a commit to `done` releases the four
// warps, which read their 32 accumulator lanes back from tensor memory.
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                float* __restrict__ C, int N, int K, int ldc, int bn, int vec4, GemmEpi E,
                int* err) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char* gsm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  const unsigned stA = (unsigned)kTcM * kKc * 2, stB = (unsigned)bn * kKc * 2;
  __shared__ __align__(8) unsigned long long full[kGemmStages], empty[kGemmStages], done;
  __shared__ unsigned tslot;
  __shared__ int issued, consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * bn;
  const unsigned ncols = bn <= 32 ? 32u : (bn <= 64 ? 64u : (bn <= 128 ? 128u : 256u));
  const int nk = (K + kKc - 1) / kKc;
  if (warp == 0) tc_alloc(&tslot, ncols);
  if (tid == 0) {
    for (int s = 0; s < kGemmStages; ++s) {
      mbar_init(&full[s], 1u);
      mbar_init(&empty[s], 1u);
    }
    mbar_init(&done, 1u);
    fence_mbar_init();
    issued = 0;
    consumed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = tslot;
  if (tid == 0) {  // producer
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kGemmStages;
      if (kc >= kGemmStages && !mbar_wait(&empty[s], (unsigned)(kc / kGemmStages - 1) & 1u)) {
        atomicOr(err, 1);
        break;
      }
      const int k0 = kc * kKc, nkb = min(8, (K - k0) / 8);
      unsigned char* a = gsm + (size_t)s * (stA + stB);
      unsigned char* b = a + stA;
      mbar_arrive_expect_tx(&full[s], (unsigned)nkb * 16u * (unsigned)(kTcM + bn));
      for (int kb = 0; kb < nkb; ++kb) {
        tma_load_2d(a + kb * kTcM * 16, &ta, k0 + 8 * kb, m0, &full[s]);
        tma_load_2d(b + kb * bn * 16, &tb, k0 + 8 * kb, n0, &full[s]);
      }
      issued = kc + 1;
    }
  } else if (tid == 32) {  // MMA issuer
    const unsigned idesc = tc_idesc_bf16(kTcM, bn);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % kGemmStages;
      if (!mbar_wait(&full[s], (unsigned)(kc / kGemmStages) & 1u)) {
        atomicOr(err, 1);
        break;
      }
      tc_fence_after();
      const int nks = min(8, (K - kc * kKc) / 8) / 2;
      const unsigned char* a = gsm + (size_t)s * (stA + stB);
      const unsigned char* b = a + stA;
      for (int ks = 0; ks < nks; ++ks)
        tc_mma_bf16(taddr, tc_smem_desc(a + ks * 2 * kTcM * 16, kTcM * 16, 128),
                    tc_smem_desc(b + ks * 2 * bn * 16, bn * 16, 128), idesc, kc > 0 || ks > 0);
      tc_commit(&empty[s]);
      consumed = kc + 1;
    }
    tc_commit(&done);
  }
  __syncwarp();
  if (!mbar_wait(&done, 0u)) {
    if (lane == 0) atomicOr(err, 1);
  }
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  for (int c = 0; c < bn && n0 + c < N; c += 16) {
    float v[16];
    tc_ld16(taddr + ((unsigned)(warp * 32) << 16) + (unsigned)c, v);
    const size_t rb = (size_t)row * ldc + n0 + c;
    const int col = n0 + c;
    if (E.mode == kEpiStore) {
      if (vec4) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(C + rb + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) C[rb + j] = v[j];
      }
    } else if (E.mode == kEpiBias) {
      if (row < E.rows)
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(C + rb + j) =
              make_float4(v[j] + E.bias[col + j], v[j + 1] + E.bias[col + j + 1],
                          v[j + 2] + E.bias[col + j + 2], v[j + 3] + E.bias[col + j + 3]);
    } else {
      // row-major outputs as 16-byte stores of this thread's 16 columns; the transposed copy
      // column by column (lanes hold consecutive rows, so each store is coalesced)
      float o[16];
      __align__(16) __nv_bfloat16 h[16];
      if (E.mode == kEpiBiasGelu) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          o[j] = v[j] + E.bias[col + j];
          h[j] = __float2bfloat16_rn(gelu(o[j]));
        }
      } else {
        float z[16];
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(z + j) = *reinterpret_cast<const float4*>(E.Zin + rb + j);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          o[j] = v[j] * gelu_grad(z[j]);
          h[j] = __float2bfloat16_rn(o[j]);
        }
      }
      float* fo = E.mode == kEpiBiasGelu ? E.Z : C;
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(fo + rb + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
      if (E.H) {
        uint4* hd = reinterpret_cast<uint4*>(E.H + rb);
        hd[0] = *reinterpret_cast<const uint4*>(h);
        hd[1] = *reinterpret_cast<const uint4*>(h + 8);
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) E.Ht[(size_t)(col + j) * E.ldt + row] = h[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0)  // copies issued but never consumed (a timed-out MMA wait) land before exit
    for (int kc = consumed; kc < issued; ++kc)
      (void)mbar_wait(&full[kc % kGemmStages], (unsigned)(kc / kGemmStages) & 1u);
  __syncthreads();
  if (warp == 0) tc_dealloc(taddr, ncols);
}

bool gemm_shape_ok(int M, int N, int K) {
  return M > 0 && M % kTcM == 0 && N >= 16 && N <= 4096 && N % 16 == 0 && K >= 16 &&
         K % 16 == 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no libcuda link).
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows x K] (K contiguous) read in boxes of 8 x box_rows.
bool make_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int box_rows) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Width of the column tiles: the whole of N (up to 256) unless halving it still leaves
// columns of at least 32 and the grid has fewer than 64 CTAs.
int gemm_bn(int M, int N) {
  auto up16 = [](int v) { return (v + 15) & ~15; };
  int bn = std::min(up16(N), kGemmMaxBn);
  while (bn > 32 && (M / kTcM) * ((N + bn - 1) / bn) < 64) bn = up16(bn / 2);
  return bn;
}

// cudaErrorInvalidValue when an operand is not 16-byte aligned (the tensor maps need it)
cudaError_t launch_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                        int K, int ldc, int* err, cudaStream_t s, const GemmEpi& epi = GemmEpi()) {
  // room for the widest B tile whatever the launch, so no stage can reach past the allocation
  static const cudaError_t configured = cudaFuncSetAttribute(
      k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)gemm_smem_bytes(kGemmMaxBn));
  if (configured != cudaSuccess) return configured;
  const int bn = gemm_bn(M, N);
  CUtensorMap ta, tb;
  if (!make_map(&ta, A, M, K, kTcM) || !make_map(&tb, B, N, K, bn)) return cudaErrorInvalidValue;
  const int vec4 = (ldc % 4 == 0 && (reinterpret_cast<uintptr_t>(C) & 15u) == 0) ? 1 : 0;
  // the fused epilogues store 16-byte vectors: row strides of 4 floats, aligned arrays
  if (epi.mode != kEpiStore) {
    const uintptr_t al = reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(epi.Z) |
                         reinterpret_cast<uintptr_t>(epi.Zin) | reinterpret_cast<uintptr_t>(epi.H);
    if (ldc % 8 != 0 || (al & 15u) != 0) return cudaErrorInvalidValue;
  }
  const dim3 grid((unsigned)(M / kTcM), (unsigned)((N + bn - 1) / bn));
  k_gemm_bf16<<<grid, kGemmThreads, gemm_smem_bytes(bn), s>>>(ta, tb, C, N, K, ldc, bn, vec4,
                                                              epi, err);
  return cudaGetLastError();
}

// ----------------------------------------------------------------- the network's kernels
constexpr int kIn = 7, kInP = 16, kHid = 256, kOut = 192;
constexpr int kNParams = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;

// x [B x 7] FP32 (rows >= n zero) -> X [Bp x 16] BF16 and its transpose [16 x Bp]
__global__ void k_pack_input(const float* __restrict__ x, int n, int Bp, __nv_bfloat16* X,
                             __nv_bfloat16* Xt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * kInP) return;
  const int b = i / kInP, k = i - b * kInP;
  const float v = (b < n && k < kIn) ? x[(size_t)b * kIn + k] : 0.0f;
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  X[i] = h;
  Xt[(size_t)k * Bp + b] = h;
}

// Mean-squared error over B x N and its gradient dY = 2 (Y - T) / (B N): FP32, BF16 row-major
// and transposed.  Per-row partial losses go to rowloss[b] (summed on the host in order).
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, int B, int N,
                       float* dY, __nv_bfloat16* dYh, __nv_bfloat16* dYt, double* rowloss) {
  const int b = blockIdx.x;
  double acc = 0.0;
  const float s = 2.0f / ((float)B * (float)N);
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const size_t i = (size_t)b * N + j;
    const float d = Y[i] - T[i];
    acc += (double)d * (double)d;
    const float g = s * d;
    dY[i] = g;
    const __nv_bfloat16 h = __float2bfloat16_rn(g);
    dYh[i] = h;
    dYt[(size_t)j * B + b] = h;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) rowloss[b] = red[0];
}

// Column sums (bias gradients), one thread per column, rows in order (deterministic)
__global__ void k_colsum(const float* __restrict__ G, int B, int N, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.0f;
  for (int b = 0; b < B; ++b) s += G[(size_t)b * N + j];
  out[j] = s;
}

// Adam on one FP32 parameter array W[rows x cols] (row-major) with gradient G, given either
// row-major (gt == 0: G[r * ldg + c]) or transposed (gt == 1: G[c * ldg + r]); then the BF16 copies:
// Wh [rows x ldh] (columns >= cols zero-padded) and, if given, Wt = W^T [cols x rows].
__global__ void k_adam(float* W, const float* __restrict__ G, int gt, int ldg, float* m,
                       float* v, int rows, int cols, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16* Wh, int ldh, __nv_bfloat16* Wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i - r * cols;
  const float g = gt ? G[(size_t)c * ldg + r] : G[(size_t)r * ldg + c];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float w = W[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  W[i] = w;
  const __nv_bfloat16 h = __float2bfloat16_rn(w);
  if (Wh) Wh[(size_t)r * ldh + c] = h;
  if (Wt) Wt[(size_t)c * rows + r] = h;
}

// BF16 copies of a parameter array (after initialisation or a host upload)
__global__ void k_to_bf16(const float* __restrict__ W, int rows, int cols, __nv_bfloat16* Wh,
                          int ldh, __nv_bfloat16* Wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i - r * cols;
  const __nv_bfloat16 h = __float2bfloat16_rn(W[i]);
  Wh[(size_t)r * ldh + c] = h;
  if (Wt) Wt[(size_t)c * rows + r] = h;
}

__device__ int g_gemm_err;  // timeout flag of the stand-alone GEMM entry point

// Offsets of the flat parameter vector: W1 [256 x 7], b1, W2 [256 x 256], b2, W3 [192 x 256], b3
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid,
              kOffB3 = kOffW3 + kOut * kHid;
static_assert(kOffB3 + kOut == kNParams, "parameter layout");

struct MlpCarver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* r = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return r;
  }
};

}  // namespace
}  // namespace pic

struct pic_mlp {
  int bmax = 0;
  cudaStream_t stream = nullptr;
  long long t = 0;  // Adam steps taken
  float *P, *M, *V;  // parameters and Adam moments, flat layout
  __nv_bfloat16 *W1h, *W2h, *W2t, *W3h, *W3t;
  __nv_bfloat16 *Xh, *Xt, *H1h, *H1t, *H2h, *H2t, *dYh, *dYt, *dZh, *dZt;
  float *Z1, *Z2, *Y, *dY, *dZ, *dZ1, *gW1, *gW2t, *gW3t, *gb1, *gb2, *gb3;
  int last_n = 0;        // rows of the last forward pass
  int last_backward = 0; // 1 if the last call also ran the backward pass
  double* rowloss;
  int* err;
};

namespace pic {
namespace {

void mlp_carve(pic_mlp* m, char* base, int bmax, size_t* total) {
  MlpCarver c{base};
  const size_t B = (size_t)bmax;
  m->P = c.take<float>(kNParams);
  m->M = c.take<float>(kNParams);
  m->V = c.take<float>(kNParams);
  m->W1h = c.take<__nv_bfloat16>((size_t)kHid * kInP);
  m->W2h = c.take<__nv_bfloat16>((size_t)kHid * kHid);
  m->W2t = c.take<__nv_bfloat16>((size_t)kHid * kHid);
  m->W3h = c.take<__nv_bfloat16>((size_t)kOut * kHid);
  m->W3t = c.take<__nv_bfloat16>((size_t)kHid * kOut);
  m->Xh = c.take<__nv_bfloat16>(B * kInP);
  m->Xt = c.take<__nv_bfloat16>(B * kInP);
  m->H1h = c.take<__nv_bfloat16>(B * kHid);
  m->H1t = c.take<__nv_bfloat16>(B * kHid);
  m->H2h = c.take<__nv_bfloat16>(B * kHid);
  m->H2t = c.take<__nv_bfloat16>(B * kHid);
  m->dYh = c.take<__nv_bfloat16>(B * kOut);
  m->dYt = c.take<__nv_bfloat16>(B * kOut);
  m->dZh = c.take<__nv_bfloat16>(B * kHid);
  m->dZt = c.take<__nv_bfloat16>(B * kHid);
  m->Z1 = c.take<float>(B * kHid);
  m->Z2 = c.take<float>(B * kHid);
  m->Y = c.take<float>(B * kOut);
  m->dY = c.take<float>(B * kOut);
  m->dZ = c.take<float>(B * kHid);
  m->dZ1 = c.take<float>(B * kHid);
  m->gW1 = c.take<float>((size_t)kHid * kInP);
  m->gW2t = c.take<float>((size_t)kHid * kHid);
  m->gW3t = c.take<float>((size_t)kHid * kOut);
  m->gb1 = c.take<float>(kHid);
  m->gb2 = c.take<float>(kHid);
  m->gb3 = c.take<float>(kOut);
  m->rowloss = c.take<double>(B);
  m->err = c.take<int>(1);
  *total = (c.off + 255) & ~size_t(255);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// BF16 copies of the weights from the FP32 parameters
cudaError_t mlp_refresh_bf16(pic_mlp* m) {
  cudaStream_t s = m->stream;
  cudaMemsetAsync(m->W1h, 0, sizeof(__nv_bfloat16) * kHid * kInP, s);
  k_to_bf16<<<blocks(kHid * kIn), 256, 0, s>>>(m->P + kOffW1, kHid, kIn, m->W1h, kInP, nullptr);
  k_to_bf16<<<blocks(kHid * kHid), 256, 0, s>>>(m->P + kOffW2, kHid, kHid, m->W2h, kHid, m->W2t);
  k_to_bf16<<<blocks(kOut * kHid), 256, 0, s>>>(m->P + kOffW3, kOut, kHid, m->W3h, kHid, m->W3t);
  return cudaGetLastError();
}

// Forward pass of n inputs x [n x 7] (device) into m->Y [n x 192]; Bp = n rounded up to 128.
// Bias and GELU run in the GEMM epilogues.
cudaError_t mlp_forward(pic_mlp* m, const float* x, int n, int Bp) {
  cudaStream_t s = m->stream;
  k_pack_input<<<blocks((long long)Bp * kInP), 256, 0, s>>>(x, n, Bp, m->Xh, m->Xt);
  GemmEpi h1;
  h1.mode = kEpiBiasGelu;
  h1.ldt = Bp;
  h1.bias = m->P + kOffB1;
  h1.Z = m->Z1;
  h1.H = m->H1h;
  h1.Ht = m->H1t;
  cudaError_t e = launch_gemm(m->Xh, m->W1h, nullptr, Bp, kHid, kInP, kHid, m->err, s, h1);
  if (e != cudaSuccess) return e;
  GemmEpi h2 = h1;
  h2.bias = m->P + kOffB2;
  h2.Z = m->Z2;
  h2.H = m->H2h;
  h2.Ht = m->H2t;
  e = launch_gemm(m->H1h, m->W2h, nullptr, Bp, kHid, kHid, kHid, m->err, s, h2);
  if (e != cudaSuccess) return e;
  GemmEpi out;
  out.mode = kEpiBias;
  out.rows = n;
  out.bias = m->P + kOffB3;
  return launch_gemm(m->H2h, m->W3h, m->Y, Bp, kOut, kHid, kOut, m->err, s, out);
}

// Loss and gradients of a batch of B (a multiple of 128) after mlp_forward(x, B, B); the
// GELU derivative runs in the epilogues of the dH products.
cudaError_t mlp_backward(pic_mlp* m, const float* t, int B) {
  cudaStream_t s = m->stream;
  k_loss<<<B, 256, 0, s>>>(m->Y, t, B, kOut, m->dY, m->dYh, m->dYt, m->rowloss);
  // dW3^T [256 x 192] = H2^T dY
  cudaError_t e = launch_gemm(m->H2t, m->dYt, m->gW3t, kHid, kOut, B, kOut, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kOut, 0, s>>>(m->dY, B, kOut, m->gb3);
  // dZ2 = (dY W3) GELU'(Z2)
  GemmEpi g2;
  g2.mode = kEpiGeluGrad;
  g2.ldt = B;
  g2.Zin = m->Z2;
  g2.H = m->dZh;
  g2.Ht = m->dZt;
  e = launch_gemm(m->dYh, m->W3t, m->dZ, B, kHid, kOut, kHid, m->err, s, g2);
  if (e != cudaSuccess) return e;
  // dW2^T = H1^T dZ2
  e = launch_gemm(m->H1t, m->dZt, m->gW2t, kHid, kHid, B, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kHid, 0, s>>>(m->dZ, B, kHid, m->gb2);
  // dZ1 = (dZ2 W2) GELU'(Z1), FP32 into its own buffer (dZ2 stays readable)
  GemmEpi g1 = g2;
  g1.Zin = m->Z1;
  g1.H = nullptr;
  e = launch_gemm(m->dZh, m->W2t, m->dZ1, B, kHid, kHid, kHid, m->err, s, g1);
  if (e != cudaSuccess) return e;
  // dW1 [256 x 16] = dZ1^T X
  e = launch_gemm(m->dZt, m->Xt, m->gW1, kHid, kInP, B, kInP, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kHid, 0, s>>>(m->dZ1, B, kHid, m->gb1);
  return cudaGetLastError();
}

// Loss of the last backward pass (synchronises) and the GEMM timeout flag
int mlp_loss(pic_mlp* m, int B, float* loss) {
  std::vector<double> r((size_t)B);
  int err = 0;
  if (cudaMemcpyAsync(r.data(), m->rowloss, sizeof(double) * B, cudaMemcpyDeviceToHost,
                      m->stream) != cudaSuccess ||
      cudaMemcpyAsync(&err, m->err, sizeof err, cudaMemcpyDeviceToHost, m->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  double sum = 0.0;
  for (double v : r) sum += v;
  if (loss) *loss = (float)(sum / ((double)B * kOut));
  return err ? PIC_ERR_TIMEOUT : PIC_OK;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" {

int pic_tc_gemm_bf16(const uint16_t* a, const uint16_t* b, float* c, int32_t m, int32_t n,
                     int32_t k, void* cuda_stream) {
  if (!a || !b || !c || !gemm_shape_ok(m, n, k)) return PIC_ERR_PARAM;
  if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) != 0)
    return PIC_ERR_PARAM;
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


int pic_mlp_workspace_bytes(int32_t batch_max, size_t* bytes) {
  if (batch_max < 128 || batch_max % 128 || !bytes) return PIC_ERR_PARAM;
  pic_mlp m;
  mlp_carve(&m, nullptr, batch_max, bytes);
  return PIC_OK;
}

int pic_mlp_init(int32_t batch_max, uint64_t seed, void* workspace, size_t workspace_bytes,
                 void* cuda_stream, pic_mlp** out) {
  if (!out) return PIC_ERR_PARAM;
  *out = nullptr;
  size_t need = 0;
  if (pic_mlp_workspace_bytes(batch_max, &need) != PIC_OK) return PIC_ERR_PARAM;
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return PIC_ERR_WORKSPACE;
  pic_mlp* m = new (std::nothrow) pic_mlp;
  if (!m) return PIC_ERR_PARAM;
  m->bmax = batch_max;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  size_t total = 0;
  mlp_carve(m, static_cast<char*>(workspace), batch_max, &total);
  // uniform initialisation with bound sqrt(6 / (fan_in + fan_out)), biases zero; a
  // splitmix64 stream of the seed (host set-up only)
  std::vector<float> P((size_t)kNParams, 0.0f);
  unsigned long long z = seed;
  auto next_u = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    unsigned long long x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return ((double)(x >> 11) + 0.5) * 0x1p-53;
  };
  auto fill = [&](int off, int rows, int cols) {
    const double a = std::sqrt(6.0 / (double)(rows + cols));
    for (int i = 0; i < rows * cols; ++i) P[(size_t)off + i] = (float)((2.0 * next_u() - 1.0) * a);
  };
  fill(kOffW1, kHid, kIn);
  fill(kOffW2, kHid, kHid);
  fill(kOffW3, kOut, kHid);
  cudaStream_t s = m->stream;
  if (cudaMemsetAsync(workspace, 0, total, s) != cudaSuccess ||
      cudaMemcpyAsync(m->P, P.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      mlp_refresh_bf16(m) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    delete m;
    return PIC_ERR_CUDA;
  }
  *out = m;
  return PIC_OK;
}

int pic_mlp_num_params(void) { return kNParams; }

int pic_mlp_get_params(pic_mlp* m, float* params) {
  if (!m || !params) return PIC_ERR_PARAM;
  if (cudaMemcpyAsync(params, m->P, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                      m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  return PIC_OK;
}

int pic_mlp_set_params(pic_mlp* m, const float* params) {
  if (!m || !params) return PIC_ERR_PARAM;
  if (cudaMemcpyAsync(m->P, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice,
                      m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->M, 0, sizeof(float) * kNParams, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->V, 0, sizeof(float) * kNParams, m->stream) != cudaSuccess ||
      mlp_refresh_bf16(m) != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  m->t = 0;
  return PIC_OK;
}

int pic_mlp_forward(pic_mlp* m, const float* x, int32_t n, float* y) {
  if (!m || !x || !y || n < 1 || n > m->bmax) return PIC_ERR_PARAM;
  const int Bp = (n + 127) / 128 * 128;
  m->last_n = n;
  m->last_backward = 0;
  if (mlp_forward(m, x, n, Bp) != cudaSuccess ||
      cudaMemcpyAsync(y, m->Y, sizeof(float) * (size_t)n * kOut, cudaMemcpyDeviceToDevice,
                      m->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  return PIC_OK;
}

int pic_mlp_gradients(pic_mlp* m, const float* x, const float* t, int32_t n, float* grads,
                      float* loss) {
  if (!m || !x || !t || !grads || n < 128 || n % 128 || n > m->bmax) return PIC_ERR_PARAM;
  m->last_n = n;
  m->last_backward = 1;
  if (mlp_forward(m, x, n, n) != cudaSuccess || mlp_backward(m, t, n) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  const int rc = mlp_loss(m, n, loss);
  if (rc != PIC_OK) return rc;
  std::vector<float> g1((size_t)kHid * kInP), g2((size_t)kHid * kHid), g3((size_t)kHid * kOut);
  cudaStream_t s = m->stream;
  if (cudaMemcpyAsync(g1.data(), m->gW1, sizeof(float) * g1.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(g2.data(), m->gW2t, sizeof(float) * g2.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(g3.data(), m->gW3t, sizeof(float) * g3.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(grads + kOffB1, m->gb1, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(grads + kOffB2, m->gb2, sizeof(float) * kHid, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(grads + kOffB3, m->gb3, sizeof(float) * kOut, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  for (int r = 0; r < kHid; ++r)
    for (int c = 0; c < kIn; ++c) grads[kOffW1 + r * kIn + c] = g1[(size_t)r * kInP + c];
  for (int r = 0; r < kHid; ++r)
    for (int c = 0; c < kHid; ++c) grads[kOffW2 + r * kHid + c] = g2[(size_t)c * kHid + r];
  for (int r = 0; r < kOut; ++r)
    for (int c = 0; c < kHid; ++c) grads[kOffW3 + r * kHid + c] = g3[(size_t)c * kOut + r];
  return PIC_OK;
}

int pic_mlp_train_step(pic_mlp* m, const float* x, const float* t, int32_t n, float lr,
                       float* loss) {
  if (!m || !x || !t || n < 128 || n % 128 || n > m->bmax || !(lr > 0.0f)) return PIC_ERR_PARAM;
  m->last_n = n;
  m->last_backward = 1;
  if (mlp_forward(m, x, n, n) != cudaSuccess || mlp_backward(m, t, n) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)m->t));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)m->t));
  cudaStream_t s = m->stream;
  float* P = m->P;
  k_adam<<<blocks(kHid * kIn), 256, 0, s>>>(P + kOffW1, m->gW1, 0, kInP, m->M + kOffW1,
                                            m->V + kOffW1, kHid, kIn, lr, b1, b2, eps, c1, c2,
                                            m->W1h, kInP, nullptr);
  k_adam<<<blocks(kHid), 256, 0, s>>>(P + kOffB1, m->gb1, 0, kHid, m->M + kOffB1, m->V + kOffB1,
                                      1, kHid, lr, b1, b2, eps, c1, c2, nullptr, 0, nullptr);
  k_adam<<<blocks(kHid * kHid), 256, 0, s>>>(P + kOffW2, m->gW2t, 1, kHid, m->M + kOffW2,
                                             m->V + kOffW2, kHid, kHid, lr, b1, b2, eps, c1, c2,
                                             m->W2h, kHid, m->W2t);
  k_adam<<<blocks(kHid), 256, 0, s>>>(P + kOffB2, m->gb2, 0, kHid, m->M + kOffB2, m->V + kOffB2,
                                      1, kHid, lr, b1, b2, eps, c1, c2, nullptr, 0, nullptr);
  k_adam<<<blocks(kOut * kHid), 256, 0, s>>>(P + kOffW3, m->gW3t, 1, kOut, m->M + kOffW3,
                                             m->V + kOffW3, kOut, kHid, lr, b1, b2, eps, c1, c2,
                                             m->W3h, kHid, m->W3t);
  k_adam<<<blocks(kOut), 256, 0, s>>>(P + kOffB3, m->gb3, 0, kOut, m->M + kOffB3, m->V + kOffB3,
                                      1, kOut, lr, b1, b2, eps, c1, c2, nullptr, 0, nullptr);
  if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
  return loss ? mlp_loss(m, n, loss) : PIC_OK;
}

int pic_mlp_get_activations(pic_mlp* m, int32_t which, int32_t n, void* host) {
  if (!m || !host || which < 0 || which > PIC_MLP_ACT_DZ1H || n < 1 || n > m->last_n)
    return PIC_ERR_PARAM;
  if (which >= PIC_MLP_ACT_DY && !m->last_backward) return PIC_ERR_PARAM;
  const void* src = nullptr;
  size_t elem = 4, cols = kHid;
  switch (which) {
    case PIC_MLP_ACT_X: src = m->Xh; elem = 2; cols = kInP; break;
    case PIC_MLP_ACT_Z1: src = m->Z1; break;
    case PIC_MLP_ACT_H1: src = m->H1h; elem = 2; break;
    case PIC_MLP_ACT_Z2: src = m->Z2; break;
    case PIC_MLP_ACT_H2: src = m->H2h; elem = 2; break;
    case PIC_MLP_ACT_Y: src = m->Y; cols = kOut; break;
    case PIC_MLP_ACT_DY: src = m->dY; cols = kOut; break;
    case PIC_MLP_ACT_DYH: src = m->dYh; elem = 2; cols = kOut; break;
    case PIC_MLP_ACT_DZ2: src = m->dZ; break;
    case PIC_MLP_ACT_DZ2H: src = m->dZh; elem = 2; break;
    case PIC_MLP_ACT_DZ1: src = m->dZ1; break;
    default: break;  // PIC_MLP_ACT_DZ1H: kept transposed [256][n] for the dW1 product
  }
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  if (src) {
    if (cudaMemcpy(host, src, elem * cols * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) {
      (void)cudaGetLastError();
      return PIC_ERR_CUDA;
    }
    return PIC_OK;
  }
  const int ldt = m->last_n;  // the backward pass ran on exactly last_n rows
  std::vector<uint16_t> t((size_t)kHid * ldt);
  if (cudaMemcpy(t.data(), m->dZt, sizeof(uint16_t) * t.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return PIC_ERR_CUDA;
  }
  uint16_t* out = static_cast<uint16_t*>(host);
  for (int b = 0; b < n; ++b)
    for (int j = 0; j < kHid; ++j) out[(size_t)b * kHid + j] = t[(size_t)j * ldt + b];
  return PIC_OK;
}

void pic_mlp_free(pic_mlp* m) { delete m; }

}  // extern "C"
