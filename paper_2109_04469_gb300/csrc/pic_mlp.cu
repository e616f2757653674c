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

// ----------------------------------------------------------------- the network's kernels
constexpr int kIn = 7, kInP = 16, kHid = 256, kOut = 192;
constexpr int kNParams = kHid * kIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;

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

// Z = C + bias; H = GELU(Z) as BF16, row-major and transposed ([N x Bp]); Z kept for backward
__global__ void k_bias_gelu(const float* __restrict__ Cm, const float* __restrict__ bias, int Bp,
                            int N, float* Z, __nv_bfloat16* H, __nv_bfloat16* Ht) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bp * N) return;
  const int b = i / N, j = i - b * N;
  const float z = Cm[i] + bias[j];
  if (Z) Z[i] = z;
  const __nv_bfloat16 h = __float2bfloat16_rn(gelu(z));
  H[i] = h;
  if (Ht) Ht[(size_t)j * Bp + b] = h;
}

// Y = C + bias (the linear output layer)
__global__ void k_bias_out(const float* __restrict__ Cm, const float* __restrict__ bias, int n,
                           int N, float* Y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * N) return;
  Y[i] = Cm[i] + bias[i % N];
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

// dZ = dH * GELU'(Z): FP32 (for the bias gradient), BF16 row-major and transposed
__global__ void k_gelu_back(const float* __restrict__ dH, const float* __restrict__ Z, int B,
                            int N, float* dZ, __nv_bfloat16* dZh, __nv_bfloat16* dZt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  const int b = i / N, j = i - b * N;
  const float g = dH[i] * gelu_grad(Z[i]);
  dZ[i] = g;
  const __nv_bfloat16 h = __float2bfloat16_rn(g);
  if (dZh) dZh[i] = h;
  dZt[(size_t)j * B + b] = h;
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
  float *Cb, *Z1, *Z2, *Y, *dY, *dH, *dZ, *gW1, *gW2t, *gW3t, *gb1, *gb2, *gb3;
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
  m->Cb = c.take<float>(B * kHid);
  m->Z1 = c.take<float>(B * kHid);
  m->Z2 = c.take<float>(B * kHid);
  m->Y = c.take<float>(B * kOut);
  m->dY = c.take<float>(B * kOut);
  m->dH = c.take<float>(B * kHid);
  m->dZ = c.take<float>(B * kHid);
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

// Forward pass of n inputs x [n x 7] (device) into m->Y [n x 192]; Bp = n rounded up to 128
cudaError_t mlp_forward(pic_mlp* m, const float* x, int n, int Bp) {
  cudaStream_t s = m->stream;
  k_pack_input<<<blocks((long long)Bp * kInP), 256, 0, s>>>(x, n, Bp, m->Xh, m->Xt);
  cudaError_t e = launch_gemm(m->Xh, m->W1h, m->Cb, Bp, kHid, kInP, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_bias_gelu<<<blocks((long long)Bp * kHid), 256, 0, s>>>(m->Cb, m->P + kOffB1, Bp, kHid, m->Z1,
                                                          m->H1h, m->H1t);
  e = launch_gemm(m->H1h, m->W2h, m->Cb, Bp, kHid, kHid, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_bias_gelu<<<blocks((long long)Bp * kHid), 256, 0, s>>>(m->Cb, m->P + kOffB2, Bp, kHid, m->Z2,
                                                          m->H2h, m->H2t);
  e = launch_gemm(m->H2h, m->W3h, m->Cb, Bp, kOut, kHid, kOut, m->err, s);
  if (e != cudaSuccess) return e;
  k_bias_out<<<blocks((long long)n * kOut), 256, 0, s>>>(m->Cb, m->P + kOffB3, n, kOut, m->Y);
  return cudaGetLastError();
}

// Loss and gradients of a batch of B (a multiple of 128) after mlp_forward(x, B, B)
cudaError_t mlp_backward(pic_mlp* m, const float* t, int B) {
  cudaStream_t s = m->stream;
  k_loss<<<B, 256, 0, s>>>(m->Y, t, B, kOut, m->dY, m->dYh, m->dYt, m->rowloss);
  // dW3^T [256 x 192] = H2^T dY
  cudaError_t e = launch_gemm(m->H2t, m->dYt, m->gW3t, kHid, kOut, B, kOut, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kOut, 0, s>>>(m->dY, B, kOut, m->gb3);
  // dH2 = dY W3
  e = launch_gemm(m->dYh, m->W3t, m->dH, B, kHid, kOut, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_gelu_back<<<blocks((long long)B * kHid), 256, 0, s>>>(m->dH, m->Z2, B, kHid, m->dZ, m->dZh,
                                                         m->dZt);
  // dW2^T = H1^T dZ2
  e = launch_gemm(m->H1t, m->dZt, m->gW2t, kHid, kHid, B, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kHid, 0, s>>>(m->dZ, B, kHid, m->gb2);
  // dH1 = dZ2 W2
  e = launch_gemm(m->dZh, m->W2t, m->dH, B, kHid, kHid, kHid, m->err, s);
  if (e != cudaSuccess) return e;
  k_gelu_back<<<blocks((long long)B * kHid), 256, 0, s>>>(m->dH, m->Z1, B, kHid, m->dZ, nullptr,
                                                         m->dZt);
  // dW1 [256 x 16] = dZ1^T X
  e = launch_gemm(m->dZt, m->Xt, m->gW1, kHid, kInP, B, kInP, m->err, s);
  if (e != cudaSuccess) return e;
  k_colsum<<<1, kHid, 0, s>>>(m->dZ, B, kHid, m->gb1);
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

void pic_mlp_free(pic_mlp* m) { delete m; }

}  // extern "C"
