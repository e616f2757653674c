// pic_field_solve_static: the field solve of §2 step 2 (exact discrete Green's function,
// reading C-23) on caller-owned device arrays, for callers that must not allocate device
// memory at all -- a process whose caching allocator has reserved the device's free memory,
// a latency-critical path that must not call cudaMalloc / cudaFree (they can synchronise the
// device), or a plug-in that is handed device pointers but no allocator or workspace.
//
// Its one scratch array (the integer sums S_j of the Green's function, one per node) lives in
// a file-scope __device__ array of fixed size instead of shared memory or a workspace, so
// grids larger than the shared-memory field solve of the simulation handle can be solved.
// The arithmetic is the FP64 simulation's field solve: exact int128 sums, then the same
// rounded FP64 operations in the same order, so phi and E agree bit for bit with
// pic_solve_field of a PIC_FP64 handle for the same charge and drive voltage (a PIC_FP32
// handle multiplies by rounded reciprocals instead of dividing: within one ulp).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "pic.h"
#include "pic_common.cuh"

namespace {

constexpr int kStaticNodes = PIC_FIELD_STATIC_MAX_CELLS + 1;
constexpr int kStaticThreads = 1024;
constexpr int kMaxDevices = 64;

// S_j of the Green's-function solve for one grid of up to kStaticNodes nodes (1 MiB).
// Every element the kernel reads is written earlier in the same launch: nothing has to start
// at zero, and nothing is left for the next call.
static __device__ __align__(256) __int128 g_field_scratch[kStaticNodes];

// Same constants as the simulation's host set-up (CODATA 2018, §2).
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kTwo32 = 4294967296.0;

struct StaticField {
  const long long* Ce;
  const long long* Ci;
  double* phi;
  double* E;
  __int128* Sg;
  int N;
  double V, rfac, den1, den2;
};

// One block: per-thread segments of the nodes, a block-wide int128 scan of
// sum j dc_j and sum (N-j) dc_j, then S_j = (N-j) sum_{k<=j} k dc_k + j sum_{k>j} (N-k) dc_k.
__global__ void __launch_bounds__(kStaticThreads, 1) k_field_static(StaticField F) {
  const int N = F.N, nx = N + 1;
  const int seg = (nx + blockDim.x - 1) / blockDim.x;
  const int j0 = min((int)threadIdx.x * seg, nx), j1 = min(j0 + seg, nx);
  __int128 sa = 0, sb = 0;
  for (int j = j0; j < j1; ++j)
    if (j >= 1 && j <= N - 1) {
      const long long dc = F.Ci[j] - F.Ce[j];
      sa += (__int128)j * dc;
      sb += (__int128)(N - j) * dc;
    }
  __int128 tb;
  pic::block_scan_i128x2(sa, sb, tb);
  for (int j = j0; j < j1; ++j) {
    if (j >= 1 && j <= N - 1) {
      const long long dc = F.Ci[j] - F.Ce[j];
      sa += (__int128)j * dc;
      sb += (__int128)(N - j) * dc;
    }
    F.Sg[j] = (__int128)(N - j) * sa + (__int128)j * (tb - sb);
  }
  __syncthreads();  // the block's global writes of Sg are visible to all its threads
  const __int128* Sg = F.Sg;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    double e, ph;
    if (j == 0) {
      const __int128 q = Sg[1] + (__int128)N * (__int128)(F.Ci[0] - F.Ce[0]);
      e = __ddiv_rn(__dsub_rn(F.V, __dmul_rn(F.rfac, pic::i128_to_f64(q))), F.den1);
      ph = F.V;
    } else if (j == N) {
      const __int128 q = Sg[N - 1] + (__int128)N * (__int128)(F.Ci[N] - F.Ce[N]);
      e = __ddiv_rn(__dadd_rn(F.V, __dmul_rn(F.rfac, pic::i128_to_f64(q))), F.den1);
      ph = 0.0;
    } else {
      e = __ddiv_rn(__dadd_rn(__dmul_rn(2.0, F.V), __dmul_rn(F.rfac, pic::i128_to_f64(Sg[j - 1] - Sg[j + 1]))),
                    F.den2);
      ph = __ddiv_rn(__dadd_rn(__dmul_rn(F.V, (double)(N - j)), __dmul_rn(F.rfac, pic::i128_to_f64(Sg[j]))),
                     (double)N);
    }
    F.E[j] = e;
    F.phi[j] = ph;
  }
}

std::mutex g_scratch_mutex;
__int128* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_field_scratch on the current device, looked up once per device (with
// that device current) and cached for the life of the process; a cudaDeviceReset invalidates
// it, which the header tells callers.
cudaError_t scratch_address(__int128** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_field_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<__int128*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Device-accessible pointer on the current device, 8-byte aligned.
bool device_array(const void* p, int dev) {
  if (p == nullptr || (reinterpret_cast<uintptr_t>(p) & 7u) != 0) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

int pic_field_solve_static(const int64_t* charge_e, const int64_t* charge_i, int32_t n_cells,
                           double gap_m, double weight, double area_m2, double v_left,
                           double* phi, double* efield, void* cuda_stream) {
  if (n_cells > PIC_FIELD_STATIC_MAX_CELLS) return PIC_ERR_SCRATCH;
  if (n_cells < 2 || !(gap_m > 0.0) || !(weight > 0.0) || !(area_m2 > 0.0) ||
      !std::isfinite(gap_m) || !std::isfinite(weight) || !std::isfinite(area_m2) ||
      !std::isfinite(v_left))
    return PIC_ERR_PARAM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ERR_CUDA;
  if (!device_array(charge_e, dev) || !device_array(charge_i, dev) || !device_array(phi, dev) ||
      !device_array(efield, dev))
    return PIC_ERR_PARAM;
  __int128* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return PIC_ERR_CUDA;
  // derived constants exactly as the simulation handle derives them (§2, reading C-23)
  const double dx = gap_m / (double)n_cells;
  const double efac = (kQe * weight) / ((area_m2 * kEps0) * kTwo32);
  StaticField F;
  F.Ce = reinterpret_cast<const long long*>(charge_e);
  F.Ci = reinterpret_cast<const long long*>(charge_i);
  F.phi = phi;
  F.E = efield;
  F.Sg = scratch;
  F.N = n_cells;
  F.V = v_left;
  F.rfac = efac * dx;
  F.den1 = dx * (double)n_cells;
  F.den2 = (2.0 * dx) * (double)n_cells;
  k_field_static<<<1, kStaticThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(F);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

}  // extern "C"
