// pic_common.cuh -- precision-independent device code of libpic: block scans, the exact field
// solve of §2 step 2 (reading C-23), the hole / birth bookkeeping of the compaction (reading
// C-15) and the placement launch.  Included by the FP64 and FP32 translation units; the FP64
// arithmetic here uses explicit round-to-nearest intrinsics so no compiler flag can contract
// it into fused multiply-adds.
#pragma once
#include <cuda_runtime.h>

#include "pic_dev.cuh"

namespace pic {

// Programmatic dependent launch between the step's two launches (and into the next step):
// a kernel launched with launch_chained may be scheduled while the previous kernel of the
// stream still runs, once every block of that kernel has called chain_release();
// chain_wait() then returns when the previous kernel has completed and its writes are
// visible.  Nothing written by an earlier kernel may be read before chain_wait().  In a
// kernel launched the ordinary way both are no-ops.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Raise (never lower) a kernel's dynamic shared-memory limit: handles with different grids
// share the kernel, and a limit set for a smaller grid must not break a larger one.
template <typename... Args>
cudaError_t raise_smem_limit(void (*kernel)(Args...), size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename... Args>
cudaError_t launch_chained(void (*kernel)(Args...), unsigned grid, unsigned block, size_t smem,
                           cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int NW>
__device__ __forceinline__ int block_excl_scan(int v, int* sWarp, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sWarp[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int t = (lane < NW) ? sWarp[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < NW) sWarp[lane] = ti - t;
    if (lane == NW - 1) sWarp[NW] = ti;
  }
  __syncthreads();
  total = sWarp[NW];
  const int r = sWarp[w] + inc - v;
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------- field (§2 step 2)
// Round-to-nearest-even conversion of a 128-bit integer to double.
__device__ __forceinline__ double i128_to_f64(__int128 v) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u =
      neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  if (msb <= 52) {
    const double d = (double)lo;  // exact
    return neg ? -d : d;
  }
  int sh = msb - 52;
  unsigned long long mant = (unsigned long long)(u >> sh);  // 53 significant bits
  const unsigned __int128 rem = u - ((unsigned __int128)mant << sh);
  const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
  if (rem > half || (rem == half && (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++sh;
    }
  }
  const unsigned long long bits =
      ((unsigned long long)(sh + 52 + 1023) << 52) | (mant & ((1ull << 52) - 1ull));
  const double d = __longlong_as_double((long long)bits);
  return neg ? -d : d;
}

__device__ __forceinline__ __int128 shfl_up_i128(__int128 v, int o) {
  unsigned long long lo = (unsigned long long)v;
  unsigned long long hi = (unsigned long long)((unsigned __int128)v >> 64);
  lo = __shfl_up_sync(0xffffffffu, lo, o);
  hi = __shfl_up_sync(0xffffffffu, hi, o);
  return (__int128)(((unsigned __int128)hi << 64) | lo);
}

// Exclusive block scan of two int128 values (exact: integer sums are order-free).
__device__ __forceinline__ void block_scan_i128x2(__int128& a, __int128& b, __int128& tb) {
  __shared__ __int128 wa[33], wb[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __int128 ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const __int128 ya = shfl_up_i128(ia, o), yb = shfl_up_i128(ib, o);
    if (lane >= o) {
      ia += ya;
      ib += yb;
    }
  }
  if (lane == 31) {
    wa[w] = ia;
    wb[w] = ib;
  }
  __syncthreads();
  if (w == 0) {
    const __int128 xa = (lane < nw) ? wa[lane] : (__int128)0;
    const __int128 xb = (lane < nw) ? wb[lane] : (__int128)0;
    __int128 sa = xa, sb = xb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const __int128 ya = shfl_up_i128(sa, o), yb = shfl_up_i128(sb, o);
      if (lane >= o) {
        sa += ya;
        sb += yb;
      }
    }
    if (lane < nw) {
      wa[lane] = sa - xa;
      wb[lane] = sb - xb;
    }
    if (lane == nw - 1) wb[32] = sb;
  }
  __syncthreads();
  const __int128 ea = wa[w] + ia - a, eb = wb[w] + ib - b;
  tb = wb[32];
  __syncthreads();
  a = ea;
  b = eb;
}

// Field of step `step` from the counts of buffer `buf` (reading C-23): the tridiagonal
// system of §2 step 2 solved through its discrete Green's function,
//   S_j = (N-j) sum_{k<=j} k dC_k + j sum_{k>j} (N-k) dC_k   (exact int128 prefix sums),
//   phi_j = (V (N-j) + rfac S_j) / N,
//   E_j = (2V + rfac (S_{j-1} - S_{j+1})) / (2 N dx)   inside,
//   E_0 = (V - rfac (S_1 + N dC_0)) / (N dx),  E_N = (V + rfac (S_{N-1} + N dC_N)) / (N dx)
// (half-cell Gauss law at the electrodes, reading C-4).  Each value rounds once, so the
// result is independent of the thread count and of how the nodes are split over blocks.
// Writes the FP64 field of nodes [jlo, jhi) (all nodes when jhi < 0), and its FP32 copy in
// cell units per step squared when K.fE is set; the exact sums S_j are formed for every node.
// With `mul` the three divisions become products with the reciprocals K.rden1, K.rden2, K.rnc
// (within an ulp of FP64, and far cheaper on a part with a low FP64 rate): for the FP32
// particle path, whose kicks are FP32; the FP64 path divides, as the oracle does.
// smem: 16 * nx bytes.
__device__ __forceinline__ void field_solve(const DevCtx& K, unsigned step, int buf,
                                            void* smem, int jlo = 0, int jhi = -1,
                                            bool mul = false) {
  const int N = K.nc, nx = K.nx;
  __int128* Sg = reinterpret_cast<__int128*>(smem);
  const unsigned long long* Ce = K.C + (size_t)(buf * 2 + 0) * nx;
  const unsigned long long* Ci = K.C + (size_t)(buf * 2 + 1) * nx;
  const double V = K.vtab[step % (unsigned)K.steps_per_rf];  // reading C-2
  const int seg = (nx + blockDim.x - 1) / blockDim.x;
  const int j0 = min((int)threadIdx.x * seg, nx), j1 = min(j0 + seg, nx);
  __int128 sa = 0, sb = 0;
  for (int j = j0; j < j1; ++j)
    if (j >= 1 && j <= N - 1) {
      const long long dc = (long long)Ci[j] - (long long)Ce[j];
      sa += (__int128)j * dc;
      sb += (__int128)(N - j) * dc;
    }
  __int128 tb;
  block_scan_i128x2(sa, sb, tb);
  for (int j = j0; j < j1; ++j) {
    if (j >= 1 && j <= N - 1) {
      const long long dc = (long long)Ci[j] - (long long)Ce[j];
      sa += (__int128)j * dc;
      sb += (__int128)(N - j) * dc;
    }
    Sg[j] = (__int128)(N - j) * sa + (__int128)j * (tb - sb);
  }
  __syncthreads();
  if (jhi < 0) jhi = nx;
  for (int j = jlo + (int)threadIdx.x; j < jhi; j += blockDim.x) {
    double e, ph;
    if (j == 0) {
      const __int128 q = Sg[1] + (__int128)N * (__int128)((long long)Ci[0] - (long long)Ce[0]);
      const double a = __dsub_rn(V, __dmul_rn(K.rfac, i128_to_f64(q)));
      e = mul ? __dmul_rn(a, K.rden1) : __ddiv_rn(a, K.den1);
      ph = V;
    } else if (j == N) {
      const __int128 q =
          Sg[N - 1] + (__int128)N * (__int128)((long long)Ci[N] - (long long)Ce[N]);
      const double a = __dadd_rn(V, __dmul_rn(K.rfac, i128_to_f64(q)));
      e = mul ? __dmul_rn(a, K.rden1) : __ddiv_rn(a, K.den1);
      ph = 0.0;
    } else {
      const double a =
          __dadd_rn(__dmul_rn(2.0, V), __dmul_rn(K.rfac, i128_to_f64(Sg[j - 1] - Sg[j + 1])));
      const double b =
          __dadd_rn(__dmul_rn(V, (double)(N - j)), __dmul_rn(K.rfac, i128_to_f64(Sg[j])));
      e = mul ? __dmul_rn(a, K.rden2) : __ddiv_rn(a, K.den2);
      ph = mul ? __dmul_rn(b, K.rnc) : __ddiv_rn(b, (double)N);
    }
    K.E[j] = e;
    K.phi[j] = ph;
    if (K.fE[0] != nullptr) {  // FP32 particle state only
      K.fE[0][j] = (float)__dmul_rn(e, K.fe_scale[0]);
      K.fE[1][j] = (float)__dmul_rn(e, K.fe_scale[1]);
    }
  }
}

// Thread 0 of block 0 of a particle pass: the step index and the counts and id counters the
// pass starts from, for the placement launch (which publishes new ones).
__device__ __forceinline__ void snapshot_pass(const DevCtx& K, unsigned step, long long ne,
                                              long long ni) {
  K.st->step_next = step + 1;
  K.st->n_snap[0] = ne;
  K.st->n_snap[1] = ni;
  K.st->id_snap[0] = K.st->next_id[0];
  K.st->id_snap[1] = K.st->next_id[1];
}

// Field block f of F in the placement launch (F = 1: the whole grid): close step n's
// accumulation (acc += C(n), counted) on its share of the nodes and clear that buffer for the
// deposit of step n+1, solve the field of step n+1 on the same share (every field block forms
// the exact sums of all nodes, so no block waits on another); block 0 advances the step index.
// The counts read (step n+1's deposit) and the buffer cleared (step n's) are different.
__device__ __forceinline__ void advance_field(const DevCtx& K, void* smem, int f = 0, int F = 1,
                                              bool mul = false) {
  const unsigned m = K.st->step_next;  // n + 1
  const int done = (m - 1u) & 1u;      // buffer of step n
  const int nx = K.nx;
  const int jlo = (int)((long long)nx * f / F), jhi = (int)((long long)nx * (f + 1) / F);
  unsigned long long* Cd = K.C + (size_t)(done * 2) * nx;
  for (int j = jlo + (int)threadIdx.x; j < jhi; j += blockDim.x) {
    K.acc[j] += (double)(long long)Cd[j];
    K.acc[nx + j] += (double)(long long)Cd[nx + j];
    Cd[j] = 0ull;
    Cd[nx + j] = 0ull;
  }
  field_solve(K, m, m & 1u, smem, jlo, jhi, mul);
  if (f == 0 && threadIdx.x == 0) {
    K.st->steps_avg += 1;
    K.st->step = m;
  }
}

// ------------------------------------------------------------ compaction (reading C-15)
// The lists of particle block b for a species with n particles start at the slot of the
// block's first particle (a block lists at most one hole and one birth per particle).
__device__ __forceinline__ long long list_base(long long n, int b, int G) {
  return range_begin(n, b, G);
}

__device__ __forceinline__ int upper_bound_i(const int* a, int n, long long v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)a[mid] <= v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Position of v in the ascending list a[0, n) (the number of entries below v) and whether v
// is in it: binary steps down to 32 entries, then one pass whose loads are all independent.
__device__ __forceinline__ int find_sorted(const int* a, int n, long long v, bool& found) {
  int lo = 0, hi = n;
  while (hi - lo > 32) {
    const int mid = (lo + hi) >> 1;
    if ((long long)a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  int lb = lo;
  bool f = false;
#pragma unroll 8
  for (int i = lo; i < hi; ++i) {
    const long long x = a[i];
    lb += x < v ? 1 : 0;
    f |= x == v;
  }
  if (lb == hi && hi < n && !f) f = (long long)a[hi] == v;  // a[hi] >= v after the binary steps
  found = f;
  return lb;
}

// Shared memory of the placement launch: the Green's-function sums of block 0, or the five
// prefix arrays of the other blocks.
__host__ __device__ __forceinline__ size_t place_smem_bytes(int nx, int nlist) {
  const size_t field = sizeof(__int128) * (size_t)nx;
  const size_t lists = sizeof(int) * 5 * (size_t)((nlist + 3) & ~3);  // 16-byte rows
  return field > lists ? field : lists;
}

// Row stride, in ints, of the five prefix arrays in shared memory (16-byte rows).
__host__ __device__ __forceinline__ int prefix_stride(int G) { return (G + 3) & ~3; }

// The single run's placement launch also keeps the list bases of its nlist owners in shared
// memory, after the five prefix arrays: sb[s * prefix_stride(G + 1) + b] = list_base(N_s, b,
// G) for b = 0..G, formed once per block (multiply-high by K.nl_div) instead of by 64-bit
// divisions in every item.  After them, per species, the hole list of the owner of the new
// count N_n when it holds at most kStagedHoles entries (the block reads it anyway to count
// the holes below N_n, and most tail positions lie in that owner): st[s] = that owner, or -1,
// and its entries at st + 4 + s * kStagedHoles.
constexpr int kStagedHoles = 256;
__host__ __device__ __forceinline__ size_t place_run_smem_bytes(int nx, int nlist) {
  const size_t field = sizeof(__int128) * (size_t)nx;
  const size_t lists = sizeof(int) * (5 * (size_t)prefix_stride(nlist) +
                                      2 * (size_t)prefix_stride(nlist + 1) + 4 +
                                      2 * (size_t)kStagedHoles);
  return field > lists ? field : lists;
}

// Reading C-15, run by every placement block into its own shared memory: the exclusive
// prefixes of the five per-owner count arrays of one simulation (sp[a * Gp + c], Gp =
// prefix_stride(G): a = 0, 1 holes of electrons / ions; 2 electron births from electron
// ranges; 3 electron births from ion ranges, whose ranks continue those of list 2; 4 ion
// births) and the totals of both species.  The count arrays lie at stride gstride from
// hole_cnt[0] (gstride >= G + 4 or the block is padded); they are read once with 16-byte
// loads; nothing waits on another block.
template <int NT, bool kSB = false>
__device__ void list_prefixes(const DevCtx& K, int G, int gstride, int* sp, CompactTot* sT) {
  constexpr int kA = 5, NW = NT / 32;
  __shared__ int wsum[NW][kA], wtot[kA];
  __shared__ int sq[2];
  const int Gp = prefix_stride(G);
  const long long N2[2] = {K.st->n_snap[0], K.st->n_snap[1]};  // loads overlap the staging
  const unsigned nid2[2] = {K.st->id_snap[0], K.st->id_snap[1]};
  if (gstride == G && (G & 3) == 0) {  // one contiguous block: 16-byte loads, all in flight
    constexpr int kBatch = 12;
    const int4* src = reinterpret_cast<const int4*>(K.hole_cnt[0]);
    int4* dst = reinterpret_cast<int4*>(sp);
    const int n4 = kA * G / 4;
    for (int i0 = threadIdx.x; i0 < n4; i0 += kBatch * NT) {
      int4 v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = i0 + u * NT;
        if (i < n4) v[u] = __ldcg(src + i);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = i0 + u * NT;
        if (i < n4) dst[i] = v[u];
      }
    }
  } else if ((gstride & 3) == 0) {  // rows on 16-byte boundaries: 16-byte loads, all in flight
    const int n4 = Gp / 4;
    for (int c0 = threadIdx.x; c0 < n4; c0 += 2 * NT) {
      int4 v[kA][2];
#pragma unroll
      for (int a = 0; a < kA; ++a)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = c0 + u * NT;
          if (c < n4)
            v[a][u] = __ldcg(reinterpret_cast<const int4*>(K.hole_cnt[0] + (size_t)a * gstride) + c);
        }
#pragma unroll
      for (int a = 0; a < kA; ++a)
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = c0 + u * NT;
          if (c < n4) reinterpret_cast<int4*>(sp + a * Gp)[c] = v[a][u];
        }
    }
  } else {
    for (int i = threadIdx.x; i < kA * G; i += NT) {
      const int a = i / G, c = i - a * G;
      sp[a * Gp + c] = __ldcg(K.hole_cnt[0] + (size_t)a * gstride + c);
    }
  }
  const int Gb = prefix_stride(G + 1);
  int* sb = sp + kA * Gp;  // list bases (kSB), formed while the staging loads are in flight
  if (kSB)
    for (int i = threadIdx.x; i < 2 * (G + 1); i += NT) {
      const int s = i > G ? 1 : 0, b = i - s * (G + 1);
      sb[s * Gb + b] = (int)range_begin_d(N2[s], b, K.nl_div);
    }
  if (threadIdx.x < 2) sq[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (G <= 32 * 32 && NW >= kA) {
    // up to 1024 owners: one warp per array, 32 lanes over contiguous segments, one warp
    // scan of the segment sums; one barrier before list 3 continues list 2's ranks
    const int per = (G + 31) >> 5;
    const int c0 = min(lane * per, G), c1 = min(c0 + per, G);
    int loc = 0, inc = 0;
    if (w < kA) {
      for (int c = c0; c < c1; ++c) loc += sp[w * Gp + c];
      inc = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) wtot[w] = inc;
    }
    __syncthreads();
    if (w < kA) {
      int run = inc - loc + (w == 3 ? wtot[2] : 0);
      for (int c = c0; c < c1; ++c) {
        const int v = sp[w * Gp + c];
        sp[w * Gp + c] = run;
        run += v;
      }
    }
  } else {
    const int seg = (G + NT - 1) / NT;
    const int c0 = min((int)threadIdx.x * seg, G), c1 = min(c0 + seg, G);
    int loc[kA], inc[kA];
#pragma unroll
    for (int a = 0; a < kA; ++a) {
      loc[a] = 0;
      for (int c = c0; c < c1; ++c) loc[a] += sp[a * Gp + c];
      inc[a] = loc[a];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc[a], o);
        if (lane >= o) inc[a] += y;
      }
      if (lane == 31) wsum[w][a] = inc[a];
    }
    __syncthreads();
    if (threadIdx.x < kA) {  // serial over the few warp sums
      int run = 0;
      for (int ww = 0; ww < NW; ++ww) {
        const int v = wsum[ww][threadIdx.x];
        wsum[ww][threadIdx.x] = run;
        run += v;
      }
      wtot[threadIdx.x] = run;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < kA; ++a) {
      int run = wsum[w][a] + inc[a] - loc[a] + (a == 3 ? wtot[2] : 0);
      for (int c = c0; c < c1; ++c) {
        const int v = sp[a * Gp + c];
        sp[a * Gp + c] = run;
        run += v;
      }
    }
  }
  __syncthreads();  // the prefixes are complete before any thread reads another's
  const int H2[2] = {wtot[0], wtot[1]};
  const int B2[2] = {wtot[2] + wtot[3], wtot[4]};
  // holes below Nn (needed when tail survivors fill holes): prefix of the owner of Nn plus
  // its list entries below Nn, counted by the whole block
  long long Nn2[2], Beff2[2];
  int owner[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const long long limit = K.cap - (N2[s] - H2[s]);
    Beff2[s] = B2[s] < limit ? B2[s] : limit;
    Nn2[s] = N2[s] - H2[s] + Beff2[s];
    owner[s] = -1;
    if (kSB && threadIdx.x == 0) sb[2 * Gb + s] = -1;  // no staged list (yet)
    if (H2[s] > Beff2[s]) {
      const int b = kSB ? upper_bound_i(sb + s * Gb, G, Nn2[s]) - 1 : range_owner(N2[s], Nn2[s], G);
      owner[s] = b;
      const int* list = K.hole_idx[s] + (kSB ? (long long)sb[s * Gb + b] : list_base(N2[s], b, G));
      const int m = (b + 1 < G ? sp[s * Gp + b + 1] : H2[s]) - sp[s * Gp + b];
      int* st = sb + 2 * Gb;  // (kSB) the staged list of this owner
      const bool stage = kSB && m <= kStagedHoles;
      if (kSB && threadIdx.x == 0) st[s] = stage ? b : -1;
      unsigned below = 0;
      for (int r = threadIdx.x; r < m; r += NT) {
        const int h = list[r];
        below += ((long long)h < Nn2[s]) ? 1u : 0u;
        if (stage) st[4 + s * kStagedHoles + r] = h;
      }
      below = __reduce_add_sync(0xffffffffu, below);
      if (lane == 0 && below) atomicAdd(&sq[s], (int)below);
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int s = threadIdx.x;
    CompactTot t;
    t.N = N2[s];
    t.H = H2[s];
    t.B = B2[s];
    t.B0 = s ? wtot[4] : wtot[2];
    t.Beff = Beff2[s];
    t.Nn = Nn2[s];
    t.q = owner[s] >= 0 ? (long long)sp[s * Gp + owner[s]] + sq[s] : 0;
    t.nid = nid2[s];
    t.pad = 0;
    sT[s] = t;
  }
  __syncthreads();
}

// Index of the hole of rank r of species s (hp: that species' hole prefixes, G owners).
// sbs: that species' list bases in shared memory (kSB), else null.
template <bool kSB>
__device__ __forceinline__ long long hole_of_rank(const DevCtx& K, int G, const int* hp, int s,
                                                  long long r, const CompactTot& t,
                                                  const int* sbs) {
  const int b = upper_bound_i(hp, G, r) - 1;
  const long long base = kSB ? (long long)sbs[b] : list_base(t.N, b, G);
  return K.hole_idx[s][base + (r - hp[b])];
}

// Births and tail survivors of one simulation to place: births into the holes by rank, then
// after N; tail survivors (index >= Nn, not a hole) into the remaining holes below Nn.
__device__ __forceinline__ long long place_count(const CompactTot* sT) {
  const CompactTot &te = sT[0], &ti = sT[1];
  const long long tle = te.H > te.Beff ? te.N - te.Nn : 0;
  const long long tli = ti.H > ti.Beff ? ti.N - ti.Nn : 0;
  return te.Beff + tle + ti.Beff + tli;
}

// The new counts and id counters of a simulation (and the births dropped at capacity).
__device__ __forceinline__ void publish_counts(const DevCtx& K, int s, const CompactTot& t) {
  K.st->n[s] = t.Nn;
  K.st->next_id[s] = t.nid + (unsigned)t.Beff;
  if (t.B > t.Beff) {
    atomicOr(&K.st->status, kStCapacity);
    atomicAdd(&K.counters[kCnDropped], (unsigned long long)(t.B - t.Beff));
  }
}

// Items u = first, first + step, ... below end of the placement of one simulation (items in
// the order: electron births, electron tail moves, ion births, ion tail moves).  P supplies
// the records of the particle representation: P::Rec, P::load_birth(K, list, slot) (a birth
// record), P::load(K, s, t) (the particle at slot t) and P::store(K, s, d, rec, id).  An
// item's record is loaded before the hole searches that give its destination, so that its
// loads are in flight during theirs (a tail position's record is loaded even when that
// position turns out to be a hole, and then dropped).
template <class P, bool kSB = false>
__device__ __forceinline__ void place_items(const DevCtx& K, int G, const int* sp,
                                            const CompactTot* sT, long long first,
                                            long long end, long long step) {
  const int Gp = prefix_stride(G);
  const int* sb = sp + 5 * Gp;  // list bases of both species (kSB)
  const int Gb = prefix_stride(G + 1);
  const CompactTot &te = sT[0], &ti = sT[1];  // shared: no per-thread copies
  const long long tle = te.H > te.Beff ? te.N - te.Nn : 0;
  for (long long u = first; u < end; u += step) {
    long long v = u;
    int s;
    bool birth;
    if (v < te.Beff) {
      s = 0; birth = true;
    } else if ((v -= te.Beff) < tle) {
      s = 0; birth = false;
    } else if ((v -= tle) < ti.Beff) {
      s = 1; birth = true;
    } else {
      v -= ti.Beff;
      s = 1; birth = false;
    }
    const CompactTot& t = sT[s];
    const int* hp = sp + s * Gp;
    const int* sbs = sb + s * Gb;
    if (birth) {
      const long long r = v;
      int list, b;
      long long slot;
      // electron births come from the owners' electron ranges (ionization) and ion ranges
      // (emission); ion births from the electron ranges
      if (s == 0 && r < t.B0) {
        list = 0;
        b = upper_bound_i(sp + 2 * Gp, G, r) - 1;
        slot = (kSB ? (long long)sb[b] : list_base(te.N, b, G)) + (r - sp[2 * Gp + b]);
      } else if (s == 0) {
        list = 1;
        b = upper_bound_i(sp + 3 * Gp, G, r) - 1;
        slot = (kSB ? (long long)sb[Gb + b] : list_base(ti.N, b, G)) + (r - sp[3 * Gp + b]);
      } else {
        list = 2;
        b = upper_bound_i(sp + 4 * Gp, G, r) - 1;
        slot = (kSB ? (long long)sb[b] : list_base(te.N, b, G)) + (r - sp[4 * Gp + b]);
      }
      const typename P::Rec rec = P::load_birth(K, list, slot);
      const long long d =
          (r < t.H) ? hole_of_rank<kSB>(K, G, hp, s, r, t, sbs) : t.N + r - t.H;
      P::store(K, s, d, rec, t.nid + (unsigned)r);
    } else {
      const long long idx = t.Nn + v;  // a tail position
      const typename P::Rec rec = P::load(K, s, idx);
      const int b = kSB ? upper_bound_i(sbs, G, idx) - 1 : range_owner(t.N, idx, G);
      const int* list = K.hole_idx[s] + (kSB ? (long long)sbs[b] : list_base(t.N, b, G));
      if (kSB && sb[2 * Gb + s] == b) list = sb + 2 * Gb + 4 + s * kStagedHoles;  // staged
      const int m = (b + 1 < G ? hp[b + 1] : (int)t.H) - hp[b];
      bool is_hole;
      const int lb = find_sorted(list, m, idx, is_hole);
      if (is_hole) continue;  // the tail position is itself a hole
      const long long before = (long long)hp[b] + lb;  // holes below idx
      const long long j = (idx - t.Nn) - (before - t.q);  // rank among survivors
      P::store(K, s, hole_of_rank<kSB>(K, G, hp, s, t.Beff + j, t, sbs), rec, rec.id);
    }
  }
}

// Placement launch: blocks [0, K.nfield) advance the field, each on its share of the nodes;
// the other blocks each total the lists and place the births and tail survivors; the first of
// them publishes the new counts and id counters.
template <class P>
__global__ void __launch_bounds__(256) k_place_field(DevCtx K) {
  extern __shared__ __align__(16) unsigned char place_smem[];
  chain_release();  // the next particle pass may take the SM room this launch leaves
  chain_wait();     // the particle pass of this step has completed
  const int F = K.nfield;
  if ((int)blockIdx.x < F) {
    advance_field(K, place_smem, blockIdx.x, F, P::kFieldMul);
    return;
  }
  __shared__ CompactTot sT[2];
  int* sp = reinterpret_cast<int*>(place_smem);
  list_prefixes<256, true>(K, K.nlist, K.nlist, sp, sT);
  const int b = blockIdx.x - F;
  if (b == 0 && threadIdx.x < 2) publish_counts(K, threadIdx.x, sT[threadIdx.x]);
  place_items<P, true>(K, K.nlist, sp, sT, (long long)b * blockDim.x + threadIdx.x, place_count(sT),
                 (long long)(gridDim.x - F) * blockDim.x);
}


}  // namespace pic
