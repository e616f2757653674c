// pic_fp64.cu -- FP64 kernels of one PIC/MCC timestep (arXiv 2109.04469, §2 steps 1-6).
//
// Compiled with -fmad=false: every product and sum rounds as written, so the kernels
// reproduce the FP64 CPU oracle bit for bit on identical inputs and random keys.
//
// Step n is two launches:
//   k_push_fp64(n)     steps 3-6 of §2 and the deposit (step 1) of x^{n+1}: one pass over
//                      the particle state, persistent grid, block-private smem grids;
//   k_compact_field(n) blocks 0/1 remove absorbed particles and insert births (one block per
//                      species); block 2 closes step n's RF-average accumulation and solves
//                      steps 1-2 (counts -> rho -> phi -> E) for step n+1, which depend only
//                      on the deposit, so the field solve overlaps the compaction.
// The counts, the step index and the particle numbers live on the device: no step needs
// the host.
#include <cuda_runtime.h>

#include "pic_dev.cuh"
#include "pic_launch.h"

namespace pic {

// ---------------------------------------------------------------- shared helpers
// Linear weighting (§2 steps 1 and 3): cell j = floor(x/dx) clamped to [0, nc-1],
// fraction f = x/dx - j.  __double2ll_rd is floor and conversion in one instruction.
__device__ __forceinline__ int cell_of(const DevCtx& K, double x, double& f) {
  const double xn = x * K.inv_dx;
  long long j = __double2ll_rd(xn);
  if (j > K.nc - 1) j = K.nc - 1;
  if (j < 0) j = 0;
  f = xn - (double)j;
  return (int)j;
}

// 32-bit fixed-point weights, round half to even, w_L = 2^32 - w_R (reading C-14): the sum
// of the counts is exact and independent of the order of the additions.
__device__ __forceinline__ void deposit_at(unsigned long long* C, int j, double f) {
  const long long wr = __double2ll_rn(f * 4294967296.0);
  const long long wl = 4294967296ll - wr;
  atomicAdd(&C[j], (unsigned long long)wl);
  atomicAdd(&C[j + 1], (unsigned long long)wr);
}

__device__ __forceinline__ void deposit_to(const DevCtx& K, unsigned long long* C, double x) {
  double f;
  const int j = cell_of(K, x, f);
  deposit_at(C, j, f);
}

// Piecewise-linear interpolant of the cumulative collision fractions (contract 2.4).
__device__ __forceinline__ void lookup(const double* __restrict__ F, double eps, double& f0,
                                       double& f1, double& f2) {
  const double t = eps * kXsInvDe;
  const double kf = floor(t);
  if (!(kf < (double)(kXsNodes - 1))) {  // also catches a non-finite energy
    const double* a = F + 4 * (kXsNodes - 1);
    f0 = __ldg(a);
    f1 = __ldg(a + 1);
    f2 = __ldg(a + 2);
    return;
  }
  const long long k = (long long)kf;
  const double fr = t - kf;
  const double2 a01 = __ldg(reinterpret_cast<const double2*>(F + 4 * k));
  const double2 a23 = __ldg(reinterpret_cast<const double2*>(F + 4 * k + 2));
  const double2 b01 = __ldg(reinterpret_cast<const double2*>(F + 4 * k + 4));
  const double2 b23 = __ldg(reinterpret_cast<const double2*>(F + 4 * k + 6));
  f0 = a01.x + fr * (b01.x - a01.x);
  f1 = a01.y + fr * (b01.y - a01.y);
  f2 = a23.x + fr * (b23.x - a23.x);
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

// ------------------------------------------------------------------ initial load
// Reading C-22: uniform x in (0, L), Maxwellian velocities, ids 0..n0-1, streams at step
// 0xFFFFFFFF.
__global__ void k_init_load(DevCtx K, int s, long long n0) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n0) return;
  Stream st(K, s, kPurLoad, (unsigned)q, 0xFFFFFFFFu);
  double ua, ub, v0, v1, v2;
  st.pair(ua, ub);
  maxwell3(st, K.sig_load[s], v0, v1, v2);
  K.x[s][q] = ua * K.L;
  K.vx[s][q] = v0;
  K.vy[s][q] = v1;
  K.vz[s][q] = v2;
  K.id[s][q] = (unsigned)q;
}

__global__ void k_deposit(DevCtx K, int s, int buf, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  deposit_to(K, K.C + (size_t)(buf * 2 + s) * K.nx, K.x[s][q]);
}

// Counts live in buffer (step & 1) and the other buffer must be zero (it receives the next
// deposit): a jump to a step of the other parity moves the counts along.
__global__ void k_set_step(DevCtx K, unsigned step) {
  const unsigned old = K.st->step;
  if ((old ^ step) & 1u) {
    unsigned long long* src = K.C + (size_t)((old & 1u) * 2) * K.nx;
    unsigned long long* dst = K.C + (size_t)((step & 1u) * 2) * K.nx;
    for (int j = threadIdx.x; j < 2 * K.nx; j += blockDim.x) {
      dst[j] = src[j];
      src[j] = 0ull;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) K.st->step = step;
}

// max |v| over n values: non-negative doubles order like their bit patterns
__global__ void k_max_abs(const double* __restrict__ v, long long n, unsigned long long* out) {
  unsigned long long m = 0ull;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)__double_as_longlong(fabs(v[q])));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// ------------------------------------------------------------------- field (§2 step 2)
// Round-to-nearest-even conversion of a 128-bit integer to double (the one rounding of each
// field value).
__device__ __forceinline__ double i128_to_f64(__int128 v) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
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
__device__ __forceinline__ void block_scan_i128x2(__int128& a, __int128& b, __int128& ta,
                                                  __int128& tb) {
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
    __int128 xa = (lane < nw) ? wa[lane] : (__int128)0, xb = (lane < nw) ? wb[lane] : (__int128)0;
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
    if (lane == nw - 1) {
      wa[32] = sa;
      wb[32] = sb;
    }
  }
  __syncthreads();
  const __int128 ea = wa[w] + ia - a, eb = wb[w] + ib - b;
  ta = wa[32];
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
// result is independent of the thread count.  smem: 16 * nx bytes.
__device__ __forceinline__ void field_solve(const DevCtx& K, unsigned step, int buf,
                                            void* smem) {
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
  __int128 ta, tb;
  block_scan_i128x2(sa, sb, ta, tb);
  for (int j = j0; j < j1; ++j) {
    if (j >= 1 && j <= N - 1) {
      const long long dc = (long long)Ci[j] - (long long)Ce[j];
      sa += (__int128)j * dc;
      sb += (__int128)(N - j) * dc;
    }
    Sg[j] = (__int128)(N - j) * sa + (__int128)j * (tb - sb);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    double e, ph;
    if (j == 0) {
      const __int128 q = Sg[1] + (__int128)N * (__int128)((long long)Ci[0] - (long long)Ce[0]);
      e = (V - K.rfac * i128_to_f64(q)) / K.den1;
      ph = V;
    } else if (j == N) {
      const __int128 q = Sg[N - 1] + (__int128)N * (__int128)((long long)Ci[N] - (long long)Ce[N]);
      e = (V + K.rfac * i128_to_f64(q)) / K.den1;
      ph = 0.0;
    } else {
      e = (2.0 * V + K.rfac * i128_to_f64(Sg[j - 1] - Sg[j + 1])) / K.den2;
      ph = (V * (double)(N - j) + K.rfac * i128_to_f64(Sg[j])) / (double)N;
    }
    K.E[j] = e;
    K.phi[j] = ph;
  }
}

// Stand-alone solve for the current step (after init, set_particles, set_step, or on
// request); touches no accumulator.
__global__ void k_field(DevCtx K) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const unsigned step = K.st->step;
  field_solve(K, step, step & 1, fsm);
}

// --------------------------------------------------------- one particle (§2 steps 3-6)
struct Births {
  bool e, i;
  double e4[4], i4[4];
};

template <int S>
__device__ __forceinline__ bool step_particle(const DevCtx& K, unsigned step, long long p,
                                              double& x, double& vx, unsigned pid,
                                              const double* sE, unsigned long long* sCe,
                                              unsigned long long* sCi, unsigned long long* sCnt,
                                              Births& b) {
  // per-step draws: u_null < P_max is decided on the 52-bit integer k of
  // u = (2k+1) 2^-53, against the exact threshold computed on the host
  const U4 w = philox4x32_10(pid, step, ((unsigned)S << 30) | ((unsigned)kPurStep << 24), 0u,
                             K.key0, K.key1);
  const unsigned long long k_null = ((unsigned long long)w.a << 20) | (w.b >> 12);
  // steps 3-4: linear gather and leapfrog (reading C-3)
  double f;
  const int j = cell_of(K, x, f);
  const double Ep = (1.0 - f) * sE[j] + f * sE[j + 1];
  vx = vx + K.qm_dt[S] * Ep;
  x = x + vx * K.dt;
  if ((((unsigned long long)__double_as_longlong(vx) >> 52) & 0x7ffull) == 0x7ffull)
    atomicOr(&K.st->status, kStNonfinite);
  double vy = 0.0, vz = 0.0;
  bool have_v = false, dirty_v = false;
  auto load_v = [&]() {
    if (!have_v) {
      vy = K.vy[S][p];
      vz = K.vz[S][p];
      have_v = true;
    }
  };
  bool dead = false;
  // step 5: surfaces (readings C-11, C-12)
  if (x <= 0.0 || x >= K.L) {
    const double u_wall = u52(w.c, w.d);
    const bool left = (x <= 0.0);
    if (S == 0) {
      bool removed = true;
      if (u_wall < K.refl) {
        x = left ? -x : 2.0 * K.L - x;
        vx = -vx;
        atomicAdd(&sCnt[kCnERefl], 1ull);
        removed = (x <= 0.0 || x >= K.L);
      }
      if (removed) {
        dead = true;
        atomicAdd(&sCnt[left ? kCnEAbsL : kCnEAbsR], 1ull);
        load_v();
        const double eps = ((vx * vx + vy * vy) + vz * vz) * K.emfac_e;
        const double t = floor(eps * K.fedf_inv_de);
        if (t < (double)K.fedf_bins) atomicAdd(&K.fedf[(int)t], 1ull);
      }
    } else {
      dead = true;
      atomicAdd(&sCnt[left ? kCnIAbsL : kCnIAbsR], 1ull);
      load_v();
      const double eps = ((vx * vx + vy * vy) + vz * vz) * K.emfac_ilab;
      const double t = floor(eps * K.fedf_inv_de);
      if (t < (double)K.fedf_bins) atomicAdd(&K.fedf[K.fedf_bins + (int)t], 1ull);
      if (u_wall < K.gamma) {
        Stream se(K, 1, kPurEmit, pid, step);
        double n0, n1, n2;
        iso_dir(se, n0, n1, n2);
        const double ax = fabs(n0) * K.v_see;
        const double xb = left ? 0.0 : K.L;
        b.e = true;
        b.e4[0] = xb;
        b.e4[1] = left ? ax : -ax;
        b.e4[2] = n1 * K.v_see;
        b.e4[3] = n2 * K.v_see;
        deposit_to(K, sCe, xb);
        atomicAdd(&sCnt[kCnSee], 1ull);
      }
    }
  }
  if (dead) return true;
  // step 6: null-collision Monte Carlo (readings C-7..C-10, C-13)
  if (k_null < K.null_kthr[S]) {
    load_v();
    Stream sc(K, S, kPurColl, pid, step);
    double up, unused;
    sc.pair(up, unused);
    if (S == 0) {
      atomicAdd(&sCnt[kCnECand], 1ull);
      const double v2 = (vx * vx + vy * vy) + vz * vz;
      const double eps = v2 * K.emfac_e;
      double F0, F1, F2;
      lookup(K.F[0], eps, F0, F1, F2);
      if (up < F0) {  // elastic, isotropic in the lab frame, cold target (C-9)
        double n0, n1, n2;
        iso_dir(sc, n0, n1, n2);
        const double vmag = sqrt(v2);
        const double cosx = (vmag > 0.0) ? ((vx * n0 + vy * n1) + vz * n2) / vmag : 0.0;
        const double sp = vmag * sqrt(1.0 - K.mr2 * (1.0 - cosx));
        vx = n0 * sp;
        vy = n1 * sp;
        vz = n2 * sp;
        dirty_v = true;
        atomicAdd(&sCnt[kCnEEla], 1ull);
      } else if (up < F1) {  // excitation
        if (eps >= kEExc) {
          double n0, n1, n2;
          iso_dir(sc, n0, n1, n2);
          const double sp = sqrt((eps - kEExc) * K.spd2_e);
          vx = n0 * sp;
          vy = n1 * sp;
          vz = n2 * sp;
          dirty_v = true;
          atomicAdd(&sCnt[kCnEExc], 1ull);
        }
      } else if (up < F2) {  // ionization (C-10)
        if (eps >= kEIon) {
          double a0, a1, a2, c0, c1, c2, w0, w1, w2;
          iso_dir(sc, a0, a1, a2);
          iso_dir(sc, c0, c1, c2);
          maxwell3(sc, K.sig_i, w0, w1, w2);
          const double e1 = 0.5 * (eps - kEIon);
          const double sp = sqrt(e1 * K.spd2_e);
          vx = a0 * sp;
          vy = a1 * sp;
          vz = a2 * sp;
          dirty_v = true;
          b.e = true;
          b.e4[0] = x;
          b.e4[1] = c0 * sp;
          b.e4[2] = c1 * sp;
          b.e4[3] = c2 * sp;
          b.i = true;
          b.i4[0] = x;
          b.i4[1] = w0;
          b.i4[2] = w1;
          b.i4[3] = w2;
          deposit_to(K, sCe, x);
          deposit_to(K, sCi, x);
          atomicAdd(&sCnt[kCnEIon], 1ull);
        }
      }
    } else {
      atomicAdd(&sCnt[kCnICand], 1ull);
      double n0, n1, n2;
      maxwell3(sc, K.sig_i, n0, n1, n2);  // target velocity
      const double gx = vx - n0, gy = vy - n1, gz = vz - n2;
      const double g2 = (gx * gx + gy * gy) + gz * gz;
      const double eps = g2 * K.emfac_rel;
      double F0, F1, F2;
      lookup(K.F[1], eps, F0, F1, F2);
      if (up < F0) {  // isotropic in the centre-of-mass frame, equal masses
        double d0, d1, d2;
        iso_dir(sc, d0, d1, d2);
        const double hg = 0.5 * sqrt(g2);
        vx = 0.5 * (vx + n0) + d0 * hg;
        vy = 0.5 * (vy + n1) + d1 * hg;
        vz = 0.5 * (vz + n2) + d2 * hg;
        dirty_v = true;
        atomicAdd(&sCnt[kCnIIso], 1ull);
      } else if (up < F1) {  // charge transfer
        vx = n0;
        vy = n1;
        vz = n2;
        dirty_v = true;
        atomicAdd(&sCnt[kCnICx], 1ull);
      }
    }
  }
  // step 1 of the next cycle: deposit at x^{n+1}
  double fd;
  const int jd = cell_of(K, x, fd);
  deposit_at(S == 0 ? sCe : sCi, jd, fd);
  // EEPF at the centre (reading C-18); the cell index only pre-selects the few candidates,
  // the window test itself is the contract's
  if (S == 0 && jd >= K.eepf_jlo && jd <= K.eepf_jhi) {
    const double d = x - K.half_L;
    if (d > -K.half_dx && d < K.half_dx) {
      load_v();
      const double eps = ((vx * vx + vy * vy) + vz * vz) * K.emfac_e;
      const double t = floor(eps * K.eepf_inv_de);
      if (t < (double)K.eepf_bins) atomicAdd(&K.eepf[(int)t], 1ull);
      atomicAdd(&sCnt[kCnEepfN], 1ull);
      atomicAdd(&sCnt[kCnEepfEsum], (unsigned long long)__double2ll_rn(eps * 1048576.0));
    }
  }
  if (dirty_v) {
    K.vy[S][p] = vy;
    K.vz[S][p] = vz;
  }
  return false;
}

// One chunk of kChunk particles of species S: two 512-particle passes; each thread moves a
// pair of neighbours with 128-bit loads/stores.  Holes and births are ranked in particle
// order with a block scan and written to the chunk's slots of the scratch lists.
template <int S>
__device__ __forceinline__ void chunk_pass(const DevCtx& K, unsigned step, int c, long long n,
                                           const double* sE, unsigned long long* sCe,
                                           unsigned long long* sCi, unsigned long long* sCnt,
                                           int* sWarp, int* sRun) {
  const long long cbase = (long long)c * kChunk;
  const size_t cap = (size_t)K.nchunk_max * kChunk;
  for (int t = 0; t < kChunk / kTile; ++t) {
    const long long p0 = cbase + (long long)t * kTile + 2 * threadIdx.x;
    bool dead0 = false, dead1 = false;
    Births b0, b1;
    b0.e = b0.i = b1.e = b1.i = false;
    if (p0 < n) {
      const bool both = (p0 + 1 < n);
      double x0, x1 = 0.0, v0, v1 = 0.0;
      unsigned id0, id1 = 0;
      if (both) {
        const double2 xx = *reinterpret_cast<const double2*>(K.x[S] + p0);
        const double2 vv = *reinterpret_cast<const double2*>(K.vx[S] + p0);
        const uint2 ii = *reinterpret_cast<const uint2*>(K.id[S] + p0);
        x0 = xx.x; x1 = xx.y; v0 = vv.x; v1 = vv.y; id0 = ii.x; id1 = ii.y;
      } else {
        x0 = K.x[S][p0];
        v0 = K.vx[S][p0];
        id0 = K.id[S][p0];
      }
      dead0 = step_particle<S>(K, step, p0, x0, v0, id0, sE, sCe, sCi, sCnt, b0);
      if (both) {
        dead1 = step_particle<S>(K, step, p0 + 1, x1, v1, id1, sE, sCe, sCi, sCnt, b1);
        *reinterpret_cast<double2*>(K.x[S] + p0) = make_double2(x0, x1);
        *reinterpret_cast<double2*>(K.vx[S] + p0) = make_double2(v0, v1);
      } else {
        K.x[S][p0] = x0;
        K.vx[S][p0] = v0;
      }
    }
    const int h = (int)dead0 + (int)dead1;
    const int e = (int)b0.e + (int)b1.e;
    const int i = (int)b0.i + (int)b1.i;
    int total;
    const int ex = block_excl_scan<kBlock / 32>(h | (e << 10) | (i << 20), sWarp, total);
    int hk = sRun[0] + (ex & 1023);
    int ek = sRun[1] + ((ex >> 10) & 1023);
    int ik = sRun[2] + ((ex >> 20) & 1023);
    if (dead0) K.hole_idx[S][cbase + hk++] = (int)p0;
    if (dead1) K.hole_idx[S][cbase + hk++] = (int)(p0 + 1);
    if (b0.e) {
      double* E4 = K.eb[S] + cbase + ek++;
      E4[0] = b0.e4[0]; E4[cap] = b0.e4[1]; E4[2 * cap] = b0.e4[2]; E4[3 * cap] = b0.e4[3];
    }
    if (b1.e) {
      double* E4 = K.eb[S] + cbase + ek++;
      E4[0] = b1.e4[0]; E4[cap] = b1.e4[1]; E4[2 * cap] = b1.e4[2]; E4[3 * cap] = b1.e4[3];
    }
    if (S == 0) {
      if (b0.i) {
        double* I4 = K.ib + cbase + ik++;
        I4[0] = b0.i4[0]; I4[cap] = b0.i4[1]; I4[2 * cap] = b0.i4[2]; I4[3 * cap] = b0.i4[3];
      }
      if (b1.i) {
        double* I4 = K.ib + cbase + ik++;
        I4[0] = b1.i4[0]; I4[cap] = b1.i4[1]; I4[2 * cap] = b1.i4[2]; I4[3 * cap] = b1.i4[3];
      }
    }
    if (threadIdx.x == 0) {
      sRun[0] += total & 1023;
      sRun[1] += (total >> 10) & 1023;
      sRun[2] += (total >> 20) & 1023;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    K.hole_cnt[S][c] = sRun[0];
    K.eb_cnt[S][c] = sRun[1];
    if (S == 0) K.ib_cnt[c] = sRun[2];
    sRun[0] = sRun[1] = sRun[2] = 0;
  }
  __syncthreads();
}

// Persistent grid over the electron chunks followed by the ion chunks.  Block-private
// shared-memory copies of E and of the two count grids; the counts are flushed to the
// global int64 grid with one atomic per touched node at the end.
__global__ void __launch_bounds__(kBlock, 2) k_push_fp64(DevCtx K) {
  extern __shared__ double psm[];
  const int nx = K.nx;
  double* sE = psm;
  unsigned long long* sC = reinterpret_cast<unsigned long long*>(sE + nx);
  unsigned long long* sCnt = sC + 2 * nx;
  __shared__ int sWarp[kBlock / 32 + 1];
  __shared__ int sRun[3];
  for (int j = threadIdx.x; j < nx; j += blockDim.x) sE[j] = K.E[j];
  for (int j = threadIdx.x; j < 2 * nx; j += blockDim.x) sC[j] = 0ull;
  if (threadIdx.x < kNumCounters) sCnt[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) sRun[0] = sRun[1] = sRun[2] = 0;
  const unsigned step = K.st->step;
  const long long ne = K.st->n[0], ni = K.st->n[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // counts and step the compaction works from
    K.st->n_snap[0] = ne;
    K.st->n_snap[1] = ni;
    K.st->step_next = step + 1;
  }
  __syncthreads();
  const int nche = (int)((ne + kChunk - 1) / kChunk);
  const int nchi = (int)((ni + kChunk - 1) / kChunk);
  for (int vc = blockIdx.x; vc < nche + nchi; vc += gridDim.x) {
    if (vc < nche)
      chunk_pass<0>(K, step, vc, ne, sE, sC, sC + nx, sCnt, sWarp, sRun);
    else
      chunk_pass<1>(K, step, vc - nche, ni, sE, sC, sC + nx, sCnt, sWarp, sRun);
  }
  __syncthreads();
  unsigned long long* Cn = K.C + (size_t)(((step + 1) & 1) * 2) * nx;
  for (int j = threadIdx.x; j < 2 * nx; j += blockDim.x) {
    const unsigned long long v = sC[j];
    if (v) atomicAdd(&Cn[j], v);
  }
  if (threadIdx.x < kNumCounters && sCnt[threadIdx.x])
    atomicAdd(&K.counters[threadIdx.x], sCnt[threadIdx.x]);
}

// ------------------------------------------------------- compaction (C-15) + next field
constexpr int kCompactThreads = 1024;

// For every chunk c < nch with cnt[c] entries at chunk-local slots, visit the entries in
// chunk order with their global rank: f(rank, slot).
template <typename Fn>
__device__ __forceinline__ int for_ranked(const int* cnt, int nch, int* sPref, int* sCnt,
                                          int* sWarp, int rank0, Fn f) {
  int carry = rank0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int b0 = 0; b0 < nch; b0 += kCompactThreads) {
    const int c = b0 + threadIdx.x;
    const int v = (c < nch) ? cnt[c] : 0;
    int total;
    const int ex = block_excl_scan<kCompactThreads / 32>(v, sWarp, total);
    sPref[threadIdx.x] = ex;
    sCnt[threadIdx.x] = v;
    __syncthreads();
    const int nb = min(kCompactThreads, nch - b0);
    for (int cc = warp; cc < nb; cc += kCompactThreads / 32) {
      const int m = sCnt[cc];
      const int base = carry + sPref[cc];
      const long long slot0 = (long long)(b0 + cc) * kChunk;
      for (int r = lane; r < m; r += 32) f(base + r, slot0 + r);
    }
    carry += total;
    __syncthreads();
  }
  return carry;
}

__device__ void compact_species(const DevCtx& K, int s, int* sPref, int* sCnt, int* sWarp) {
  const long long N = K.st->n_snap[s];
  const long long Ne = K.st->n_snap[0], Ni = K.st->n_snap[1];
  const int nch = (int)((N + kChunk - 1) / kChunk);
  const int nche = (int)((Ne + kChunk - 1) / kChunk), nchi = (int)((Ni + kChunk - 1) / kChunk);
  const size_t cap = (size_t)K.nchunk_max * kChunk;
  int* hs = K.hole_sorted[s];
  const int* hidx = K.hole_idx[s];
  // 1. all holes in ascending order
  const int H = for_ranked(K.hole_cnt[s], nch, sPref, sCnt, sWarp, 0,
                           [&](int rank, long long slot) { hs[rank] = hidx[slot]; });
  __syncthreads();
  // 2. births in rank order: into the holes, then appended after N
  const long long limit = K.cap - (N - H);
  const unsigned nid = K.st->next_id[s];
  double* X = K.x[s];
  double* VX = K.vx[s];
  double* VY = K.vy[s];
  double* VZ = K.vz[s];
  unsigned* ID = K.id[s];
  auto place = [&](const double* rec) {
    return [=](int rank, long long slot) {
      if (rank >= limit) return;
      const long long d = (rank < H) ? (long long)hs[rank] : N + rank - H;
      X[d] = rec[slot];
      VX[d] = rec[slot + cap];
      VY[d] = rec[slot + 2 * cap];
      VZ[d] = rec[slot + 3 * cap];
      ID[d] = nid + (unsigned)rank;
    };
  };
  int B;
  if (s == 0) {
    B = for_ranked(K.eb_cnt[0], nche, sPref, sCnt, sWarp, 0, place(K.eb[0]));
    B = for_ranked(K.eb_cnt[1], nchi, sPref, sCnt, sWarp, B, place(K.eb[1]));
  } else {
    B = for_ranked(K.ib_cnt, nche, sPref, sCnt, sWarp, 0, place(K.ib));
  }
  const long long Beff = (B < limit) ? (long long)B : limit;
  const long long Nn = N - H + Beff;
  // 3. tail survivors (indices >= Nn that are not holes) fill the remaining holes below Nn
  //    in ascending order.  The holes at or above Nn are the sorted suffix hs[q..H); each
  //    1024-index tile of the tail marks its holes in shared memory.
  if (H > Beff) {
    int* sFlag = sCnt;
    int q = 0;
    {  // first hole index >= Nn: count of holes below Nn, by a block reduction
      int below = 0;
      for (int r = threadIdx.x; r < H; r += kCompactThreads) below += (hs[r] < Nn) ? 1 : 0;
      int total;
      (void)block_excl_scan<kCompactThreads / 32>(below, sWarp, total);
      q = total;
    }
    int carry = 0, hq = q;
    for (long long b0 = Nn; b0 < N; b0 += kCompactThreads) {
      sFlag[threadIdx.x] = 0;
      __syncthreads();
      // holes in [b0, b0 + 1024) are hs[hq .. hq + m): at most 1024 of them
      const int r = hq + threadIdx.x;
      const bool inr = r < H && (long long)hs[r] < b0 + kCompactThreads;
      if (inr) sFlag[hs[r] - b0] = 1;
      int m;
      (void)block_excl_scan<kCompactThreads / 32>((int)inr, sWarp, m);
      const long long idx = b0 + threadIdx.x;
      const bool surv = idx < N && !sFlag[threadIdx.x];
      int total;
      const int ex = block_excl_scan<kCompactThreads / 32>((int)surv, sWarp, total);
      if (surv) {
        const long long d = hs[Beff + carry + ex];
        X[d] = X[idx];
        VX[d] = VX[idx];
        VY[d] = VY[idx];
        VZ[d] = VZ[idx];
        ID[d] = ID[idx];
      }
      carry += total;
      hq += m;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    K.st->n[s] = Nn;
    K.st->next_id[s] = nid + (unsigned)Beff;
    if (B > Beff) {
      atomicOr(&K.st->status, kStCapacity);
      atomicAdd(&K.counters[kCnDropped], (unsigned long long)(B - Beff));
    }
  }
}

// Block 2: close step n's accumulation (acc += C(n), counted) and clear that buffer for the
// deposit of step n+1, then solve the field of step n+1.
__device__ void advance_field(const DevCtx& K, void* smem) {
  const unsigned m = K.st->step_next;  // n + 1
  const int done = (m - 1u) & 1u;      // buffer of step n
  const int nx = K.nx;
  unsigned long long* Cd = K.C + (size_t)(done * 2) * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    K.acc[j] += (double)(long long)Cd[j];
    K.acc[nx + j] += (double)(long long)Cd[nx + j];
    Cd[j] = 0ull;
    Cd[nx + j] = 0ull;
  }
  if (threadIdx.x == 0) K.st->steps_avg += 1;
  field_solve(K, m, m & 1u, smem);
}

__global__ void __launch_bounds__(kCompactThreads) k_compact_field(DevCtx K) {
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ int sPref[kCompactThreads], sCnt[kCompactThreads];
  __shared__ int sWarp[kCompactThreads / 32 + 1];
  if (blockIdx.x < 2) {
    compact_species(K, blockIdx.x, sPref, sCnt, sWarp);
    if (blockIdx.x == 0 && threadIdx.x == 0) K.st->step = K.st->step_next;
  } else {
    advance_field(K, csm);
  }
}

// ------------------------------------------------------------------------ launchers
size_t field_smem_bytes(int nx) { return sizeof(__int128) * (size_t)nx; }
size_t push_smem_bytes(int nx) {
  return sizeof(double) * (size_t)nx + sizeof(unsigned long long) * (2 * (size_t)nx + kNumCounters);
}

cudaError_t launch_init_load(const DevCtx& K, int species, long long n0, cudaStream_t s) {
  if (n0 <= 0) return cudaSuccess;
  const int bs = 256;
  k_init_load<<<(unsigned)((n0 + bs - 1) / bs), bs, 0, s>>>(K, species, n0);
  return cudaGetLastError();
}

cudaError_t launch_deposit(const DevCtx& K, int species, int buf, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int bs = 256;
  k_deposit<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(K, species, buf, n);
  return cudaGetLastError();
}

cudaError_t launch_field(const DevCtx& K, cudaStream_t s) {
  k_field<<<1, 256, field_smem_bytes(K.nx), s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_push_fp64(const DevCtx& K, int grid, cudaStream_t s) {
  k_push_fp64<<<grid, kBlock, push_smem_bytes(K.nx), s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_compact_field(const DevCtx& K, cudaStream_t s) {
  k_compact_field<<<3, kCompactThreads, field_smem_bytes(K.nx), s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_set_step(const DevCtx& K, unsigned step, cudaStream_t s) {
  k_set_step<<<1, 256, 0, s>>>(K, step);
  return cudaGetLastError();
}

cudaError_t launch_max_abs(const double* v, long long n, unsigned long long* out,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const unsigned grid = (unsigned)(want < 1024 ? want : 1024);
  k_max_abs<<<grid, 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t configure_kernels(int nx) {
  cudaError_t e = cudaFuncSetAttribute(k_push_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)push_smem_bytes(nx));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_compact_field, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)field_smem_bytes(nx));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)field_smem_bytes(nx));
}

int push_fp64_blocks_per_sm(int nx) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_fp64, kBlock,
                                                    push_smem_bytes(nx)) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace pic
