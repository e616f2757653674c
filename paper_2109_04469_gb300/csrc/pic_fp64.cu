// pic_fp64.cu -- FP64 kernels of one PIC/MCC timestep (arXiv 2109.04469, §2 steps 1-6).
//
// Compiled with -fmad=false: every product and sum rounds as written, so the kernels
// reproduce the FP64 CPU oracle bit for bit on identical inputs and random keys.
//
// Step n is two launches:
//   k_push_fp64(n)   steps 3-6 of §2 and the deposit (step 1) of x^{n+1}: one pass over the
//                    particle state, persistent grid, block-private smem grids; each block
//                    owns a contiguous range of chunks and lists its holes and births in
//                    particle order; the last block to finish totals the lists;
//   k_place_field(n) places births and tail survivors (reading C-15) in parallel, while
//                    block 0 closes step n's RF average and solves the field of step n+1
//                    (§2 steps 1-2), which depends only on the deposit.
// The counts, the step index and the particle numbers live on the device: no step needs
// the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "pic_common.cuh"
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

// Piecewise-linear interpolant of the cumulative collision fractions between table nodes.
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
  // block-private counts over a grid-stride loop, then one global atomic per touched node
  // (integer sums, so the order of the additions does not matter); buf < 0: the counts
  // buffer of the current step
  if (buf < 0) buf = (int)(K.st->step & 1u);
  extern __shared__ unsigned long long dsm[];
  const int nx = K.nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) dsm[j] = 0ull;
  __syncthreads();
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    deposit_to(K, dsm, K.x[s][q]);
  __syncthreads();
  unsigned long long* C = K.C + (size_t)(buf * 2 + s) * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x)
    if (dsm[j]) atomicAdd(&C[j], dsm[j]);
}

// A species' population replaced (pic_set_particles): its count, the count the next particle
// pass starts from, its next id, and its counts in the current step's buffer cleared for the
// deposit that follows.
__global__ void k_set_counts(DevCtx K, int s, long long n, unsigned next_id) {
  if (threadIdx.x == 0) {
    K.st->n[s] = n;
    K.st->n_snap[s] = n;
    K.st->next_id[s] = next_id;
  }
  unsigned long long* C = K.C + (size_t)((K.st->step & 1u) * 2 + s) * K.nx;
  for (int j = threadIdx.x; j < K.nx; j += blockDim.x) C[j] = 0ull;
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

// Stand-alone field solve for the current step (after init, set_particles, set_step, or on
// request); touches no accumulator.
// Block f of F writes nodes [nx f / F, nx (f + 1) / F), like the field blocks of a step.
__global__ void k_field(DevCtx K) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const unsigned step = K.st->step;
  const int F = gridDim.x, f = blockIdx.x, nx = K.nx;
  const int jlo = (int)((long long)nx * f / F), jhi = (int)((long long)nx * (f + 1) / F);
  // an FP32 particle state (K.fE set) takes the field in the form its steps use
  field_solve(K, step, step & 1, fsm, jlo, jhi, K.fE[0] != nullptr);
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

// The block's particles [pb, pe) of species S (pb even), in 512-particle passes; each thread
// moves a pair of neighbours with 128-bit loads/stores.  Holes and births are ranked in
// particle order with a block scan and appended to the block's lists (which start at pb).
template <int S>
__device__ __forceinline__ void range_pass(const DevCtx& K, unsigned step, long long pb,
                                           long long pe, const double* sE,
                                           unsigned long long* sCe, unsigned long long* sCi,
                                           unsigned long long* sCnt, int* sWarp, int* sRun) {
  const size_t cap = (size_t)K.nchunk_max * kChunk;
  const long long lbase = pb;
  for (long long tile = pb; tile < pe; tile += kTile) {
    const long long p0 = tile + 2 * threadIdx.x;
    bool dead0 = false, dead1 = false;
    Births b0, b1;
    b0.e = b0.i = b1.e = b1.i = false;
    if (p0 < pe) {
      const bool both = (p0 + 1 < pe);
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
    long long hk = lbase + sRun[0] + (ex & 1023);
    long long ek = lbase + sRun[1] + ((ex >> 10) & 1023);
    long long ik = lbase + sRun[2] + ((ex >> 20) & 1023);
    if (dead0) K.hole_idx[S][hk++] = (int)p0;
    if (dead1) K.hole_idx[S][hk++] = (int)(p0 + 1);
    if (b0.e) {
      double* E4 = K.eb[S] + ek++;
      E4[0] = b0.e4[0]; E4[cap] = b0.e4[1]; E4[2 * cap] = b0.e4[2]; E4[3 * cap] = b0.e4[3];
    }
    if (b1.e) {
      double* E4 = K.eb[S] + ek++;
      E4[0] = b1.e4[0]; E4[cap] = b1.e4[1]; E4[2 * cap] = b1.e4[2]; E4[3 * cap] = b1.e4[3];
    }
    if (S == 0) {
      if (b0.i) {
        double* I4 = K.ib + ik++;
        I4[0] = b0.i4[0]; I4[cap] = b0.i4[1]; I4[2 * cap] = b0.i4[2]; I4[3 * cap] = b0.i4[3];
      }
      if (b1.i) {
        double* I4 = K.ib + ik++;
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
}

// Persistent grid: block b takes its balanced contiguous range of the electrons, then of the
// ions.  Block-private shared-memory copies of E and of the two count grids, flushed to the
// global int64 grid with one atomic per touched node.
__global__ void __launch_bounds__(kBlock, 2) k_push_fp64(DevCtx K) {
  extern __shared__ double psm[];
  const int nx = K.nx;
  double* sE = psm;
  unsigned long long* sC = reinterpret_cast<unsigned long long*>(sE + nx);
  unsigned long long* sCnt = sC + 2 * nx;
  __shared__ int sWarp[kBlock / 32 + 1];
  __shared__ int sRun[3];
  chain_release();  // the placement launch may take the SM room this pass leaves
  for (int j = threadIdx.x; j < 2 * nx; j += blockDim.x) sC[j] = 0ull;
  if (threadIdx.x < kNumCounters) sCnt[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) sRun[0] = sRun[1] = sRun[2] = 0;
  chain_wait();  // the field and counts of the previous launch are complete
  for (int j = threadIdx.x; j < nx; j += blockDim.x) sE[j] = K.E[j];
  const unsigned step = K.st->step;
  const long long ne = K.st->n[0], ni = K.st->n[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) snapshot_pass(K, step, ne, ni);
  __syncthreads();
  const int G = gridDim.x, b = blockIdx.x;
  range_pass<0>(K, step, range_begin(ne, b, G), range_begin(ne, b + 1, G), sE, sC, sC + nx,
                sCnt, sWarp, sRun);
  if (threadIdx.x == 0) {
    K.hole_cnt[0][blockIdx.x] = sRun[0];
    K.eb_cnt[0][blockIdx.x] = sRun[1];
    K.ib_cnt[blockIdx.x] = sRun[2];
    sRun[0] = sRun[1] = sRun[2] = 0;
  }
  __syncthreads();
  range_pass<1>(K, step, range_begin(ni, b, G), range_begin(ni, b + 1, G), sE, sC, sC + nx,
                sCnt, sWarp, sRun);
  if (threadIdx.x == 0) {
    K.hole_cnt[1][blockIdx.x] = sRun[0];
    K.eb_cnt[1][blockIdx.x] = sRun[1];
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

// Record moves of the FP64 representation for the placement launch.
struct Fp64Moves {
  static constexpr bool kFieldMul = false;  // bit-exact with the oracle: the field solve divides
  struct Rec {
    double x, vx, vy, vz;
    unsigned id;
  };
  // every field is loaded before the first use, so the loads are in flight together
  static __device__ __forceinline__ Rec load_birth(const DevCtx& K, int list, long long slot) {
    const double* rec = list == 0 ? K.eb[0] : (list == 1 ? K.eb[1] : K.ib);
    const size_t cap = (size_t)K.nchunk_max * kChunk;
    return Rec{rec[slot], rec[slot + cap], rec[slot + 2 * cap], rec[slot + 3 * cap], 0u};
  }
  static __device__ __forceinline__ Rec load(const DevCtx& K, int s, long long t) {
    return Rec{K.x[s][t], K.vx[s][t], K.vy[s][t], K.vz[s][t], K.id[s][t]};
  }
  static __device__ __forceinline__ void store(const DevCtx& K, int s, long long d,
                                               const Rec& r, unsigned id) {
    K.x[s][d] = r.x;
    K.vx[s][d] = r.vx;
    K.vy[s][d] = r.vy;
    K.vz[s][d] = r.vz;
    K.id[s][d] = id;
  }
};

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
  const long long blocks = std::min<long long>((n + bs - 1) / bs, kDepositBlocks);
  k_deposit<<<(unsigned)blocks, bs, sizeof(unsigned long long) * K.nx, s>>>(K, species, buf, n);
  return cudaGetLastError();
}

cudaError_t launch_field(const DevCtx& K, cudaStream_t s) {
  k_field<<<(unsigned)(K.nfield > 0 ? K.nfield : 1), 256, field_smem_bytes(K.nx), s>>>(K);
  return cudaGetLastError();
}

cudaError_t launch_push_fp64(const DevCtx& K, int grid, cudaStream_t s) {
  return launch_chained(k_push_fp64, (unsigned)grid, kBlock, push_smem_bytes(K.nx), s, K);
}

cudaError_t launch_place_fp64(const DevCtx& K, int grid, cudaStream_t s) {
  return launch_chained(k_place_field<Fp64Moves>, (unsigned)grid, 256u,
                        place_run_smem_bytes(K.nx, K.nlist), s, K);
}

cudaError_t launch_set_step(const DevCtx& K, unsigned step, cudaStream_t s) {
  k_set_step<<<1, 256, 0, s>>>(K, step);
  return cudaGetLastError();
}

cudaError_t launch_set_counts(const DevCtx& K, int species, long long n, unsigned next_id,
                              cudaStream_t s) {
  k_set_counts<<<1, 256, 0, s>>>(K, species, n, next_id);
  return cudaGetLastError();
}

// FP64 pipe probe: kChains independent chains per thread of x <- x * a + b, either as a
// separate multiply and add (what this translation unit's -fmad=false code issues: the
// particle pass's mix) or as fused multiply-adds.  Each chain step is 2 FP64 operations.
constexpr int kProbeChains = 8;
__device__ double g_probe_sink;  // written only if the chains' sum hits an impossible value
template <bool FMA>
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double a, double b) {
  double x[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k)
      x[k] = FMA ? __fma_rn(x[k], a, b) : __dadd_rn(__dmul_rn(x[k], a), b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += x[k];
  if (s == 12345.678) g_probe_sink = s;  // never true for these inputs; keeps the chains live
}

cudaError_t fp64_probe(bool fma, int sms, int iters, double* ms, double* ops, cudaStream_t s) {
  const unsigned grid = (unsigned)(8 * sms);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  float t = 0.0f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(a, s);
    if (fma)
      k_fp64_probe<true><<<grid, 256, 0, s>>>(iters, 0.999999, 1e-7);
    else
      k_fp64_probe<false><<<grid, 256, 0, s>>>(iters, 0.999999, 1e-7);
    cudaEventRecord(b, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = t;
  *ops = 2.0 * (double)grid * 256.0 * (double)iters * kProbeChains;
  return e;
}

cudaError_t configure_kernels(int nx) {
  cudaError_t e = raise_smem_limit(k_push_fp64, (int)push_smem_bytes(nx));
  if (e != cudaSuccess) return e;
  return raise_smem_limit(k_field, (int)field_smem_bytes(nx));
}

cudaError_t configure_place_fp64(int nx, int nlist) {
  return raise_smem_limit(k_place_field<Fp64Moves>, (int)place_run_smem_bytes(nx, nlist));
}

int push_fp64_blocks_per_sm(int nx) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_fp64, kBlock,
                                                    push_smem_bytes(nx)) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace pic
