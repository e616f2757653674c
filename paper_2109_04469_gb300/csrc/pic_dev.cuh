// pic_dev.cuh -- device-side layout and random-number / sampling helpers of libpic.
//
// Everything here implements the step contract of the PIC/MCC cycle of arXiv 2109.04469 §2
// (readings C-16 and the sampling rules) for the CUDA path.  FP64 translation units that
// include it are compiled with -fmad=false so every product and sum rounds exactly as
// written (IEEE division and square root, no contraction).
#pragma once
#include <cstdint>

namespace pic {

constexpr int kChunk = 1024;       // particles per chunk (hole / birth bookkeeping unit)
constexpr int kBlock = 256;        // threads per block of the particle kernels
constexpr int kTile = 2 * kBlock;  // particles per block-wide pass (two per thread)
constexpr int kDepositBlocks = 304; // grid of the stand-alone deposits (shared counts per block)
constexpr int kXsNodes = 100001;   // collision table nodes at eps_k = k / 100 eV
constexpr double kXsInvDe = 100.0;
constexpr int kMaxTries = 64;      // rejection-sampling attempts before the fixed fallback
constexpr int kNumCounters = 16;
constexpr double kEExc = 11.55;    // eV, lumped excitation threshold
constexpr double kEIon = 15.76;    // eV, ionization threshold (§3.1)

enum : int { kStCapacity = 1, kStNonfinite = 2, kStTimeout = 4 };
enum : int { kPurStep = 0, kPurColl = 1, kPurEmit = 2, kPurLoad = 3 };
enum : int {
  kCnEAbsL = 0, kCnEAbsR, kCnIAbsL, kCnIAbsR, kCnERefl, kCnSee, kCnEEla, kCnEExc, kCnEIon,
  kCnIIso, kCnICx, kCnECand, kCnICand, kCnEepfN, kCnEepfEsum, kCnDropped
};

// Exact floor(x / d) for 0 <= x < 2^62 and 1 <= d < 2^32 with no 64-bit division: with
// m = ceil(2^64 / d) (0 for d = 1), umulhi(x, m) exceeds x / d by less than x / 2^64 < 1, so
// it is the quotient or one more, and one multiply tells which.
struct Divider {
  unsigned long long m;
  long long d;
};
__host__ __device__ __forceinline__ Divider make_divider(long long d) {
  return Divider{d <= 1 ? 0ull : ~0ull / (unsigned long long)d + 1ull, d};
}

// Compaction totals of one species for the current step (written by the last particle
// block, read by the placement launch).
struct CompactTot {
  long long N;     // particles before the step
  long long H;     // holes (removed particles)
  long long B;     // births (all sources)
  long long B0;    // births of the first source (electrons: ionization; ions: all)
  long long Beff;  // births that fit the capacity
  long long Nn;    // particles after the step
  long long q;     // holes below Nn
  unsigned nid;    // id of the first birth
  int pad;
};

// Particle block b of a grid of G blocks owns the particles [range_begin(b), range_begin(b+1))
// of each species: contiguous, balanced to one 32-particle unit, starting on an even index.
constexpr int kUnit = 32;
__host__ __device__ __forceinline__ long long range_begin(long long n, int b, int G) {
  const long long units = (n + kUnit - 1) / kUnit;
  const long long u = (units * (long long)b) / G;
  const long long p = u * kUnit;
  return p < n ? p : n;
}
#ifdef __CUDACC__
__device__ __forceinline__ long long div_floor(long long x, const Divider& v) {
  if (v.m == 0ull) return x;
  long long q = (long long)__umul64hi((unsigned long long)x, v.m);
  if (q * v.d > x) --q;
  return q;
}
// range_begin(n, b, G) with dG = make_divider(G)
__device__ __forceinline__ long long range_begin_d(long long n, int b, const Divider& dG) {
  const long long units = (n + kUnit - 1) / kUnit;
  const long long p = div_floor(units * (long long)b, dG) * kUnit;
  return p < n ? p : n;
}
#endif
// The block whose range holds particle index t (0 <= t < n).
__host__ __device__ __forceinline__ int range_owner(long long n, long long t, int G) {
  const long long units = (n + kUnit - 1) / kUnit;
  const long long u = t / kUnit;
  // smallest b with range_begin(b+1) > t, i.e. floor(units (b+1) / G) > u
  long long b = ((u + 1) * (long long)G + units - 1) / units - 1;
  if (b < 0) b = 0;
  if (b > G - 1) b = G - 1;
  while (b > 0 && range_begin(n, (int)b, G) > t) --b;
  while (b < G - 1 && range_begin(n, (int)b + 1, G) <= t) ++b;
  return (int)b;
}

// Field blocks of the placement launch: about 64 nodes each (the FP64 divisions of a node
// set are what one block spends its time on), at most 16.
__host__ __device__ __forceinline__ int place_field_blocks(int nx) {
  const int f = (nx + 63) / 64;
  return f < 1 ? 1 : (f > 16 ? 16 : f);
}

// Device-resident scalars that change every step.
struct DevState {
  long long n[2];       // live particles per species
  long long n_snap[2];  // counts at the start of the current step's particle pass
  unsigned next_id[2];  // next id per species (reading C-15)
  unsigned step;        // step index n
  unsigned step_next;   // n + 1, written by the particle pass for the compaction launch
  int status;           // sticky kSt* bits
  long long steps_avg;  // steps added to the RF-average accumulators
  unsigned long long vmax_bits;  // scratch of the |vx| maximum reduction
  double v2sum;                  // scratch of the electrons' sum of |v|^2 (diagnostics)
  unsigned id_snap[2];           // next_id at the start of the current step's particle pass
  unsigned diag_ticket;          // blocks of the diagnostics launch done (zero between calls)
};

// Device-side state of an ensemble of FP32 simulations advanced by one launch per step (the
// paper's parameter scans, §3): the simulations' own contexts and states, and the few words
// the launch shares between its blocks.
constexpr int kMaxEnsemble = 128;
constexpr int kMaxEnsUnit = 16000;  // most particles (both species) per list owner
// Particles of one species a warp of the ensemble handles between flushes of its block's
// 32-bit counts: 8 warps x 8000 particles x 2^16 stays below 2^32 (a particle adds at most
// 2^16 to one count of its own species; births add theirs straight to the 64-bit counts).
constexpr int kEnsSpeciesRound = 8000;
struct DevCtx;
struct EnsDev {
  unsigned estep;      // launches so far (parity selects the totals buffer)
  unsigned bar_count;  // grid barrier: arrivals of the current generation
  unsigned bar_gen;    // grid barrier: generation
  int status;          // kSt* bits of the ensemble (a barrier that timed out)
  int n;               // simulations
  int unit;            // particles (both species) per list owner, <= kMaxEnsUnit
  int pipes_off;       // byte offset of the warps' staging pipes in dynamic shared memory
  int pad;
  const DevCtx* sims[kMaxEnsemble];  // each simulation's context (device copy)
  DevState* st[kMaxEnsemble];        // each simulation's state
  long long target[kMaxEnsemble];    // step index at which a simulation stops
  int gcap[kMaxEnsemble];            // most list owners a simulation may use
  int gstride[kMaxEnsemble];         // row stride of its five list-count arrays
  int tot[2][kMaxEnsemble][5];       // list totals per simulation, by launch parity
  int order[kMaxEnsemble];           // phase-1 order of the members: costliest first
  unsigned next_chunk[2];            // phase-1 work counter, by launch parity
};

// Everything a kernel needs, passed by value (constant bank).  Pointers address the
// caller's workspace.
struct DevCtx {
  int nc, nx, steps_per_rf, eepf_bins, fedf_bins, nchunk_max;
  long long cap;
  double L, dx, inv_dx, inv_2dx, dt, efac, rfac, den1, den2, half_L, half_dx;
  double rden1, rden2, rnc;  // 1 / den1, 1 / den2, 1 / N: the FP32 path's field multiplies
  double qm_dt[2], emfac_e, spd2_e, emfac_rel, spd2_rel, emfac_ilab, mr2, sig_i, v_see;
  double sig_load[2];
  double pmax[2], refl, gamma, eepf_inv_de, fedf_inv_de;
  // u < P_max  <=>  k < null_kthr for u = (2k+1) 2^-53 (exact integer threshold)
  unsigned long long null_kthr[2];
  int eepf_jlo, eepf_jhi;  // cells that can hold a particle of the EEPF window
  unsigned key0, key1;
  // particle state (FP64 path)
  double *x[2], *vx[2], *vy[2], *vz[2];
  unsigned *id[2];
  // grid: counts C[buf][species][nx], potential, field, density accumulators [2][nx]
  unsigned long long *C;
  double *phi, *E, *acc;
  float* fE[2];        // FP32 path: per-species velocity kick per step in cells/step (or null)
  double fe_scale[2];  // E [V/m] -> kick: (q/m) dt^2 / dx
  const double *inv_den, *vtab, *F[2];
  unsigned long long *eepf, *fedf, *counters;  // fedf [2][fedf_bins]
  DevState *st;
  // per-step scratch (hole / birth bookkeeping).  List owner b (a particle block of the
  // FP64 pass, a warp of the FP32 pass) owns a contiguous range of each species; its lists
  // start at the slot of its first particle and are in particle order.  The counts are per
  // owner ([nlist] entries); the placement launch forms their prefixes in shared memory.
  int nlist;            // list owners of the particle pass
  Divider gw_div;       // divider of the FP32 particle grid's warp count
  Divider nl_div;       // divider of nlist
  int nfield;           // field blocks of the placement launch
  int *hole_idx[2];     // [cap]: hole indices
  int *hole_cnt[2];
  int *eb_cnt[2];       // electron births from owners' species-s ranges
  int *ib_cnt;          // ion births from owners' electron ranges
  double *eb[2];        // [4][cap] records x, vx, vy, vz of electron births (FP64 state)
  double *ib;           // [4][cap] ion births (FP64 state)
  // FP32 particle state (precision PIC_FP32): position = cell + off in cells, off in [0, 1]
  // (1 only for a particle born on x = L), velocities in cells per step
  // ccd: cell | countdown << 16, the countdown counting the steps to the next null-collision
  // candidate (bit 15: the count ran out without a candidate); ov: (off, vx).  The two
  // arrays the particle pass reads and writes for every particle; vy, vz only on rare paths.
  unsigned* ccd[2];
  float2* ov[2];
  float *fvy[2], *fvz[2];
  float *feb[2], *fib;  // [6][cap] birth records: cell (int bits), off, vx, vy, vz, countdown
  float f_lnq[2];       // ln(1 - P_max) per species (0 without gas)
  const float* fF[2];   // FP32 cumulative collision fractions [kXsNodes][4]
  float f_emfac_e, f_emfac_rel, f_emfac_ilab;  // (cells/step)^2 -> eV
  float f_spd2_e;                              // eV -> (cells/step)^2 of an electron
  float f_sig_i, f_v_see, f_mr2;               // thermal ion speed, emitted speed, 2m/M
  float f_refl, f_gamma, f_eepf_inv_de, f_fedf_inv_de;
  unsigned f_null_thr[2];  // u < P_max <=> (w >> 8) < f_null_thr for u = (2k+1) 2^-25
  double to_si_v;          // cells/step -> m/s
  // a copy of this struct in device memory, for out-of-line device functions (taking the
  // address of a kernel parameter would copy the struct into every thread's local memory)
  const struct DevCtx* self;
};

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of the 4x32 Philox bijection with the
// published round multipliers and Weyl key increments.
struct U4 { unsigned a, b, c, d; };

__device__ __forceinline__ U4 philox4x32_10(unsigned c0, unsigned c1, unsigned c2, unsigned c3,
                                            unsigned k0, unsigned k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// (2k+1) 2^-53 with k the top 52 bits of (hi, lo): strictly inside (0, 1)
__device__ __forceinline__ double u52(unsigned hi, unsigned lo) {
  const unsigned long long k = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  return (double)(2ull * k + 1ull) * 0x1p-53;
}

// A counter-addressed stream: counter (id, step, species<<30 | purpose<<24 | block, 0).
struct Stream {
  unsigned k0, k1, id, step, base, block;
  __device__ __forceinline__ Stream(const DevCtx& K, int species, int purpose, unsigned pid,
                                    unsigned stp)
      : k0(K.key0), k1(K.key1), id(pid), step(stp),
        base(((unsigned)species << 30) | ((unsigned)purpose << 24)), block(0) {}
  __device__ __forceinline__ void pair(double& ua, double& ub) {
    const U4 w = philox4x32_10(id, step, base | block, 0u, k0, k1);
    ++block;
    ua = u52(w.a, w.b);
    ub = u52(w.c, w.d);
  }
};

// Natural logarithm of a positive normal double: binary exponent reduction to
// m in [sqrt(1/2), sqrt(2)) and ln m = 2 artanh t, t = (m-1)/(m+1), summed to t^23.
__device__ __forceinline__ double own_log(double x) {
  const long long b = __double_as_longlong(x);
  int k = (int)((b >> 52) & 0x7ff) - 1023;
  double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    k = k + 1;
  }
  const double t = (m - 1.0) / (m + 1.0);
  const double t2 = t * t;
  double s = 1.0 / 23.0;
  s = s * t2 + 1.0 / 21.0;
  s = s * t2 + 1.0 / 19.0;
  s = s * t2 + 1.0 / 17.0;
  s = s * t2 + 1.0 / 15.0;
  s = s * t2 + 1.0 / 13.0;
  s = s * t2 + 1.0 / 11.0;
  s = s * t2 + 1.0 / 9.0;
  s = s * t2 + 1.0 / 7.0;
  s = s * t2 + 1.0 / 5.0;
  s = s * t2 + 1.0 / 3.0;
  s = s * t2 + 1.0;
  return (double)k * 0.6931471805599453 + 2.0 * t * s;
}

// Marsaglia (1972): uniform direction by rejection of a point of the square.
__device__ __forceinline__ void iso_dir(Stream& st, double& n0, double& n1, double& n2) {
  for (int a = 0; a < kMaxTries; ++a) {
    double ua, ub;
    st.pair(ua, ub);
    const double v1 = 2.0 * ua - 1.0, v2 = 2.0 * ub - 1.0;
    const double s = v1 * v1 + v2 * v2;
    if (s < 1.0) {
      const double q = 2.0 * sqrt(1.0 - s);
      n0 = v1 * q;
      n1 = v2 * q;
      n2 = 1.0 - 2.0 * s;
      return;
    }
  }
  n0 = 0.0; n1 = 0.0; n2 = 1.0;
}

// Marsaglia polar method: two independent standard normal deviates.
__device__ __forceinline__ void gauss_pair(Stream& st, double& g0, double& g1) {
  for (int a = 0; a < kMaxTries; ++a) {
    double ua, ub;
    st.pair(ua, ub);
    const double v1 = 2.0 * ua - 1.0, v2 = 2.0 * ub - 1.0;
    const double s = v1 * v1 + v2 * v2;
    if (s < 1.0) {
      const double fac = sqrt((-2.0 * own_log(s)) / s);
      g0 = v1 * fac;
      g1 = v2 * fac;
      return;
    }
  }
  g0 = 0.0; g1 = 0.0;
}

__device__ __forceinline__ void maxwell3(Stream& st, double sig, double& v0, double& v1,
                                         double& v2) {
  double a0, a1, b0, b1;
  gauss_pair(st, a0, a1);
  gauss_pair(st, b0, b1);
  v0 = sig * a0;
  v1 = sig * a1;
  v2 = sig * b0;
}

}  // namespace pic
