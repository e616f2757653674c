// pic_fp32.cu -- FP32 particle path of one PIC/MCC timestep (arXiv 2109.04469, §2 steps
// 3-6 and the deposit of step 1), GB300.
//
// Particles are stored as a 16-bit cell index plus an FP32 offset in the cell and FP32
// velocities in cells per step, so the push is one kick and one drift per particle:
//   vx += kick(x),  off += vx,  cell += floor(off),  off -= floor(off).
// The field solve stays FP64 (pic_common.cuh) and writes the kick table fE[s][j] =
// (q/m) dt^2/dx E_j.  The deposit uses 16-bit linear weights accumulated in block-private
// 32-bit shared counters and flushed (<< 16) into the same int64 grid as the FP64 path, so
// charge stays exact and order-free.  Compaction and births follow the same hole-filling
// rule (reading C-15) through the common placement launch.  Results are statistical
// matches of the FP64 oracle, not bitwise ones.
//
// Null collisions (§3.5, reading C-7): a per-step Bernoulli(P_max) candidate test is the same
// in distribution as a geometric waiting time between candidates, so each particle carries a
// 16-bit countdown of the steps to its next candidate, drawn again at every candidate.  The
// counter-based generator then runs only at candidates, surfaces and births.
//
// Work split: every warp owns a contiguous, balanced range of each species and walks it in
// 128-particle tiles staged in shared memory by bulk asynchronous copies (stages - 1 tiles
// in flight per warp); a lane holds two neighbouring particles of each 64-particle half of a
// tile, so ballots and popcounts rank holes, births and queued work in particle order and
// warps never wait for one another.  The hole and birth lists are per warp.  The rare work
// (surfaces, collisions, EEPF samples) is queued and drained 32 entries at a time through
// out-of-line calls, so the hot loop stays small.
#include <cuda_runtime.h>

#include <algorithm>

#include "pic_common.cuh"
#include "pic_dev.cuh"
#include "pic_launch.h"
#include "pic_tma.cuh"

namespace pic {

// Resident blocks per SM the particle pass is compiled for (register budget 65536 /
// (256 x this)); the rare out-of-line branches may spill under a tight budget.
#ifndef PIC_FP32_MIN_BLOCKS
#define PIC_FP32_MIN_BLOCKS 2
#endif

constexpr int kWarps32 = kBlock / 32;
constexpr int kRoundPerWarp = 8160;  // particles a warp handles between counter flushes
// A block's 32-bit counters of species s take one full weight (2^16) at most per particle of
// species s (births add their charge straight to the 64-bit counts), so 8 warps x 8160
// particles x 2^16 < 2^32: they cannot overflow between flushes, and the electron counters
// are left alone by the ion pass (and the ion counters by the electron pass).  8160 is a
// multiple of 32, so every round starts on a tile boundary.
constexpr unsigned short kCdFlag = 0x8000;  // countdown expires without a candidate
constexpr int kPurCount = 4;                 // stream purpose: countdown of a new particle

__device__ __forceinline__ float u24(unsigned w) {  // (2k+1) 2^-25, k = top 24 bits
  return (float)((w >> 8) * 2u + 1u) * 0x1p-25f;
}

// Steps to the next null-collision candidate of a per-step Bernoulli(P) trial (geometric,
// >= 1), from a uniform u in (0, 1) and lnq = ln(1 - P) < 0.  Waits beyond 32766 steps are
// split: the countdown then expires with the flag set and is drawn again (memoryless).
__device__ __forceinline__ unsigned short draw_countdown(float u, float lnq) {
  if (!(lnq < 0.0f)) return (unsigned short)(kCdFlag | 0x7FFF);
  const float t = floorf(logf(u) / lnq);
  if (!(t < 32766.0f)) return (unsigned short)(kCdFlag | 0x7FFF);
  return (unsigned short)(t + 1.0f);
}

// Uniform direction (Marsaglia 1972); each Philox block offers two attempts.
__device__ __forceinline__ void iso_dir_f(Stream& st, float& n0, float& n1, float& n2) {
  for (int a = 0; a < kMaxTries / 2; ++a) {
    const U4 w = philox4x32_10(st.id, st.step, st.base | st.block, 0u, st.k0, st.k1);
    ++st.block;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float v1 = 2.0f * u24(h ? w.c : w.a) - 1.0f, v2 = 2.0f * u24(h ? w.d : w.b) - 1.0f;
      const float s = v1 * v1 + v2 * v2;
      if (s < 1.0f) {
        const float q = 2.0f * sqrtf(1.0f - s);
        n0 = v1 * q;
        n1 = v2 * q;
        n2 = 1.0f - 2.0f * s;
        return;
      }
    }
  }
  n0 = 0.0f; n1 = 0.0f; n2 = 1.0f;
}

// Two standard normal deviates (Marsaglia polar method).
__device__ __forceinline__ void gauss_pair_f(Stream& st, float& g0, float& g1) {
  for (int a = 0; a < kMaxTries / 2; ++a) {
    const U4 w = philox4x32_10(st.id, st.step, st.base | st.block, 0u, st.k0, st.k1);
    ++st.block;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float v1 = 2.0f * u24(h ? w.c : w.a) - 1.0f, v2 = 2.0f * u24(h ? w.d : w.b) - 1.0f;
      const float s = v1 * v1 + v2 * v2;
      if (s < 1.0f) {
        const float fac = sqrtf(-2.0f * logf(s) / s);
        g0 = v1 * fac;
        g1 = v2 * fac;
        return;
      }
    }
  }
  g0 = 0.0f; g1 = 0.0f;
}

__device__ __forceinline__ float next_u(Stream& st) {  // one more uniform of a stream
  const U4 w = philox4x32_10(st.id, st.step, st.base | st.block, 0u, st.k0, st.k1);
  ++st.block;
  return u24(w.a);
}

__device__ __forceinline__ void lookup_f(const float* __restrict__ F, float eps, float& f0,
                                         float& f1, float& f2) {
  const float t = eps * (float)kXsInvDe;
  if (!(t < (float)(kXsNodes - 1))) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(F) + (kXsNodes - 1));
    f0 = a.x; f1 = a.y; f2 = a.z;
    return;
  }
  const int k = (int)t;  // t >= 0
  const float fr = t - (float)k;
  const float4 a = __ldg(reinterpret_cast<const float4*>(F) + k);
  const float4 b = __ldg(reinterpret_cast<const float4*>(F) + k + 1);
  f0 = a.x + fr * (b.x - a.x);
  f1 = a.y + fr * (b.y - a.y);
  f2 = a.z + fr * (b.z - a.z);
}

// 16-bit linear weights into the block's 32-bit counters (w_L + w_R = 2^16 exactly).
__device__ __forceinline__ void deposit32(unsigned* C, int j, float f) {
  const int wr = __float2int_rn(f * 65536.0f);
  atomicAdd(&C[j], (unsigned)(65536 - wr));
  atomicAdd(&C[j + 1], (unsigned)wr);
}

// A newborn particle of species s (rare) whose charge does not go into the block's counters:
// the same weights, straight into the next step's 64-bit counts (the block's counters hold
// the units of 2^-16 that a flush shifts by 16 bits).
__device__ __forceinline__ void deposit_birth64(const DevCtx* G, unsigned step, int s, int j,
                                                float f) {
  unsigned long long* Cn = G->C + (size_t)(((step + 1) & 1) * 2 + s) * G->nx;
  const int wr = __float2int_rn(f * 65536.0f);
  if (wr != 65536) atomicAdd(&Cn[j], (unsigned long long)(65536 - wr) << 16);
  if (wr != 0) atomicAdd(&Cn[j + 1], (unsigned long long)wr << 16);
}

// (cell, off) with off brought back into [0, 1)
__device__ __forceinline__ void renorm(int& c, float& off) {
  const float k = floorf(off);
  c += (int)k;
  off -= k;
}

// A birth: position and velocity in cell units, countdown.
struct Rec32 {
  int cell;
  float off, vx, vy, vz;
  unsigned cd;
};

struct SurfOut {  // state after step 5; flags: bit 0 removed, bit 1 electron emitted
  int cell;
  float off, vx;
  int flags;
  unsigned ev;  // events: bit k adds one to event counter k
};

// Step 5 for a particle that left the gap (x <= 0 or x >= L).  An emitted electron is
// written to *em (this lane's slot in shared memory).  The events it counts are returned as
// bits, for the drain to add up over the warp.
template <int S>
__device__ __noinline__ SurfOut surface32(const DevCtx* __restrict__ G, unsigned step, long long p,
                                          int cell, float off, float vx, bool left,
                                          Rec32* em) {
  const int nc = G->nc;
  unsigned ev = 0u;
  const unsigned pid = G->id[S][p];
  const float vy = G->fvy[S][p], vz = G->fvz[S][p];  // in flight during the draw below
  // the per-step block of the FP64 contract: its third word decides the surface event
  const U4 w = philox4x32_10(pid, step, ((unsigned)S << 30) | ((unsigned)kPurStep << 24), 0u,
                             G->key0, G->key1);
  const float u_wall = u24(w.c);
  if (S == 0) {
    if (u_wall < G->f_refl) {  // specular reflection
      if (off > 0.0f) {
        cell = left ? -cell - 1 : 2 * nc - cell - 1;
        off = 1.0f - off;
      } else {
        cell = left ? -cell : 2 * nc - cell;
      }
      renorm(cell, off);
      vx = -vx;
      ev |= 1u << kCnERefl;
      if (!(cell < 0 || (cell == 0 && off == 0.0f) || cell >= nc))
        return SurfOut{cell, off, vx, 0, ev};
    }
    ev |= 1u << (left ? kCnEAbsL : kCnEAbsR);
    const float t = (vx * vx + vy * vy + vz * vz) * G->f_emfac_e * G->f_fedf_inv_de;
    if (t < (float)G->fedf_bins) atomicAdd(&G->fedf[(int)t], 1ull);
    return SurfOut{cell, off, vx, 1, ev};
  }
  ev |= 1u << (left ? kCnIAbsL : kCnIAbsR);
  const float t = (vx * vx + vy * vy + vz * vz) * G->f_emfac_ilab * G->f_fedf_inv_de;
  if (t < (float)G->fedf_bins) atomicAdd(&G->fedf[G->fedf_bins + (int)t], 1ull);
  int flags = 1;
  if (u_wall < G->f_gamma) {  // ion-induced electron at the struck electrode
    Stream se(*G, 1, kPurEmit, pid, step);
    float n0, n1, n2;
    iso_dir_f(se, n0, n1, n2);
    const float ax = fabsf(n0) * G->f_v_see;
    Rec32 r;
    r.cell = left ? 0 : nc - 1;
    r.off = left ? 0.0f : 1.0f;
    r.vx = left ? ax : -ax;
    r.vy = n1 * G->f_v_see;
    r.vz = n2 * G->f_v_see;
    r.cd = draw_countdown(next_u(se), G->f_lnq[0]);
    *em = r;
    flags |= 2;
    ev |= 1u << kCnSee;
  }
  return SurfOut{cell, off, vx, flags, ev};
}

struct CollOut {  // state after step 6; born: an ionization pair was written
  float vx;
  unsigned cd;
  int born;
  unsigned ev;  // events: bit k adds one to event counter k
};

// Countdown expiry: a null-collision candidate unless the flag is set (readings C-7..C-10,
// C-13), then the next countdown.  An ionization writes the pair to *re / *ri (this lane's
// slots in shared memory).  The events it counts are returned as bits.
template <int S>
__device__ __noinline__ CollOut collide32(const DevCtx* __restrict__ G, unsigned step, long long p,
                                          int cell, float off, float vx, unsigned cd,
                                          Rec32* re, Rec32* ri) {
  const unsigned pid = G->id[S][p];  // one round trip with vy, vz
  float vy = G->fvy[S][p], vz = G->fvz[S][p];  // in flight during the draws below
  Stream sc(*G, S, kPurColl, pid, step);
  const U4 wp = philox4x32_10(sc.id, sc.step, sc.base | sc.block, 0u, sc.k0, sc.k1);
  ++sc.block;
  const bool candidate = !(cd & kCdFlag);
  const unsigned cd_next = draw_countdown(u24(wp.b), G->f_lnq[S]);
  if (!candidate) return CollOut{vx, cd_next, 0, 0u};
  unsigned ev = 0u;
  bool dirty = false;
  int born = 0;
  const float up = u24(wp.a);
  if (S == 0) {
    ev |= 1u << kCnECand;
    const float v2 = vx * vx + vy * vy + vz * vz;
    const float eps = v2 * G->f_emfac_e;
    float F0, F1, F2;
    lookup_f(G->fF[0], eps, F0, F1, F2);
    if (up < F0) {  // elastic (C-9)
      float n0, n1, n2;
      iso_dir_f(sc, n0, n1, n2);
      const float vmag = sqrtf(v2);
      const float cosx = vmag > 0.0f ? (vx * n0 + vy * n1 + vz * n2) / vmag : 0.0f;
      const float sp = vmag * sqrtf(1.0f - G->f_mr2 * (1.0f - cosx));
      vx = n0 * sp; vy = n1 * sp; vz = n2 * sp;
      dirty = true;
      ev |= 1u << kCnEEla;
    } else if (up < F1) {  // excitation
      if (eps >= (float)kEExc) {
        float n0, n1, n2;
        iso_dir_f(sc, n0, n1, n2);
        const float sp = sqrtf((eps - (float)kEExc) * G->f_spd2_e);
        vx = n0 * sp; vy = n1 * sp; vz = n2 * sp;
        dirty = true;
        ev |= 1u << kCnEExc;
      }
    } else if (up < F2) {  // ionization (C-10)
      if (eps >= (float)kEIon) {
        float a0, a1, a2, c0, c1, c2, g0, g1, g2, g3;
        iso_dir_f(sc, a0, a1, a2);
        iso_dir_f(sc, c0, c1, c2);
        gauss_pair_f(sc, g0, g1);
        gauss_pair_f(sc, g2, g3);
        const float sp = sqrtf(0.5f * (eps - (float)kEIon) * G->f_spd2_e);
        vx = a0 * sp; vy = a1 * sp; vz = a2 * sp;
        dirty = true;
        *re = Rec32{cell, off, c0 * sp, c1 * sp, c2 * sp, draw_countdown(next_u(sc), G->f_lnq[0])};
        *ri = Rec32{cell, off, g0 * G->f_sig_i, g1 * G->f_sig_i, g2 * G->f_sig_i,
                    draw_countdown(next_u(sc), G->f_lnq[1])};
        born = 1;
        ev |= 1u << kCnEIon;
      }
    }
  } else {
    ev |= 1u << kCnICand;
    float g0, g1, g2, g3;
    gauss_pair_f(sc, g0, g1);
    gauss_pair_f(sc, g2, g3);
    const float n0 = g0 * G->f_sig_i, n1 = g1 * G->f_sig_i, n2 = g2 * G->f_sig_i;
    const float gx = vx - n0, gy = vy - n1, gz = vz - n2;
    const float g2s = gx * gx + gy * gy + gz * gz;
    float F0, F1, F2;
    lookup_f(G->fF[1], g2s * G->f_emfac_rel, F0, F1, F2);
    if (up < F0) {  // isotropic in the centre-of-mass frame
      float d0, d1, d2;
      iso_dir_f(sc, d0, d1, d2);
      const float hg = 0.5f * sqrtf(g2s);
      vx = 0.5f * (vx + n0) + d0 * hg;
      vy = 0.5f * (vy + n1) + d1 * hg;
      vz = 0.5f * (vz + n2) + d2 * hg;
      dirty = true;
      ev |= 1u << kCnIIso;
    } else if (up < F1) {  // charge transfer
      vx = n0; vy = n1; vz = n2;
      dirty = true;
      ev |= 1u << kCnICx;
    }
  }
  if (dirty) {
    G->fvy[S][p] = vy;
    G->fvz[S][p] = vz;
  }
  return CollOut{vx, cd_next, born, ev};
}

// EEPF sample of an electron in the centre window (reading C-18).  Returns the sample's
// energy in units of 2^-20 eV (rounded from FP32), or exactly -1 if the electron is outside
// the window.
__device__ __noinline__ long long eepf32(const DevCtx* __restrict__ G, long long p, int cell,
                                         float off, float vx) {
  const float d = ((float)cell - 0.5f * (float)G->nc) + off;
  if (!(d > -0.5f && d < 0.5f)) return -1ll;
  const float vy = G->fvy[0][p], vz = G->fvz[0][p];
  const float eps = (vx * vx + vy * vy + vz * vz) * G->f_emfac_e;
  if (eps * G->f_eepf_inv_de < (float)G->eepf_bins)
    atomicAdd(&G->eepf[(int)(eps * G->f_eepf_inv_de)], 1ull);
  return __float2ll_rn(eps * 1048576.0f);
}

__device__ __forceinline__ void put_rec(float* list, size_t cap, long long slot, const Rec32& r) {
  list[slot] = __int_as_float(r.cell);
  list[slot + cap] = r.off;
  list[slot + 2 * cap] = r.vx;
  list[slot + 3 * cap] = r.vy;
  list[slot + 4 * cap] = r.vz;
  list[slot + 5 * cap] = __int_as_float((int)r.cd);
}

// A warp's staging of one 128-particle tile (bulk-copy destination; 16-byte aligned fields).
// Only the two words every particle needs are staged; the id is read by the rare paths.
// Tile stages per warp: the single run keeps two tiles in flight; the ensemble one, since a
// third stage would take from the L1 that its members' collision tables are read through.
constexpr int kStagesRun = 3, kStagesEns = 2;
struct WarpTile {
  unsigned ccd[128];  // cell | countdown << 16
  float2 ov[128];     // off, vx
};
// The rare work of a particle, queued in particle order until 32 entries (or the end of the
// warp's range) are handled together, one per lane, so that their scattered loads and
// latency chains overlap: a particle that left the gap (surface, then for a survivor the
// countdown, deposit and possibly a collision), a particle whose countdown ran out (a
// null-collision candidate), or an electron of the EEPF cells.  pk = index | out << 31
// (indices stay below 2^31); aux = cell | countdown << 16, the countdown decremented for this
// step unless the particle left the gap, whose cell is kept as a signed 16-bit value
// saturated at +-32767 (with at most 4096 cells a saturated cell is still outside after a
// mirror reflection, so every surface decision is the unsaturated one's).
struct __align__(16) Cand {  // one 16-byte shared-memory access
  unsigned pk;
  unsigned aux;
  float off, vx;
};
constexpr int kCandQ = 160;  // up to 31 waiting + 128 from one tile
struct __align__(16) WarpRare {
  Rec32 recE[32], recI[32];  // the lanes' births of the current drain
  Cand cq[kCandQ];
  // births' charge goes into the block's counters while the warp's budget lasts (nb birth
  // deposits there since its last flush, at most bud), else into the 64-bit counts; the
  // budget keeps the counters' bound (bud = 0 in the single run, whose counter rounds fill
  // the bound with particles of the counter's own species)
  int nb, bud;
};
template <int NS>
struct __align__(128) WarpPipe {  // one per warp, back to back in shared memory
  WarpTile t[NS];
  unsigned long long bar[NS];
  WarpRare r;
};
struct PipeCount {         // per-warp, warp-uniform, in registers
  unsigned issued, waited;  // tiles issued / consumed by this warp so far
};

__device__ __forceinline__ unsigned round16(unsigned b) { return (b + 15u) & ~15u; }

// The cells an electron of the EEPF window |x / dx - N / 2| < 1/2 can sit in: (N - 1) / 2 to
// N / 2.  With the offset in [0, 1] (renorm can round it up to 1) and the cell a small integer,
// the window test of eepf32 is exact in FP32 and fails in every other cell.
__device__ __forceinline__ bool in_eepf_cells(int nc, int cell) {
  return (unsigned)(cell - (nc - 1) / 2) <= (unsigned)(nc / 2 - (nc - 1) / 2);
}

// Handle the first n queued entries (n <= 32, of nq queued), one per lane, in queue order
// (particle order): for an outgoing particle the surface event (step 5) and, if it stays, its
// countdown and deposit; then for an expired countdown the collision and next countdown
// (step 6); then the EEPF sample of an electron in the centre window.  Holes and births are
// ranked by ballot into the warp's lists (electrons: ionization pairs; ions: ion-induced
// electrons).  The remaining nq - n entries move to the front of the queue.  Returns (holes,
// births) listed: the caller advances hk by the first and ek (and, for electrons, ik) by the
// second.
template <int S>
__device__ __noinline__ int2 drain32(const DevCtx* __restrict__ G, unsigned step, WarpRare& P,
                                     int n, int nq, unsigned* sCe, unsigned* sCi,
                                     unsigned long long* sCnt, long long hk, long long ek,
                                     long long ik) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  bool dead = false, born = false;
  long long p = 0;
  unsigned ev = 0u;  // this lane's events, bit k for event counter k
  if (lane < n) {
    const Cand c = P.cq[lane];
    p = (long long)(c.pk & 0x7FFFFFFFu);
    int cell;
    float off = c.off, vx = c.vx;
    unsigned cd;
    bool moved = false;
    if (c.pk >> 31) {  // step 5: left the gap
      cell = (int)(short)(c.aux & 0xFFFFu);
      const bool left = cell < 0 || (cell == 0 && off == 0.0f);
      const SurfOut r = surface32<S>(G, step, p, cell, off, vx, left, &P.recE[lane]);
      ev |= r.ev;
      cell = r.cell;
      off = r.off;
      vx = r.vx;
      dead = r.flags & 1;
      born = (r.flags >> 1) & 1;  // an ion-induced electron (ions only)
      cd = (c.aux >> 16) - 1u;  // this step's countdown decrement, for a survivor
      if (!dead) deposit32(S == 0 ? sCe : sCi, cell, off);
      moved = true;
    } else {
      cell = (int)(c.aux & 0xFFFFu);
      cd = c.aux >> 16;
    }
    if (!dead) {
      if ((cd & 0x7FFFu) == 0u) {  // the countdown ran out: step 6
        const CollOut o =
            collide32<S>(G, step, p, cell, off, vx, cd, &P.recE[lane], &P.recI[lane]);
        ev |= o.ev;
        vx = o.vx;
        cd = o.cd;
        born = born || o.born != 0;  // an ionization pair (electrons only)
        moved = true;
      }
      if (moved) {
        G->ov[S][p] = make_float2(off, vx);
        G->ccd[S][p] = ((unsigned)cell & 0xFFFFu) | (cd << 16);
      }
      if (S == 0 && in_eepf_cells(G->nc, cell)) {
        const long long e = eepf32(G, p, cell, off, vx);
        if (e != -1ll) {  // rare: one lane of a few, so the 64-bit sum is added directly
          ev |= 1u << kCnEepfN;
          atomicAdd(&sCnt[kCnEepfEsum], (unsigned long long)e);
        }
      }
    }
  }
  // the drain's events into the block's counters: one shared atomic per counter that
  // occurred (lanes adding one by one would all hit the same address)
  const unsigned evs = __reduce_or_sync(0xffffffffu, ev);
  for (unsigned b = evs; b != 0u; b &= b - 1u) {
    const int k = __ffs(b) - 1;
    const unsigned m = __ballot_sync(0xffffffffu, (ev >> k) & 1u);
    if (lane == 0) atomicAdd(&sCnt[k], (unsigned long long)__popc(m));
  }
  const unsigned mh = __ballot_sync(0xffffffffu, dead);
  const unsigned mb = __ballot_sync(0xffffffffu, born);
  if (mb) {  // the births' charge: an ionization pair at the electron, an emitted electron
    const int nd = __popc(mb) * (S == 0 ? 2 : 1);  // deposits
    int nb = 0;
    if (lane == 0) nb = P.nb;
    nb = __shfl_sync(0xffffffffu, nb, 0);
    const bool blk = nb + nd <= P.bud;  // warp-uniform
    if (born) {
      const Rec32& re = P.recE[lane];
      if (blk) {
        deposit32(sCe, re.cell, re.off);
        if (S == 0) deposit32(sCi, re.cell, re.off);  // the ion is born at the electron
      } else {
        deposit_birth64(G, step, 0, re.cell, re.off);
        if (S == 0) deposit_birth64(G, step, 1, re.cell, re.off);
      }
    }
    __syncwarp();
    if (blk && lane == 0) P.nb = nb + nd;
  }
  if (dead) G->hole_idx[S][hk + __popc(mh & lt)] = (int)p;
  if (born) {
    const size_t cap = (size_t)G->nchunk_max * kChunk;
    put_rec(G->feb[S], cap, ek + __popc(mb & lt), P.recE[lane]);
    if (S == 0) put_rec(G->fib, cap, ik + __popc(mb & lt), P.recI[lane]);
  }
  __syncwarp();
  // the remaining nq - n entries move to the front (n == 32 here), 32 per round, every load
  // of a round before its stores; nq and n are warp-uniform, so every lane runs every round
  for (int i0 = 0; i0 < nq - n; i0 += 32) {
    const int i = i0 + lane;
    Cand c;
    if (i < nq - n) c = P.cq[i + n];
    __syncwarp();
    if (i < nq - n) P.cq[i] = c;
    __syncwarp();
  }
  return make_int2(__popc(mh), __popc(mb));
}

// Lane 0 starts the bulk copies of particles [t0, t0 + n) into the next stage (t0 is a
// multiple of 32, so every source starts on a 16-byte boundary).
template <int S, int NS>
__device__ __forceinline__ void issue_tile(const DevCtx& K, WarpPipe<NS>& P, PipeCount& Q,
                                           long long t0, int n) {
  if ((threadIdx.x & 31) == 0) {
    const unsigned st = Q.issued % NS;
    WarpTile& T = P.t[st];
    const unsigned b4 = round16(4u * n), b8 = round16(8u * n);
    fence_proxy_async_smem();  // the lanes' earlier reads of this stage come first
    mbar_arrive_expect_tx(&P.bar[st], b4 + b8);
    bulk_g2s(T.ccd, K.ccd[S] + t0, b4, &P.bar[st]);
    bulk_g2s(T.ov, K.ov[S] + t0, b8, &P.bar[st]);
  }
  ++Q.issued;
}

// Ranks in particle order of the flagged particles of a half tile (lane L holds particles
// 2L and 2L + 1 of the half): m0, m1 the ballots of the lanes' first and second particles.
// Returns the rank of the lane's first particle; the second one's is that plus its flag.
__device__ __forceinline__ int half_rank(unsigned m0, unsigned m1, unsigned lt) {
  return __popc(m0 & lt) + __popc(m1 & lt);
}

// Tile index of this lane's particle q (q = 2h + k: half h, k-th of the lane's two).
__device__ __forceinline__ int tile_index(int q, int lane) {
  return 64 * (q >> 1) + 2 * lane + (q & 1);
}

// One 128-particle tile of a warp's range.  Lane L holds particles 2L, 2L + 1 of each
// 64-particle half of the tile: its two (cell | countdown) words are one 8-byte shared load
// and one 8-byte global store, its two (off, vx) pairs one 16-byte load and store, all
// contiguous across the warp.  Ranks in particle order (holes, births, queue slots) are two
// ballots and two popcounts per half.  Expired countdowns and electrons of the EEPF cells
// are appended to the warp's queue (drained between tiles).  FULL: the tile holds 128
// particles of the range, so no bounds tests.
template <int S, bool FULL>
__device__ __forceinline__ void tile32_body(const DevCtx& K, long long tile, int nv,
                                            const WarpTile& T, const float2* sE, unsigned* sCe,
                                            unsigned* sCi, WarpRare& P, int& nq, float& fin) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int nc = K.nc;
  int cell[4];
  float off[4], vx[4];
  unsigned cd[4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i0 = 64 * h + 2 * lane;
    const uint2 cc = *reinterpret_cast<const uint2*>(&T.ccd[i0]);
    const float4 o = *reinterpret_cast<const float4*>(&T.ov[i0]);
    cell[2 * h] = (int)(cc.x & 0xFFFFu);
    cell[2 * h + 1] = (int)(cc.y & 0xFFFFu);
    cd[2 * h] = cc.x >> 16;
    cd[2 * h + 1] = cc.y >> 16;
    off[2 * h] = o.x;
    vx[2 * h] = o.y;
    off[2 * h + 1] = o.z;
    vx[2 * h + 1] = o.w;
  }
  // steps 3-4: linear gather and leapfrog in cell units
  bool out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool valid = FULL || tile_index(q, lane) < nv;
    if (!FULL && !valid) cell[q] = 0;  // staged words past nv are not this range's
    const float2 e = sE[cell[q]];
    vx[q] += e.x + off[q] * e.y;
    off[q] += vx[q];
    renorm(cell[q], off[q]);
    if (FULL || valid) fin = fmaf(vx[q], 0.0f, fin);
    out[q] = valid && ((unsigned)cell[q] >= (unsigned)nc ||
                       (__float_as_uint(off[q]) | (unsigned)cell[q]) == 0u);
  }
  // step 6 for the particles still in the gap: the countdown to the next null-collision
  // candidate, then the deposit (a collision changes neither cell nor offset).  Queued for the
  // drain, in particle order: an outgoing particle (surface first, step 5), an expired
  // countdown, an electron in the EEPF cells.
  bool qd[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    qd[q] = out[q];
    if ((FULL || tile_index(q, lane) < nv) && !out[q]) {
      --cd[q];
      deposit32(S == 0 ? sCe : sCi, cell[q], off[q]);
      qd[q] = (cd[q] & 0x7FFFu) == 0u || (S == 0 && in_eepf_cells(nc, cell[q]));
    }
  }
  unsigned* __restrict__ gccd = K.ccd[S] + tile;
  float2* __restrict__ gov = K.ov[S] + tile;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i0 = 64 * h + 2 * lane;
    const unsigned w0 = ((unsigned)cell[2 * h] & 0xFFFFu) | (cd[2 * h] << 16);
    const unsigned w1 = ((unsigned)cell[2 * h + 1] & 0xFFFFu) | (cd[2 * h + 1] << 16);
    const float4 o = make_float4(off[2 * h], vx[2 * h], off[2 * h + 1], vx[2 * h + 1]);
    if (FULL || i0 + 1 < nv) {
      *reinterpret_cast<uint2*>(gccd + i0) = make_uint2(w0, w1);
      *reinterpret_cast<float4*>(gov + i0) = o;
    } else if (i0 < nv) {
      gccd[i0] = w0;
      gov[i0] = make_float2(o.x, o.y);
    }
  }
  if (__any_sync(0xffffffffu, qd[0] | qd[1] | qd[2] | qd[3])) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned m0 = __ballot_sync(0xffffffffu, qd[2 * h]);
      const unsigned m1 = __ballot_sync(0xffffffffu, qd[2 * h + 1]);
      const int r = nq + half_rank(m0, m1, lt);
      const unsigned p0 = (unsigned)(tile + 64 * h + 2 * lane);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = 2 * h + k;
        if (qd[q])
          P.cq[r + (k ? (int)qd[2 * h] : 0)] =
              Cand{(p0 + (unsigned)k) | ((unsigned)out[q] << 31),
                   ((unsigned)max(-32767, min(32767, cell[q])) & 0xFFFFu) | (cd[q] << 16),
                   off[q], vx[q]};
      }
      nq += __popc(m0) + __popc(m1);
    }
  }
}

// One warp walks particles [q, qe) of species S (q a multiple of 32) in 128-particle tiles
// staged in shared memory by bulk copies, NS - 1 tiles in flight.  Holes and births go
// to the warp's lists at hk / ek / ik (running offsets, warp-uniform).  Returns false if a
// staged tile never arrived.
template <int S, int NS>
__device__ __forceinline__ bool warp_pass32(const DevCtx& K, unsigned step, long long q,
                                            long long qe, const float2* sE, unsigned* sCe,
                                            unsigned* sCi, unsigned long long* sCnt,
                                            WarpPipe<NS>& P, PipeCount& Q, long long& hk,
                                            long long& ek, long long& ik) {
  const int lane = threadIdx.x & 31;
  const DevCtx* __restrict__ G = K.self;
  const int ntiles = (int)((qe - q + 127) / 128);
  int nq = 0;          // queued entries (warp-uniform)
  float fin = 0.0f;    // stays finite unless a velocity was not: v * 0 + fin
  for (int t = 0; t < NS - 1 && t < ntiles; ++t)
    issue_tile<S>(K, P, Q, q + 128 * t, (int)min(128ll, qe - q - 128ll * t));
  for (int t = 0; t < ntiles; ++t) {
    if (t + NS - 1 < ntiles) {
      const int u = t + NS - 1;
      issue_tile<S>(K, P, Q, q + 128ll * u, (int)min(128ll, qe - q - 128ll * u));
    }
    const unsigned st = Q.waited % NS;
    if (!mbar_wait(&P.bar[st], (Q.waited / NS) & 1u)) {
      atomicOr(&K.st->status, kStTimeout);
      for (unsigned w = Q.waited + 1; w < Q.issued; ++w)  // let the copies in flight land
        (void)mbar_wait(&P.bar[w % NS], (w / NS) & 1u);
      Q.waited = Q.issued;
      return false;
    }
    ++Q.waited;
    const long long tile = q + 128ll * t;
    const int nv = (int)min(128ll, qe - tile);  // particles of this tile
    if (nv == 128)
      tile32_body<S, true>(K, tile, 128, P.t[st], sE, sCe, sCi, P.r, nq, fin);
    else
      tile32_body<S, false>(K, tile, nv, P.t[st], sE, sCe, sCi, P.r, nq, fin);
    while (nq >= 32) {  // the rare work, 32 entries at a time, in queue order
      const int2 r = drain32<S>(G, step, P.r, 32, nq, sCe, sCi, sCnt, hk, ek, ik);
      hk += r.x;
      ek += r.y;
      if (S == 0) ik += r.y;
      nq -= 32;
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
  }
  if (nq > 0) {
    const int2 r = drain32<S>(G, step, P.r, nq, nq, sCe, sCi, sCnt, hk, ek, ik);
    hk += r.x;
    ek += r.y;
    if (S == 0) ik += r.y;
  }
  if (__any_sync(0xffffffffu, !isfinite(fin)) && lane == 0) atomicOr(&K.st->status, kStNonfinite);
  return true;
}

__device__ __forceinline__ void flush32(const DevCtx& K, unsigned* sC, unsigned long long* Cn) {
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * K.nx; j += blockDim.x) {
    const unsigned v = sC[j];
    if (v) {
      atomicAdd(&Cn[j], (unsigned long long)v << 16);
      sC[j] = 0u;
    }
  }
  __syncthreads();
}

// The longest range a warp of the grid gets out of n particles: range_begin floors
// units g / GW, so no range exceeds ceil(units / GW) units of kUnit particles.
__device__ __forceinline__ long long warp_range_max(long long n) {
  const long long GW = (long long)gridDim.x * kWarps32;
  const long long units = (n + kUnit - 1) / kUnit;
  return (units + GW - 1) / GW * kUnit;
}

// Species S for the whole block: each warp its own range, in rounds that bound the 32-bit
// counters.  The warp's list lengths go to wc[list][warp] (lists: 0, 1 holes of electrons /
// ions; 2, 3 electron births from electron / ion ranges; 4 ion births), its first particle of
// species S to wb[S][warp].
template <int S>
__device__ __forceinline__ void block_pass32(const DevCtx& K, unsigned step, long long n,
                                             const float2* sE, unsigned* sC,
                                             unsigned long long* sCnt, unsigned long long* Cn,
                                             WarpPipe<kStagesRun>& P, PipeCount& Q,
                                             int (*wc)[kWarps32],
                                             long long (*wb)[kWarps32]) {
  const int gw = blockIdx.x * kWarps32 + (threadIdx.x >> 5);
  const long long q0 = range_begin_d(n, gw, K.gw_div), q1 = range_begin_d(n, gw + 1, K.gw_div);
  long long hk = q0, ek = q0, ik = q0;  // list slots of this warp
  // rounds: uniform across the grid (every warp's range is within warp_range_max), and an
  // empty round only costs a flush
  const long long wmax = warp_range_max(n);
  const int rounds = (int)((wmax + kRoundPerWarp - 1) / kRoundPerWarp);
  bool ok = true;
  for (int r = 0; r < rounds; ++r) {
    const long long a = q0 + (long long)r * kRoundPerWarp;
    const long long e = min(q1, a + kRoundPerWarp);
    if (ok && a < e)
      ok = warp_pass32<S>(K, step, a, e, sE, sC, sC + K.nx, sCnt, P, Q, hk, ek, ik);
    if (r + 1 < rounds) flush32(K, sC, Cn);
  }
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    wb[S][w] = q0;
    wc[S][w] = (int)(hk - q0);
    wc[2 + S][w] = (int)(ek - q0);
    if (S == 0) wc[4][w] = (int)(ik - q0);
  }
}

// The lists of the block's warps, each written from its warp's first particle on, packed into
// one list per block from the block's first particle on (warp b 8 + w of the grid's warps
// starts where block b starts for w = 0; the block's range is the union of its warps'), and
// the block's list lengths in K.hole_cnt rows of stride gridDim.x.  Warp order is particle
// order, so every list stays in particle order (reading C-15 ranks births and holes by it).
// An entry only moves down (a warp lists at most one entry per particle of its range).  When
// every destination lies below the first entry that moves (the usual case: a list is much
// shorter than a warp's range), each warp moves its own entries with no further barrier;
// otherwise the block moves them in rounds of one entry per thread -- every load of a round
// before a barrier, every store after it -- so no store reaches an entry still to be loaded.
// Called by the whole block after both species passes.
__device__ void pack_block_lists(const DevCtx& K, const int (*wc)[kWarps32],
                                 const long long (*wb)[kWarps32]) {
  __shared__ int off[5][kWarps32 + 1];
  __shared__ int direct[5];
  const int G = gridDim.x, b = blockIdx.x;
  const size_t cap = (size_t)K.nchunk_max * kChunk;
  if (threadIdx.x < 5) {
    const int a = threadIdx.x, sp = (a == 1 || a == 3) ? 1 : 0;
    int run = 0, first = -1;
    for (int w = 0; w < kWarps32; ++w) {
      off[a][w] = run;
      if (w > 0 && first < 0 && wc[a][w] > 0) first = w;
      run += wc[a][w];
    }
    off[a][kWarps32] = run;
    direct[a] = first < 0 || wb[sp][0] + run <= wb[sp][first];
  }
  __syncthreads();
  if (direct[0] & direct[1] & direct[2] & direct[3] & direct[4]) {
    // each warp its own entries, 32 per round of every list: all loads, then all stores
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 0) goto counts;  // warp 0's entries are in place
    {
      int mmax = 0;
#pragma unroll
      for (int a = 0; a < 5; ++a) mmax = max(mmax, off[a][w + 1] - off[a][w]);
      for (int e0 = 0; e0 < mmax; e0 += 32) {
        const int e = e0 + lane;
        int hv[2];
        float rv[3][6];
        bool mv[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          const int sp = (a == 1 || a == 3) ? 1 : 0;
          mv[a] = e < off[a][w + 1] - off[a][w];
          if (!mv[a]) continue;
          const long long src = wb[sp][w] + e;
          if (a < 2) {
            hv[a] = K.hole_idx[a][src];
          } else {
            const float* rec = a == 2 ? K.feb[0] : (a == 3 ? K.feb[1] : K.fib);
#pragma unroll
            for (int k = 0; k < 6; ++k) rv[a - 2][k] = rec[src + k * cap];
          }
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          if (!mv[a]) continue;
          const int sp = (a == 1 || a == 3) ? 1 : 0;
          const long long dst = wb[sp][0] + off[a][w] + e;
          if (a < 2) {
            K.hole_idx[a][dst] = hv[a];
          } else {
            float* rec = a == 2 ? K.feb[0] : (a == 3 ? K.feb[1] : K.fib);
#pragma unroll
            for (int k = 0; k < 6; ++k) rec[dst + k * cap] = rv[a - 2][k];
          }
        }
      }
    }
  counts:
    if (threadIdx.x < 5) K.hole_cnt[0][(size_t)threadIdx.x * G + b] = off[threadIdx.x][kWarps32];
    return;
  }
  int rounds = 0;
#pragma unroll
  for (int a = 0; a < 5; ++a)
    rounds = max(rounds, (off[a][kWarps32] + (int)blockDim.x - 1) / (int)blockDim.x);
  for (int r = 0; r < rounds; ++r) {
    const int i = r * blockDim.x + threadIdx.x;
    long long dst[5];
    int hv[2];
    float rv[3][6];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      dst[a] = -1;
      if (i < off[a][kWarps32]) {
        const int sp = (a == 1 || a == 3) ? 1 : 0;
        int w = 0;
        while (w + 1 < kWarps32 && off[a][w + 1] <= i) ++w;
        const long long src = wb[sp][w] + (i - off[a][w]);
        const long long d = wb[sp][0] + i;
        if (src != d) {
          dst[a] = d;
          if (a < 2) {
            hv[a] = K.hole_idx[a][src];
          } else {
            const float* rec = a == 2 ? K.feb[0] : (a == 3 ? K.feb[1] : K.fib);
#pragma unroll
            for (int k = 0; k < 6; ++k) rv[a - 2][k] = rec[src + k * cap];
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      if (dst[a] < 0) continue;
      if (a < 2) {
        K.hole_idx[a][dst[a]] = hv[a];
      } else {
        float* rec = a == 2 ? K.feb[0] : (a == 3 ? K.feb[1] : K.fib);
#pragma unroll
        for (int k = 0; k < 6; ++k) rec[dst[a] + k * cap] = rv[a - 2][k];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 5) K.hole_cnt[0][(size_t)threadIdx.x * G + b] = off[threadIdx.x][kWarps32];
}

__host__ __device__ __forceinline__ size_t pipes_offset(int nx) {
  return ((sizeof(float2) * 2 * (size_t)nx + sizeof(unsigned) * 2 * (size_t)nx) + 127) &
         ~size_t(127);
}

__global__ void __launch_bounds__(kBlock, PIC_FP32_MIN_BLOCKS) k_push_fp32(DevCtx K) {
  extern __shared__ __align__(128) unsigned char smem32[];
  const int nx = K.nx;
  float2* sE = reinterpret_cast<float2*>(smem32);           // [2][nx] kick, kick difference
  unsigned* sC = reinterpret_cast<unsigned*>(sE + 2 * nx);  // [2][nx] 32-bit counts
  WarpPipe<kStagesRun>& P =
      reinterpret_cast<WarpPipe<kStagesRun>*>(smem32 + pipes_offset(nx))[threadIdx.x >> 5];
  __shared__ unsigned long long sCnt[kNumCounters];
  chain_release();  // the placement launch may take the SM room this pass leaves
  if ((threadIdx.x & 31) == 0) {
    for (int s = 0; s < kStagesRun; ++s) mbar_init(&P.bar[s], 1u);
    fence_mbar_init();
    P.r.nb = 0;
    P.r.bud = 0;  // births to the 64-bit counts
  }
  PipeCount Q{0u, 0u};
  for (int j = threadIdx.x; j < 2 * nx; j += blockDim.x) sC[j] = 0u;
  if (threadIdx.x < kNumCounters) sCnt[threadIdx.x] = 0ull;
  chain_wait();  // the kick tables and counts of the previous launch are complete
  for (int s = 0; s < 2; ++s)
    for (int j = threadIdx.x; j < nx; j += blockDim.x) {
      const float a = K.fE[s][j];
      const float b = (j + 1 < nx) ? K.fE[s][j + 1] : a;
      sE[s * nx + j] = make_float2(a, b - a);
    }
  const unsigned step = K.st->step;
  const long long ne = K.st->n[0], ni = K.st->n[1];
  if (blockIdx.x == 0 && threadIdx.x == 0) snapshot_pass(K, step, ne, ni);
  __syncthreads();
  unsigned long long* Cn = K.C + (size_t)(((step + 1) & 1) * 2) * nx;
  __shared__ int wc[5][kWarps32];
  __shared__ long long wb[2][kWarps32];
  block_pass32<0>(K, step, ne, sE, sC, sCnt, Cn, P, Q, wc, wb);
  // no flush between the species: the ion pass adds nothing to the electron counters, so
  // each warp goes on to its ions without waiting for the block
  block_pass32<1>(K, step, ni, sE + nx, sC, sCnt, Cn, P, Q, wc, wb);
  flush32(K, sC, Cn);  // ends with a block barrier: every warp's lists are complete
  if (threadIdx.x < kNumCounters && sCnt[threadIdx.x])
    atomicAdd(&K.counters[threadIdx.x], sCnt[threadIdx.x]);
  pack_block_lists(K, wc, wb);
}

// Record moves of the FP32 representation for the placement launch.
struct Fp32Moves {
  static constexpr bool kFieldMul = true;  // FP32 kicks: the field solve multiplies
  struct Rec {
    unsigned ccd, id;
    float2 ov;
    float vy, vz;
  };
  // every field is loaded before the first use, so the loads are in flight together
  static __device__ __forceinline__ Rec load_birth(const DevCtx& K, int list, long long slot) {
    const float* rec = list == 0 ? K.feb[0] : (list == 1 ? K.feb[1] : K.fib);
    const size_t cap = (size_t)K.nchunk_max * kChunk;
    const float c = rec[slot], o = rec[slot + cap], vx = rec[slot + 2 * cap],
                vy = rec[slot + 3 * cap], vz = rec[slot + 4 * cap], cd = rec[slot + 5 * cap];
    return Rec{(unsigned)__float_as_int(c) | ((unsigned)__float_as_int(cd) << 16), 0u,
               make_float2(o, vx), vy, vz};
  }
  static __device__ __forceinline__ Rec load(const DevCtx& K, int s, long long t) {
    return Rec{K.ccd[s][t], K.id[s][t], K.ov[s][t], K.fvy[s][t], K.fvz[s][t]};
  }
  static __device__ __forceinline__ void store(const DevCtx& K, int s, long long d,
                                               const Rec& r, unsigned id) {
    K.ccd[s][d] = r.ccd;
    K.ov[s][d] = r.ov;
    K.fvy[s][d] = r.vy;
    K.fvz[s][d] = r.vz;
    K.id[s][d] = id;
  }
};

// FP64 SI state (x, v) -> FP32 cell units of particles [0, n) of species s, for the initial
// load and pic_set_particles, with their charge deposited in the same pass (16-bit weights of
// the stored offset into block-private 64-bit counts, one global atomic per touched node and
// block, into the current step's buffer, which the caller has cleared); draws each particle's
// countdown from its own stream at the current step.  The SI arrays x, vx, vy, vz, id are the
// FP64 buffers or device-readable host memory; ids read from elsewhere are stored into the
// species' id array.
__global__ void k_to_fp32(DevCtx K, int s, long long n, const double* __restrict__ x,
                          const double* __restrict__ vx, const double* __restrict__ vy,
                          const double* __restrict__ vz, const unsigned* __restrict__ id) {
  extern __shared__ unsigned long long csm[];
  const int nx = K.nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) csm[j] = 0ull;
  __syncthreads();
  const unsigned step = K.st->step;
  const double sc = K.dt * K.inv_dx;  // m/s -> cells per step
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const double xn = x[q] * K.inv_dx;
    long long j = __double2ll_rd(xn);
    if (j > K.nc - 1) j = K.nc - 1;
    if (j < 0) j = 0;
    const float off = (float)(xn - (double)j);
    K.ov[s][q] = make_float2(off, (float)(vx[q] * sc));
    K.fvy[s][q] = (float)(vy[q] * sc);
    K.fvz[s][q] = (float)(vz[q] * sc);
    const unsigned pid = id[q];
    if (id != K.id[s]) K.id[s][q] = pid;
    Stream st(K, s, kPurCount, pid, step);
    K.ccd[s][q] = (unsigned)j | ((unsigned)draw_countdown(next_u(st), K.f_lnq[s]) << 16);
    const int wr = __float2int_rn(off * 65536.0f);
    atomicAdd(&csm[j], (unsigned long long)(65536 - wr) << 16);
    atomicAdd(&csm[j + 1], (unsigned long long)wr << 16);
  }
  __syncthreads();
  unsigned long long* C = K.C + (size_t)((step & 1u) * 2 + s) * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x)
    if (csm[j]) atomicAdd(&C[j], csm[j]);
}

// pic_diag in one launch.  Every block reduces the electrons' max |vx| (as the bits of a
// non-negative float or double, which order like the values; a non-finite value wins) and
// sum of |v|^2 over the live count into the state's reduction words; the last block to finish
// (by a ticket) then writes the state, the event counters, the averages and the
// distributions into `out` (the handle's pinned host buffer, device-mapped) at the byte
// offsets off[0..4], and clears the reduction words and the ticket for the next call.
template <bool F32>
__global__ void __launch_bounds__(256) k_diag(DevCtx K, char* __restrict__ out, DiagOffsets off) {
  __shared__ unsigned long long wm[8];
  __shared__ double wsum[8];
  __shared__ int last;
  const long long n = K.st->n[0];
  unsigned long long m = 0ull;
  double acc = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    double a, b, c;
    if (F32) {
      const float ax = K.ov[0][q].y;
      m = max(m, (unsigned long long)__float_as_uint(fabsf(ax)));
      a = ax;
      b = K.fvy[0][q];
      c = K.fvz[0][q];
    } else {
      a = K.vx[0][q];
      m = max(m, (unsigned long long)__double_as_longlong(fabs(a)));
      b = K.vy[0][q];
      c = K.vz[0][q];
    }
    acc += (a * a + b * b) + c * c;
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    wm[w] = m;
    wsum[w] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      m = max(m, wm[i]);
      acc += wsum[i];
    }
    if (m) atomicMax(&K.st->vmax_bits, m);
    if (acc != 0.0) atomicAdd(&K.st->v2sum, acc);
    __threadfence();
    last = atomicAdd(&K.st->diag_ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // L2 reads (__ldcg): this block read the state's line at its start
  auto put = [&](size_t at, const void* src, size_t bytes) {
    const unsigned long long* s8 = static_cast<const unsigned long long*>(src);
    unsigned long long* d8 = reinterpret_cast<unsigned long long*>(out + at);
    for (size_t i = threadIdx.x; i < bytes / 8; i += blockDim.x) d8[i] = __ldcg(s8 + i);
  };
  static_assert(sizeof(DevState) % 8 == 0, "the state is copied in 8-byte words");
  put(off.state, K.st, sizeof(DevState));
  put(off.counters, K.counters, sizeof(unsigned long long) * kNumCounters);
  put(off.acc, K.acc, sizeof(double) * 2 * (size_t)K.nx);
  put(off.eepf, K.eepf, sizeof(unsigned long long) * (size_t)K.eepf_bins);
  put(off.fedf, K.fedf, sizeof(unsigned long long) * 2 * (size_t)K.fedf_bins);
  __syncthreads();
  if (threadIdx.x == 0) {
    K.st->vmax_bits = 0ull;
    K.st->v2sum = 0.0;
    K.st->diag_ticket = 0u;
  }
}

__global__ void k_to_fp64(DevCtx K, int s, long long n) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float2 ov = K.ov[s][q];
  K.x[s][q] = ((double)(K.ccd[s][q] & 0xFFFFu) + (double)ov.x) * K.dx;
  K.vx[s][q] = (double)ov.y * K.to_si_v;
  K.vy[s][q] = (double)K.fvy[s][q] * K.to_si_v;
  K.vz[s][q] = (double)K.fvz[s][q] * K.to_si_v;
}

// Deposit of the FP32 state with the FP32 rule (16-bit weights), after a load or a set.

// ------------------------------------------------------------ ensemble (one launch a step)
// All blocks of the ensemble launch are resident together (cooperative launch), so they can
// meet at a grid barrier; the wait is bounded and reports kStTimeout instead of hanging.
constexpr long long kGridSpinLimit = 1ll << 22;  // polls, ~128 ns apart (~0.5 s)

__device__ bool grid_barrier(EnsDev* E, unsigned expected = 0u) {
  __shared__ int sOk;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &E->bar_gen;
    const unsigned g0 = *gen;
    __threadfence();
    int ok = 1;
    const unsigned arrivals = expected ? expected : gridDim.x;
    if (atomicAdd(&E->bar_count, 1u) == arrivals - 1) {
      E->bar_count = 0u;
      __threadfence();
      atomicAdd(&E->bar_gen, 1u);
    } else {
      long long it = 0;
      while (*gen == g0 && it < kGridSpinLimit) {
        __nanosleep(128);
        ++it;
      }
      if (*gen == g0) {
        ok = 0;
        atomicOr(&E->status, kStTimeout);
      }
    }
    __threadfence();
    sOk = ok;
  }
  __syncthreads();
  return sOk != 0;
}

// Phase 2 of an ensemble step (after the grid barrier), out of line so that its registers do
// not add to the particle phase's.
__device__ __noinline__ void ensemble_phase2(EnsDev* E, unsigned par, unsigned sEstep, int n,
                                             const long long* sNe, const long long* sNi,
                                             long long* sIt, const int* sG, unsigned char* esm,
                                             CompactTot* sT) {
  // phase 2
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) E->estep = sEstep + 1u;
    for (int i = threadIdx.x; i < n * 5; i += blockDim.x) E->tot[par ^ 1u][i / 5][i % 5] = 0;
    if (threadIdx.x == 0) E->next_chunk[par ^ 1u] = 0u;
  }
  // items of every simulation, from the totals
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    long long items = 0;
    if (sG[s] > 0) {
      const int* t = E->tot[par][s];
      const long long cap = E->sims[s]->cap;
      const long long N2[2] = {sNe[s], sNi[s]};
      const long long H2[2] = {t[0], t[1]}, B2[2] = {(long long)t[2] + t[3], t[4]};
      for (int sp = 0; sp < 2; ++sp) {
        const long long limit = cap - (N2[sp] - H2[sp]);
        const long long beff = B2[sp] < limit ? B2[sp] : limit;
        const long long nn = N2[sp] - H2[sp] + beff;
        items += beff + (H2[sp] > beff ? N2[sp] - nn : 0);
      }
    }
    sIt[s] = items;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int s = 0; s < n; ++s) {
      const long long v = sIt[s];
      sIt[s] = run;
      run += v;
    }
    sIt[n] = run;
  }
  __syncthreads();
  if ((int)blockIdx.x < n) {
    const int s = blockIdx.x;
    if (sG[s] > 0) {
      const DevCtx& K = *E->sims[s];
      if (threadIdx.x < 2) {
        const int sp = threadIdx.x;
        const int* t = E->tot[par][s];
        CompactTot c;
        c.N = sp ? sNi[s] : sNe[s];
        c.H = t[sp];
        c.B = sp ? t[4] : (long long)t[2] + t[3];
        const long long limit = K.cap - (c.N - c.H);
        c.Beff = c.B < limit ? c.B : limit;
        c.Nn = c.N - c.H + c.Beff;
        c.nid = K.st->id_snap[sp];
        publish_counts(K, sp, c);
      }
      advance_field(K, esm, 0, 1, Fp32Moves::kFieldMul);
    }
    return;
  }
  const int nb = gridDim.x - n, j = blockIdx.x - n;
  const long long I = sIt[n];
  const long long lo = I * j / nb, hi = I * (j + 1) / nb;
  int* sp = reinterpret_cast<int*>(esm);
  for (int s = 0; s < n && lo < hi; ++s) {
    const long long a = max(lo, sIt[s]) - sIt[s], b = min(hi, sIt[s + 1]) - sIt[s];
    if (a >= b) continue;
    const DevCtx& K = *E->sims[s];
    list_prefixes<kBlock>(K, sG[s], E->gstride[s], sp, sT);
    place_items<Fp32Moves>(K, sG[s], sp, sT, a + threadIdx.x, b, (long long)blockDim.x);
    __syncthreads();
  }
}

// One step of every simulation of the ensemble that has not reached its target step.
// Phase 1: the particle passes.  Each simulation's particles (both species) are cut into G_s
// list owners of about E->unit particles, grouped in chunks of one owner per warp; blocks
// take chunks from a shared counter (members costliest first) and load a member's tables
// into shared memory when their chunk changes member.  The owners
// play the role of the single-run warps: lists in particle order at the owner's first slot,
// five counts per owner, and per-simulation totals by atomics.
// Phase 2 (after the grid barrier): block s < n closes simulation s's step and solves its
// next field; the other blocks split all simulations' births and tail moves evenly, forming
// the list prefixes of each simulation they touch in shared memory.
// Results do not depend on E->unit or on the grid: the compaction rule fixes every slot.
__global__ void __launch_bounds__(kBlock, PIC_FP32_MIN_BLOCKS) k_ensemble_step(EnsDev* E) {
  extern __shared__ __align__(128) unsigned char esm[];
  __shared__ long long sNe[kMaxEnsemble], sNi[kMaxEnsemble], sIt[kMaxEnsemble + 1];
  __shared__ unsigned sStep[kMaxEnsemble];
  __shared__ int sG[kMaxEnsemble], sC0[kMaxEnsemble + 1], sOrd[kMaxEnsemble];
  __shared__ Divider sGd[kMaxEnsemble];  // dividers of the owner counts
  __shared__ int sBud[kMaxEnsemble];     // births an owner may deposit into the block's counts
  __shared__ unsigned sChunk;
  __shared__ unsigned long long sCnt[kNumCounters];
  __shared__ CompactTot sT[2];
  __shared__ unsigned sEstep;
  const int n = E->n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // phase 0: the step's owners of every simulation
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const DevState* st = E->st[s];
    const unsigned step = st->step;
    const long long ne = st->n[0], ni = st->n[1];
    const bool active = (long long)step < E->target[s];
    // owners of about E->unit particles, and enough of them that no owner holds more than
    // kEnsSpeciesRound - 64 particles of one species before the 32-particle rounding
    const long long nmax = ne > ni ? ne : ni;
    long long g = (ne + ni + E->unit - 1) / E->unit;
    g = max(g, (nmax + kEnsSpeciesRound - 65) / (kEnsSpeciesRound - 64));
    g = g < 1 ? 1 : (g > E->gcap[s] ? E->gcap[s] : g);
    sNe[s] = ne;
    sNi[s] = ni;
    sStep[s] = step;
    sG[s] = active ? (int)g : 0;
    sGd[s] = make_divider(g);
    // a count of species s takes per chunk at most 2^16 per particle of that species (fewer
    // than ceil(n_s / G) + 64 of them per owner, 32-particle rounding) and per birth in the
    // block's counts: 8 owners x (per + budget) <= 8 x 8191 keeps it below 2^32
    sBud[s] = 8191 - (int)((nmax + g - 1) / g + 64);
    if (active && blockIdx.x == 0) snapshot_pass(*E->sims[s], step, ne, ni);
  }
  if (threadIdx.x < kNumCounters) sCnt[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) sEstep = E->estep;
  __syncthreads();
  if (threadIdx.x == 0) {  // chunks of kWarps32 owners (one round), members costliest first
    int run = 0;
    for (int k = 0; k < n; ++k) {
      const int s = E->order[k];
      sOrd[k] = s;
      sC0[k] = run;
      run += (sG[s] + kWarps32 - 1) / kWarps32;
    }
    sC0[n] = run;
  }
  __syncthreads();
  const unsigned par = sEstep & 1u;
  // phase 1: blocks take chunks (one owner per warp) from a shared counter until none is left,
  // so members whose particles cost more (more collision candidates) do not hold back a
  // block that a static split would have given too much
  {
    const unsigned TC = (unsigned)sC0[n];
    PipeCount Q{0u, 0u};
    bool ok = true;
    WarpPipe<kStagesEns>& P =
        reinterpret_cast<WarpPipe<kStagesEns>*>(esm + (size_t)E->pipes_off)[warp];
    if (lane == 0) {
      for (int k = 0; k < kStagesEns; ++k) mbar_init(&P.bar[k], 1u);
      fence_mbar_init();
    }
    int cur = -1;  // member (position in the order) whose tables are in shared memory
    float2* sE = reinterpret_cast<float2*>(esm);
    for (;;) {
      if (threadIdx.x == 0) sChunk = atomicAdd(&E->next_chunk[par], 1u);
      __syncthreads();
      const unsigned c = sChunk;
      if (c >= TC) break;
      int k = 0;  // the member holding chunk c: last k with sC0[k] <= c
      for (int lo2 = 0, hi2 = n; lo2 < hi2;) {
        const int mid = (lo2 + hi2) >> 1;
        if ((unsigned)sC0[mid] <= c) {
          k = mid;
          lo2 = mid + 1;
        } else {
          hi2 = mid;
        }
      }
      const int s = sOrd[k];
      const DevCtx& K = *E->sims[s];
      const int nx = K.nx;
      unsigned* sC = reinterpret_cast<unsigned*>(sE + 2 * nx);
      if (k != cur) {
        if (cur >= 0 && threadIdx.x < kNumCounters && sCnt[threadIdx.x]) {
          atomicAdd(&E->sims[sOrd[cur]]->counters[threadIdx.x], sCnt[threadIdx.x]);
          sCnt[threadIdx.x] = 0ull;
        }
        for (int sp = 0; sp < 2; ++sp)
          for (int j = threadIdx.x; j < nx; j += blockDim.x) {
            const float a = K.fE[sp][j];
            const float b = (j + 1 < nx) ? K.fE[sp][j + 1] : a;
            sE[sp * nx + j] = make_float2(a, b - a);
          }
        for (int j = threadIdx.x; j < 2 * nx; j += blockDim.x) sC[j] = 0u;
        cur = k;
        __syncthreads();
      }
      const unsigned step = sStep[s];
      const long long ne = sNe[s], ni = sNi[s];
      const int G = sG[s], gs = E->gstride[s];
      unsigned long long* Cn = K.C + (size_t)(((step + 1) & 1) * 2) * nx;
      const long long g = (long long)(c - (unsigned)sC0[k]) * kWarps32 + warp;
      if (g < G) {
        if (lane == 0) {
          P.r.nb = 0;
          P.r.bud = sBud[s];
        }
        __syncwarp();
        // after a timed-out wait (status set) the warp's remaining owners list nothing
        const Divider& dG = sGd[s];
        const long long q0 = range_begin_d(ne, (int)g, dG), q1 = range_begin_d(ne, (int)g + 1, dG);
        long long hk = q0, ek = q0, ik = q0;
        if (ok) ok = warp_pass32<0>(K, step, q0, q1, sE, sC, sC + nx, sCnt, P, Q, hk, ek, ik);
        const int he = (int)(hk - q0), be0 = (int)(ek - q0), bi = (int)(ik - q0);
        const long long r0 = range_begin_d(ni, (int)g, dG), r1 = range_begin_d(ni, (int)g + 1, dG);
        hk = ek = ik = r0;
        if (ok) ok = warp_pass32<1>(K, step, r0, r1, sE + nx, sC, sC + nx, sCnt, P, Q, hk, ek, ik);
        const int hi_ = (int)(hk - r0), be1 = (int)(ek - r0);
        if (lane == 0) {
          int* rows = K.hole_cnt[0];
          rows[g] = he;
          rows[(size_t)gs + g] = hi_;
          rows[2 * (size_t)gs + g] = be0;
          rows[3 * (size_t)gs + g] = be1;
          rows[4 * (size_t)gs + g] = bi;
          int* t = E->tot[par][s];
          if (he) atomicAdd(&t[0], he);
          if (hi_) atomicAdd(&t[1], hi_);
          if (be0) atomicAdd(&t[2], be0);
          if (be1) atomicAdd(&t[3], be1);
          if (bi) atomicAdd(&t[4], bi);
        }
      }
      // one owner per warp per chunk: an owner's range of species s holds fewer than
      // ceil(n_s / G) + 64 <= kEnsSpeciesRound particles (32-particle rounding; the owner
      // count above and the capacity check at creation), so the 32-bit counts stay in range
      flush32(K, sC, Cn);
    }
    if (cur >= 0 && threadIdx.x < kNumCounters && sCnt[threadIdx.x])
      atomicAdd(&E->sims[sOrd[cur]]->counters[threadIdx.x], sCnt[threadIdx.x]);
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < kStagesEns; ++k) mbar_inval(&P.bar[k]);
  }
  if (!grid_barrier(E)) return;
  ensemble_phase2(E, par, sEstep, n, sNe, sNi, sIt, sG, esm, sT);
}

// Self-test of the bounded waits (failure detection without a fault): a bulk-copy barrier
// that is told to expect bytes no copy will deliver, and a grid barrier that is told to expect
// one block more than the launch has.  Both must give up and record kStTimeout.
__global__ void k_selftest_waits(EnsDev* E, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1u);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16u);  // 16 bytes announced, none will arrive
    if (!mbar_wait(&bar, 0u, 200)) atomicOr(&status[0], kStTimeout);  // ~0.1 s of polls
  }
  __syncthreads();
  if (!grid_barrier(E, gridDim.x + 1u)) atomicOr(&status[1], kStTimeout);
}

cudaError_t launch_selftest_waits(EnsDev* E, int* status, cudaStream_t s) {
  k_selftest_waits<<<1, 32, 0, s>>>(E, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ launchers
size_t push32_smem_bytes(int nx) {
  return pipes_offset(nx) + sizeof(WarpPipe<kStagesRun>) * kWarps32;
}

cudaError_t launch_push_fp32(const DevCtx& K, int grid, cudaStream_t s) {
  return launch_chained(k_push_fp32, (unsigned)grid, (unsigned)kBlock, push32_smem_bytes(K.nx),
                        s, K);
}

cudaError_t launch_place_fp32(const DevCtx& K, int grid, cudaStream_t s) {
  return launch_chained(k_place_field<Fp32Moves>, (unsigned)grid, 256u,
                        place_run_smem_bytes(K.nx, K.nlist), s, K);
}

size_t ensemble_pipes_offset(int nx_max) { return pipes_offset(nx_max); }
size_t ensemble_smem_bytes(int nx_max, int gcap_max) {
  const size_t p1 = pipes_offset(nx_max) + sizeof(WarpPipe<kStagesEns>) * kWarps32;
  const size_t p2 = place_smem_bytes(nx_max, gcap_max);
  return p1 > p2 ? p1 : p2;
}

cudaError_t configure_ensemble(size_t smem) {
  return raise_smem_limit(k_ensemble_step, (int)smem);
}

int ensemble_blocks_per_sm(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ensemble_step, kBlock, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

// Cooperative launch: every block resident at once, so the grid barrier can complete.
cudaError_t launch_ensemble(EnsDev* E, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)kBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ensemble_step, E);
}

cudaError_t launch_convert(const DevCtx& K, int species, long long n, bool to_fp32,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = (unsigned)((n + 255) / 256);
  if (to_fp32)
    return launch_convert_from(K, species, n, K.x[species], K.vx[species], K.vy[species],
                               K.vz[species], K.id[species], s);
  k_to_fp64<<<g, 256, 0, s>>>(K, species, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_from(const DevCtx& K, int species, long long n, const double* x,
                                const double* vx, const double* vy, const double* vz,
                                const unsigned* id, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 2 * kDepositBlocks);
  k_to_fp32<<<(unsigned)blocks, 256, sizeof(unsigned long long) * K.nx, s>>>(K, species, n, x,
                                                                            vx, vy, vz, id);
  return cudaGetLastError();
}

cudaError_t launch_diag(const DevCtx& K, bool fp32, char* out_dev, const DiagOffsets& off,
                        cudaStream_t s) {
  const long long want = (K.cap + 255) / 256;
  const unsigned grid = (unsigned)(want < 1024 ? (want > 0 ? want : 1) : 1024);
  if (fp32)
    k_diag<true><<<grid, 256, 0, s>>>(K, out_dev, off);
  else
    k_diag<false><<<grid, 256, 0, s>>>(K, out_dev, off);
  return cudaGetLastError();
}

cudaError_t configure_kernels32(int nx) {
  cudaError_t e = raise_smem_limit(k_push_fp32, (int)push32_smem_bytes(nx));
  return e;
}

cudaError_t configure_place_fp32(int nx, int nlist) {
  return raise_smem_limit(k_place_field<Fp32Moves>, (int)place_run_smem_bytes(nx, nlist));
}

int push_fp32_blocks_per_sm(int nx) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_fp32, kBlock,
                                                    push32_smem_bytes(nx)) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace pic
