/*
 * pic_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the 1D3V PIC/MCC
 * timestep of Vass, Palla & Hartmann (arXiv 2109.04469), §2 steps 1-6.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code, header, table or constant
 * generator with the CUDA path; both implement the same written step contract
 * independently.  Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (the flag
 * matters: contracted multiply-adds would change the rounding).
 *
 * Every routine cites the passage of the paper it follows.  Where the paper is silent the
 * reading it takes is named (listed below).  Pins (tests that fix this code to something
 * other than itself) live in tests/test_oracle_*.py.
 *
 * Readings of the paper used in these sources (where §2 leaves a detail open; comments cite
 * them as "reading C-n"):
 *  C-1  N_c cells, N_x = N_c + 1 nodes, dx = L / N_c.
 *  C-2  Drive V(t_n) = V_rf cos(2 pi f n dt) on x = 0 at the start of step n; x = L grounded.
 *  C-3  Loaded velocities are taken at n - 1/2 (no half-step push back).
 *  C-4  Field at the electrodes from the half-cell Gauss law:
 *       E_0 = (phi_0 - phi_1)/dx - rho_0 dx/(2 eps0), E_N = (phi_N-1 - phi_N)/dx + rho_N dx/(2 eps0).
 *  C-5  An electrode node owns half a cell of volume.
 *  C-7  One null-collision trial per particle and step: a candidate if u < P_max =
 *       1 - exp(-nu_max dt).
 *  C-8  nu_max is the largest total collision frequency over the cross-section table.
 *  C-9  Electron elastic scattering: isotropic in the lab frame off a cold atom, with the
 *       recoil loss of a fraction (2 m_e / M)(1 - cos chi) of the energy.
 *  C-10 Ionization: the energy above threshold shared equally by the two electrons, both
 *       isotropic; the new ion drawn from the gas Maxwellian.
 *  C-11 An ion-induced electron starts at the struck electrode with see_energy_ev, isotropic
 *       into the gap.
 *  C-12 Absorbed iff x <= 0 or x >= L; a reflected electron has x mirrored and vx negated and
 *       is removed if still outside.
 *  C-13 Ar+ - Ar: isotropic scattering in the centre-of-mass frame, or charge transfer (the ion
 *       takes the sampled atom's velocity).
 *  C-14 Deposit in fixed point: 2^32 per superparticle, w_R = rint(f 2^32) (ties to even),
 *       w_L = 2^32 - w_R.
 *  C-15 Compaction: removed particles leave holes; births, ranked in particle order and given
 *       ids next_id + rank, fill the holes in rank order and then follow the last particle;
 *       survivors beyond the new count fill the holes that remain below it.
 *  C-16 Random numbers: Philox4x32-10, key (seed, instance), counter (id, step,
 *       species | purpose | block, 0).
 *  C-18 EEPF: electrons with |x - L/2| < dx/2, sampled every step.
 *  C-19 omega_pe and lambda_D from the time-averaged centre density and k T_e = (2/3) <eps>
 *       of the centre EEPF.
 *  C-20 N_D = n_e(L/2) A lambda_D / W, superparticles per Debye length.
 *  C-21 Gamma = W x ions absorbed at an electrode / (A x time), the mean of both electrodes.
 *  C-22 Initial load: x uniform in (0, L), Maxwellian velocities, ids 0 .. N-1.
 *  C-23 The tridiagonal Poisson system solved exactly through its discrete Green's function in
 *       integer arithmetic, each output value rounded once.
 *  C-XS Closed-form cross sections (Phelps' tables are not available): electron elastic,
 *       excitation at 11.55 eV, Lotz-type ionization at 15.76 eV; Ar+ - Ar isotropic and
 *       charge transfer.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants (CODATA 2018) */
#define Q_E 1.602176634e-19
#define M_EL 9.1093837015e-31
#define AMU 1.66053906660e-27
#define EPS_0 8.8541878128e-12
#define K_BOLTZ 1.380649e-23
#define E_EXC 11.55 /* eV, excitation threshold (C-XS) */
#define E_ION 15.76 /* eV, ionization threshold, §3.1 */
#define TWO32 4294967296.0
#define TWO20 1048576.0

#define XS_NODES 100001 /* eps_k = k/100 eV, 0..1000 eV */
#define XS_INV_DE 100.0
#define MAX_TRIES 64

/* status bits */
#define ORC_ST_CAPACITY 1
#define ORC_ST_NONFINITE 2

enum { SP_E = 0, SP_I = 1 };
enum { PUR_STEP = 0, PUR_COLL = 1, PUR_EMIT = 2, PUR_LOAD = 3 };
enum {
  CN_E_ABS_L = 0, CN_E_ABS_R, CN_I_ABS_L, CN_I_ABS_R, CN_E_REFL, CN_SEE, CN_E_ELA, CN_E_EXC,
  CN_E_ION, CN_I_ISO, CN_I_CX, CN_E_CAND, CN_I_CAND, CN_EEPF_N, CN_EEPF_ESUM, CN_DROPPED,
  N_COUNTERS
};

/* The oracle's own parameter record (the CUDA library declares its own). */
typedef struct {
  double gap_m, pressure_pa, gas_temp_k, v_rf_amp_v, f_rf_hz;
  int32_t steps_per_rf, n_cells;
  double weight, refl_e, gamma_see, area_m2, init_te_ev, see_energy_ev;
  int64_t init_per_species, capacity_per_species;
  uint64_t seed;
  uint32_t instance;
  int32_t eepf_bins;
  double eepf_emax_ev;
  int32_t fedf_bins;
  double fedf_emax_ev;
} orc_params;

typedef struct {
  orc_params p;
  /* derived quantities (§2), computed once in this order */
  int nc, nx;
  double dx, inv_dx, inv_2dx, dt, ng, qm_dt[2], emfac_e, spd2_e, mu, emfac_rel, spd2_rel,
      emfac_ilab, mr2, sig_e, sig_i, v_see, efac, rfac, den1, den2, mass[2];
  double *inv_den; /* Poisson pivots, index 1..nc-1 */
  double *vtab;    /* drive table, N_t entries */
  double *F[2];    /* cumulative collision fractions, XS_NODES x 4 */
  double numax[2], pmax[2];
  /* state */
  int64_t n[2], cap;
  uint32_t next_id[2];
  uint32_t step;
  double *x[2], *vx[2], *vy[2], *vz[2];
  uint32_t *id[2];
  int64_t *C[2];  /* counts at the current positions */
  double *phi, *E;
  /* accumulators */
  double *acc[2];
  int64_t steps_avg;
  uint64_t *eepf, *fedf[2];
  uint64_t cnt[N_COUNTERS];
  int status;
  /* scratch for one step */
  int64_t *holes[2];
  double *bx[2], *bvx[2], *bvy[2], *bvz[2]; /* births in rank order */
  int64_t nb[2];
  unsigned char *dead[2];
} orc_sim;

/* ------------------------------------------------------------ Philox4x32-10 (C-16)
 * Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11:
 * ten rounds of the 4x32 Philox bijection with the published multipliers and Weyl
 * key increments.  Replaces the paper's MT19937 (§2 step 5) so draws are addressable
 * by (particle id, step, purpose). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* two uniforms in (0,1) from one block: (2k+1)*2^-53 with k 52 bits */
static double u52(uint32_t hi, uint32_t lo) {
  uint64_t k = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);
  return (double)(2 * k + 1) * 0x1p-53;
}

typedef struct {
  uint32_t key[2];
  uint32_t id, step, base; /* base = species<<30 | purpose<<24 */
  uint32_t block;
} orc_stream;

static orc_stream stream_open(const orc_sim *S, int species, int purpose, uint32_t id,
                              uint32_t step) {
  orc_stream st;
  st.key[0] = (uint32_t)S->p.seed;
  st.key[1] = (uint32_t)(S->p.seed >> 32) ^ S->p.instance;
  st.id = id;
  st.step = step;
  st.base = ((uint32_t)species << 30) | ((uint32_t)purpose << 24);
  st.block = 0;
  return st;
}

static void stream_pair(orc_stream *st, double *ua, double *ub) {
  uint32_t c[4] = {st->id, st->step, st->base | st->block, 0u}, w[4];
  orc_philox4x32_10(c, st->key, w);
  st->block++;
  *ua = u52(w[0], w[1]);
  *ub = u52(w[2], w[3]);
}

void orc_uniform_pair(uint64_t seed, uint32_t instance, int species, int purpose, uint32_t id,
                      uint32_t step, uint32_t block, double out[2]) {
  orc_sim tmp;
  tmp.p.seed = seed;
  tmp.p.instance = instance;
  orc_stream st = stream_open(&tmp, species, purpose, id, step);
  st.block = block;
  stream_pair(&st, &out[0], &out[1]);
}

/* --------------------------------------------------------------- natural logarithm
 * Own implementation: binary-exponent argument reduction to
 * m in [sqrt(1/2), sqrt(2)) and the series ln m = 2 artanh t, t = (m-1)/(m+1),
 * summed to t^23.  Used only by the polar Gaussian sampler; the input is a positive
 * normal number there. */
double orc_log(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  int k = (int)((b >> 52) & 0x7ff) - 1023;
  uint64_t mb = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
  double m;
  memcpy(&m, &mb, sizeof m);
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    k = k + 1;
  }
  double t = (m - 1.0) / (m + 1.0);
  double t2 = t * t;
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

/* Marsaglia (1972) uniform direction on the sphere by rejection from the square. */
static void iso_dir(orc_stream *st, double n[3]) {
  for (int a = 0; a < MAX_TRIES; ++a) {
    double ua, ub;
    stream_pair(st, &ua, &ub);
    double v1 = 2.0 * ua - 1.0, v2 = 2.0 * ub - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s < 1.0) {
      double q = 2.0 * sqrt(1.0 - s);
      n[0] = v1 * q;
      n[1] = v2 * q;
      n[2] = 1.0 - 2.0 * s;
      return;
    }
  }
  n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
}

/* Marsaglia polar method: a pair of independent standard normal deviates. */
static void gauss_pair(orc_stream *st, double g[2]) {
  for (int a = 0; a < MAX_TRIES; ++a) {
    double ua, ub;
    stream_pair(st, &ua, &ub);
    double v1 = 2.0 * ua - 1.0, v2 = 2.0 * ub - 1.0;
    double s = v1 * v1 + v2 * v2;
    if (s < 1.0) {
      double fac = sqrt((-2.0 * orc_log(s)) / s);
      g[0] = v1 * fac;
      g[1] = v2 * fac;
      return;
    }
  }
  g[0] = 0.0; g[1] = 0.0;
}

static void maxwell3(orc_stream *st, double sig, double v[3]) {
  double a[2], b[2];
  gauss_pair(st, a);
  gauss_pair(st, b);
  v[0] = sig * a[0];
  v[1] = sig * a[1];
  v[2] = sig * b[0];
}

/* ------------------------------------------------------- cross sections (C-XS, §2 step 6)
 * The paper takes e-Ar and Ar+-Ar data from Phelps' compilations, which are not available
 * here; these closed forms keep its process list (elastic, one excitation at 11.55 eV,
 * ionization at 15.76 eV; isotropic and charge transfer for ions). */
double orc_sigma_e(int proc, double eps) {
  if (proc == 0) {
    double x = eps / 10.0;
    return 1e-20 * (6.0 * exp(-eps / 0.07) + 25.0 * (x * x) / pow(1.0 + x * x, 1.3));
  }
  if (proc == 1) {
    if (eps <= E_EXC) return 0.0;
    return 1.6e-20 * log(eps / E_EXC) / (eps / E_EXC);
  }
  if (eps <= E_ION) return 0.0; /* Lotz (1967), a = 4.5e-14 cm^2 eV^2, q = 6 */
  return 2.7e-17 * log(eps / E_ION) / (eps * E_ION);
}

/* sigma*g for Ar+-Ar as a function of the centre-of-mass energy eps [eV] */
double orc_sigma_g_i(int proc, double eps, double spd2_rel) {
  if (proc == 0) return 1e-19 * sqrt((0.5 + eps) * spd2_rel) / sqrt(1.0 + eps / 100.0);
  if (eps <= 0.0) return 0.0;
  double a = 7.0 - 0.55 * log(eps);
  return 1e-20 * (a * a) * sqrt(eps * spd2_rel);
}

/* nu tables and nu_max (C-8), cumulative fractions stored per node */
static void build_tables(orc_sim *S) {
  for (int s = 0; s < 2; ++s) {
    double *nu = (double *)malloc(sizeof(double) * XS_NODES * 3);
    double numax = 0.0;
    for (int k = 0; k < XS_NODES; ++k) {
      double eps = (double)k / XS_INV_DE;
      if (s == SP_E) {
        double v = sqrt(eps * S->spd2_e);
        for (int m = 0; m < 3; ++m) nu[3 * k + m] = S->ng * orc_sigma_e(m, eps) * v;
      } else {
        nu[3 * k + 0] = S->ng * orc_sigma_g_i(0, eps, S->spd2_rel);
        nu[3 * k + 1] = S->ng * orc_sigma_g_i(1, eps, S->spd2_rel);
        nu[3 * k + 2] = 0.0;
      }
      double tot = (nu[3 * k] + nu[3 * k + 1]) + nu[3 * k + 2];
      if (tot > numax) numax = tot;
    }
    S->numax[s] = numax;
    S->pmax[s] = 1.0 - exp(-numax * S->dt); /* §3.5 */
    double *F = S->F[s];
    for (int k = 0; k < XS_NODES; ++k) {
      double c1 = nu[3 * k];
      double c2 = c1 + nu[3 * k + 1];
      double c3 = c2 + nu[3 * k + 2];
      /* a gas-free run (n_g = 0) has nu_max = 0: no candidate is ever drawn */
      F[4 * k + 0] = numax > 0.0 ? c1 / numax : 0.0;
      F[4 * k + 1] = numax > 0.0 ? c2 / numax : 0.0;
      F[4 * k + 2] = numax > 0.0 ? c3 / numax : 0.0;
      F[4 * k + 3] = 0.0;
    }
    free(nu);
  }
}

/* piecewise-linear interpolant of the cumulative fractions between table nodes */
static void lookup(const double *F, double eps, double out[3]) {
  double t = eps * XS_INV_DE;
  double kf = floor(t);
  if (!(kf < (double)(XS_NODES - 1))) { /* also catches a non-finite energy */
    const double *a = F + 4 * (XS_NODES - 1);
    out[0] = a[0]; out[1] = a[1]; out[2] = a[2];
    return;
  }
  int64_t k = (int64_t)kf;
  double fr = t - kf;
  const double *a = F + 4 * k, *b = F + 4 * (k + 1);
  for (int m = 0; m < 3; ++m) out[m] = a[m] + fr * (b[m] - a[m]);
}

/* -------------------------------------------------------------- linear weighting (§2 step 1,3) */
static int64_t cell_of(const orc_sim *S, double x, double *f) {
  double xn = x * S->inv_dx;
  double jf = floor(xn);
  int64_t j = (int64_t)jf;
  if (j > S->nc - 1) j = S->nc - 1;
  if (j < 0) j = 0;
  *f = xn - (double)j;
  return j;
}

static void deposit(const orc_sim *S, int64_t *C, double x) {
  double f;
  int64_t j = cell_of(S, x, &f);
  int64_t wr = llrint(f * TWO32); /* round half to even (default rounding mode) */
  int64_t wl = (int64_t)4294967296LL - wr;
  C[j] += wl;
  C[j + 1] += wr;
}

/* ----------------------------------------------------------------- field (§2 step 2) */
/* The Thomas algorithm named in §2 step 2, on the constant tridiagonal matrix (-1, 2, -1)
 * with pivots precomputed: kept as the pin of field() below (both solve the same system). */
void orc_thomas_phi(const orc_sim *S, double V, double *phi) {
  int nc = S->nc;
  const int64_t *Ce = S->C[SP_E], *Ci = S->C[SP_I];
  double *g = (double *)malloc(sizeof(double) * (size_t)(nc + 1));
  phi[0] = V;
  phi[nc] = 0.0;
  for (int j = 1; j <= nc - 1; ++j) {
    double r = (double)(Ci[j] - Ce[j]) * S->rfac;
    if (j == 1)
      g[j] = (r + V) * S->inv_den[j];
    else
      g[j] = (r + g[j - 1]) * S->inv_den[j];
  }
  for (int j = nc - 1; j >= 1; --j) {
    if (j == nc - 1)
      phi[j] = g[j];
    else
      phi[j] = g[j] + S->inv_den[j] * phi[j + 1];
  }
  free(g);
}

/* §2 step 2 (reading C-23).  The finite-difference system 2 phi_j - phi_{j-1} - phi_{j+1} =
 * r_j (j = 1..N-1), phi_0 = V, phi_N = 0, r_j = rfac (C_i,j - C_e,j), has the solution
 *   phi_j = V (N-j)/N + sum_k G(j,k) r_k,  G(j,k) = min(j,k) (N - max(j,k)) / N
 * (the discrete Green's function of the Dirichlet matrix).  With integer counts,
 *   S_j = N sum_k G(j,k) dC_k = (N-j) sum_{k<=j} k dC_k + j sum_{k>j} (N-k) dC_k
 * is an exact integer, so phi_j = (V (N-j) + rfac S_j) / N rounds once.  The field follows
 * from the same exact sums: E_j = N(phi_{j-1} - phi_{j+1}) / (2 N dx) inside, and the
 * half-cell Gauss law at the electrodes (reading C-4). */
static void field(orc_sim *S, double V, int accumulate) {
  const int N = S->nc;
  const int64_t *Ce = S->C[SP_E], *Ci = S->C[SP_I];
  __int128 *A = (__int128 *)malloc(sizeof(__int128) * (size_t)(N + 1));
  __int128 *B = (__int128 *)malloc(sizeof(__int128) * (size_t)(N + 1));
  __int128 *Sg = (__int128 *)malloc(sizeof(__int128) * (size_t)(N + 1));
  A[0] = 0;
  for (int k = 1; k <= N - 1; ++k) A[k] = A[k - 1] + (__int128)k * (__int128)(Ci[k] - Ce[k]);
  A[N] = A[N - 1];
  B[N] = 0;
  B[N - 1] = 0;
  for (int k = N - 2; k >= 0; --k)
    B[k] = B[k + 1] + (__int128)(N - (k + 1)) * (__int128)(Ci[k + 1] - Ce[k + 1]);
  for (int j = 0; j <= N; ++j) Sg[j] = (__int128)(N - j) * A[j] + (__int128)j * B[j];
  double *phi = S->phi, *E = S->E;
  phi[0] = V;
  phi[N] = 0.0;
  for (int j = 1; j <= N - 1; ++j)
    phi[j] = (V * (double)(N - j) + S->rfac * (double)Sg[j]) / (double)N;
  for (int j = 1; j <= N - 1; ++j)
    E[j] = (2.0 * V + S->rfac * (double)(Sg[j - 1] - Sg[j + 1])) / S->den2;
  E[0] = (V - S->rfac * (double)(Sg[1] + (__int128)N * (__int128)(Ci[0] - Ce[0]))) / S->den1;
  E[N] = (V + S->rfac * (double)(Sg[N - 1] + (__int128)N * (__int128)(Ci[N] - Ce[N]))) / S->den1;
  free(A);
  free(B);
  free(Sg);
  if (accumulate) {
    for (int j = 0; j <= N; ++j) {
      S->acc[SP_E][j] += (double)Ce[j];
      S->acc[SP_I][j] += (double)Ci[j];
    }
    S->steps_avg += 1;
  }
}

/* ------------------------------------------------------------------ construction */
static void derive(orc_sim *S) {
  const orc_params *p = &S->p;
  S->nc = p->n_cells;
  S->nx = p->n_cells + 1;
  S->dx = p->gap_m / (double)p->n_cells;
  S->inv_dx = 1.0 / S->dx;
  S->inv_2dx = 0.5 * S->inv_dx;
  S->dt = 1.0 / (p->f_rf_hz * (double)p->steps_per_rf);
  S->ng = p->pressure_pa / (K_BOLTZ * p->gas_temp_k);
  S->mass[SP_E] = M_EL;
  S->mass[SP_I] = 39.948 * AMU;
  S->qm_dt[SP_E] = (-Q_E / M_EL) * S->dt;
  S->qm_dt[SP_I] = (Q_E / S->mass[SP_I]) * S->dt;
  S->emfac_e = (0.5 * M_EL) / Q_E;
  S->spd2_e = (2.0 * Q_E) / M_EL;
  S->mu = 0.5 * S->mass[SP_I];
  S->emfac_rel = (0.5 * S->mu) / Q_E;
  S->spd2_rel = (2.0 * Q_E) / S->mu;
  S->emfac_ilab = (0.5 * S->mass[SP_I]) / Q_E;
  S->mr2 = (2.0 * M_EL) / S->mass[SP_I];
  S->sig_e = sqrt((p->init_te_ev * Q_E) / M_EL);
  S->sig_i = sqrt((K_BOLTZ * p->gas_temp_k) / S->mass[SP_I]);
  S->v_see = sqrt(p->see_energy_ev * S->spd2_e);
  S->efac = (Q_E * p->weight) / ((p->area_m2 * EPS_0) * TWO32);
  S->rfac = S->efac * S->dx;
  S->den1 = S->dx * (double)S->nc;
  S->den2 = (2.0 * S->dx) * (double)S->nc;
  S->inv_den = (double *)calloc((size_t)S->nc + 1, sizeof(double));
  double den = 2.0;
  for (int j = 1; j <= S->nc - 1; ++j) {
    S->inv_den[j] = 1.0 / den;
    den = 2.0 - S->inv_den[j];
  }
  S->vtab = (double *)malloc(sizeof(double) * (size_t)p->steps_per_rf);
  for (int k = 0; k < p->steps_per_rf; ++k)
    S->vtab[k] = p->v_rf_amp_v * cos((6.283185307179586 * (double)k) / (double)p->steps_per_rf);
}

static void redeposit(orc_sim *S, int s) {
  memset(S->C[s], 0, sizeof(int64_t) * (size_t)S->nx);
  for (int64_t q = 0; q < S->n[s]; ++q) deposit(S, S->C[s], S->x[s][q]);
}

orc_sim *orc_create(const orc_params *p) {
  if (p->n_cells < 2 || p->steps_per_rf < 1 || p->capacity_per_species < p->init_per_species ||
      p->init_per_species < 0 || p->eepf_bins < 1 || p->fedf_bins < 1)
    return NULL;
  orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
  S->p = *p;
  derive(S);
  S->cap = p->capacity_per_species;
  for (int s = 0; s < 2; ++s) {
    size_t c = (size_t)S->cap + 1;
    S->x[s] = (double *)calloc(c, sizeof(double));
    S->vx[s] = (double *)calloc(c, sizeof(double));
    S->vy[s] = (double *)calloc(c, sizeof(double));
    S->vz[s] = (double *)calloc(c, sizeof(double));
    S->id[s] = (uint32_t *)calloc(c, sizeof(uint32_t));
    S->C[s] = (int64_t *)calloc((size_t)S->nx, sizeof(int64_t));
    S->acc[s] = (double *)calloc((size_t)S->nx, sizeof(double));
    S->F[s] = (double *)malloc(sizeof(double) * XS_NODES * 4);
    S->fedf[s] = (uint64_t *)calloc((size_t)p->fedf_bins, sizeof(uint64_t));
    S->holes[s] = (int64_t *)malloc(sizeof(int64_t) * c);
    S->bx[s] = (double *)malloc(sizeof(double) * 2 * c);
    S->bvx[s] = (double *)malloc(sizeof(double) * 2 * c);
    S->bvy[s] = (double *)malloc(sizeof(double) * 2 * c);
    S->bvz[s] = (double *)malloc(sizeof(double) * 2 * c);
  }
  S->dead[0] = (unsigned char *)malloc((size_t)S->cap + 1);
  S->dead[1] = (unsigned char *)malloc((size_t)S->cap + 1);
  S->phi = (double *)calloc((size_t)S->nx, sizeof(double));
  S->E = (double *)calloc((size_t)S->nx, sizeof(double));
  S->eepf = (uint64_t *)calloc((size_t)p->eepf_bins, sizeof(uint64_t));
  build_tables(S);
  /* initial load (C-22): uniform x, Maxwellian v, ids 0..N-1, stream step 0xFFFFFFFF */
  for (int s = 0; s < 2; ++s) {
    double sig = (s == SP_E) ? S->sig_e : S->sig_i;
    for (int64_t q = 0; q < p->init_per_species; ++q) {
      orc_stream st = stream_open(S, s, PUR_LOAD, (uint32_t)q, 0xFFFFFFFFu);
      double ua, ub, v[3];
      stream_pair(&st, &ua, &ub);
      maxwell3(&st, sig, v);
      S->x[s][q] = ua * p->gap_m;
      S->vx[s][q] = v[0];
      S->vy[s][q] = v[1];
      S->vz[s][q] = v[2];
      S->id[s][q] = (uint32_t)q;
    }
    S->n[s] = p->init_per_species;
    S->next_id[s] = (uint32_t)p->init_per_species;
    redeposit(S, s);
  }
  return S;
}

void orc_destroy(orc_sim *S) {
  if (!S) return;
  for (int s = 0; s < 2; ++s) {
    free(S->x[s]); free(S->vx[s]); free(S->vy[s]); free(S->vz[s]); free(S->id[s]);
    free(S->C[s]); free(S->acc[s]); free(S->F[s]); free(S->fedf[s]); free(S->holes[s]);
    free(S->bx[s]); free(S->bvx[s]); free(S->bvy[s]); free(S->bvz[s]);
  }
  free(S->dead[0]); free(S->dead[1]); free(S->phi); free(S->E); free(S->eepf); free(S->inv_den); free(S->vtab);
  free(S);
}

/* --------------------------------------------------------------------- one timestep */
static void add_birth(orc_sim *S, int s, double x, double vx, double vy, double vz) {
  int64_t b = S->nb[s]++;
  S->bx[s][b] = x;
  S->bvx[s][b] = vx;
  S->bvy[s][b] = vy;
  S->bvz[s][b] = vz;
}

static void fedf_add(orc_sim *S, int s, double eps) {
  double t = floor(eps * ((double)S->p.fedf_bins / S->p.fedf_emax_ev));
  if (t < (double)S->p.fedf_bins) S->fedf[s][(int64_t)t] += 1;
}

/* §2 step 6 for one electron (C-7, C-9, C-10); returns nothing, may append births */
static void collide_electron(orc_sim *S, int64_t q, int64_t *Cn_e, int64_t *Cn_i) {
  double *vx = &S->vx[SP_E][q], *vy = &S->vy[SP_E][q], *vz = &S->vz[SP_E][q];
  double v2 = ((*vx) * (*vx) + (*vy) * (*vy)) + (*vz) * (*vz);
  double eps = v2 * S->emfac_e;
  double F[3];
  lookup(S->F[SP_E], eps, F);
  orc_stream st = stream_open(S, SP_E, PUR_COLL, S->id[SP_E][q], S->step);
  double up, unused;
  stream_pair(&st, &up, &unused);
  S->cnt[CN_E_CAND] += 1;
  if (up < F[0]) { /* elastic, isotropic in the lab frame, cold target */
    double n[3];
    iso_dir(&st, n);
    double vmag = sqrt(v2);
    double cosx = (vmag > 0.0) ? (((*vx) * n[0] + (*vy) * n[1]) + (*vz) * n[2]) / vmag : 0.0;
    double sp = vmag * sqrt(1.0 - S->mr2 * (1.0 - cosx));
    *vx = n[0] * sp; *vy = n[1] * sp; *vz = n[2] * sp;
    S->cnt[CN_E_ELA] += 1;
  } else if (up < F[1]) { /* excitation */
    if (eps >= E_EXC) {
      double n[3];
      iso_dir(&st, n);
      double sp = sqrt((eps - E_EXC) * S->spd2_e);
      *vx = n[0] * sp; *vy = n[1] * sp; *vz = n[2] * sp;
      S->cnt[CN_E_EXC] += 1;
    }
  } else if (up < F[2]) { /* ionization */
    if (eps >= E_ION) {
      double n1[3], n2[3], vi[3];
      iso_dir(&st, n1);
      iso_dir(&st, n2);
      maxwell3(&st, S->sig_i, vi);
      double e1 = 0.5 * (eps - E_ION);
      double sp = sqrt(e1 * S->spd2_e);
      *vx = n1[0] * sp; *vy = n1[1] * sp; *vz = n1[2] * sp;
      double xb = S->x[SP_E][q];
      add_birth(S, SP_E, xb, n2[0] * sp, n2[1] * sp, n2[2] * sp);
      add_birth(S, SP_I, xb, vi[0], vi[1], vi[2]);
      deposit(S, Cn_e, xb);
      deposit(S, Cn_i, xb);
      S->cnt[CN_E_ION] += 1;
    }
  }
}

/* §2 step 6 for one ion (C-13): moving-target null collision */
static void collide_ion(orc_sim *S, int64_t q) {
  double *vx = &S->vx[SP_I][q], *vy = &S->vy[SP_I][q], *vz = &S->vz[SP_I][q];
  orc_stream st = stream_open(S, SP_I, PUR_COLL, S->id[SP_I][q], S->step);
  double up, unused, vn[3];
  stream_pair(&st, &up, &unused);
  maxwell3(&st, S->sig_i, vn);
  double gx = *vx - vn[0], gy = *vy - vn[1], gz = *vz - vn[2];
  double g2 = (gx * gx + gy * gy) + gz * gz;
  double eps = g2 * S->emfac_rel;
  double F[3];
  lookup(S->F[SP_I], eps, F);
  S->cnt[CN_I_CAND] += 1;
  if (up < F[0]) { /* isotropic scattering in the centre-of-mass frame, equal masses */
    double n[3];
    iso_dir(&st, n);
    double hg = 0.5 * sqrt(g2);
    *vx = 0.5 * (*vx + vn[0]) + n[0] * hg;
    *vy = 0.5 * (*vy + vn[1]) + n[1] * hg;
    *vz = 0.5 * (*vz + vn[2]) + n[2] * hg;
    S->cnt[CN_I_ISO] += 1;
  } else if (up < F[1]) { /* charge transfer: the ion takes the neutral's velocity */
    *vx = vn[0]; *vy = vn[1]; *vz = vn[2];
    S->cnt[CN_I_CX] += 1;
  }
}

static void compact(orc_sim *S, int s) {
  int64_t N = S->n[s], H = 0, B = S->nb[s];
  int64_t *holes = S->holes[s];
  for (int64_t q = 0; q < N; ++q)
    if (S->dead[s][q]) holes[H++] = q;
  int64_t Beff = B;
  if (N - H + B > S->cap) {
    Beff = S->cap - (N - H);
    S->status |= ORC_ST_CAPACITY;
    S->cnt[CN_DROPPED] += (uint64_t)(B - Beff);
  }
  for (int64_t r = 0; r < Beff; ++r) {
    int64_t d = (r < H) ? holes[r] : N + r - H;
    S->x[s][d] = S->bx[s][r];
    S->vx[s][d] = S->bvx[s][r];
    S->vy[s][d] = S->bvy[s][r];
    S->vz[s][d] = S->bvz[s][r];
    S->id[s][d] = S->next_id[s] + (uint32_t)r;
  }
  S->next_id[s] += (uint32_t)Beff;
  int64_t Nn = N - H + Beff;
  if (H > Beff) {
    /* tail survivors at indices >= Nn fill the remaining holes below Nn, ascending */
    int64_t hk = Beff;
    for (int64_t t = Nn; t < N; ++t) {
      if (S->dead[s][t]) continue;
      int64_t d = holes[hk++];
      S->x[s][d] = S->x[s][t];
      S->vx[s][d] = S->vx[s][t];
      S->vy[s][d] = S->vy[s][t];
      S->vz[s][d] = S->vz[s][t];
      S->id[s][d] = S->id[s][t];
    }
  }
  S->n[s] = Nn;
}

static void process_species(orc_sim *S, int s, int64_t *Cn[2]) {
  const orc_params *p = &S->p;
  double L = p->gap_m;
  int64_t N = S->n[s];
  unsigned char *dead = S->dead[s];
  memset(dead, 0, (size_t)N + 1);
  for (int64_t q = 0; q < N; ++q) {
    orc_stream st = stream_open(S, s, PUR_STEP, S->id[s][q], S->step);
    double u_null, u_wall;
    stream_pair(&st, &u_null, &u_wall);
    /* §2 steps 3-4: linear gather and leapfrog */
    double f;
    int64_t j = cell_of(S, S->x[s][q], &f);
    double Ep = (1.0 - f) * S->E[j] + f * S->E[j + 1];
    S->vx[s][q] = S->vx[s][q] + S->qm_dt[s] * Ep;
    S->x[s][q] = S->x[s][q] + S->vx[s][q] * S->dt;
    if (!isfinite(S->vx[s][q])) S->status |= ORC_ST_NONFINITE;
    double x = S->x[s][q];
    /* §2 step 5: surfaces (C-11, C-12) */
    if (x <= 0.0 || x >= L) {
      int left = (x <= 0.0);
      if (s == SP_E) {
        int removed = 1;
        if (u_wall < p->refl_e) {
          S->x[s][q] = left ? -x : 2.0 * L - x;
          S->vx[s][q] = -S->vx[s][q];
          S->cnt[CN_E_REFL] += 1;
          removed = (S->x[s][q] <= 0.0 || S->x[s][q] >= L);
        }
        if (removed) {
          dead[q] = 1;
          S->cnt[left ? CN_E_ABS_L : CN_E_ABS_R] += 1;
          double v2 = (S->vx[s][q] * S->vx[s][q] + S->vy[s][q] * S->vy[s][q]) +
                      S->vz[s][q] * S->vz[s][q];
          fedf_add(S, SP_E, v2 * S->emfac_e);
        }
      } else {
        dead[q] = 1;
        S->cnt[left ? CN_I_ABS_L : CN_I_ABS_R] += 1;
        double v2 = (S->vx[s][q] * S->vx[s][q] + S->vy[s][q] * S->vy[s][q]) +
                    S->vz[s][q] * S->vz[s][q];
        fedf_add(S, SP_I, v2 * S->emfac_ilab);
        if (u_wall < p->gamma_see) {
          orc_stream se = stream_open(S, SP_I, PUR_EMIT, S->id[s][q], S->step);
          double n[3];
          iso_dir(&se, n);
          double ax = fabs(n[0]) * S->v_see;
          double xb = left ? 0.0 : L;
          add_birth(S, SP_E, xb, left ? ax : -ax, n[1] * S->v_see, n[2] * S->v_see);
          deposit(S, Cn[SP_E], xb);
          S->cnt[CN_SEE] += 1;
        }
      }
    }
    if (dead[q]) continue;
    /* §2 step 6: null-collision Monte Carlo */
    if (u_null < S->pmax[s]) {
      if (s == SP_E)
        collide_electron(S, q, Cn[SP_E], Cn[SP_I]);
      else
        collide_ion(S, q);
    }
    /* §2 step 1 for the next step: linear deposit at x^{n+1} */
    deposit(S, Cn[s], S->x[s][q]);
    /* EEPF sample at the centre (C-18) */
    if (s == SP_E) {
      double d = S->x[s][q] - 0.5 * L;
      double h = 0.5 * S->dx;
      if (d > -h && d < h) {
        double v2 = (S->vx[s][q] * S->vx[s][q] + S->vy[s][q] * S->vy[s][q]) +
                    S->vz[s][q] * S->vz[s][q];
        double eps = v2 * S->emfac_e;
        double t = floor(eps * ((double)p->eepf_bins / p->eepf_emax_ev));
        if (t < (double)p->eepf_bins) S->eepf[(int64_t)t] += 1;
        S->cnt[CN_EEPF_N] += 1;
        S->cnt[CN_EEPF_ESUM] += (uint64_t)llrint(eps * TWO20);
      }
    }
  }
}

int orc_step(orc_sim *S, int64_t nsteps) {
  for (int64_t it = 0; it < nsteps; ++it) {
    double V = S->vtab[S->step % (uint32_t)S->p.steps_per_rf]; /* C-2 */
    field(S, V, 1);
    int64_t *Cn[2];
    for (int s = 0; s < 2; ++s) Cn[s] = (int64_t *)calloc((size_t)S->nx, sizeof(int64_t));
    S->nb[SP_E] = 0;
    S->nb[SP_I] = 0;
    /* electrons, then ions; electron births = ionization births then gamma electrons */
    process_species(S, SP_E, Cn);
    process_species(S, SP_I, Cn);
    compact(S, SP_E);
    compact(S, SP_I);
    for (int s = 0; s < 2; ++s) {
      memcpy(S->C[s], Cn[s], sizeof(int64_t) * (size_t)S->nx);
      free(Cn[s]);
    }
    S->step += 1;
  }
  return S->status;
}

/* ------------------------------------------------------------------ accessors */
int64_t orc_count(const orc_sim *S, int s) { return S->n[s]; }
uint32_t orc_next_id(const orc_sim *S, int s) { return S->next_id[s]; }
uint32_t orc_step_index(const orc_sim *S) { return S->step; }
int orc_status(const orc_sim *S) { return S->status; }

int64_t orc_get_particles(const orc_sim *S, int s, double *x, double *vx, double *vy, double *vz,
                          uint32_t *id, int64_t cap) {
  int64_t n = S->n[s] < cap ? S->n[s] : cap;
  memcpy(x, S->x[s], sizeof(double) * (size_t)n);
  memcpy(vx, S->vx[s], sizeof(double) * (size_t)n);
  memcpy(vy, S->vy[s], sizeof(double) * (size_t)n);
  memcpy(vz, S->vz[s], sizeof(double) * (size_t)n);
  memcpy(id, S->id[s], sizeof(uint32_t) * (size_t)n);
  return S->n[s];
}

/* replace the particles of one species and redeposit its charge (§2 step 1) */
int orc_set_particles(orc_sim *S, int s, const double *x, const double *vx, const double *vy,
                      const double *vz, const uint32_t *id, int64_t n, uint32_t next_id) {
  if (n < 0 || n > S->cap) return -1;
  memcpy(S->x[s], x, sizeof(double) * (size_t)n);
  memcpy(S->vx[s], vx, sizeof(double) * (size_t)n);
  memcpy(S->vy[s], vy, sizeof(double) * (size_t)n);
  memcpy(S->vz[s], vz, sizeof(double) * (size_t)n);
  memcpy(S->id[s], id, sizeof(uint32_t) * (size_t)n);
  S->n[s] = n;
  S->next_id[s] = next_id;
  redeposit(S, s);
  return 0;
}

void orc_set_step(orc_sim *S, uint32_t step) { S->step = step; }

/* field of the current charge at V(t_step), without touching the accumulators */
void orc_solve_field(orc_sim *S) {
  field(S, S->vtab[S->step % (uint32_t)S->p.steps_per_rf], 0);
}

void orc_get_grid(const orc_sim *S, int64_t *Ce, int64_t *Ci, double *phi, double *E) {
  memcpy(Ce, S->C[SP_E], sizeof(int64_t) * (size_t)S->nx);
  memcpy(Ci, S->C[SP_I], sizeof(int64_t) * (size_t)S->nx);
  memcpy(phi, S->phi, sizeof(double) * (size_t)S->nx);
  memcpy(E, S->E, sizeof(double) * (size_t)S->nx);
}

/* raw accumulators: acc_e, acc_i [nx], eepf [eepf_bins], fedf_e, fedf_i [fedf_bins],
   counters [16]; returns the number of averaged steps */
int64_t orc_get_accum(const orc_sim *S, double *acc_e, double *acc_i, uint64_t *eepf,
                      uint64_t *fedf_e, uint64_t *fedf_i, uint64_t *counters) {
  memcpy(acc_e, S->acc[SP_E], sizeof(double) * (size_t)S->nx);
  memcpy(acc_i, S->acc[SP_I], sizeof(double) * (size_t)S->nx);
  memcpy(eepf, S->eepf, sizeof(uint64_t) * (size_t)S->p.eepf_bins);
  memcpy(fedf_e, S->fedf[SP_E], sizeof(uint64_t) * (size_t)S->p.fedf_bins);
  memcpy(fedf_i, S->fedf[SP_I], sizeof(uint64_t) * (size_t)S->p.fedf_bins);
  memcpy(counters, S->cnt, sizeof(uint64_t) * N_COUNTERS);
  return S->steps_avg;
}

void orc_reset_averages(orc_sim *S) {
  for (int s = 0; s < 2; ++s) {
    memset(S->acc[s], 0, sizeof(double) * (size_t)S->nx);
    memset(S->fedf[s], 0, sizeof(uint64_t) * (size_t)S->p.fedf_bins);
  }
  memset(S->eepf, 0, sizeof(uint64_t) * (size_t)S->p.eepf_bins);
  memset(S->cnt, 0, sizeof S->cnt);
  S->steps_avg = 0;
}

/* derived constants for the pins: dt, dx, ng, numax_e, numax_i, pmax_e, pmax_i, efac, rfac,
   qm_dt_e, qm_dt_i, emfac_e, spd2_e, emfac_rel, spd2_rel, sig_e, sig_i, v_see, mr2 */
void orc_get_derived(const orc_sim *S, double *out) {
  double d[19] = {S->dt, S->dx, S->ng, S->numax[0], S->numax[1], S->pmax[0], S->pmax[1],
                  S->efac, S->rfac, S->qm_dt[0], S->qm_dt[1], S->emfac_e, S->spd2_e,
                  S->emfac_rel, S->spd2_rel, S->sig_e, S->sig_i, S->v_see, S->mr2};
  memcpy(out, d, sizeof d);
}

/* pins: replace a species' cumulative table (XS_NODES x 4) and nu_max */
void orc_override_table(orc_sim *S, int s, const double *F, double numax) {
  memcpy(S->F[s], F, sizeof(double) * XS_NODES * 4);
  S->numax[s] = numax;
  S->pmax[s] = 1.0 - exp(-numax * S->dt);
}

void orc_get_table(const orc_sim *S, int s, double *F) {
  memcpy(F, S->F[s], sizeof(double) * XS_NODES * 4);
}

/* pins: the oracle's Gaussian / direction samplers on one stream */
void orc_sample_dirs(uint64_t seed, uint32_t instance, uint32_t id0, int64_t n, double *out) {
  orc_sim tmp;
  tmp.p.seed = seed;
  tmp.p.instance = instance;
  for (int64_t q = 0; q < n; ++q) {
    orc_stream st = stream_open(&tmp, 0, PUR_COLL, id0 + (uint32_t)q, 0);
    iso_dir(&st, out + 3 * q);
  }
}

void orc_sample_gauss(uint64_t seed, uint32_t instance, uint32_t id0, int64_t n, double *out) {
  orc_sim tmp;
  tmp.p.seed = seed;
  tmp.p.instance = instance;
  for (int64_t q = 0; q < n; ++q) {
    orc_stream st = stream_open(&tmp, 0, PUR_COLL, id0 + (uint32_t)q, 0);
    gauss_pair(&st, out + 2 * q);
  }
}

/* pins: overwrite the charge counts that the next field solve reads */
void orc_set_counts(orc_sim *S, const int64_t *Ce, const int64_t *Ci) {
  memcpy(S->C[SP_E], Ce, sizeof(int64_t) * (size_t)S->nx);
  memcpy(S->C[SP_I], Ci, sizeof(int64_t) * (size_t)S->nx);
}
