// pic_capi.cu -- the C-ABI of libpic (include/pic.h): parameter checks, the derived
// constants and host tables of the step contract, workspace layout, launches, diagnostics.
//
// Host arithmetic that feeds the FP64 kernels (constants, pivots, drive and collision
// tables) is compiled with -ffp-contract=off and follows the contract's operation order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "pic.h"
#include "pic_dev.cuh"
#include "pic_launch.h"

namespace {

using namespace pic;

// CODATA 2018
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKb = 1.380649e-23;
constexpr double kTwo32 = 4294967296.0;

// Closed-form cross sections of the project (reading C-XS; Phelps' data of §2 step 6 is not
// available).  eps in eV, sigma in m^2.
double sigma_e(int proc, double eps) {
  if (proc == 0) {
    const double x = eps / 10.0;
    return 1e-20 * (6.0 * std::exp(-eps / 0.07) + 25.0 * (x * x) / std::pow(1.0 + x * x, 1.3));
  }
  if (proc == 1) {
    if (eps <= kEExc) return 0.0;
    return 1.6e-20 * std::log(eps / kEExc) / (eps / kEExc);
  }
  if (eps <= kEIon) return 0.0;  // Lotz (1967), a = 4.5e-14 cm^2 eV^2, q = 6
  return 2.7e-17 * std::log(eps / kEIon) / (eps * kEIon);
}

// sigma * g of Ar+ - Ar against the centre-of-mass energy eps (eV)
double sigma_g_i(int proc, double eps, double spd2_rel) {
  if (proc == 0) return 1e-19 * std::sqrt((0.5 + eps) * spd2_rel) / std::sqrt(1.0 + eps / 100.0);
  if (eps <= 0.0) return 0.0;
  const double a = 7.0 - 0.55 * std::log(eps);
  return 1e-20 * (a * a) * std::sqrt(eps * spd2_rel);
}

struct Derived {
  double dx, inv_dx, inv_2dx, dt, ng, qm_dt[2], emfac_e, spd2_e, mu, emfac_rel, spd2_rel,
      emfac_ilab, mr2, sig_e, sig_i, v_see, efac, rfac, mi;
  double numax[2], pmax[2];
};

Derived derive(const pic_params& p) {
  Derived d;
  d.dx = p.gap_m / (double)p.n_cells;
  d.inv_dx = 1.0 / d.dx;
  d.inv_2dx = 0.5 * d.inv_dx;
  d.dt = 1.0 / (p.f_rf_hz * (double)p.steps_per_rf);
  d.ng = p.pressure_pa / (kKb * p.gas_temp_k);
  d.mi = 39.948 * kAmu;
  d.qm_dt[0] = (-kQe / kMe) * d.dt;
  d.qm_dt[1] = (kQe / d.mi) * d.dt;
  d.emfac_e = (0.5 * kMe) / kQe;
  d.spd2_e = (2.0 * kQe) / kMe;
  d.mu = 0.5 * d.mi;
  d.emfac_rel = (0.5 * d.mu) / kQe;
  d.spd2_rel = (2.0 * kQe) / d.mu;
  d.emfac_ilab = (0.5 * d.mi) / kQe;
  d.mr2 = (2.0 * kMe) / d.mi;
  d.sig_e = std::sqrt((p.init_te_ev * kQe) / kMe);
  d.sig_i = std::sqrt((kKb * p.gas_temp_k) / d.mi);
  d.v_see = std::sqrt(p.see_energy_ev * d.spd2_e);
  d.efac = (kQe * p.weight) / ((p.area_m2 * kEps0) * kTwo32);
  d.rfac = d.efac * d.dx;
  return d;
}

// nu_m at the table nodes, nu_max (reading C-8), cumulative fractions [k][4]
void build_tables(Derived& d, std::vector<double>& Fe, std::vector<double>& Fi) {
  std::vector<double> nu((size_t)kXsNodes * 3);
  for (int s = 0; s < 2; ++s) {
    double numax = 0.0;
    for (int k = 0; k < kXsNodes; ++k) {
      const double eps = (double)k / kXsInvDe;
      double* n = &nu[(size_t)3 * k];
      if (s == 0) {
        const double v = std::sqrt(eps * d.spd2_e);
        for (int m = 0; m < 3; ++m) n[m] = d.ng * sigma_e(m, eps) * v;
      } else {
        n[0] = d.ng * sigma_g_i(0, eps, d.spd2_rel);
        n[1] = d.ng * sigma_g_i(1, eps, d.spd2_rel);
        n[2] = 0.0;
      }
      const double tot = (n[0] + n[1]) + n[2];
      if (tot > numax) numax = tot;
    }
    d.numax[s] = numax;
    d.pmax[s] = 1.0 - std::exp(-numax * d.dt);  // §3.5
    std::vector<double>& F = (s == 0) ? Fe : Fi;
    F.assign((size_t)kXsNodes * 4, 0.0);
    for (int k = 0; k < kXsNodes; ++k) {
      const double* n = &nu[(size_t)3 * k];
      const double c1 = n[0];
      const double c2 = c1 + n[1];
      const double c3 = c2 + n[2];
      F[(size_t)4 * k + 0] = numax > 0.0 ? c1 / numax : 0.0;
      F[(size_t)4 * k + 1] = numax > 0.0 ? c2 / numax : 0.0;
      F[(size_t)4 * k + 2] = numax > 0.0 ? c3 / numax : 0.0;
    }
  }
}

bool valid(const pic_params* p) {
  if (!p) return false;
  const bool fin = std::isfinite(p->gap_m) && std::isfinite(p->pressure_pa) &&
                   std::isfinite(p->gas_temp_k) && std::isfinite(p->v_rf_amp_v) &&
                   std::isfinite(p->f_rf_hz) && std::isfinite(p->weight) &&
                   std::isfinite(p->refl_e) && std::isfinite(p->gamma_see) &&
                   std::isfinite(p->area_m2) && std::isfinite(p->init_te_ev) &&
                   std::isfinite(p->see_energy_ev) && std::isfinite(p->eepf_emax_ev) &&
                   std::isfinite(p->fedf_emax_ev);
  return fin && p->gap_m > 0 && p->pressure_pa >= 0 && p->gas_temp_k > 0 && p->f_rf_hz > 0 &&
         p->steps_per_rf >= 1 && p->n_cells >= 2 && p->n_cells <= 4096 && p->weight > 0 &&
         p->refl_e >= 0 && p->refl_e <= 1 && p->gamma_see >= 0 && p->gamma_see <= 1 &&
         p->area_m2 > 0 && p->init_te_ev >= 0 && p->see_energy_ev >= 0 &&
         p->init_per_species >= 0 && p->capacity_per_species >= p->init_per_species &&
         p->capacity_per_species >= 1 && p->capacity_per_species < (int64_t(1) << 31) - kChunk &&
         (p->precision == PIC_FP64 || p->precision == PIC_FP32) && p->eepf_bins >= 1 &&
         p->eepf_bins <= (1 << 20) &&
         p->eepf_emax_ev > 0 && p->fedf_bins >= 1 && p->fedf_bins <= (1 << 20) &&
         p->fedf_emax_ev > 0;
}

// Bump allocator over the workspace (first pass with base 0 measures the size).
struct Carver {
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

// Upper bound of the particle grid size (entries of the per-block count arrays).
// (FP32 handles keep one list per warp: 8 per block of at most capacity/256 blocks.)
long long max_list_blocks(const pic_params& p) { return p.capacity_per_species / 32 + 8192; }

// Count arrays of the lists (reading C-15) at stride G inside their block:
// holes e, holes i, electron births from e / i ranges, ion births.
void set_list_counts(DevCtx& K, int G) {
  int* base = K.hole_cnt[0];
  K.hole_cnt[1] = base + G;
  K.eb_cnt[0] = base + 2 * (size_t)G;
  K.eb_cnt[1] = base + 3 * (size_t)G;
  K.ib_cnt = base + 4 * (size_t)G;
}

void carve(const pic_params& p, char* base, DevCtx& K, size_t* total) {
  Carver c{base};
  const int nx = p.n_cells + 1;
  const int nch = (int)((p.capacity_per_species + kChunk - 1) / kChunk);
  const size_t cap = (size_t)nch * kChunk;
  K.nchunk_max = nch;
  K.st = c.take<DevState>(1);
  K.self = c.take<DevCtx>(1);
  for (int s = 0; s < 2; ++s) {
    K.x[s] = c.take<double>(cap);
    K.vx[s] = c.take<double>(cap);
    K.vy[s] = c.take<double>(cap);
    K.vz[s] = c.take<double>(cap);
    K.id[s] = c.take<unsigned>(cap + 64);  // tail padding for rounded bulk copies
  }
  K.C = c.take<unsigned long long>((size_t)4 * nx);
  K.phi = c.take<double>(nx);
  K.E = c.take<double>(nx);
  K.acc = c.take<double>((size_t)2 * nx);
  K.inv_den = c.take<double>(nx);
  K.vtab = c.take<double>((size_t)p.steps_per_rf);
  K.F[0] = c.take<double>((size_t)kXsNodes * 4);
  K.F[1] = c.take<double>((size_t)kXsNodes * 4);
  K.eepf = c.take<unsigned long long>((size_t)p.eepf_bins);
  K.fedf = c.take<unsigned long long>((size_t)2 * p.fedf_bins);
  K.counters = c.take<unsigned long long>(kNumCounters);
  // per-block list counts: the particle grid has at most max_list_blocks(p) blocks
  const size_t nl = (size_t)max_list_blocks(p);
  const bool fp32 = p.precision == PIC_FP32;
  // the five count arrays are one contiguous block (placed with stride nlist by
  // set_list_counts once the grid is known), so the placement launch stages them with
  // 16-byte loads; 4 ints of padding for the last rounded load
  K.hole_cnt[0] = c.take<int>(5 * nl + 4);
  set_list_counts(K, (int)nl);
  for (int s = 0; s < 2; ++s) {
    K.hole_idx[s] = c.take<int>(cap);
    K.eb[s] = fp32 ? nullptr : c.take<double>(4 * cap);
  }
  K.ib = fp32 ? nullptr : c.take<double>(4 * cap);
  if (fp32) {
    for (int s = 0; s < 2; ++s) {
      // 64 elements of tail padding: a bulk copy of a last tile is rounded up to 16 bytes
      K.ccd[s] = c.take<unsigned>(cap + 64);
      K.ov[s] = c.take<float2>(cap + 64);
      K.fvy[s] = c.take<float>(cap);
      K.fvz[s] = c.take<float>(cap);
      K.feb[s] = c.take<float>(6 * cap);
      K.fF[s] = c.take<float>((size_t)kXsNodes * 4);
      K.fE[s] = c.take<float>(nx);
    }
    K.fib = c.take<float>(6 * cap);
  }
  *total = (c.off + 255) & ~size_t(255);
}

// The null-collision test u < P_max with u = (2k+1) 2^-53 (k a 52-bit integer) holds exactly
// when 2k+1 < C, C = ceil(P_max 2^53) (an integer, exact in double), i.e. k < floor(C/2).
unsigned long long null_threshold(double pmax) {
  const double c = std::ceil(std::ldexp(pmax, 53));
  return (unsigned long long)c / 2ull;
}

// FP32 path: u = (2k+1) 2^-25 with k a 24-bit integer; u < P_max <=> k < floor(C/2),
// C = ceil(P_max 2^25).
unsigned null_threshold24(double pmax) {
  const double c = std::ceil(std::ldexp(pmax, 25));
  return (unsigned)((unsigned long long)c / 2ull);
}

int status_code(int st) {
  if (st & kStTimeout) return PIC_ERR_TIMEOUT;
  if (st & kStNonfinite) return PIC_ERR_NONFINITE;
  if (st & kStCapacity) return PIC_ERR_CAPACITY;
  return PIC_OK;
}

}  // namespace

struct pic_handle {
  pic_params p;
  Derived d;
  DevCtx K;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  int push_grid;
  int place_grid;
  int last_status;
  // pinned host staging of pic_diag's read-back (state, counters, averages, distributions),
  // written by the diagnostics launch through its device mapping (stage_dev)
  char* stage = nullptr;
  char* stage_dev = nullptr;
  ~pic_handle() {
    if (stage) cudaFreeHost(stage);
  }
};

namespace {
// If *p is host memory the device can address (pinned or registered), replace it by its
// device address and return true; false for other memory (then it is copied instead).
template <class T>
bool device_view(const T** p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, *p) != cudaSuccess) {
    (void)cudaGetLastError();  // not a CUDA-known pointer: not an error of this call
    return false;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
  *p = static_cast<const T*>(a.devicePointer);
  return true;
}

// Byte offsets of pic_diag's read-back in the pinned staging buffer.
struct StageLayout {
  size_t state, counters, acc, eepf, fedf, bytes;
};
StageLayout stage_layout(const pic_params& p) {
  StageLayout L;
  auto up = [](size_t b) { return (b + 15) & ~size_t(15); };
  const size_t nx = (size_t)p.n_cells + 1;
  L.state = 0;
  L.counters = up(sizeof(DevState));
  L.acc = L.counters + up(sizeof(uint64_t) * kNumCounters);
  L.eepf = L.acc + up(sizeof(double) * 2 * nx);
  L.fedf = L.eepf + up(sizeof(uint64_t) * (size_t)p.eepf_bins);
  L.bytes = L.fedf + up(sizeof(uint64_t) * 2 * (size_t)p.fedf_bins);
  return L;
}
}  // namespace

namespace {
bool is_fp32(const pic_handle* h) { return h->p.precision == PIC_FP32; }

cudaError_t launch_particles(const pic_handle* h) {
  return is_fp32(h) ? launch_push_fp32(h->K, h->push_grid, h->stream)
                    : launch_push_fp64(h->K, h->push_grid, h->stream);
}

cudaError_t launch_place(const pic_handle* h) {
  return is_fp32(h) ? launch_place_fp32(h->K, h->place_grid, h->stream)
                    : launch_place_fp64(h->K, h->place_grid, h->stream);
}
}  // namespace

namespace {
// The last CUDA error a call of this thread turned into PIC_ERR_CUDA (pic_last_cuda_error).
thread_local cudaError_t g_last_cuda = cudaSuccess;
void note_cuda(cudaError_t e) {
  if (e != cudaSuccess) g_last_cuda = e;
}
}  // namespace

#define PIC_CUDA(call)                        \
  do {                                        \
    const cudaError_t pic_e_ = (call);        \
    if (pic_e_ != cudaSuccess) {              \
      note_cuda(pic_e_);                      \
      (void)cudaGetLastError();               \
      return PIC_ERR_CUDA;                    \
    }                                         \
  } while (0)

extern "C" {

int pic_workspace_bytes(const pic_params* p, size_t* bytes) {
  if (!valid(p) || !bytes) return PIC_ERR_PARAM;
  DevCtx K;
  carve(*p, nullptr, K, bytes);
  return PIC_OK;
}

int pic_init(const pic_params* p, void* workspace, size_t workspace_bytes, void* cuda_stream,
             pic_handle** out) {
  if (!valid(p) || !out) return PIC_ERR_PARAM;
  *out = nullptr;
  size_t need = 0;
  DevCtx K;
  std::memset(&K, 0, sizeof K);
  carve(*p, nullptr, K, &need);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return PIC_ERR_WORKSPACE;
  pic_handle* h = new (std::nothrow) pic_handle;
  if (!h) return PIC_ERR_PARAM;
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->ws = static_cast<char*>(workspace);
  h->ws_bytes = workspace_bytes;
  h->last_status = PIC_OK;
  carve(*p, h->ws, K, &need);
  Derived& d = h->d;
  d = derive(*p);
  std::vector<double> Fe, Fi;
  build_tables(d, Fe, Fi);
  const int nc = p->n_cells, nx = nc + 1;
  std::vector<double> inv_den((size_t)nx, 0.0);
  double den = 2.0;
  for (int j = 1; j <= nc - 1; ++j) {
    inv_den[j] = 1.0 / den;
    den = 2.0 - inv_den[j];
  }
  std::vector<double> vtab((size_t)p->steps_per_rf);
  for (int k = 0; k < p->steps_per_rf; ++k)
    vtab[k] = p->v_rf_amp_v * std::cos((6.283185307179586 * (double)k) / (double)p->steps_per_rf);

  K.nc = nc;
  K.nx = nx;
  K.steps_per_rf = p->steps_per_rf;
  K.eepf_bins = p->eepf_bins;
  K.fedf_bins = p->fedf_bins;
  K.cap = p->capacity_per_species;
  K.L = p->gap_m;
  K.dx = d.dx;
  K.inv_dx = d.inv_dx;
  K.inv_2dx = d.inv_2dx;
  K.dt = d.dt;
  K.efac = d.efac;
  K.rfac = d.rfac;
  K.den1 = d.dx * (double)nc;  // N dx and 2 N dx of the field solve (reading C-23)
  K.den2 = (2.0 * d.dx) * (double)nc;
  K.rden1 = 1.0 / K.den1;
  K.rden2 = 1.0 / K.den2;
  K.rnc = 1.0 / (double)nc;
  K.half_L = 0.5 * p->gap_m;
  K.half_dx = 0.5 * d.dx;
  K.qm_dt[0] = d.qm_dt[0];
  K.qm_dt[1] = d.qm_dt[1];
  K.emfac_e = d.emfac_e;
  K.spd2_e = d.spd2_e;
  K.emfac_rel = d.emfac_rel;
  K.spd2_rel = d.spd2_rel;
  K.emfac_ilab = d.emfac_ilab;
  K.mr2 = d.mr2;
  K.sig_i = d.sig_i;
  K.v_see = d.v_see;
  K.sig_load[0] = d.sig_e;
  K.sig_load[1] = d.sig_i;
  K.pmax[0] = d.pmax[0];
  K.pmax[1] = d.pmax[1];
  K.null_kthr[0] = null_threshold(d.pmax[0]);
  K.null_kthr[1] = null_threshold(d.pmax[1]);
  // the EEPF window |x - L/2| < dx/2 lies in cells (nc-1)/2 .. nc/2, one cell of margin
  K.eepf_jlo = std::max(0, (nc - 1) / 2 - 1);
  K.eepf_jhi = std::min(nc - 1, nc / 2 + 1);
  K.refl = p->refl_e;
  K.gamma = p->gamma_see;
  K.eepf_inv_de = (double)p->eepf_bins / p->eepf_emax_ev;
  K.fedf_inv_de = (double)p->fedf_bins / p->fedf_emax_ev;
  K.key0 = (unsigned)p->seed;
  K.key1 = (unsigned)(p->seed >> 32) ^ p->instance;
  const bool fp32 = p->precision == PIC_FP32;
  std::vector<float> fFe, fFi;
  if (fp32) {  // cell units: x / dx, v dt / dx
    const double vs = d.dt * d.inv_dx, vs2 = vs * vs;
    K.f_emfac_e = (float)(d.emfac_e / vs2);
    K.f_emfac_rel = (float)(d.emfac_rel / vs2);
    K.f_emfac_ilab = (float)(d.emfac_ilab / vs2);
    K.f_spd2_e = (float)(d.spd2_e * vs2);
    K.f_sig_i = (float)(d.sig_i * vs);
    K.f_v_see = (float)(d.v_see * vs);
    K.f_mr2 = (float)d.mr2;
    K.f_refl = (float)p->refl_e;
    K.f_gamma = (float)p->gamma_see;
    K.f_eepf_inv_de = (float)K.eepf_inv_de;
    K.f_fedf_inv_de = (float)K.fedf_inv_de;
    K.f_null_thr[0] = null_threshold24(d.pmax[0]);
    K.f_null_thr[1] = null_threshold24(d.pmax[1]);
    K.f_lnq[0] = (float)std::log1p(-d.pmax[0]);  // geometric countdown of the FP32 pass
    K.f_lnq[1] = (float)std::log1p(-d.pmax[1]);
    K.to_si_v = d.dx / d.dt;
    K.fe_scale[0] = d.qm_dt[0] * d.dt * d.inv_dx;  // E -> kick in cells per step
    K.fe_scale[1] = d.qm_dt[1] * d.dt * d.inv_dx;
    fFe.assign(Fe.begin(), Fe.end());
    fFi.assign(Fi.begin(), Fi.end());
  }
  h->K = K;

  int dev = 0, sms = 0;
  cudaStream_t st = h->stream;
  auto fail = [&](int code) {
    note_cuda(cudaGetLastError());
    delete h;
    return code;
  };
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      configure_kernels(nx) != cudaSuccess || (fp32 && configure_kernels32(nx) != cudaSuccess) ||
      cudaMallocHost(reinterpret_cast<void**>(&h->stage), stage_layout(*p).bytes) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->stage_dev), h->stage, 0) !=
          cudaSuccess)
    return fail(PIC_ERR_CUDA);
  // persistent particle grid: resident blocks on all SMs, fewer for small populations
  const int bps = fp32 ? push_fp32_blocks_per_sm(nx) : push_fp64_blocks_per_sm(nx);
  const long long by_size = (p->capacity_per_species + 255) / 256;
  h->push_grid = (int)std::max(1LL, std::min<long long>({(long long)sms * bps, by_size,
                                                          max_list_blocks(*p) / 8}));
  K.nfield = place_field_blocks(nx);
  h->place_grid = K.nfield + sms;
  // hole / birth list owners: the particle blocks (the FP32 pass packs its warps' lists)
  K.nlist = h->push_grid;
  K.gw_div = make_divider((long long)h->push_grid * (kBlock / 32));
  K.nl_div = make_divider(K.nlist);
  set_list_counts(K, K.nlist);
  h->K = K;
  if ((fp32 ? configure_place_fp32(nx, K.nlist) : configure_place_fp64(nx, K.nlist)) !=
      cudaSuccess)
    return fail(PIC_ERR_CUDA);

  DevState s0;
  std::memset(&s0, 0, sizeof s0);
  s0.n[0] = s0.n[1] = p->init_per_species;
  s0.n_snap[0] = s0.n_snap[1] = p->init_per_species;
  s0.next_id[0] = s0.next_id[1] = (unsigned)p->init_per_species;
  if (cudaMemsetAsync(h->ws, 0, need, st) != cudaSuccess ||
      cudaMemcpyAsync(K.st, &s0, sizeof s0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)K.inv_den, inv_den.data(), sizeof(double) * nx,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)K.vtab, vtab.data(), sizeof(double) * vtab.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)K.F[0], Fe.data(), sizeof(double) * Fe.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync((void*)K.F[1], Fi.data(), sizeof(double) * Fi.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      // the device copy of the context (read by out-of-line device functions)
      cudaMemcpyAsync((void*)K.self, &h->K, sizeof(DevCtx), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return fail(PIC_ERR_CUDA);
  if (fp32 && (cudaMemcpyAsync((void*)K.fF[0], fFe.data(), sizeof(float) * fFe.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess ||
               cudaMemcpyAsync((void*)K.fF[1], fFi.data(), sizeof(float) * fFi.size(),
                               cudaMemcpyHostToDevice, st) != cudaSuccess))
    return fail(PIC_ERR_CUDA);
  for (int s = 0; s < 2; ++s) {
    // the FP32 state is the FP64 load rounded, so both precisions start from one sample (the
    // FP32 conversion deposits the charge as it goes)
    if (launch_init_load(K, s, p->init_per_species, st) != cudaSuccess ||
        (fp32 ? launch_convert(K, s, p->init_per_species, true, st) != cudaSuccess
              : launch_deposit(K, s, 0, p->init_per_species, st) != cudaSuccess))
      return fail(PIC_ERR_CUDA);
  }
  if (launch_field(K, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return fail(PIC_ERR_CUDA);
  *out = h;
  return PIC_OK;
}

int pic_step(pic_handle* h, int64_t n_steps) {
  if (!h || n_steps < 0) return PIC_ERR_PARAM;
  for (int64_t i = 0; i < n_steps; ++i) {
    if (launch_particles(h) != cudaSuccess || launch_place(h) != cudaSuccess) {
      note_cuda(cudaGetLastError());
      return PIC_ERR_CUDA;
    }
  }
  return h->last_status;
}

int pic_step_profiled(pic_handle* h, int64_t n_steps, double* ms_out) {
  if (!h || n_steps < 0 || !ms_out) return PIC_ERR_PARAM;
  cudaEvent_t ev[3];
  for (int k = 0; k < 3; ++k)
    if (cudaEventCreate(&ev[k]) != cudaSuccess) {
      for (int m = 0; m < k; ++m) cudaEventDestroy(ev[m]);
      note_cuda(cudaGetLastError());
      return PIC_ERR_CUDA;
    }
  int rc = PIC_OK;
  for (int64_t i = 0; i < n_steps && rc == PIC_OK; ++i) {
    float t[2];
    if (cudaEventRecord(ev[0], h->stream) != cudaSuccess ||
        launch_particles(h) != cudaSuccess ||
        cudaEventRecord(ev[1], h->stream) != cudaSuccess ||
        launch_place(h) != cudaSuccess ||
        cudaEventRecord(ev[2], h->stream) != cudaSuccess ||
        cudaEventSynchronize(ev[2]) != cudaSuccess ||
        cudaEventElapsedTime(&t[0], ev[0], ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t[1], ev[1], ev[2]) != cudaSuccess) {
      rc = PIC_ERR_CUDA;
      break;
    }
    ms_out[0] += (double)t[0];
    ms_out[1] += (double)t[1];
  }
  for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
  if (rc != PIC_OK) {
    note_cuda(cudaGetLastError());
    return rc;
  }
  return h->last_status;
}

int pic_sync(pic_handle* h) {
  if (!h) return PIC_ERR_PARAM;
  int st = 0;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&st, &h->K.st->status, sizeof st, cudaMemcpyDeviceToHost));
  h->last_status = status_code(st);
  return h->last_status;
}

int pic_counts(pic_handle* h, int64_t* n_e, int64_t* n_i) {
  if (!h) return PIC_ERR_PARAM;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  if (n_e) *n_e = s.n[0];
  if (n_i) *n_i = s.n[1];
  return PIC_OK;
}

int pic_counts_async(pic_handle* h, int64_t* counts2) {
  if (!h || !counts2) return PIC_ERR_PARAM;
  static_assert(offsetof(DevState, n) == 0, "counts lead the device state");
  PIC_CUDA(cudaMemcpyAsync(counts2, h->K.st, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                           h->stream));
  return PIC_OK;
}

int pic_get_step(pic_handle* h, uint32_t* step, uint32_t* next_id_e, uint32_t* next_id_i) {
  if (!h) return PIC_ERR_PARAM;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  if (step) *step = s.step;
  if (next_id_e) *next_id_e = s.next_id[0];
  if (next_id_i) *next_id_i = s.next_id[1];
  return PIC_OK;
}

int pic_get_particles(pic_handle* h, int species, double* x, double* vx, double* vy,
                      double* vz, uint32_t* id, int64_t capacity, int64_t* n_out) {
  if (!h || species < 0 || species > 1 || capacity < 0) return PIC_ERR_PARAM;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  const int64_t n = s.n[species];
  if (n_out) *n_out = n;
  const int64_t m = std::min(n, capacity);
  if (m > 0) {
    const DevCtx& K = h->K;
    cudaStream_t st = h->stream;
    if (is_fp32(h)) PIC_CUDA(launch_convert(K, species, n, false, st));
    if (x) PIC_CUDA(cudaMemcpyAsync(x, K.x[species], m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (vx) PIC_CUDA(cudaMemcpyAsync(vx, K.vx[species], m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (vy) PIC_CUDA(cudaMemcpyAsync(vy, K.vy[species], m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (vz) PIC_CUDA(cudaMemcpyAsync(vz, K.vz[species], m * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (id) PIC_CUDA(cudaMemcpyAsync(id, K.id[species], m * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PIC_CUDA(cudaStreamSynchronize(st));
  }
  return n > capacity ? PIC_ERR_PARAM : PIC_OK;
}

int pic_set_particles(pic_handle* h, int species, const double* x, const double* vx,
                      const double* vy, const double* vz, const uint32_t* id, int64_t n,
                      uint32_t next_id) {
  if (!h || species < 0 || species > 1 || n < 0 || n > h->p.capacity_per_species)
    return PIC_ERR_PARAM;
  if (n > 0 && (!x || !vx || !vy || !vz || !id)) return PIC_ERR_PARAM;
  const DevCtx& K = h->K;
  cudaStream_t st = h->stream;
  // An FP32 handle reads host arrays the device can address (pinned or registered memory)
  // straight from its conversion kernel; otherwise they are copied into the FP64 buffers
  // first.  Either way the state, the counts and the charge are then set on the device, in
  // stream order, and one synchronization returns the host arrays to the caller.
  const double* dx_ = x;
  const double* dvx = vx;
  const double* dvy = vy;
  const double* dvz = vz;
  const uint32_t* did = id;
  const bool direct = is_fp32(h) && n > 0 && device_view(&dx_) && device_view(&dvx) &&
                      device_view(&dvy) && device_view(&dvz) && device_view(&did);
  if (n > 0 && !direct) {
    PIC_CUDA(cudaMemcpyAsync(K.x[species], x, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PIC_CUDA(cudaMemcpyAsync(K.vx[species], vx, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PIC_CUDA(cudaMemcpyAsync(K.vy[species], vy, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PIC_CUDA(cudaMemcpyAsync(K.vz[species], vz, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PIC_CUDA(cudaMemcpyAsync(K.id[species], id, n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  }
  PIC_CUDA(launch_set_counts(K, species, n, next_id, st));
  if (is_fp32(h)) {
    // the conversion deposits the charge as it goes
    if (direct)
      PIC_CUDA(launch_convert_from(K, species, n, dx_, dvx, dvy, dvz, did, st));
    else
      PIC_CUDA(launch_convert(K, species, n, true, st));
  } else {
    PIC_CUDA(launch_deposit(K, species, -1, n, st));
  }
  PIC_CUDA(launch_field(K, st));
  PIC_CUDA(cudaStreamSynchronize(st));
  return PIC_OK;
}

int pic_get_grid(pic_handle* h, int64_t* charge_e, int64_t* charge_i, double* phi,
                 double* efield) {
  if (!h) return PIC_ERR_PARAM;
  const DevCtx& K = h->K;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, K.st, sizeof s, cudaMemcpyDeviceToHost));
  const int buf = s.step & 1;
  const size_t nb = sizeof(int64_t) * K.nx;
  if (charge_e) PIC_CUDA(cudaMemcpy(charge_e, K.C + (size_t)(buf * 2) * K.nx, nb, cudaMemcpyDeviceToHost));
  if (charge_i) PIC_CUDA(cudaMemcpy(charge_i, K.C + (size_t)(buf * 2 + 1) * K.nx, nb, cudaMemcpyDeviceToHost));
  if (phi) PIC_CUDA(cudaMemcpy(phi, K.phi, sizeof(double) * K.nx, cudaMemcpyDeviceToHost));
  if (efield) PIC_CUDA(cudaMemcpy(efield, K.E, sizeof(double) * K.nx, cudaMemcpyDeviceToHost));
  return PIC_OK;
}

int pic_solve_field(pic_handle* h) {
  if (!h) return PIC_ERR_PARAM;
  PIC_CUDA(launch_field(h->K, h->stream));
  return PIC_OK;
}

int pic_get_accum(pic_handle* h, double* acc_e, double* acc_i, uint64_t* eepf,
                  uint64_t* fedf_e, uint64_t* fedf_i, uint64_t* counters, int64_t* steps) {
  if (!h) return PIC_ERR_PARAM;
  const DevCtx& K = h->K;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  if (acc_e) PIC_CUDA(cudaMemcpy(acc_e, K.acc, sizeof(double) * K.nx, cudaMemcpyDeviceToHost));
  if (acc_i) PIC_CUDA(cudaMemcpy(acc_i, K.acc + K.nx, sizeof(double) * K.nx, cudaMemcpyDeviceToHost));
  if (eepf) PIC_CUDA(cudaMemcpy(eepf, K.eepf, sizeof(uint64_t) * K.eepf_bins, cudaMemcpyDeviceToHost));
  if (fedf_e) PIC_CUDA(cudaMemcpy(fedf_e, K.fedf, sizeof(uint64_t) * K.fedf_bins, cudaMemcpyDeviceToHost));
  if (fedf_i) PIC_CUDA(cudaMemcpy(fedf_i, K.fedf + K.fedf_bins, sizeof(uint64_t) * K.fedf_bins, cudaMemcpyDeviceToHost));
  if (counters) PIC_CUDA(cudaMemcpy(counters, K.counters, sizeof(uint64_t) * kNumCounters, cudaMemcpyDeviceToHost));
  if (steps) {
    DevState s;
    PIC_CUDA(cudaMemcpy(&s, K.st, sizeof s, cudaMemcpyDeviceToHost));
    *steps = s.steps_avg;
  }
  return PIC_OK;
}

int pic_reset_averages(pic_handle* h) {
  if (!h) return PIC_ERR_PARAM;
  const DevCtx& K = h->K;
  cudaStream_t st = h->stream;
  PIC_CUDA(cudaMemsetAsync(K.acc, 0, sizeof(double) * 2 * K.nx, st));
  PIC_CUDA(cudaMemsetAsync(K.eepf, 0, sizeof(uint64_t) * K.eepf_bins, st));
  PIC_CUDA(cudaMemsetAsync(K.fedf, 0, sizeof(uint64_t) * 2 * K.fedf_bins, st));
  PIC_CUDA(cudaMemsetAsync(K.counters, 0, sizeof(uint64_t) * kNumCounters, st));
  PIC_CUDA(cudaMemsetAsync(&K.st->steps_avg, 0, sizeof(long long), st));
  return PIC_OK;
}

int pic_set_step(pic_handle* h, uint32_t step) {
  if (!h) return PIC_ERR_PARAM;
  PIC_CUDA(launch_set_step(h->K, step, h->stream));
  PIC_CUDA(launch_field(h->K, h->stream));  // the field of the new step's drive value
  return PIC_OK;
}

int pic_override_table(pic_handle* h, int species, const double* table, double nu_max) {
  if (!h || species < 0 || species > 1 || !table || !(nu_max >= 0) || !std::isfinite(nu_max))
    return PIC_ERR_PARAM;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy((void*)h->K.F[species], table, sizeof(double) * kXsNodes * 4,
                      cudaMemcpyHostToDevice));
  h->d.numax[species] = nu_max;
  h->d.pmax[species] = 1.0 - std::exp(-nu_max * h->d.dt);
  h->K.pmax[species] = h->d.pmax[species];
  h->K.null_kthr[species] = null_threshold(h->d.pmax[species]);
  if (is_fp32(h)) {
    std::vector<float> f(table, table + (size_t)kXsNodes * 4);
    PIC_CUDA(cudaMemcpy((void*)h->K.fF[species], f.data(), sizeof(float) * f.size(),
                        cudaMemcpyHostToDevice));
    h->K.f_null_thr[species] = null_threshold24(h->d.pmax[species]);
    h->K.f_lnq[species] = (float)std::log1p(-h->d.pmax[species]);
    PIC_CUDA(cudaMemcpy((void*)h->K.self, &h->K, sizeof(DevCtx), cudaMemcpyHostToDevice));
  }
  return PIC_OK;
}

int pic_get_derived(pic_handle* h, double* out) {
  if (!h || !out) return PIC_ERR_PARAM;
  const double v[7] = {h->d.dt, h->d.dx, h->d.ng, h->d.numax[0], h->d.numax[1],
                       h->d.pmax[0], h->d.pmax[1]};
  std::memcpy(out, v, sizeof v);
  return PIC_OK;
}

int pic_diag(pic_handle* h, pic_diag_out* out) {
  if (!h || !out) return PIC_ERR_PARAM;
  const pic_params& p = h->p;
  const DevCtx& K = h->K;
  const int nc = p.n_cells, nx = nc + 1;
  if ((out->n_e || out->n_i) && out->n_x != nx) return PIC_ERR_PARAM;
  if ((out->eepf || out->eepf_energy) && out->eepf_bins != p.eepf_bins) return PIC_ERR_PARAM;
  if ((out->fedf_e || out->fedf_i || out->fedf_energy) && out->fedf_bins != p.fedf_bins)
    return PIC_ERR_PARAM;
  // one launch and one synchronization: the electrons' max |vx| and sum of |v|^2 reduced on
  // the device (FP32 handles straight from the FP32 state, in cells per step), after which
  // its last block writes the state, counters, averages and distributions into the pinned
  // staging buffer
  cudaStream_t st = h->stream;
  const StageLayout L = stage_layout(p);
  char* hs = h->stage;
  PIC_CUDA(launch_diag(K, is_fp32(h), h->stage_dev,
                       DiagOffsets{L.state, L.counters, L.acc, L.eepf, L.fedf}, st));
  PIC_CUDA(cudaStreamSynchronize(st));
  DevState s;
  std::memcpy(&s, hs + L.state, sizeof s);
  const int rc = status_code(s.status);
  h->last_status = rc;
  std::memcpy(out->counters, hs + L.counters, sizeof(uint64_t) * kNumCounters);
  const double* acc = reinterpret_cast<const double*>(hs + L.acc);
  const uint64_t* eepf = reinterpret_cast<const uint64_t*>(hs + L.eepf);
  const uint64_t* fedf = reinterpret_cast<const uint64_t*>(hs + L.fedf);
  const unsigned long long vbits = s.vmax_bits;
  double v2sum = s.v2sum;
  double vmax;
  if (is_fp32(h)) {
    float f;
    const uint32_t b = (uint32_t)vbits;
    std::memcpy(&f, &b, sizeof f);
    vmax = (double)f * K.to_si_v;
    v2sum *= K.to_si_v * K.to_si_v;
  } else {
    std::memcpy(&vmax, &vbits, sizeof vmax);
  }

  const Derived& d = h->d;
  const int64_t steps = s.steps_avg;
  out->steps_averaged = steps;
  out->count_e = s.n[0];
  out->count_i = s.n[1];
  out->status = rc;
  const double W = p.weight, A = p.area_m2;
  const double dens_fac = W / ((A * d.dx) * kTwo32);
  std::vector<double> ne((size_t)nx);
  for (int j = 0; j < nx; ++j) {
    const double vol = (j == 0 || j == nc) ? 0.5 : 1.0;  // reading C-5
    const double st = steps > 0 ? (double)steps : 1.0;
    ne[j] = (acc[j] / st) * dens_fac / vol;
    if (out->n_e) out->n_e[j] = ne[j];
    if (out->n_i) out->n_i[j] = (acc[nx + j] / st) * dens_fac / vol;
  }
  // EEPF with sum sqrt(e) f de = 1 (§3.1)
  const double de = p.eepf_emax_ev / p.eepf_bins;
  double tot = 0.0;
  for (int b = 0; b < p.eepf_bins; ++b) tot += (double)eepf[b];
  for (int b = 0; b < p.eepf_bins; ++b) {
    const double ec = (b + 0.5) * de;
    if (out->eepf_energy) out->eepf_energy[b] = ec;
    if (out->eepf) out->eepf[b] = tot > 0 ? (double)eepf[b] / (std::sqrt(ec) * de * tot) : 0.0;
  }
  // flux-energy distributions with sum f de = 1 (§3.4)
  const double fde = p.fedf_emax_ev / p.fedf_bins;
  double tf[2] = {0.0, 0.0};
  for (int sp = 0; sp < 2; ++sp)
    for (int b = 0; b < p.fedf_bins; ++b) tf[sp] += (double)fedf[(size_t)sp * p.fedf_bins + b];
  for (int b = 0; b < p.fedf_bins; ++b) {
    if (out->fedf_energy) out->fedf_energy[b] = (b + 0.5) * fde;
    if (out->fedf_e) out->fedf_e[b] = tf[0] > 0 ? (double)fedf[b] / (fde * tf[0]) : 0.0;
    if (out->fedf_i)
      out->fedf_i[b] = tf[1] > 0 ? (double)fedf[(size_t)p.fedf_bins + b] / (fde * tf[1]) : 0.0;
  }
  // ion flux (reading C-21)
  const double T = (double)steps * d.dt;
  out->ion_flux_left = T > 0 ? (double)out->counters[kCnIAbsL] * W / (A * T) : 0.0;
  out->ion_flux_right = T > 0 ? (double)out->counters[kCnIAbsR] * W / (A * T) : 0.0;
  out->ion_flux = 0.5 * (out->ion_flux_left + out->ion_flux_right);
  // centre density and temperature (reading C-19), criteria of §3.5
  const double xc = 0.5 * nc;
  const int j = (int)std::floor(xc);
  const double f = xc - j;
  const double n_c = (1 - f) * ne[j] + f * ne[std::min(j + 1, nc)];
  const double ns = (double)out->counters[kCnEepfN];
  const double mean_eps = ns > 0 ? ((double)out->counters[kCnEepfEsum] / 1048576.0) / ns : 0.0;
  const double te = (2.0 / 3.0) * mean_eps;
  out->n_e_center = n_c;
  out->te_center_ev = te;
  const double wfac = kQe * kQe / (kEps0 * kMe);
  out->omega_pe_dt = std::sqrt(std::max(n_c, 0.0) * wfac) * d.dt;
  const double nmax = *std::max_element(ne.begin(), ne.end());
  out->omega_pe_dt_max = std::sqrt(std::max(nmax, 0.0) * wfac) * d.dt;
  out->p_coll_e = d.pmax[0];
  out->p_coll_i = d.pmax[1];
  out->cfl_max = vmax * d.dt / d.dx;
  const double lam = (n_c > 0 && te > 0) ? std::sqrt(kEps0 * te / (n_c * kQe)) : INFINITY;
  out->lambda_d = lam;
  out->dx_over_lambda_d = d.dx / lam;
  out->n_debye = std::isfinite(lam) ? n_c * A * lam / W : INFINITY;  // reading C-20
  // runaway check: mean electron kinetic energy against the largest energy the drive can
  // give (e |V_rf|), with a floor for undriven runs
  out->mean_energy_e_ev = s.n[0] > 0 ? (v2sum / (double)s.n[0]) * (0.5 * kMe / kQe) : 0.0;
  if (rc != PIC_OK) return rc;
  const double runaway_ev = std::max(std::fabs(p.v_rf_amp_v), PIC_RUNAWAY_FLOOR_EV);
  const bool unstable = out->omega_pe_dt_max > 2.0 || !(out->mean_energy_e_ev <= runaway_ev);
  return unstable ? PIC_WARN_UNSTABLE : PIC_OK;
}

int pic_fp64_rate(void* cuda_stream, double* rates) {
  if (!rates) return PIC_ERR_PARAM;
  int dev = 0, sms = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  PIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  for (int k = 0; k < 2; ++k) {
    double ms = 0.0, ops = 0.0;
    PIC_CUDA(fp64_probe(k == 1, sms, 2048, &ms, &ops, s));
    rates[k] = ms > 0.0 ? ops / (ms * 1e-3) : 0.0;
  }
  return PIC_OK;
}

// ------------------------------------------------------------ checkpoint / resume
}  // extern "C"

namespace {

constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  pic_params p;
  int64_t n[2];
  uint32_t next_id[2];
  uint32_t step;
  int32_t status;
  int64_t steps_avg;
  uint64_t payload_bytes;
};

struct Seg {
  void* dev;
  size_t bytes;
};

// The device arrays a checkpoint holds, in file order, for counts n[2]: each species'
// particles in the handle's own representation (so a resumed run is bit for bit the same),
// then the charge counts of both parity buffers, the field, the kick table (FP32), the
// accumulators, EEPF, FEDFs and counters.
std::vector<Seg> ckpt_segments(const pic_handle* h, const int64_t n[2]) {
  const DevCtx& K = h->K;
  std::vector<Seg> v;
  for (int s = 0; s < 2; ++s) {
    const size_t m = (size_t)n[s];
    if (is_fp32(h)) {
      v.push_back({K.ccd[s], 4 * m});
      v.push_back({K.ov[s], 8 * m});
      v.push_back({K.fvy[s], 4 * m});
      v.push_back({K.fvz[s], 4 * m});
    } else {
      v.push_back({K.x[s], 8 * m});
      v.push_back({K.vx[s], 8 * m});
      v.push_back({K.vy[s], 8 * m});
      v.push_back({K.vz[s], 8 * m});
    }
    v.push_back({K.id[s], 4 * m});
  }
  const size_t nx = (size_t)K.nx;
  v.push_back({K.C, 8 * 4 * nx});
  v.push_back({K.phi, 8 * nx});
  v.push_back({K.E, 8 * nx});
  if (is_fp32(h)) {
    v.push_back({K.fE[0], 4 * nx});
    v.push_back({K.fE[1], 4 * nx});
  }
  v.push_back({K.acc, 8 * 2 * nx});
  v.push_back({K.eepf, 8 * (size_t)K.eepf_bins});
  v.push_back({K.fedf, 8 * 2 * (size_t)K.fedf_bins});
  v.push_back({K.counters, 8 * (size_t)kNumCounters});
  return v;
}

size_t ckpt_payload(const std::vector<Seg>& v) {
  size_t b = 0;
  for (const Seg& s : v) b += s.bytes;
  return b;
}

// Everything but the initial load size and the capacity must agree for a resume.
bool same_physics(const pic_params& a, const pic_params& b) {
  return a.gap_m == b.gap_m && a.pressure_pa == b.pressure_pa &&
         a.gas_temp_k == b.gas_temp_k && a.v_rf_amp_v == b.v_rf_amp_v &&
         a.f_rf_hz == b.f_rf_hz && a.steps_per_rf == b.steps_per_rf &&
         a.n_cells == b.n_cells && a.weight == b.weight && a.refl_e == b.refl_e &&
         a.gamma_see == b.gamma_see && a.area_m2 == b.area_m2 && a.init_te_ev == b.init_te_ev &&
         a.see_energy_ev == b.see_energy_ev && a.seed == b.seed && a.instance == b.instance &&
         a.precision == b.precision && a.eepf_bins == b.eepf_bins &&
         a.eepf_emax_ev == b.eepf_emax_ev && a.fedf_bins == b.fedf_bins &&
         a.fedf_emax_ev == b.fedf_emax_ev;
}

}  // namespace

extern "C" {

int pic_checkpoint_bytes(pic_handle* h, size_t* bytes) {
  if (!h || !bytes) return PIC_ERR_PARAM;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  const int64_t n[2] = {s.n[0], s.n[1]};
  *bytes = sizeof(CkptHeader) + ckpt_payload(ckpt_segments(h, n));
  return PIC_OK;
}

int pic_checkpoint_save(pic_handle* h, void* buffer, size_t bytes) {
  if (!h || !buffer) return PIC_ERR_PARAM;
  DevState s;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  const int64_t n[2] = {s.n[0], s.n[1]};
  const std::vector<Seg> segs = ckpt_segments(h, n);
  const size_t payload = ckpt_payload(segs);
  if (bytes < sizeof(CkptHeader) + payload) return PIC_ERR_PARAM;
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = kCkptVersion;
  hd.header_bytes = sizeof(CkptHeader);
  hd.p = h->p;
  hd.n[0] = n[0];
  hd.n[1] = n[1];
  hd.next_id[0] = s.next_id[0];
  hd.next_id[1] = s.next_id[1];
  hd.step = s.step;
  hd.status = s.status;
  hd.steps_avg = s.steps_avg;
  hd.payload_bytes = payload;
  char* out = static_cast<char*>(buffer);
  std::memcpy(out, &hd, sizeof hd);
  size_t off = sizeof hd;
  for (const Seg& g : segs) {
    if (g.bytes) PIC_CUDA(cudaMemcpy(out + off, g.dev, g.bytes, cudaMemcpyDeviceToHost));
    off += g.bytes;
  }
  return PIC_OK;
}

int pic_checkpoint_load(pic_handle* h, const void* buffer, size_t bytes) {
  if (!h || !buffer || bytes < sizeof(CkptHeader)) return PIC_ERR_PARAM;
  CkptHeader hd;
  std::memcpy(&hd, buffer, sizeof hd);
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion ||
      hd.header_bytes != sizeof(CkptHeader) || !same_physics(hd.p, h->p))
    return PIC_ERR_PARAM;
  const int64_t cap = h->p.capacity_per_species;
  if (hd.n[0] < 0 || hd.n[1] < 0 || hd.n[0] > cap || hd.n[1] > cap) return PIC_ERR_PARAM;
  const std::vector<Seg> segs = ckpt_segments(h, hd.n);
  const size_t payload = ckpt_payload(segs);
  if (hd.payload_bytes != payload || bytes < sizeof(CkptHeader) + payload) return PIC_ERR_PARAM;
  PIC_CUDA(cudaStreamSynchronize(h->stream));
  const char* in = static_cast<const char*>(buffer);
  size_t off = sizeof hd;
  for (const Seg& g : segs) {
    if (g.bytes) PIC_CUDA(cudaMemcpy(g.dev, in + off, g.bytes, cudaMemcpyHostToDevice));
    off += g.bytes;
  }
  DevState s;
  PIC_CUDA(cudaMemcpy(&s, h->K.st, sizeof s, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 2; ++k) {
    s.n[k] = s.n_snap[k] = hd.n[k];
    s.next_id[k] = s.id_snap[k] = hd.next_id[k];
  }
  s.step = s.step_next = hd.step;
  s.status = hd.status;
  s.steps_avg = hd.steps_avg;
  PIC_CUDA(cudaMemcpy(h->K.st, &s, sizeof s, cudaMemcpyHostToDevice));
  h->last_status = status_code(hd.status);
  return PIC_OK;
}

// ------------------------------------------------------------------- ensemble (§3 scans)
}  // extern "C"

struct pic_ensemble {
  std::vector<pic_handle*> sims;
  EnsDev* E = nullptr;  // in the caller's ensemble workspace
  cudaStream_t stream = nullptr;
  size_t smem = 0;
  int sms = 0, max_bps = 0, bps = 0, unit = 2048;
  bool want_graph = true, have_graph = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int last_status = PIC_OK;
};

namespace {

void drop_graph(pic_ensemble* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  e->exec = nullptr;
  e->graph = nullptr;
  e->have_graph = false;
}

// Record one step's launch as a CUDA graph (replayed by pic_ensemble_step); on any failure
// the ensemble falls back to direct launches.
void build_graph(pic_ensemble* e) {
  drop_graph(e);
  if (!e->want_graph) return;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    note_cuda(cudaGetLastError());
    return;
  }
  const cudaError_t le = launch_ensemble(e->E, e->sms * e->bps, e->smem, e->stream);
  const cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess || !g) {
    note_cuda(cudaGetLastError());
    if (g) cudaGraphDestroy(g);
    return;
  }
  cudaGraphExec_t x = nullptr;
  if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    note_cuda(cudaGetLastError());
    cudaGraphDestroy(g);
    return;
  }
  e->graph = g;
  e->exec = x;
  e->have_graph = true;
}

cudaError_t ensemble_launch(pic_ensemble* e) {
  if (e->have_graph) return cudaGraphLaunch(e->exec, e->stream);
  return launch_ensemble(e->E, e->sms * e->bps, e->smem, e->stream);
}

}  // namespace

extern "C" {

static_assert(PIC_MAX_ENSEMBLE == kMaxEnsemble, "header and device limits agree");

int pic_ensemble_workspace_bytes(int n, size_t* bytes) {
  if (n < 1 || n > kMaxEnsemble || !bytes) return PIC_ERR_PARAM;
  *bytes = (sizeof(EnsDev) + 255) & ~size_t(255);
  return PIC_OK;
}

int pic_ensemble_create(pic_handle* const* sims, int n, const int64_t* target_steps,
                        void* workspace, size_t workspace_bytes, pic_ensemble** out) {
  if (!out || !sims || !target_steps || n < 1 || n > kMaxEnsemble) return PIC_ERR_PARAM;
  *out = nullptr;
  size_t need = 0;
  pic_ensemble_workspace_bytes(n, &need);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return PIC_ERR_WORKSPACE;
  int nx_max = 0;
  for (int i = 0; i < n; ++i) {
    if (!sims[i] || sims[i]->p.precision != PIC_FP32 || sims[i]->stream != sims[0]->stream ||
        target_steps[i] < 0)
      return PIC_ERR_PARAM;
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return PIC_ERR_PARAM;
    nx_max = std::max(nx_max, sims[i]->K.nx);
  }
  pic_ensemble* e = new (std::nothrow) pic_ensemble;
  if (!e) return PIC_ERR_PARAM;
  e->sims.assign(sims, sims + n);
  e->stream = sims[0]->stream;
  e->E = static_cast<EnsDev*>(workspace);
  auto fail = [&](int code) {
    note_cuda(cudaGetLastError());
    delete e;
    return code;
  };
  // shared memory: the particle phase's tables and pipes; the placement prefixes of one
  // simulation are kept within the same room, which bounds its list owners
  const size_t p1 = ensemble_smem_bytes(nx_max, 0);
  const int gcap_lim = (int)(p1 / (5 * sizeof(int))) & ~3;
  e->smem = ensemble_smem_bytes(nx_max, gcap_lim);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      configure_ensemble(e->smem) != cudaSuccess)
    return fail(PIC_ERR_CUDA);
  e->max_bps = std::min(ensemble_blocks_per_sm(e->smem), 2);
  if (e->max_bps < 1 || e->sms * 1 <= n) return fail(PIC_ERR_PARAM);
  e->bps = e->max_bps;
  std::vector<char> hbuf(sizeof(EnsDev), 0);
  EnsDev* h = reinterpret_cast<EnsDev*>(hbuf.data());
  h->n = n;
  h->unit = e->unit;
  h->pipes_off = (int)ensemble_pipes_offset(nx_max);
  for (int i = 0; i < n; ++i) {
    const long long nl = max_list_blocks(sims[i]->p);
    h->sims[i] = sims[i]->K.self;
    h->st[i] = sims[i]->K.st;
    h->target[i] = target_steps[i];
    h->gcap[i] = (int)std::min<long long>(nl - 4, gcap_lim);
    h->gstride[i] = (int)nl;
    // with at most gcap owners, an owner must still fit the shared counters' bound
    if ((sims[i]->p.capacity_per_species + h->gcap[i] - 1) / h->gcap[i] + 64 > kEnsSpeciesRound)
      return fail(PIC_ERR_PARAM);
  }
  // phase-1 order: members whose electrons are collision candidates most often (the costly
  // particles) first, so the last chunks taken are cheap ones
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return sims[a]->d.pmax[0] > sims[b]->d.pmax[0];
  });
  for (int i = 0; i < n; ++i) h->order[i] = ord[i];
  if (cudaMemcpyAsync(e->E, h, sizeof(EnsDev), cudaMemcpyHostToDevice, e->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(e->stream) != cudaSuccess)
    return fail(PIC_ERR_CUDA);
  build_graph(e);
  *out = e;
  return PIC_OK;
}

int pic_ensemble_configure(pic_ensemble* e, int32_t unit, int32_t blocks_per_sm,
                           int32_t use_graph) {
  if (!e || unit < 256 || unit > kMaxEnsUnit || blocks_per_sm < 1 || blocks_per_sm > e->max_bps)
    return PIC_ERR_PARAM;
  PIC_CUDA(cudaStreamSynchronize(e->stream));
  e->unit = unit;
  e->bps = blocks_per_sm;
  e->want_graph = use_graph != 0;
  PIC_CUDA(cudaMemcpy(&e->E->unit, &e->unit, sizeof(int), cudaMemcpyHostToDevice));
  build_graph(e);
  return PIC_OK;
}

int pic_ensemble_step(pic_ensemble* e, int64_t n_steps) {
  if (!e || n_steps < 0) return PIC_ERR_PARAM;
  for (int64_t i = 0; i < n_steps; ++i) PIC_CUDA(ensemble_launch(e));
  return e->last_status;
}

int pic_ensemble_sync(pic_ensemble* e) {
  if (!e) return PIC_ERR_PARAM;
  PIC_CUDA(cudaStreamSynchronize(e->stream));
  int st = 0;
  PIC_CUDA(cudaMemcpy(&st, &e->E->status, sizeof st, cudaMemcpyDeviceToHost));
  int code = status_code(st);  // the ensemble's own (barrier) status first
  for (pic_handle* h : e->sims) {
    const int c = pic_sync(h);
    if (code == PIC_OK && c != PIC_OK) code = c;
  }
  e->last_status = code;
  return code;
}

int pic_ensemble_autotune(pic_ensemble* e, int32_t trial_steps, int32_t* chosen) {
  if (!e || trial_steps < 1) return PIC_ERR_PARAM;
  const int32_t units[3] = {4000, 8000, 16000};
  float best = 0.0f;
  int32_t bu = e->unit, bb = e->bps;
  cudaEvent_t a = nullptr, b = nullptr;
  PIC_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return PIC_ERR_CUDA;
  }
  int rc = PIC_OK;
  for (int bps = 1; bps <= e->max_bps && rc == PIC_OK; ++bps)
    for (int k = 0; k < 3 && rc == PIC_OK; ++k) {
      rc = pic_ensemble_configure(e, units[k], bps, e->want_graph ? 1 : 0);
      if (rc != PIC_OK) break;
      float ms = 0.0f;
      if (ensemble_launch(e) != cudaSuccess || cudaEventRecord(a, e->stream) != cudaSuccess) {
        rc = PIC_ERR_CUDA;
        break;
      }
      for (int t = 0; t < trial_steps && rc == PIC_OK; ++t)
        if (ensemble_launch(e) != cudaSuccess) rc = PIC_ERR_CUDA;
      if (rc != PIC_OK || cudaEventRecord(b, e->stream) != cudaSuccess ||
          cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        rc = PIC_ERR_CUDA;
        break;
      }
      if (best == 0.0f || ms < best) {
        best = ms;
        bu = units[k];
        bb = bps;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != PIC_OK) {
    note_cuda(cudaGetLastError());
    return rc;
  }
  rc = pic_ensemble_configure(e, bu, bb, e->want_graph ? 1 : 0);
  if (rc == PIC_OK && chosen) {
    chosen[0] = bu;
    chosen[1] = bb;
  }
  return rc;
}

int pic_ensemble_info(pic_ensemble* e, int32_t* out) {
  if (!e || !out) return PIC_ERR_PARAM;
  out[0] = e->unit;
  out[1] = e->bps;
  out[2] = e->sms * e->bps;
  out[3] = e->have_graph ? 1 : 0;
  out[4] = (int32_t)e->smem;
  return PIC_OK;
}

int pic_selftest_waits(void* workspace, size_t workspace_bytes, void* cuda_stream,
                       int32_t* codes) {
  size_t need = 0;
  pic_ensemble_workspace_bytes(1, &need);
  need += 256;
  if (!codes || !workspace || workspace_bytes < need ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return PIC_ERR_PARAM;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  EnsDev* E = static_cast<EnsDev*>(workspace);
  int* st = reinterpret_cast<int*>(static_cast<char*>(workspace) + need - 256);
  int h[2] = {0, 0};
  PIC_CUDA(cudaMemsetAsync(workspace, 0, need, s));
  PIC_CUDA(launch_selftest_waits(E, st, s));
  PIC_CUDA(cudaMemcpyAsync(h, st, sizeof h, cudaMemcpyDeviceToHost, s));
  PIC_CUDA(cudaStreamSynchronize(s));
  codes[0] = status_code(h[0]);
  codes[1] = status_code(h[1]);
  return PIC_OK;
}

void pic_ensemble_free(pic_ensemble* e) {
  if (!e) return;
  drop_graph(e);
  delete e;
}

void pic_free(pic_handle* h) { delete h; }

const char* pic_last_cuda_error(void) {
  return g_last_cuda == cudaSuccess ? "no CUDA error" : cudaGetErrorString(g_last_cuda);
}

const char* pic_strerror(int code) {
  switch (code) {
    case PIC_OK: return "ok";
    case PIC_ERR_PARAM: return "invalid parameter or argument";
    case PIC_ERR_CUDA: return "CUDA error";
    case PIC_ERR_CAPACITY: return "particle capacity exceeded (births dropped)";
    case PIC_ERR_NONFINITE: return "non-finite particle velocity";
    case PIC_ERR_WORKSPACE: return "workspace missing, too small or not 256-byte aligned";
    case PIC_ERR_TIMEOUT: return "a bounded device wait ran out (staged data never arrived)";
    case PIC_ERR_SCRATCH:
      return "n_cells above PIC_FIELD_STATIC_MAX_CELLS, the static scratch of pic_field_solve_static";
    case PIC_WARN_UNSTABLE:
      return "numerically unstable: omega_pe*dt above the leapfrog bound 2, or runaway "
             "electron energy";
    default: return "unknown code";
  }
}

}  // extern "C"
