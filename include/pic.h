/*
 * pic.h -- C-ABI of libpic.so, the GB300 (sm_103a) hot path of the explicit electrostatic
 * 1D3V PIC/MCC simulation of a capacitively coupled RF argon discharge
 * (Vass, Palla & Hartmann, arXiv 2109.04469, §2 "Computational method", steps 1-6).
 *
 * Conventions for every entry point:
 *  - Return 0 (PIC_OK) on success, a negative PIC_ERR_* code on failure, or a positive
 *    PIC_WARN_* code.  No exception or abort crosses the ABI.  pic_strerror() names a code.
 *  - A handle works on one CUDA stream (given at pic_init) and is not thread-safe.
 *  - Device memory: the caller allocates ONE device workspace of pic_workspace_bytes()
 *    bytes (256-byte aligned) and keeps it alive until pic_free(); the library allocates no
 *    device memory.  Host memory of the handle itself is owned by the library.
 *  - Arrays passed to pic_get_* / pic_set_* / pic_diag are HOST arrays owned by the caller.
 *  - Units are SI unless a name says otherwise (_ev: electronvolt).
 *  - Species index: 0 = electrons, 1 = Ar+ ions.
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
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_OK 0
#define PIC_ERR_PARAM (-1)      /* invalid parameter or argument */
#define PIC_ERR_CUDA (-2)       /* a CUDA call failed; the handle should be freed */
#define PIC_ERR_CAPACITY (-3)   /* births exceeded capacity_per_species; excess dropped */
#define PIC_ERR_NONFINITE (-4)  /* a velocity became NaN or infinite */
#define PIC_ERR_WORKSPACE (-5)  /* workspace missing, too small or misaligned */
#define PIC_ERR_TIMEOUT (-6)    /* a bounded device wait ran out; results of the step invalid */
#define PIC_ERR_SCRATCH (-7)    /* n_cells above PIC_FIELD_STATIC_MAX_CELLS (pic_field_solve_static) */
#define PIC_WARN_UNSTABLE 1     /* a numerically unstable run (§3.5): omega_pe*dt above the
                                   leapfrog stability bound 2, or a runaway electron energy:
                                   the mean kinetic energy of the electrons above
                                   max(e |V_rf|, PIC_RUNAWAY_FLOOR_EV) */
#define PIC_RUNAWAY_FLOOR_EV 100.0

#define PIC_FP64 0 /* FP64 particle state; bit-for-bit the oracle's step contract */
#define PIC_FP32 1 /* FP32 cell + offset particle state, FP64 field solve and diagnostics */

#define PIC_N_COUNTERS 16
/* counter slots of pic_diag_out.counters / pic_get_accum():
 * 0,1 electrons absorbed at x=0 / x=L; 2,3 ions absorbed at x=0 / x=L; 4 electron
 * reflections; 5 ion-induced electrons emitted; 6,7,8 electron elastic / excitation /
 * ionization events; 9,10 ion isotropic / charge-transfer events; 11,12 electron / ion
 * null-collision candidates; 13 EEPF samples; 14 sum of sampled energies in 2^-20 eV;
 * 15 births dropped for lack of capacity. */

/* The problem statement of §2 and Table 1 (gap, pressure, gas temperature, RF amplitude
 * and frequency, N_t, grid, weight W, R, gamma, nominal 1 cm^2 area of §3) plus the
 * synthetic initial load and diagnostic layout. */
typedef struct pic_params {
  double gap_m;           /* L, electrode gap (§2 step 1) */
  double pressure_pa;     /* p, argon pressure (Table 1); 0 = no gas */
  double gas_temp_k;      /* T_g (Table 1) */
  double v_rf_amp_v;      /* phi_0 of V(t) = phi_0 cos(2 pi f t) at x = 0 (§2) */
  double f_rf_hz;         /* f (§2) */
  int32_t steps_per_rf;   /* N_t, dt = 1/(f N_t) (§2) */
  int32_t n_cells;        /* N_x - 1 >= 2, dx = L/n_cells (§2 step 1) */
  double weight;          /* W, real particles per superparticle (§3.4), > 0 */
  double refl_e;          /* R, electron reflection probability in [0,1] (§2 step 5) */
  double gamma_see;       /* gamma, ion-induced emission yield in [0,1] (§2 step 5) */
  double area_m2;         /* nominal electrode area (§3: 1 cm^2) */
  double init_te_ev;      /* initial electron temperature of the uniform load */
  double see_energy_ev;   /* energy of ion-induced electrons (reading C-11) */
  int64_t init_per_species;     /* superparticles of each species in the initial load */
  int64_t capacity_per_species; /* array capacity, >= init_per_species, < 2^31 */
  uint64_t seed;          /* Philox key: (lo32(seed), hi32(seed) xor instance) */
  uint32_t instance;      /* simulation index within an ensemble */
  int32_t precision;      /* PIC_FP64 or PIC_FP32 */
  int32_t eepf_bins;      /* EEPF histogram bins over [0, eepf_emax_ev) */
  double eepf_emax_ev;
  int32_t fedf_bins;      /* wall flux-energy histogram bins over [0, fedf_emax_ev) */
  double fedf_emax_ev;
} pic_params;

typedef struct pic_handle pic_handle;

/* Output of pic_diag().  The caller sets the three sizes and the array pointers (host
 * memory it owns, or NULL to skip an array); the library fills everything else. */
typedef struct pic_diag_out {
  int32_t n_x;        /* must equal n_cells + 1 when n_e / n_i are given */
  int32_t eepf_bins;  /* must equal the handle's eepf_bins when eepf arrays are given */
  int32_t fedf_bins;  /* must equal the handle's fedf_bins when fedf arrays are given */
  double *n_e, *n_i;                 /* [n_x] time-averaged densities, m^-3 (§3.1) */
  double *eepf_energy, *eepf;        /* [eepf_bins] bin centres (eV) and EEPF, with
                                        sum sqrt(e) f de = 1 (§3.1) */
  double *fedf_energy, *fedf_e, *fedf_i; /* [fedf_bins] wall flux-energy distributions,
                                            sum f de = 1 (§3.4) */
  uint64_t counters[PIC_N_COUNTERS];
  int64_t steps_averaged, count_e, count_i;
  double ion_flux_left, ion_flux_right, ion_flux; /* m^-2 s^-1 (§3.4 Fig. 11; C-21) */
  double n_e_center, te_center_ev;                /* at L/2 (reading C-19) */
  double omega_pe_dt, omega_pe_dt_max;            /* §3.5 (centre / peak density) */
  double p_coll_e, p_coll_i;                      /* 1 - exp(-nu_max dt) (§3.5) */
  double cfl_max;                                 /* max |vx| dt/dx over electrons (§1, §3.5) */
  double lambda_d, dx_over_lambda_d, n_debye;     /* §3.5 (readings C-19, C-20) */
  double mean_energy_e_ev;                        /* mean kinetic energy of all electrons
                                                     now (runaway check of PIC_WARN_UNSTABLE) */
  int32_t status;                                 /* sticky device status (PIC_OK or error) */
} pic_diag_out;

/* Device workspace size for p (validates p).  Returns PIC_ERR_PARAM on invalid p. */
int pic_workspace_bytes(const pic_params* p, size_t* bytes);

/* Create a simulation in the caller's workspace on cuda_stream (a cudaStream_t, or NULL
 * for the legacy default stream): derives the constants of §2, builds the collision tables
 * (reading C-XS) and drive table on the host, loads the initial uniform Maxwellian
 * population (reading C-22) and deposits it.  Besides the handle it allocates one small
 * pinned host buffer (a few tens of KB: pic_diag's read-back), freed by pic_free; device
 * memory is the caller's workspace only.  Synchronises the stream before returning. */
int pic_init(const pic_params* p, void* workspace, size_t workspace_bytes, void* cuda_stream,
             pic_handle** out);

/* Enqueue n_steps timesteps (§2 steps 1-6, in that order) on the handle's stream without
 * synchronising.  Returns the sticky status observed at the end of an earlier call. */
int pic_step(pic_handle* h, int64_t n_steps);

/* Wait for the stream and return the sticky device status. */
int pic_sync(pic_handle* h);

/* Timing variant of pic_step for benchmarks: runs n_steps steps with CUDA events recorded on
 * the handle's stream around each of the step's two launches, waits for each step, and ADDS
 * the measured device milliseconds to ms_out[0] (particle pass: §2 steps 3-6 and the deposit
 * of step 1) and ms_out[1] (compaction, with the field solve of §2 steps 1-2 for the next
 * step running beside it in the same launch).  Same results as pic_step. */
int pic_step_profiled(pic_handle* h, int64_t n_steps, double* ms_out);

/* Reduce the accumulators into physical diagnostics (host side).  The electrons' max |vx|
 * and sum of |v|^2 are reduced on the device and everything is read back into the handle's
 * pinned buffer with one stream synchronization.  Returns the sticky device status if it is
 * an error, else PIC_WARN_UNSTABLE when the run is numerically unstable (see
 * PIC_WARN_UNSTABLE; §3.5 names such runs), else PIC_OK. */
int pic_diag(pic_handle* h, pic_diag_out* out);

/* Copy one species' particles to host arrays of length >= capacity; *n_out = count.
 * FP32 handles convert to FP64 at this boundary. */
int pic_get_particles(pic_handle* h, int species, double* x, double* vx, double* vy,
                      double* vz, uint32_t* id, int64_t capacity, int64_t* n_out);

/* Replace one species' particles from host arrays of length n and set its id counter,
 * then redeposit its charge (§2 step 1).  An FP32 handle reads arrays in pinned or
 * registered host memory directly from its conversion kernel (over the host link, no device
 * copy of the FP64 values); other arrays, and every array of an FP64 handle, are copied to
 * the device first.  Synchronises once, after which the host arrays may be reused. */
int pic_set_particles(pic_handle* h, int species, const double* x, const double* vx,
                      const double* vy, const double* vz, const uint32_t* id, int64_t n,
                      uint32_t next_id);

/* Number of particles of each species (synchronises). */
int pic_counts(pic_handle* h, int64_t* n_e, int64_t* n_i);

/* Enqueue on the handle's stream a copy of the two particle counts (electrons, ions) as they
 * stand when the stream reaches it into counts2[2], without synchronising.  counts2 should be
 * pinned host memory (cudaHostAlloc), else the copy is synchronous; it must stay valid until
 * the stream has passed the copy. */
int pic_counts_async(pic_handle* h, int64_t* counts2);

/* Copy the current charge counts (int64, 2^32 per superparticle, [n_cells+1] each) and the
 * potential / field of the current step (solved from those counts at the end of the
 * previous step, at init, or by pic_solve_field) to host arrays (any may be NULL).
 * Synchronises. */
int pic_get_grid(pic_handle* h, int64_t* charge_e, int64_t* charge_i, double* phi,
                 double* efield);

/* Solve the field (§2 step 2) of the current charge at V(t_n) of the current step index,
 * without advancing time or touching the accumulators.  Enqueued on the stream. */
int pic_solve_field(pic_handle* h);

/* Raw accumulators for bit-exact comparison: acc_e / acc_i [n_x] (sums of the counts per
 * averaged step), eepf [eepf_bins], fedf_e / fedf_i [fedf_bins], counters [16];
 * *steps = averaged steps.  Any pointer may be NULL.  Synchronises. */
int pic_get_accum(pic_handle* h, double* acc_e, double* acc_i, uint64_t* eepf,
                  uint64_t* fedf_e, uint64_t* fedf_i, uint64_t* counters, int64_t* steps);

/* Zero the accumulators (start of a measurement window after convergence, §2). */
int pic_reset_averages(pic_handle* h);

/* Set the step index n (selects V(t_n) and the random streams).  Enqueued. */
int pic_set_step(pic_handle* h, uint32_t step);

/* Current step index and id counters (synchronises). */
int pic_get_step(pic_handle* h, uint32_t* step, uint32_t* next_id_e, uint32_t* next_id_i);

/* Replace a species' cumulative collision-fraction table ([100001][4] doubles, contract of
 * the cross-section lookup) and nu_max; for statistical tests with synthetic rates. */
int pic_override_table(pic_handle* h, int species, const double* table, double nu_max);

/* Derived constants (dt, dx, n_g, nu_max e/i, P_max e/i) into out[7]. */
int pic_get_derived(pic_handle* h, double* out);

/* Measured FP64 pipe rate of the current device (the paper has no counterpart: the roofline
 * of the FP64 particle pass, which GB300's reduced FP64 rate bounds): rates[0] = FP64
 * operations per second issued as separate multiplies and adds (the FP64 path's own mix,
 * compiled without contraction), rates[1] = FP64 operations per second as fused multiply-adds
 * (2 per instruction).  Two timed launches of about 10-20 ms each on cuda_stream (NULL:
 * legacy default stream), 8 blocks per SM.  Synchronises. */
int pic_fp64_rate(void* cuda_stream, double* rates);

/* Release the handle and its pinned read-back buffer (host memory only; the caller frees
 * the workspace afterwards). */
void pic_free(pic_handle* h);

/* Static string for a return code. */
const char* pic_strerror(int code);

/* Description of the last CUDA error that a call made on this thread turned into
 * PIC_ERR_CUDA ("no CUDA error" if none). */
const char* pic_last_cuda_error(void);

/* ---------------------------------------------------------------------------------------
 * Checkpoint / resume.  The paper's runs converge over thousands of RF periods (§3); a
 * checkpoint holds the whole simulation state at a step boundary -- each species' particles
 * in the handle's own representation, charge counts, field, accumulators, EEPF, FEDFs,
 * counters, ids, step index and status -- so a handle resumed from it continues bit for bit
 * as the saved one would have.  Collision tables are not saved: they follow from the
 * parameters (a table replaced with pic_override_table must be replaced again).
 * --------------------------------------------------------------------------------------- */

/* Size in bytes of a checkpoint of the current state (it grows with the particle counts).
 * Synchronises. */
int pic_checkpoint_bytes(pic_handle* h, size_t* bytes);

/* Write the current state into the caller's HOST buffer of >= pic_checkpoint_bytes bytes
 * (a self-describing blob: magic "PICCKPT1", version, the parameters, then the arrays).
 * Synchronises.  PIC_ERR_PARAM if the buffer is too small. */
int pic_checkpoint_save(pic_handle* h, void* buffer, size_t bytes);

/* Replace the handle's state by a checkpoint.  The handle must have been made with the same
 * parameters (the initial load size and the capacity may differ; the capacity must hold the
 * saved counts).  Synchronises.  PIC_ERR_PARAM for a foreign, damaged or truncated blob or
 * other parameters; the handle is unchanged then. */
int pic_checkpoint_load(pic_handle* h, const void* buffer, size_t bytes);

/* ---------------------------------------------------------------------------------------
 * Ensembles: the paper's parameter scans (§3 varies N_t, N_x, W, R and γ around its base
 * cases) as many independent FP32 simulations advanced together, one cooperative launch per
 * step (replayed from a CUDA graph).  Each member is an ordinary PIC_FP32 handle made by
 * pic_init (its own parameters and workspace); all members must share one CUDA stream.
 * Every single-run call (pic_diag, pic_get_particles, ...) still works on a member.  A member
 * is advanced by pic_ensemble_step until its step index reaches its target, then left alone.
 * The results do not depend on the ensemble's schedule (owner size, grid, graph): the
 * compaction rule fixes every slot, and deposits are integer sums, so a member advanced in an
 * ensemble is bit for bit the same simulation advanced alone with pic_step.
 * --------------------------------------------------------------------------------------- */
typedef struct pic_ensemble pic_ensemble;
#define PIC_MAX_ENSEMBLE 128

/* Device workspace of an ensemble of n members (1 <= n <= PIC_MAX_ENSEMBLE). */
int pic_ensemble_workspace_bytes(int n, size_t* bytes);

/* Make an ensemble of the n handles sims[] (PIC_FP32, one stream, distinct) in the caller's
 * DEVICE workspace (256-byte aligned, kept alive until pic_ensemble_free; the members'
 * workspaces likewise).  target_steps[i] >= 0: the step index at which member i stops.
 * Records the step launch as a CUDA graph (falls back to direct launches if recording
 * fails).  Synchronises the stream.  PIC_ERR_PARAM for a member that is not PIC_FP32, on
 * another stream, repeated, or too large for the launch's shared memory (more than about
 * 7900 x 3800 superparticles of capacity per species); PIC_ERR_WORKSPACE for a missing
 * or small workspace. */
int pic_ensemble_create(pic_handle* const* sims, int n, const int64_t* target_steps,
                        void* workspace, size_t workspace_bytes, pic_ensemble** out);

/* Enqueue n_steps ensemble steps (each advances every member below its target by one step,
 * §2 steps 1-6) without synchronising; returns the status seen by an earlier sync. */
int pic_ensemble_step(pic_ensemble* e, int64_t n_steps);

/* Wait for the stream; the ensemble's status (PIC_ERR_TIMEOUT if its grid barrier ran out),
 * else the first non-OK member status. */
int pic_ensemble_sync(pic_ensemble* e);

/* Schedule: particles per list owner (256..16000), blocks per SM (1 or 2, as resources allow)
 * and whether to replay a CUDA graph.  Synchronises.  Results do not depend on it. */
int pic_ensemble_configure(pic_ensemble* e, int32_t unit, int32_t blocks_per_sm,
                           int32_t use_graph);

/* Time each schedule of the tuning space (unit 4000 / 8000 / 16000 x 1..2 blocks per SM)
 * over trial_steps real steps of the ensemble (the members advance by those steps) and keep
 * the fastest; chosen[0] = unit, chosen[1] = blocks per SM (chosen may be NULL). */
int pic_ensemble_autotune(pic_ensemble* e, int32_t trial_steps, int32_t* chosen);

/* out[5]: unit, blocks per SM, grid size, graph replay (0/1), dynamic shared memory bytes. */
int pic_ensemble_info(pic_ensemble* e, int32_t* out);

/* Release the ensemble (host memory and its graph; members and workspaces stay). */
void pic_ensemble_free(pic_ensemble* e);

/* Failure detection without a fault: runs one bulk-copy barrier wait that no copy will
 * complete (about 0.1 s of polls) and one grid barrier that expects one block more than
 * launched (about 0.5 s), in the caller's DEVICE workspace of at least
 * pic_ensemble_workspace_bytes(1) + 256 bytes.  codes[0], codes[1] receive the status each
 * wait reported: PIC_ERR_TIMEOUT when the bound works.  Synchronises. */
int pic_selftest_waits(void* workspace, size_t workspace_bytes, void* cuda_stream,
                       int32_t* codes);

/* ---------------------------------------------------------------------------------------
 * Surrogate network of the §3 parameter scans (the paper has none): BF16 tensor-core kernels.
 * --------------------------------------------------------------------------------------- */

/* C[m x n] = A[m x k] * B[n x k]^T on the tcgen05 tensor cores: A, B DEVICE arrays of BF16
 * (raw 16-bit patterns), row-major with k contiguous; C a DEVICE FP32 array, row-major.
 * FP32 accumulation.  m % 128 == 0, n % 16 == 0 with 16 <= n <= 4096, k % 16 == 0, k >= 16,
 * a and b 16-byte aligned (PIC_ERR_PARAM otherwise).  Operands are read by TMA tensor copies
 * into a 4-stage shared-memory ring; one CTA per 128 rows x (up to 256) columns.
 * Synchronises; PIC_ERR_TIMEOUT if a pipeline wait or the MMAs never completed. */
int pic_tc_gemm_bf16(const uint16_t* a, const uint16_t* b, float* c, int32_t m, int32_t n,
                     int32_t k, void* cuda_stream);

/* The network: inputs x[7] (pressure, voltage, dt, dx, weight, R, gamma, as the caller
 * normalises them), two hidden layers of 256 with GELU (tanh form), 192 linear outputs (a
 * 128-point density profile and a 64-bin log EEPF).  FP32 master parameters, BF16 copies
 * for the tensor-core GEMMs, BF16 activations, FP32 accumulation, Adam (0.9, 0.999, 1e-8),
 * mean-squared-error loss.  Flat parameter layout (pic_mlp_num_params() floats):
 * W1[256][7], b1[256], W2[256][256], b2[256], W3[192][256], b3[192].  The caller owns one
 * DEVICE workspace (pic_mlp_workspace_bytes, 256-byte aligned) sized for batches of up to
 * batch_max (a multiple of 128) rows; all x / t / y arrays below are DEVICE arrays, row-major. */
typedef struct pic_mlp pic_mlp;
int pic_mlp_num_params(void);
int pic_mlp_workspace_bytes(int32_t batch_max, size_t* bytes);
/* Uniform initialisation (bound sqrt(6 / (fan_in + fan_out)), biases 0) from seed.
 * Synchronises. */
int pic_mlp_init(int32_t batch_max, uint64_t seed, void* workspace, size_t workspace_bytes,
                 void* cuda_stream, pic_mlp** out);
/* HOST arrays of pic_mlp_num_params() floats; set also clears the Adam state.  Synchronise. */
int pic_mlp_get_params(pic_mlp* m, float* params);
int pic_mlp_set_params(pic_mlp* m, const float* params);
/* y[n][192] = network(x[n][7]), 1 <= n <= batch_max.  Enqueued. */
int pic_mlp_forward(pic_mlp* m, const float* x, int32_t n, float* y);
/* Loss and the gradient of the mean-squared error of targets t[n][192] with respect to every
 * parameter (HOST array, flat layout), without updating; n % 128 == 0.  Synchronises. */
int pic_mlp_gradients(pic_mlp* m, const float* x, const float* t, int32_t n, float* grads,
                      float* loss);
/* One Adam step with learning rate lr on a batch (n % 128 == 0).  If loss is not NULL, the
 * batch's loss before the step is returned (synchronises); otherwise only enqueued. */
int pic_mlp_train_step(pic_mlp* m, const float* x, const float* t, int32_t n, float lr,
                       float* loss);
/* Copy an intermediate array of the last pic_mlp_forward / _gradients / _train_step call to
 * a HOST buffer, first n rows (n <= the rows of that call), row-major: the values each
 * kernel stage consumed or produced, so that a test can check every stage on its own inputs.
 * BF16 arrays are raw 16-bit patterns.  Columns: X 16 (7 inputs, zero padded), Y / dY / dYh
 * 192, all others 256.  The backward arrays (which >= PIC_MLP_ACT_DY) need a last call that
 * ran the backward pass.  Synchronises.  PIC_ERR_PARAM for another `which`, n out of range,
 * or a backward array after a forward-only call. */
#define PIC_MLP_ACT_X 0     /* BF16 inputs */
#define PIC_MLP_ACT_Z1 1    /* FP32 pre-activations of layer 1 (bias added) */
#define PIC_MLP_ACT_H1 2    /* BF16 GELU(Z1) */
#define PIC_MLP_ACT_Z2 3    /* FP32 pre-activations of layer 2 */
#define PIC_MLP_ACT_H2 4    /* BF16 GELU(Z2) */
#define PIC_MLP_ACT_Y 5     /* FP32 outputs */
#define PIC_MLP_ACT_DY 6    /* FP32 loss gradient 2 (Y - T) / (n 192) */
#define PIC_MLP_ACT_DYH 7   /* its BF16 copy */
#define PIC_MLP_ACT_DZ2 8   /* FP32 gradient at Z2: (dYh W3) GELU'(Z2) */
#define PIC_MLP_ACT_DZ2H 9  /* its BF16 copy */
#define PIC_MLP_ACT_DZ1 10  /* FP32 gradient at Z1: (dZ2h W2) GELU'(Z1) */
#define PIC_MLP_ACT_DZ1H 11 /* its BF16 copy */
int pic_mlp_get_activations(pic_mlp* m, int32_t which, int32_t n, void* host);
void pic_mlp_free(pic_mlp* m);

/* ---------------------------------------------------------------------------------------
 * Allocation-free field solve.  The paper has no counterpart: it is a deployment variant of
 * the field solve of §2 step 2 (exact discrete Green's function, reading C-23) for callers
 * that cannot allocate device memory: processes whose caching allocator has already reserved
 * the device's free memory (a further cudaMalloc fails or forces the pool to release
 * memory), code on latency-critical paths that must not call cudaMalloc / cudaFree (they can
 * synchronise the whole device and stall other streams), and plug-ins whose host gives them
 * device pointers but no allocator or workspace to hand over.  It uses no handle, no
 * workspace and no allocating call (CUDA or otherwise): its one scratch array, the int128
 * sums S_j (16 bytes per node), is a file-scope device array of
 * PIC_FIELD_STATIC_MAX_CELLS + 1 nodes (1 MiB) inside libpic.so, held by every device that
 * loads the library until the process exits.
 *
 * charge_e, charge_i  DEVICE int64 arrays [n_cells + 1], the charge counts at the nodes in
 *                     units of 2^-32 superparticles (the layout pic_get_grid returns).
 * n_cells             N, 2 <= N <= PIC_FIELD_STATIC_MAX_CELLS.
 * gap_m, weight, area_m2, v_left
 *                     electrode gap L, superparticle weight W, electrode area A, and the
 *                     potential of the driven electrode at x = 0 (the one at x = L is 0 V).
 * phi, efield         DEVICE double arrays [n_cells + 1] written by the call (caller-owned).
 * cuda_stream         cudaStream_t to enqueue on (NULL: legacy default stream).
 *
 * All four arrays must be device (or managed) memory of the current device, 8-byte aligned,
 * and must not overlap each other.  For the same counts and voltage the result is bit for
 * bit that of pic_solve_field / pic_get_grid of a PIC_FP64 handle with the same gap, weight,
 * area and n_cells.  A PIC_FP32 handle's field solve multiplies by rounded reciprocals where
 * this one divides, so its phi and E agree with these within one unit in the last place.
 * Nothing has to be zeroed beforehand: every scratch element read is written earlier in the
 * same launch.
 *
 * Returns PIC_ERR_SCRATCH for n_cells > PIC_FIELD_STATIC_MAX_CELLS (nothing is launched),
 * PIC_ERR_PARAM for other invalid arguments (non-device or misaligned pointer, N < 2,
 * non-positive or non-finite sizes), PIC_ERR_CUDA if the set-up or the launch fails.
 * Enqueued only: the results are ready when the stream reaches them.
 *
 * Set-up: the first call on each device, with that device current, looks up the scratch
 * array's device address (cudaGetSymbolAddress) and caches it for later calls; that first
 * call should come before any stream capture.  The cached address belongs to the device's
 * current context: after cudaDeviceReset, unload and reload the library before calling again.
 * Concurrency: all calls on one device share the scratch array, which keeps the last call's
 * contents, so two calls whose launches can run at the same time (on different streams) race
 * and give wrong results.  Order them on one stream or with events.
 * --------------------------------------------------------------------------------------- */
#define PIC_FIELD_STATIC_MAX_CELLS 65536
int pic_field_solve_static(const int64_t* charge_e, const int64_t* charge_i, int32_t n_cells,
                           double gap_m, double weight, double area_m2, double v_left,
                           double* phi, double* efield, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
