// pic_launch.h -- host-side launchers of the libpic kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include "pic_dev.cuh"

namespace pic {

size_t field_smem_bytes(int nx);
size_t push_smem_bytes(int nx);

cudaError_t launch_init_load(const DevCtx& K, int species, long long n0, cudaStream_t s);
// deposit of the first n particles of species s into counts buffer buf (buf < 0: the
// current step's)
cudaError_t launch_deposit(const DevCtx& K, int species, int buf, long long n, cudaStream_t s);
// a replaced population's count, next id and cleared counts of the current step, on the device
cudaError_t launch_set_counts(const DevCtx& K, int species, long long n, unsigned next_id,
                              cudaStream_t s);
// field of the current step from the current counts (no accumulation)
cudaError_t launch_field(const DevCtx& K, cudaStream_t s);
// particle pass of the current step
cudaError_t launch_push_fp64(const DevCtx& K, int grid, cudaStream_t s);
// placement of births and tail survivors of the current step; block 0 closes the step's
// accumulation, solves the field of the next step and advances the step index
cudaError_t launch_place_fp64(const DevCtx& K, int grid, cudaStream_t s);
cudaError_t launch_set_step(const DevCtx& K, unsigned step, cudaStream_t s);
// pic_diag's device side in one launch: the electrons' max |vx| and sum of |v|^2 (the
// handle's velocity units) over the live count, then the state, counters, averages and
// distributions written to out_dev (device-mapped host memory) at these byte offsets
struct DiagOffsets {
  size_t state, counters, acc, eepf, fedf;
};
cudaError_t launch_diag(const DevCtx& K, bool fp32, char* out_dev, const DiagOffsets& off,
                        cudaStream_t s);
int push_fp64_blocks_per_sm(int nx);
// FP64 pipe probe (8 x SMs blocks of 256 threads, iters steps of 8 chains): elapsed ms of the
// timed launch and the FP64 operations it executed
cudaError_t fp64_probe(bool fma, int sms, int iters, double* ms, double* ops, cudaStream_t s);
// raise the dynamic shared-memory limit of the grid-sized kernels for nx nodes
cudaError_t configure_kernels(int nx);
// the placement launch's shared memory for nx nodes and nlist list owners
cudaError_t configure_place_fp64(int nx, int nlist);

// FP32 particle path (pic_fp32.cu)
cudaError_t launch_push_fp32(const DevCtx& K, int grid, cudaStream_t s);
cudaError_t launch_place_fp32(const DevCtx& K, int grid, cudaStream_t s);
// FP64 SI arrays <-> FP32 cell-unit state of one species (n particles)
// FP64 SI arrays (device-readable: the FP64 buffers or mapped host memory) -> FP32 state
cudaError_t launch_convert_from(const DevCtx& K, int species, long long n, const double* x,
                                const double* vx, const double* vy, const double* vz,
                                const unsigned* id, cudaStream_t s);
cudaError_t launch_convert(const DevCtx& K, int species, long long n, bool to_fp32,
                           cudaStream_t s);
cudaError_t configure_kernels32(int nx);
cudaError_t configure_place_fp32(int nx, int nlist);
// ensemble of FP32 simulations, one cooperative launch per step (pic_fp32.cu)
size_t ensemble_pipes_offset(int nx_max);
size_t ensemble_smem_bytes(int nx_max, int gcap_max);
cudaError_t configure_ensemble(size_t smem);
int ensemble_blocks_per_sm(size_t smem);
cudaError_t launch_ensemble(EnsDev* E, int grid, size_t smem, cudaStream_t s);
// bounded-wait self-test: status[0] bulk-copy barrier, status[1] grid barrier (kStTimeout)
cudaError_t launch_selftest_waits(EnsDev* E, int* status, cudaStream_t s);
int push_fp32_blocks_per_sm(int nx);

}  // namespace pic
