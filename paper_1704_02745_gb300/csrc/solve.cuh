// solve.cuh -- launchers of the phase kernels (solve.cu) and the helper
// kernels (ops.cu).
#pragma once
#include "pb_internal.cuh"

namespace pb {

struct KernelGrid {  // persistent grid sizes of the phase kernels
  int stencil_blocks, update_blocks;
};

// One tick: the stencil pass then the update pass over every instance.
cudaError_t launch_tick(const Batch &B, int mode, int coef, const KernelGrid &kg, cudaStream_t st);
// which: 1 = stencil pass only, 2 = update pass only, 3 = both.
cudaError_t launch_phase(const Batch &B, int mode, int coef, const KernelGrid &kg, int which,
                         cudaStream_t st);
KernelGrid kernel_grid(int mode, int coef, int num_sms);

// ops.cu
cudaError_t launch_pack(const double *dense, double *padded, int nx, int ny, int nz, int px,
                        cudaStream_t st);
cudaError_t launch_unpack(const double *padded, double *dense, int nx, int ny, int nz, int px,
                          cudaStream_t st);
cudaError_t launch_apply(const Inst &I, const Inst *dI, const void *u, void *au, int dtype,
                         cudaStream_t st);
cudaError_t launch_energy(const dbl4 *xyzq, int n_atoms, int nx, int ny, int nz, double h,
                          double ox, double oy, double oz, const double *phi, double *scratch,
                          double *out, cudaStream_t st);

}  // namespace pb
