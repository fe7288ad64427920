// setup.cuh -- launchers of the grid setup kernels (setup.cu).
#pragma once
#include "pb_internal.cuh"

namespace pb {

struct Geom {  // grid geometry as the setup kernels see it
  int nx, ny, nz, px;
  double h, ox, oy, oz;
  int periodic;  // every axis periodic with period n*h
};

struct SetupArgs {
  Geom g;
  int n_atoms;
  const dbl4 *atoms_xyzr;  // x, y, z, radius
  const dbl4 *atoms_xyzq;  // x, y, z, charge
  uint8_t *code;              // n_pad bytes
  double *b;                  // n_pad, zeroed by the caller
  double *ghost;              // 2(ny nz + nx nz + nx ny)
  double *scratch;            // >= 256 doubles
  double *bnorm2;             // one double: ||b||^2
  int *err;                   // device error word
  double kappa, ein, eout, c4pi_h;
  double q_scale;             // fixed-point scale of the charge accumulation (power of two)
  int kappa_mask, dh_f32;
};

cudaError_t launch_setup(const SetupArgs &a, cudaStream_t st);
cudaError_t launch_expand(const uint8_t *code, const Geom &g, double ein, double eout, double kbh2,
                          int coef, void *ex, void *ey, void *ez, void *diag, cudaStream_t st);
cudaError_t launch_export_lambda(const uint8_t *code, const Geom &g, uint8_t *lam, cudaStream_t st);

}  // namespace pb
