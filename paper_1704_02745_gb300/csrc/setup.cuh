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
  // weighted harmonic-average dielectric (Sec. 2.7): when ex64 is not NULL the
  // setup fills the FP64 edge arrays (layouts of pb_internal.cuh, pads 1) from
  // the fraction of each edge inside the atoms, and folds the boundary with them
  double *ex64 = nullptr, *ey64 = nullptr, *ez64 = nullptr;
  void *cell_buf = nullptr;   // cell_buffer_bytes(plan, n_atoms) bytes
  double r_max = 0;           // largest atom radius
};

// Cells of the harmonic-average setup for a grid and the largest atom radius:
// cubes of side r_max + h from one cube below the ghost layer.
struct CellPlan {
  double size;
  int ncx, ncy, ncz;
  long n() const { return (long)ncx * ncy * ncz; }
};
CellPlan cell_plan(const Geom &g, double r_max);
size_t cell_buffer_bytes(const CellPlan &p, int n_atoms);

cudaError_t launch_setup(const SetupArgs &a, cudaStream_t st);
cudaError_t launch_expand(const uint8_t *code, const Geom &g, double ein, double eout, double kbh2,
                          int coef, void *ex, void *ey, void *ez, void *diag, cudaStream_t st);
cudaError_t launch_export_lambda(const uint8_t *code, const Geom &g, uint8_t *lam, cudaStream_t st);
// Harmonic-average grids: diag64 = the six FP64 edges + kbh2 * lambda, and the
// inner solve's copies (coef PB_COEF_F32 / PB_COEF_BF16) of the FP64 arrays.
cudaError_t launch_harmonic_finish(const uint8_t *code, const Geom &g, double kbh2, const double *ex64,
                                   const double *ey64, const double *ez64, double *diag64, int coef,
                                   void *ex, void *ey, void *ez, void *diag, cudaStream_t st);

}  // namespace pb
