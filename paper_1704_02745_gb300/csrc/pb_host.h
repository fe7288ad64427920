// pb_host.h -- host-side objects of libpb shared by the C-ABI translation units.
#pragma once
#include <atomic>
#include <string>
#include <vector>

#include "pb.h"
#include "pb_internal.cuh"
#include "setup.cuh"
#include "solve.cuh"

struct pb_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 1;
  pb::Scal *host_scal = nullptr;  // pinned, for convergence polls
  // pb_ctx_stats counters; a server's internal context counts into its parent's
  std::atomic<unsigned long long> launches{0}, h2d{0}, d2h{0};
  pb_ctx *stats = this;
};

struct pb_grid {
  pb_ctx *ctx = nullptr;
  pb_grid_desc d{};
  pb::Geom g{};
  size_t n_pad = 0;
  long n_ghost = 0;
  int n_atoms = 0, atom_cap = 0;
  pb::dbl4 *h_atoms = nullptr;  // pinned host staging of the atoms: xyzq, then xyzr
  double kappa = 0, kbh2 = 0, bnorm = 0;
  // setup arrays
  uint8_t *code = nullptr;
  double *b = nullptr, *ghost = nullptr, *scratch = nullptr;
  pb::dbl4 *xyzq = nullptr, *xyzr = nullptr;
  int *err = nullptr;
  // explicit coefficients (FP32 / BF16 eps with an FP32 diagonal, or FP64)
  void *ex = nullptr, *ey = nullptr, *ez = nullptr, *diag = nullptr;
  void *ex64 = nullptr, *ey64 = nullptr, *ez64 = nullptr, *diag64 = nullptr;
  // solve workspace
  double *x64 = nullptr, *x64b = nullptr;
  void *d32 = nullptr, *z32 = nullptr, *p032 = nullptr, *p132 = nullptr, *ap32 = nullptr;
  double *z64 = nullptr, *p064 = nullptr, *p164 = nullptr, *ap64 = nullptr;
  pb::Scal *scal = nullptr;  // own allocation, or a slot of a server's scalar array
  bool own_scal = true;
  int *counts = nullptr;     // device: stencil and update item counts of the single-grid batch
  bool batch = false;        // a server's grid: its work lists and scalars are the server's
  void *cell_buf = nullptr;  // harmonic-average setup: cell list of the atoms
  size_t cell_cap = 0;
  struct pb_mg *mg = nullptr;  // multigrid hierarchy (built by the first GMG solve)
  pb::Inst *dinst = nullptr;
  pb::Item *st_items = nullptr, *ch_items = nullptr;
  double *st_part = nullptr, *ch_part = nullptr, *rs_part = nullptr;
  int W = 0, H = 0, tiles_x = 0, tiles_y = 0, tiles_z = 0, tz = 0, n_st = 0, n_ch = 0;
  int rtz = 0, n_rs = 0;  // residual-pass z pieces
  int rows_per_chunk = 0;
  // cached device graph of `graph_ticks` ticks
  cudaGraphExec_t graph = nullptr;
  int graph_mode = -1, graph_coef = -1, graph_ticks = 0;
};

pb_status pb_fail(pb_status s, const std::string &msg);
pb_status pb_dalloc(void **p, size_t bytes);
void pb_grid_release(pb_grid *g);
int pb_inner_coef(const pb_grid *g, int mode);
pb_status pb_ensure_workspace(pb_grid *g, int mode);
pb_status pb_make_inst(const pb_grid *g, const pb_solve_opts *o, int mode, int coef, pb::Inst &I);
pb::Scal pb_initial_scal(double bnorm);
pb_status pb_check_desc(const pb_grid_desc *d);
pb_status pb_check_atoms(int n_atoms, const double *xyz, const double *q, const double *radius);
// Return a pb_status from a CUDA error (in functions returning pb_status).
#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return pb_fail(e_ == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA,            \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

// gmg.cu: geometric-multigrid preconditioned CG, and the hierarchy's release.
pb_status pb_gmg_solve(pb_grid *g, const pb_solve_opts *o, double *phi, pb_solve_info *info);
void pb_mg_release(struct pb_mg *m);
pb_status pb_grid_create(pb_ctx *ctx, const pb_grid_desc *desc, bool batch, pb_grid **out);
// Tile plan of a server grid: fewest x tiles, height_pct percent of the
// tallest tile height, z chunks of at least min_planes planes filling the
// resident stencil CTAs of kg.
void pb_batch_plan_grid(pb_grid *g, const pb::KernelGrid &kg, int min_planes, int height_pct);
// st: the stream of the setup work (NULL: the grid's context stream)
pb_status pb_run_setup(pb_grid *g, int n_atoms, const double *xyz, const double *q,
                       const double *radius, bool sync, cudaStream_t st = nullptr);
pb_status pb_run_ticks(pb_grid *g, int mode, int coef, int ticks);

// Layout of a grid's FP64 scratch buffer.
enum : size_t {
  SCR_ENERGY = 0,        // energy result
  SCR_BNORM2 = 1,        // ||b||^2 from the setup
  SCR_SETUP = 8,                        // PB_FOLD_CTAS partials of the setup's norm reduction
  SCR_ENERGY_PART = 8 + PB_FOLD_CTAS    // per-CTA partials of the energy (one per 256 atoms)
};
