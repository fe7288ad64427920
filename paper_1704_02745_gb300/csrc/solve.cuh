// solve.cuh -- launchers of the phase kernels (solve.cu) and the helper
// kernels (ops.cu).
#pragma once
#include "pb_internal.cuh"

namespace pb {

struct KernelGrid {  // persistent grid sizes of the phase kernels
  int stencil_blocks, update_blocks, resid_blocks, update_tile_blocks;
  int update_fast_blocks;  // the fast build of the tile update pass
  int stencil_per_sm, update_per_sm;  // resident CTAs per SM
  int tile_update;  // 1: the update pass runs over the stencil tiles and forms Ap
                    // again (k_update_tile; the stencil pass stores no Ap, Inst.ap
                    // is NULL); 0: over row chunks, reading the stored Ap (k_update)
  int fast;         // 1: every grid of the launch is FP32 with packed codes and no wrap:
                    // the stencil and tile update passes run their fast builds
  int single;       // 1: launches over one grid (the lean stencil pass then runs its
                    // single-grid configuration)
};

// Shared-memory layout of one TMA stage of the stencil pass for a W x H tile
// of elements of `es` bytes: r and p_old boxes (W + 2*NV) x (H + 2) starting
// NV columns left of the tile (16-byte aligned for FP32 and FP64), the code box
// cw x (H + 2) bytes, the x box W x H; every box 128-byte aligned.
struct StageLayout {
  int rw, cw, rows, off_p, off_c, off_x, stage_bytes, tma_bytes, tma_bytes_upd;
  int off_c_upd, off_x_upd, stage_bytes_upd;  // update pass: p box, codes, z centre
};
inline StageLayout stage_layout(int W, int H, int es) {
  StageLayout L;
  L.rw = W + 2 * NV;
  L.rows = H + 2;
  L.cw = round_up(W + 17, 16);  // covers x0-1 .. x0+W from a 16-aligned start
  const int rbytes = L.rw * L.rows * es, cbytes = L.cw * L.rows, xbytes = W * H * es;
  L.off_p = round_up(rbytes, 128);
  L.off_c = L.off_p + round_up(rbytes, 128);
  L.off_x = L.off_c + round_up(cbytes, 128);
  L.stage_bytes = L.off_x + round_up(xbytes, 128);
  L.tma_bytes = 2 * rbytes + cbytes + xbytes;
  L.tma_bytes_upd = rbytes + cbytes + xbytes;  // update pass: p, codes, z centre
  L.off_c_upd = round_up(rbytes, 128);
  L.off_x_upd = L.off_c_upd + round_up(cbytes, 128);
  L.stage_bytes_upd = L.off_x_upd + round_up(xbytes, 128);
  return L;
}
// Largest stage over every tile the planner may choose.
inline int max_stage_bytes(int es) {
  int m = 0;
  for (int W = NV; W <= WMAX; W += NV)
    for (int H = 1; H <= HMAX && W * H <= TILE_NODES; H++) {
      const int b = stage_layout(W, H, es).stage_bytes;
      m = b > m ? b : m;
    }
  return m;
}
inline int max_stage_bytes_upd(int es) {
  int m = 0;
  for (int W = NV; W <= WMAX; W += NV)
    for (int H = 1; H <= HMAX && W * H <= TILE_NODES; H++) {
      const int b = stage_layout(W, H, es).stage_bytes_upd;
      m = b > m ? b : m;
    }
  return m;
}
// Largest ring plane ((W + 2*NV) x (H + 2) cells) over the same tiles.
constexpr int max_ring_cells() {
  int m = 0;
  for (int W = NV; W <= WMAX; W += NV)
    for (int H = 1; H <= HMAX && W * H <= TILE_NODES; H++) {
      const int c = (W + 2 * NV) * (H + 2);
      m = c > m ? c : m;
    }
  return m;
}

// One tick: the residual pass (instances that asked for one), the stencil
// pass, then the update pass over every instance.
cudaError_t launch_tick(const Batch &B, int mode, int coef, const KernelGrid &kg, cudaStream_t st);
// which: bit 2 = residual pass, bit 0 = stencil pass, bit 1 = update pass
// (launched in that order).
cudaError_t launch_phase(const Batch &B, int mode, int coef, const KernelGrid &kg, int which,
                         cudaStream_t st);
KernelGrid kernel_grid(int mode, int coef, int num_sms, bool single);
// Start solves on the listed instances from their device-side setup state
// (each one that has work asks for a residual pass: appended to resid_list,
// counted in *resid_pending).
cudaError_t launch_start(const Inst *inst, const int *list, int n, int *resid_pending,
                         int *resid_list, cudaStream_t st);

// ops.cu
cudaError_t launch_pack(const double *dense, double *padded, int nx, int ny, int nz, int px,
                        cudaStream_t st);
cudaError_t launch_unpack(const double *padded, double *dense, int nx, int ny, int nz, int px,
                          cudaStream_t st);
cudaError_t launch_apply(const Inst &I, const Inst *dI, const void *u, void *au, int dtype,
                         cudaStream_t st);
// phi: nz x ny rows of px elements (px = nx: dense).  An atom whose
// trilinear cell leaves the grid makes the energy NaN (periodic: corners wrap).
cudaError_t launch_energy(const dbl4 *xyzq, int n_atoms, int nx, int ny, int nz, int px,
                          int periodic, double h, double ox, double oy, double oz,
                          const double *phi, double *scratch, double *out, cudaStream_t st);

}  // namespace pb
