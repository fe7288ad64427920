// pb_internal.cuh -- device data layout and shared definitions of libpb.
//
// HBM layout of one grid (all node arrays padded in x to a pitch px, a
// multiple of 16 elements with px >= nx + 1, so every row of every array
// starts 16-byte aligned -- a TMA requirement, also for the one-byte codes --
// and the (nx+1)-th x-edge fits in the row):
//   code   uint8  [nz][ny][px]   packed coefficients, one byte per node:
//                                bit 0/1 x-/x+ edge inside (eps_in), bit 2/3 y-/y+,
//                                bit 4/5 z-/z+, bit 6 node inside an atom (lambda = 0
//                                when the ion-exclusion mask is on);
//                                pad bytes are 0
//   b      f64    [nz][ny][px]   right-hand side of Eq. (4) with the boundary folded in
//   x64    f64    [nz][ny][px]   solution (FP64)
//   d,z,p0,p1,ap  T [nz][ny][px] CG work vectors in the inner precision T: inner
//                                x increment, z = M^-1 r, directions, A p
//   ex     C      [nz][ny][px]   explicit modes only: edge (i-1, i) at column i, i = 0..nx
//   ey     C      [nz][ny+1][px] edge (j-1, j) at row j
//   ez     C      [nz+1][ny][px] edge (k-1, k) at plane k
//   diag   C      [nz][ny][px]   explicit modes only (pads hold 1)
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace pb {

struct __align__(32) dbl4 {  // four doubles, 32-byte aligned (atoms: x, y, z, q or radius)
  double x, y, z, w;
};

// Stencil tiles: W x H columns (W a multiple of NV, W <= WMAX, H <= HMAX,
// W*H <= NV*NT) marching over a z range; one CTA of NT threads per tile, each
// thread owning NV consecutive x columns.
constexpr int NT = 256;        // threads per stencil CTA
constexpr int NV = 4;          // x columns per thread (16-byte vectors of FP32)
constexpr int WMAX = 64;       // widest tile
constexpr int HMAX = 24;       // tallest tile
#ifndef PB_TILE_NODES
#define PB_TILE_NODES 1024
#endif
constexpr int TILE_NODES = PB_TILE_NODES;  // W*H at most (<= NV*NT)
constexpr int NT_UPD = 256;    // threads per update CTA
constexpr int CH = 2048;       // fewest elements per chunk of the update pass
// CTAs of the right-hand-side fold (each writes one partial of ||b||^2;
// 256 measured 33% slower on the serving stream's grids)
#ifndef PB_FOLD_CTAS
#define PB_FOLD_CTAS 1024
#endif
#ifndef PB_RESID_TZ
#define PB_RESID_TZ 4
#endif
constexpr int RESID_TZ = PB_RESID_TZ;  // z planes per item of the residual pass
constexpr int NDTAB = 14;      // diagonal table entries: (#inside edges 0..6) x (lambda 0/1)
constexpr int PITCH_ALIGN = 16;  // node-array pitch in elements (TMA: 16-byte strides for bytes)

enum Phase : int { PH_RESID = 0, PH_INNER = 1, PH_DONE = 2, PH_START = 3 };
enum Mode : int { MODE_F64 = 0, MODE_F32 = 1, MODE_F32_REFINE = 2 };
enum Coef : int { COEF_PACKED = 0, COEF_F32 = 1, COEF_BF16 = 2, COEF_F64 = 3 };

// Per-instance scalars of the CG recurrences (device resident, written only
// by the finalising CTA of each phase kernel).
struct Scal {
  double alpha;        // alpha of the latest step; folded into x by the next kernel
  double beta;         // beta for the next direction update
  double rz_old;       // r.z of the current residual
  double ref_norm;     // ||rhs|| of the current inner solve
  double relres;       // recursive residual / ref_norm
  double relres_true;  // ||b - A x|| / ||b|| (FP64)
  double bnorm;        // ||b||
  double itol;         // tolerance of the current inner solve
  int phase;           // Phase
  int pbuf;            // index of the buffer holding the latest direction p
  int iter;            // iterations of the current inner solve
  int total_iter;      // iterations over all inner solves
  int outer;           // inner solves started
  int status;          // pb_status
  unsigned cnt2, cnt3;  // tile-completion counters (last-CTA-done pattern)
  int xbuf;             // which of x64 / x64b holds the current solution
};

// Everything a phase kernel needs to know about one instance (one grid).
// The TMA descriptors come first (64-byte aligned).
struct alignas(64) Inst {
  CUtensorMap tm_z, tm_p0, tm_p1, tm_code, tm_x0, tm_x1;  // z, p buffers, codes, inner x
  CUtensorMap tm_zc;                  // z, centre box (the update pass)
  int W, H;                           // stencil tile
  int cw;                             // width of the code box (bytes, multiple of 16)
  int stage_bytes, off_p, off_c, off_x, tma_bytes;  // TMA stage layout and bytes per stage
  int tma_bytes_upd;                  // ... per stage of the update pass (no second halo box)
  int stage_bytes_upd, off_c_upd, off_x_upd;  // its stage layout: p box, codes, z centre
  int rows_per_chunk;                 // update-pass chunk
  uint32_t vx_magic;                  // ceil(2^32 / vectors per row), for row = f*magic >> 32
  int nx, ny, nz, px;
  int tiles_x, tiles_y, tiles_z, tz;  // stencil tile decomposition
  int n_st, n_ch;                     // stencil tiles, elementwise chunks
  int st_base, ch_base;               // offsets into the partial-sum arrays
  int rtz, n_rs, rs_base;             // residual pass: the stencil tiles cut into z
                                      // pieces of rtz planes, their count, partials
  int mode, precond, coef, max_iter, max_outer, periodic;
  double tol, inner_tol, bnorm;
  size_t n_pad;                       // nz*ny*px
  const uint8_t *code;
  const void *ex, *ey, *ez, *diag;    // explicit coefficient arrays (inner precision)
  const double *rx, *ry, *rz, *rdiag; // FP64 arrays for the residual pass when the inner
                                      // arrays are rounded copies (harmonic-average
                                      // dielectric); NULL: the codes are exact
  double *x64, *x64b;                 // solution, double-buffered across RESID passes
  const double *b;
  void *d, *z, *p0, *p1, *ap;         // inner work vectors (z = M^-1 r)
  Scal *s;
  const int *err;                     // the grid's setup error word
  const double *bnorm2;               // ||b||^2 as the setup left it
  double ein, eout, kbh2;
  double dtab[NDTAB], idtab[NDTAB];   // FP64 diagonal and its inverse by (n_in, lambda)
  float dtab32[NDTAB], idtab32[NDTAB];
  float ein32, eout32;
};

struct Item {  // one unit of work of a phase kernel
  int inst;
  int tile;
};

// Ints of the count block of a batch: [0] stencil items, [1] update items,
// [2] residual passes pending, [3] unused, [4..9] work counters, [10] the
// residual list of a single grid (its instance 0).
constexpr int PB_COUNTS = 12;

struct Batch {  // device pointers describing a batch of instances
  const Inst *inst;
  const Item *st_items;  // stencil tiles of all instances
  const Item *ch_items;  // elementwise chunks of all instances
  const int *n_items;    // [0]: stencil items, [1]: update items (device memory, so a
                         // captured device graph serves any active set)
  unsigned *work;        // [0] next stencil item, [1] stencil CTAs done, [2] next update
                         // item, [3] update CTAs done, [4] next residual item, [5]
                         // residual CTAs done: zero between launches
  int *resid_pending;    // instances waiting for a residual pass (0 skips the pass)
  int *resid_list;       // ... which ones, in the order they asked
  double *rs_part;       // 2 doubles per residual item
  double *st_part;       // 3 doubles per stencil tile
  double *ch_part;       // 2 doubles per chunk
  int *error;            // device error word
};

// Index of a code byte in the diagonal tables: 2 * (#edges inside) + lambda.
__host__ __device__ inline int dtab_index(uint32_t c) {
#ifdef __CUDA_ARCH__
  return 2 * __popc(c & 63u) + (((c >> 6) & 1u) ^ 1u);
#else
  return 2 * __builtin_popcount(c & 63u) + (((c >> 6) & 1u) ^ 1u);
#endif
}

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
inline int pitch_of(int nx) { return round_up(nx + 1, PITCH_ALIGN); }

}  // namespace pb
