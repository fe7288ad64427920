// api.cu -- C ABI of libpb (declared in include/pb.h): contexts, grid setup,
// operator application, the Jacobi-PCG solve driver and the energy.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include <mutex>

#include "pb.h"
#include "pb_host.h"
#include "pb_internal.cuh"
#include "setup.cuh"
#include "solve.cuh"

using namespace pb;

static thread_local std::string g_err;

pb_status pb_fail(pb_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

extern "C" const char *pb_last_error(void) { return g_err.c_str(); }

#ifdef PB_FAULT_TEST
// Test builds only (-DPB_FAULT_TEST, never the product library): the next
// `count` device allocations of the library fail as an exhausted device would.
static std::atomic<int> g_fault_fail_allocs{0};
extern "C" int pb_test_fail_allocs(int count) {
  g_fault_fail_allocs.store(count);
  return 0;
}
#endif

pb_status pb_dalloc(void **p, size_t bytes) {
  *p = nullptr;
#ifdef PB_FAULT_TEST
  if (g_fault_fail_allocs.load() > 0 && g_fault_fail_allocs.fetch_sub(1) > 0)
    return pb_fail(PB_ERR_OOM, "cudaMalloc(" + std::to_string(bytes) + "): injected failure");
#endif
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return pb_fail(e == cudaErrorMemoryAllocation ? PB_ERR_OOM : PB_ERR_CUDA,
                   std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return PB_OK;
}

static void dfree(void *p) {
  if (p) cudaFree(p);
}

// ---------------------------------------------------------------------------
// Context

extern "C" pb_status pb_create(pb_ctx **out, int device, void *cuda_stream) {
  if (!out) return pb_fail(PB_ERR_ARG, "pb_create: out is NULL");
  *out = nullptr;
  int n = 0;
  CK(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return pb_fail(PB_ERR_ARG, "pb_create: no such device");
  CK(cudaSetDevice(device));
  pb_ctx *c = new pb_ctx();
  c->device = device;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return pb_fail(PB_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMallocHost((void **)&c->host_scal, sizeof(Scal) * 64) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return pb_fail(PB_ERR_CUDA, "cudaMallocHost failed");
  }
  *out = c;
  return PB_OK;
}

extern "C" pb_status pb_destroy(pb_ctx *c) {
  if (!c) return PB_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  cudaFreeHost(c->host_scal);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return PB_OK;
}

extern "C" pb_status pb_ctx_stats(pb_ctx *c, uint64_t *launches, uint64_t *h2d, uint64_t *d2h) {
  if (!c) return pb_fail(PB_ERR_ARG, "pb_ctx_stats: NULL ctx");
  if (launches) *launches = c->launches.load();
  if (h2d) *h2d = c->h2d.load();
  if (d2h) *d2h = c->d2h.load();
  return PB_OK;
}

// ---------------------------------------------------------------------------
// Physics constants of the host side.

// Inverse Debye length squared (1/A^2) of a 1:1 salt of ionic strength I
// (mol/L) at temperature T in a solvent of relative permittivity eps:
// 2 N_A e^2 (1000 I) / (eps0 eps k_B T) m^-2.
static double debye_kappa2(double ionic, double temp, double eps) {
  const double avogadro = 6.02214076e23, charge = 1.602176634e-19;
  const double vacuum_perm = 8.8541878128e-12, boltzmann = 1.380649e-23;
  return 2.0 * avogadro * charge * charge * (1000.0 * ionic) /
         (vacuum_perm * eps * boltzmann * temp) * 1e-20;
}

static bool finite_all(const double *a, size_t n) {
  for (size_t t = 0; t < n; t++)
    if (!std::isfinite(a[t])) return false;
  return true;
}

pb_status pb_check_desc(const pb_grid_desc *d) {
  if (!d) return pb_fail(PB_ERR_ARG, "grid desc is NULL");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return pb_fail(PB_ERR_ARG, "empty grid");
  if ((double)d->nx * d->ny * d->nz > 2.0e9) return pb_fail(PB_ERR_ARG, "grid too large");
  if (!(d->h > 0) || !std::isfinite(d->h)) return pb_fail(PB_ERR_ARG, "h must be > 0");
  if (!(d->eps_in > 0) || !(d->eps_out > 0)) return pb_fail(PB_ERR_ARG, "eps must be > 0");
  if (!(d->ionic_strength >= 0) || !(d->temperature > 0))
    return pb_fail(PB_ERR_ARG, "ionic strength must be >= 0 and temperature > 0");
  if (!finite_all(d->origin, 3)) return pb_fail(PB_ERR_ARG, "origin not finite");
  if (d->coef < PB_COEF_PACKED || d->coef > PB_COEF_F64) return pb_fail(PB_ERR_ARG, "bad coef");
  if (d->dh_precision != PB_F64 && d->dh_precision != PB_F32)
    return pb_fail(PB_ERR_ARG, "bad dh_precision");
  if (d->periodic != 0 && d->periodic != 1) return pb_fail(PB_ERR_ARG, "bad periodic flag");
  if (d->periodic && (d->nx < 3 || d->ny < 3 || d->nz < 3))
    return pb_fail(PB_ERR_ARG, "a periodic grid needs at least 3 nodes per axis");
  if (d->periodic && !(d->ionic_strength > 0))
    return pb_fail(PB_ERR_ARG, "a periodic grid needs salt (ionic_strength > 0): without it A is singular");
  if (d->eps_model != PB_EPS_MIDPOINT && d->eps_model != PB_EPS_HARMONIC)
    return pb_fail(PB_ERR_ARG, "bad eps_model");
  if (d->eps_model == PB_EPS_HARMONIC && d->coef == PB_COEF_PACKED)
    return pb_fail(PB_ERR_ARG, "the harmonic-average dielectric needs explicit coefficients (coef f32, bf16 or f64)");
  if (d->eps_model == PB_EPS_HARMONIC && d->periodic)
    return pb_fail(PB_ERR_ARG, "the harmonic-average dielectric is for the free-space boundary");
  return PB_OK;
}

// ---------------------------------------------------------------------------
// Grid

void pb_grid_release(pb_grid *g) {
  if (!g) return;
  if (g->graph) cudaGraphExecDestroy(g->graph);
  void *ptrs[] = {g->code, g->b, g->ghost, g->xyzq, g->xyzr, g->err, g->counts, g->scratch, g->ex, g->ey,
                  g->ez, g->diag, g->ex64, g->ey64, g->ez64, g->diag64, g->x64, g->x64b, g->d32,
                  g->z32, g->p032, g->p132, g->ap32, g->z64, g->p064, g->p164, g->ap64,
                  g->own_scal ? (void *)g->scal : nullptr, g->dinst, g->st_items, g->ch_items, g->st_part,
                  g->ch_part, g->rs_part};
  for (void *p : ptrs) dfree(p);
  dfree(g->cell_buf);
  pb_mg_release(g->mg);
  if (g->h_atoms) cudaFreeHost(g->h_atoms);
  delete g;
}

extern "C" pb_status pb_free_grid(pb_grid *g) {
  if (!g) return PB_OK;
  cudaSetDevice(g->ctx->device);
  cudaStreamSynchronize(g->ctx->stream);
  pb_grid_release(g);
  return PB_OK;
}

// Stencil tiles: the fewest x tiles of width <= WMAX, then the tallest H with
// W*H <= NV*NT, then z chunks so that a single grid's tiles fill
// PB_PLAN_PER_SM CTAs per SM in one wave (a tile per CTA; fewer, longer
// tiles than the resident limit allows balance better across the SMs).
// batch = true (grids of a server): z chunks of at least 32 planes and update
// chunks of at least 16*CH elements, since many grids share each launch and
// each chunk ends with a CTA-wide reduction.
#ifndef PB_PLAN_PER_SM
#define PB_PLAN_PER_SM 2
#endif
// Row chunks of the update pass per resident update CTA (taken dynamically;
// 2 and 4 measured slower than one wave of one chunk each).
#ifndef PB_UPD_CHUNKS_PER_CTA
#define PB_UPD_CHUNKS_PER_CTA 1
#endif
// A tile plan given its x tiles, tile height and z chunks (clamped to what the
// tiles allow); the residual pieces and update chunks follow from it.
void pb_apply_plan(pb_grid *g, const KernelGrid &kg, bool batch, int tiles_x, int h, int zc) {
  const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz;
  tiles_x = std::max(tiles_x, (nx + WMAX - 1) / WMAX);
  g->tiles_x = tiles_x;
  g->W = round_up((nx + tiles_x - 1) / tiles_x, NV);
  h = std::max(1, std::min(h, std::min(HMAX, TILE_NODES / g->W)));
  g->tiles_y = (ny + h - 1) / h;
  g->H = (ny + g->tiles_y - 1) / g->tiles_y;
  const int cols = g->tiles_x * g->tiles_y;
  zc = std::max(1, std::min(zc, nz));
  g->tz = (nz + zc - 1) / zc;
  g->tiles_z = (nz + g->tz - 1) / g->tz;
  g->n_st = cols * g->tiles_z;
  // residual pass (FP64 arithmetic, not memory bound): pieces of RESID_TZ
  // planes, so that even one grid's pass spreads over every SM
  g->rtz = std::min(g->tz, RESID_TZ);
  g->n_rs = cols * ((nz + g->rtz - 1) / g->rtz);
  // update chunks: one wave of resident update CTAs on large grids, never
  // fewer than CH elements per chunk
  const long rows = (long)ny * nz;
  const long by_count = (rows + (long)PB_UPD_CHUNKS_PER_CTA * kg.update_blocks - 1) /
                        ((long)PB_UPD_CHUNKS_PER_CTA * kg.update_blocks);
  g->rows_per_chunk = (int)std::max<long>(std::max(1, (batch ? 16 * CH : CH) / nx), by_count);
  g->n_ch = (int)((rows + g->rows_per_chunk - 1) / g->rows_per_chunk);
}

void pb_batch_plan_grid(pb_grid *g, const KernelGrid &kg, int min_planes, int height_pct) {
  const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz;
  const int tiles_x = (nx + WMAX - 1) / WMAX;
  const int W = round_up((nx + tiles_x - 1) / tiles_x, NV);
  const int hmax = std::min(HMAX, TILE_NODES / W);
  const int h = std::max(1, (hmax * std::max(1, std::min(height_pct, 100)) + 50) / 100);
  const int tiles_y = (ny + h - 1) / h;
  const int cols = tiles_x * tiles_y;
  const int resident = std::max(kg.stencil_blocks, 2 * g->ctx->num_sms);
  int zc = std::max(1, resident / cols);
  zc = std::min(zc, std::max(1, nz / std::max(1, min_planes)));
  pb_apply_plan(g, kg, true, tiles_x, (ny + tiles_y - 1) / tiles_y, zc);
}

void pb_tile_plan(pb_grid *g, const KernelGrid &kg, bool batch) {
  if (batch) {
    pb_batch_plan_grid(g, kg, 32, 100);
    return;
  }
  const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz;
  const int tiles_x = (nx + WMAX - 1) / WMAX;
  const int W = round_up((nx + tiles_x - 1) / tiles_x, NV);
  const int hmax = std::min(HMAX, TILE_NODES / W);
  const int tiles_y = (ny + hmax - 1) / hmax;
  const int cols = tiles_x * tiles_y;
  const int resident = batch ? std::max(kg.stencil_blocks, 2 * g->ctx->num_sms)
                             : std::min(kg.stencil_blocks, PB_PLAN_PER_SM * g->ctx->num_sms);
  int zc = std::max(1, resident / cols);
  zc = std::min(zc, std::max(1, nz / (batch ? 32 : 4)));
  pb_apply_plan(g, kg, batch, tiles_x, (ny + tiles_y - 1) / tiles_y, zc);
}

// (Re)run the setup kernels of a grid for the given host atoms.
pb_status pb_run_setup(pb_grid *g, int n_atoms, const double *xyz, const double *q,
                       const double *radius, bool sync, cudaStream_t st_in) {
  cudaStream_t s = st_in ? st_in : g->ctx->stream;
  const pb_grid_desc *desc = &g->d;
  if (!g->scratch || n_atoms > g->atom_cap) {  // first call (also with no atoms) or growth
    if (g->xyzq) cudaFree(g->xyzq);
    if (g->xyzr) cudaFree(g->xyzr);
    if (g->scratch) cudaFree(g->scratch);
    if (g->h_atoms) cudaFreeHost(g->h_atoms);
    g->xyzq = g->xyzr = nullptr;
    g->scratch = nullptr;
    g->h_atoms = nullptr;
    g->atom_cap = 0;
    pb_status st;
    // pinned, so that the uploads below never wait for earlier work on the stream
    if (cudaMallocHost((void **)&g->h_atoms, 2 * (size_t)(n_atoms + 1) * sizeof(dbl4)) != cudaSuccess) {
      g->h_atoms = nullptr;
      cudaGetLastError();
      return pb_fail(PB_ERR_OOM, "pinned host staging of the atoms");
    }
    if ((st = pb_dalloc((void **)&g->xyzq, (size_t)(n_atoms + 1) * sizeof(dbl4)))) return st;
    if ((st = pb_dalloc((void **)&g->xyzr, (size_t)(n_atoms + 1) * sizeof(dbl4)))) return st;
    if ((st = pb_dalloc((void **)&g->scratch,
                        (SCR_ENERGY_PART + (size_t)n_atoms / 256 + 1) * sizeof(double))))
      return st;
    g->atom_cap = n_atoms;
  }
  g->n_atoms = n_atoms;
  if (g->mg) {  // the operator changes: the multigrid hierarchy is rebuilt on the next GMG solve
    cudaStreamSynchronize(s);
    pb_mg_release(g->mg);
    g->mg = nullptr;
  }
  // The staging is rewritten only by a later setup of this grid, which comes
  // after the grid's solve (a server) or after a synchronisation.
  dbl4 *hq = g->h_atoms, *hr = g->h_atoms + g->atom_cap + 1;
  for (int a = 0; a < n_atoms; a++) {
    hq[a] = dbl4{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2], q[a]};
    hr[a] = dbl4{xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2], radius[a]};
  }
  CK(cudaMemcpyAsync(g->xyzq, hq, n_atoms * sizeof(dbl4), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g->xyzr, hr, n_atoms * sizeof(dbl4), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(g->b, 0, g->n_pad * sizeof(double), s));
  CK(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, s));
  SetupArgs a;
  a.g = g->g;
  a.n_atoms = n_atoms;
  a.atoms_xyzr = g->xyzr;
  a.atoms_xyzq = g->xyzq;
  a.code = g->code;
  a.b = g->b;
  a.ghost = g->ghost;
  a.scratch = g->scratch + SCR_SETUP;  // PB_FOLD_CTAS partials of ||b||^2
  a.bnorm2 = g->scratch + SCR_BNORM2;
  a.err = g->err;
  a.kappa = g->kappa;
  a.ein = desc->eps_in;
  a.eout = desc->eps_out;
  a.c4pi_h = 4.0 * M_PI / desc->h;
  {
    double qsum = 0;
    for (int t = 0; t < n_atoms; t++) qsum += std::fabs(q[t]);
    int ex2 = 0;
    std::frexp(qsum + 1.0, &ex2);  // qsum + 1 < 2^ex2
    a.q_scale = std::ldexp(1.0, 62 - ex2);
  }
  a.kappa_mask = desc->kappa_mask ? 1 : 0;
  a.dh_f32 = desc->dh_precision == PB_F32;
  const bool harmonic = desc->eps_model == PB_EPS_HARMONIC;
  if (harmonic) {  // edge fractions from a cell list of the atoms
    double r_max = 0;
    for (int t = 0; t < n_atoms; t++) r_max = std::max(r_max, radius[t]);
    const size_t bytes = cell_buffer_bytes(cell_plan(g->g, r_max), n_atoms);
    if (bytes > g->cell_cap) {
      dfree(g->cell_buf);
      g->cell_buf = nullptr;
      g->cell_cap = 0;
      pb_status st;
      if ((st = pb_dalloc(&g->cell_buf, bytes))) return st;
      g->cell_cap = bytes;
    }
    a.ex64 = (double *)g->ex64; a.ey64 = (double *)g->ey64; a.ez64 = (double *)g->ez64;
    a.cell_buf = g->cell_buf;
    a.r_max = r_max;
  }
  CK(launch_setup(a, s));
  if (harmonic)
    CK(launch_harmonic_finish(g->code, g->g, g->kbh2, (const double *)g->ex64, (const double *)g->ey64,
                              (const double *)g->ez64, (double *)g->diag64,
                              desc->coef == PB_COEF_BF16 ? COEF_BF16 : COEF_F32, g->ex, g->ey,
                              g->ez, g->diag, s));
  else if (desc->coef == PB_COEF_F64)
    CK(launch_expand(g->code, g->g, desc->eps_in, desc->eps_out, g->kbh2, COEF_F64, g->ex64,
                     g->ey64, g->ez64, g->diag64, s));
  else if (desc->coef != PB_COEF_PACKED)
    CK(launch_expand(g->code, g->g, desc->eps_in, desc->eps_out, g->kbh2, desc->coef, g->ex, g->ey,
                     g->ez, g->diag, s));
  g->ctx->stats->launches += 3 + (n_atoms > 0 ? 3 : 0) +
                             (harmonic ? 5 + (n_atoms > 0 ? 3 : 0) : desc->coef != PB_COEF_PACKED ? 1 : 0);
  g->ctx->stats->h2d += 2 * (unsigned long long)n_atoms * sizeof(dbl4);
  if (!sync) return PB_OK;  // the error word and ||b||^2 stay on the device
  int *hbuf = (int *)g->ctx->host_scal;  // pinned staging: error word, then ||b||^2
  CK(cudaMemcpyAsync(hbuf, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync((double *)hbuf + 1, a.bnorm2, sizeof(double), cudaMemcpyDeviceToHost, s));
  g->ctx->stats->d2h += sizeof(int) + sizeof(double);
  CK(cudaStreamSynchronize(s));
  if (hbuf[0]) return pb_fail(PB_ERR_ARG, "an atom's trilinear cell leaves the grid");
  g->bnorm = std::sqrt(((double *)hbuf)[1]);
  return PB_OK;
}

pb_status pb_check_atoms(int n_atoms, const double *xyz, const double *q, const double *radius) {
  if (n_atoms < 0) return pb_fail(PB_ERR_ARG, "n_atoms < 0");
  if (n_atoms > 0 && (!xyz || !q || !radius)) return pb_fail(PB_ERR_ARG, "atom arrays are NULL");
  if (n_atoms > 0 && (!finite_all(xyz, 3 * (size_t)n_atoms) || !finite_all(q, n_atoms) ||
                      !finite_all(radius, n_atoms)))
    return pb_fail(PB_ERR_ARG, "atom arrays hold a non-finite value");
  return PB_OK;
}

extern "C" pb_status pb_grid_update_atoms(pb_grid *g, int n_atoms, const double *xyz,
                                          const double *q, const double *radius) {
  if (!g) return pb_fail(PB_ERR_ARG, "pb_grid_update_atoms: NULL grid");
  pb_status st = pb_check_atoms(n_atoms, xyz, q, radius);
  if (st) return st;
  CK(cudaSetDevice(g->ctx->device));
  return pb_run_setup(g, n_atoms, xyz, q, radius, true);
}

// Allocate a grid and plan its tiles (no atoms yet).
pb_status pb_grid_create(pb_ctx *ctx, const pb_grid_desc *desc, bool batch, pb_grid **out) {
  *out = nullptr;
  pb_status st = pb_check_desc(desc);
  if (st) return st;
  CK(cudaSetDevice(ctx->device));
  pb_grid *g = new pb_grid();
  g->ctx = ctx;
  g->d = *desc;
  const int px = pitch_of(desc->nx);
  g->g = Geom{desc->nx, desc->ny, desc->nz, px, desc->h, desc->origin[0], desc->origin[1],
              desc->origin[2], desc->periodic};
  g->n_pad = (size_t)px * desc->ny * desc->nz;
  const double kd2 = debye_kappa2(desc->ionic_strength, desc->temperature, desc->eps_out);
  g->kappa = std::sqrt(kd2);
  g->kbh2 = desc->eps_out * kd2 * desc->h * desc->h;
  g->n_ghost = 2L * ((long)desc->ny * desc->nz + (long)desc->nx * desc->nz + (long)desc->nx * desc->ny);
#define ALLOC(ptr, bytes)                                  \
  do {                                                     \
    pb_status a_ = pb_dalloc((void **)&(ptr), (bytes));    \
    if (a_) { pb_grid_release(g); return a_; }             \
  } while (0)
  ALLOC(g->code, g->n_pad);
  ALLOC(g->b, g->n_pad * sizeof(double));
  ALLOC(g->ghost, g->n_ghost * sizeof(double));
  ALLOC(g->err, sizeof(int) * 4);
  ALLOC(g->counts, sizeof(int) * PB_COUNTS);
  if (cudaMemsetAsync(g->counts, 0, sizeof(int) * PB_COUNTS, ctx->stream) != cudaSuccess) {
    pb_grid_release(g);
    return pb_fail(PB_ERR_CUDA, "clear work counters");
  }
  if (desc->coef != PB_COEF_PACKED) {
    const size_t nc = (size_t)px * (desc->ny + 1) * (desc->nz + 1);
    const bool harmonic = desc->eps_model == PB_EPS_HARMONIC;
    if (desc->coef == PB_COEF_F64 || harmonic) {
      ALLOC(g->ex64, g->n_pad * 8); ALLOC(g->ey64, nc * 8); ALLOC(g->ez64, nc * 8);
      ALLOC(g->diag64, g->n_pad * 8);
    }
    if (desc->coef != PB_COEF_F64 || harmonic) {  // the FP32 inner solve's copies
      const size_t es = desc->coef == PB_COEF_BF16 ? 2 : 4;
      ALLOC(g->ex, g->n_pad * es); ALLOC(g->ey, nc * es); ALLOC(g->ez, nc * es);
      ALLOC(g->diag, g->n_pad * 4);
    }
  }
#undef ALLOC
  pb_tile_plan(g, kernel_grid(MODE_F32, COEF_PACKED, ctx->num_sms, !batch), batch);
  g->batch = batch;
  *out = g;
  return PB_OK;
}

extern "C" pb_status pb_setup_grid(pb_ctx *ctx, const pb_grid_desc *desc, int n_atoms,
                                   const double *xyz, const double *q, const double *radius,
                                   pb_grid **out) {
  if (!ctx || !out) return pb_fail(PB_ERR_ARG, "pb_setup_grid: NULL ctx or out");
  *out = nullptr;
  pb_status st = pb_check_desc(desc);
  if (st) return st;
  if ((st = pb_check_atoms(n_atoms, xyz, q, radius))) return st;
  pb_grid *g = nullptr;
  if ((st = pb_grid_create(ctx, desc, false, &g))) return st;
  if ((st = pb_run_setup(g, n_atoms, xyz, q, radius, true))) {
    pb_grid_release(g);
    return st;
  }
  *out = g;
  return PB_OK;
}

extern "C" size_t pb_grid_bytes(const pb_grid_desc *d, int precision) {
  if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1) return 0;
  const size_t px = pitch_of(d->nx), n = px * d->ny * d->nz;
  const size_t nc = px * (d->ny + 1) * (d->nz + 1);
  size_t bytes = n * (1 + 8) + 8 * 2 * ((size_t)d->ny * d->nz + (size_t)d->nx * d->nz + (size_t)d->nx * d->ny);
  if (d->coef == PB_COEF_F64) bytes += 8 * (2 * n + 2 * nc);
  else if (d->coef == PB_COEF_F32) bytes += 4 * (2 * n + 2 * nc);
  else if (d->coef == PB_COEF_BF16) bytes += 2 * (n + 2 * nc) + 4 * n;
  bytes += 16 * n;  // x64 pair
  bytes += precision == PB_PREC_F64 ? 32 * n : 20 * n;
  bytes += n / CH * 16 + n / 256 * 16 + n / 64 + (1 << 16);
  return bytes;
}

// ---------------------------------------------------------------------------
// Instance descriptor of a grid for a solve of (mode, coef).

int pb_inner_coef(const pb_grid *g, int mode) {
  if (g->d.eps_model == PB_EPS_HARMONIC)  // FP64 edges, and FP32 / BF16 copies
    return mode == MODE_F64 ? COEF_F64 : g->d.coef == PB_COEF_BF16 ? COEF_BF16 : COEF_F32;
  if (mode == MODE_F64) return g->d.coef == PB_COEF_F64 ? COEF_F64 : COEF_PACKED;
  if (g->d.coef == PB_COEF_F32 || g->d.coef == PB_COEF_BF16) return g->d.coef;
  return COEF_PACKED;
}

pb_status pb_ensure_workspace(pb_grid *g, int mode) {
  cudaStream_t s = g->ctx->stream;
  auto alloc0 = [&](void **p, size_t bytes) -> pb_status {
    if (*p) return PB_OK;
    pb_status st = pb_dalloc(p, bytes);
    if (st) return st;
    if (cudaMemsetAsync(*p, 0, bytes, s) != cudaSuccess) return pb_fail(PB_ERR_CUDA, "memset");
    return PB_OK;
  };
  pb_status st;
  const size_t n = g->n_pad;
  if ((st = alloc0((void **)&g->x64, n * 8))) return st;
  if ((st = alloc0((void **)&g->x64b, n * 8))) return st;
  if (mode == MODE_F64) {
    if ((st = alloc0((void **)&g->z64, n * 8))) return st;
    if ((st = alloc0((void **)&g->p064, n * 8))) return st;
    if ((st = alloc0((void **)&g->p164, n * 8))) return st;
    if (!g->batch && (st = alloc0((void **)&g->ap64, n * 8))) return st;
  } else {
    if ((st = alloc0(&g->d32, n * 4))) return st;
    if ((st = alloc0(&g->z32, n * 4))) return st;
    if ((st = alloc0(&g->p032, n * 4))) return st;
    if ((st = alloc0(&g->p132, n * 4))) return st;
    if (!g->batch && (st = alloc0(&g->ap32, n * 4))) return st;
  }
  // (a server's grids hold no Ap: its update pass forms Ap again from p)
  if (g->batch) return PB_OK;  // scalars, descriptor and work lists are the server's
  if ((st = alloc0((void **)&g->scal, sizeof(Scal)))) return st;
  if ((st = alloc0((void **)&g->dinst, sizeof(Inst)))) return st;
  if (!g->st_items) {
    std::vector<Item> si(g->n_st), ci(g->n_ch);
    for (int t = 0; t < g->n_st; t++) si[t] = Item{0, t};
    for (int t = 0; t < g->n_ch; t++) ci[t] = Item{0, t};
    if ((st = pb_dalloc((void **)&g->st_items, si.size() * sizeof(Item)))) return st;
    if ((st = pb_dalloc((void **)&g->ch_items, ci.size() * sizeof(Item)))) return st;
    if ((st = pb_dalloc((void **)&g->st_part, 2 * sizeof(double) * g->n_st))) return st;
    if ((st = pb_dalloc((void **)&g->ch_part, 2 * sizeof(double) * g->n_ch))) return st;
    if ((st = pb_dalloc((void **)&g->rs_part, 2 * sizeof(double) * g->n_rs))) return st;
    const int counts[2] = {g->n_st, g->n_ch};
    if (cudaMemcpy(g->st_items, si.data(), si.size() * sizeof(Item), cudaMemcpyHostToDevice) ||
        cudaMemcpy(g->ch_items, ci.data(), ci.size() * sizeof(Item), cudaMemcpyHostToDevice) ||
        cudaMemcpy(g->counts, counts, sizeof(counts), cudaMemcpyHostToDevice))
      return pb_fail(PB_ERR_CUDA, "copy work items");
  }
  return PB_OK;
}

// TMA descriptors are encoded through the driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 3-D map of a padded node array [nz][ny][px]; extent nx in x, so elements
// beyond nx (and outside the grid in y, z) read as zero.
static bool encode_map(CUtensorMap *m, const void *base, CUtensorMapDataType dt, int es,
                       const pb_grid *g, int box_w, int box_h) {
  auto fn = tmap_encoder();
  if (!fn || !base) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g->d.nx, (cuuint64_t)g->d.ny, (cuuint64_t)g->d.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g->g.px * es, (cuuint64_t)g->g.px * g->d.ny * es};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, dt, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

pb_status pb_make_inst(const pb_grid *g, const pb_solve_opts *o, int mode, int coef, Inst &I) {
  memset(&I, 0, sizeof(I));
  I.nx = g->d.nx; I.ny = g->d.ny; I.nz = g->d.nz; I.px = g->g.px;
  I.W = g->W; I.H = g->H;
  I.tiles_x = g->tiles_x; I.tiles_y = g->tiles_y; I.tiles_z = g->tiles_z; I.tz = g->tz;
  I.n_st = g->n_st; I.n_ch = g->n_ch; I.rows_per_chunk = g->rows_per_chunk;
  I.rtz = g->rtz; I.n_rs = g->n_rs; I.rs_base = 0;
  {
    const uint64_t vx = (uint64_t)(g->d.nx + (mode == MODE_F64 ? 2 : 4) - 1) / (mode == MODE_F64 ? 2 : 4);
    I.vx_magic = vx > 1 ? (uint32_t)(((1ull << 32) + vx - 1) / vx) : 0u;
  }
  I.st_base = 0; I.ch_base = 0;
  I.mode = mode;
  I.periodic = g->d.periodic;
  I.precond = o ? (o->precond == PB_PRECOND_JACOBI) : 1;
  I.coef = coef;
  I.max_iter = o ? o->max_iter : 0;
  I.max_outer = o ? o->max_outer : 0;
  I.tol = o ? o->rel_tol : 0;
  I.inner_tol = o ? o->inner_tol : 0;
  I.bnorm = g->bnorm;
  I.err = g->err;
  I.bnorm2 = g->scratch + SCR_BNORM2;
  I.n_pad = g->n_pad;
  I.code = g->code;
  if (coef == COEF_F64) {
    I.ex = g->ex64; I.ey = g->ey64; I.ez = g->ez64; I.diag = g->diag64;
  } else if (coef == COEF_F32 || coef == COEF_BF16) {
    I.ex = g->ex; I.ey = g->ey; I.ez = g->ez; I.diag = g->diag;
  }
  I.rx = I.ry = I.rz = I.rdiag = nullptr;
  if (g->d.eps_model == PB_EPS_HARMONIC && coef != COEF_F64) {
    I.rx = (const double *)g->ex64; I.ry = (const double *)g->ey64; I.rz = (const double *)g->ez64;
    I.rdiag = (const double *)g->diag64;
  }
  I.x64 = g->x64; I.x64b = g->x64b;
  I.b = g->b;
  if (mode == MODE_F64) {
    I.d = nullptr; I.z = g->z64; I.p0 = g->p064; I.p1 = g->p164; I.ap = g->ap64;
  } else {
    I.d = g->d32; I.z = g->z32; I.p0 = g->p032; I.p1 = g->p132; I.ap = g->ap32;
  }
  I.s = g->scal;
  const double ein = g->d.eps_in, eout = g->d.eps_out;
  I.ein = ein; I.eout = eout; I.kbh2 = g->kbh2;
  I.ein32 = (float)ein; I.eout32 = (float)eout;
  for (int nin = 0; nin <= 6; nin++)
    for (int lam = 0; lam <= 1; lam++) {
      double s = 0;
      float s32 = 0;
      for (int t = 0; t < 6; t++) {
        s = s + (t < nin ? ein : eout);
        s32 = s32 + (t < nin ? (float)ein : (float)eout);
      }
      s = s + g->kbh2 * lam;
      s32 = s32 + (float)g->kbh2 * (float)lam;
      I.dtab[2 * nin + lam] = s;
      I.idtab[2 * nin + lam] = 1.0 / s;
      I.dtab32[2 * nin + lam] = s32;
      I.idtab32[2 * nin + lam] = 1.0f / s32;
    }
  // TMA stage layout and descriptors for the stencil pass
  const int es = mode == MODE_F64 ? 8 : 4;
  const StageLayout L = stage_layout(g->W, g->H, es);
  I.cw = L.cw;
  I.stage_bytes = L.stage_bytes;
  I.off_p = L.off_p;
  I.off_c = L.off_c;
  I.off_x = L.off_x;
  I.tma_bytes = L.tma_bytes;
  I.tma_bytes_upd = L.tma_bytes_upd;
  I.stage_bytes_upd = L.stage_bytes_upd;
  I.off_c_upd = L.off_c_upd;
  I.off_x_upd = L.off_x_upd;
  if (!o) return PB_OK;  // operator application needs no descriptors
  const CUtensorMapDataType dt = es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const void *x0 = mode == MODE_F64 ? (const void *)g->x64 : g->d32;
  const void *x1 = mode == MODE_F64 ? (const void *)g->x64b : g->d32;
  if (!encode_map(&I.tm_z, I.z, dt, es, g, L.rw, L.rows) ||
      !encode_map(&I.tm_p0, I.p0, dt, es, g, L.rw, L.rows) ||
      !encode_map(&I.tm_p1, I.p1, dt, es, g, L.rw, L.rows) ||
      !encode_map(&I.tm_code, g->code, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g, L.cw, L.rows) ||
      !encode_map(&I.tm_x0, x0, dt, es, g, g->W, g->H) ||
      !encode_map(&I.tm_x1, x1, dt, es, g, g->W, g->H) ||
      !encode_map(&I.tm_zc, I.z, dt, es, g, g->W, g->H))
    return pb_fail(PB_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return PB_OK;
}

Scal pb_initial_scal(double bnorm) {
  Scal S;
  memset(&S, 0, sizeof(S));
  S.bnorm = bnorm;
  S.phase = PH_RESID;
  S.ref_norm = 1.0;
  S.rz_old = 1.0;
  return S;
}

// ---------------------------------------------------------------------------
// Operator, solve, energy

extern "C" pb_status pb_apply_operator(pb_grid *g, const void *u, void *au, int dtype) {
  if (!g || !u || !au) return pb_fail(PB_ERR_ARG, "pb_apply_operator: NULL argument");
  if (dtype != PB_F64 && dtype != PB_F32) return pb_fail(PB_ERR_ARG, "bad dtype");
  CK(cudaSetDevice(g->ctx->device));
  const int mode = dtype == PB_F64 ? MODE_F64 : MODE_F32;
  pb_status st = pb_ensure_workspace(g, mode);
  if (st) return st;
  Inst I;
  if ((st = pb_make_inst(g, nullptr, mode, pb_inner_coef(g, mode), I))) return st;
  cudaStream_t s = g->ctx->stream;
  CK(cudaMemcpyAsync(g->dinst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
  CK(launch_apply(I, g->dinst, u, au, dtype == PB_F64 ? 0 : 1, s));
  g->ctx->stats->launches += 1;
  CK(cudaStreamSynchronize(s));
  return PB_OK;
}

static pb_status check_opts(const pb_solve_opts *o) {
  if (!o) return pb_fail(PB_ERR_ARG, "opts is NULL");
  if (o->precision < PB_PREC_F64 || o->precision > PB_PREC_F32_REFINE)
    return pb_fail(PB_ERR_ARG, "bad precision");
  if (o->precond != PB_PRECOND_NONE && o->precond != PB_PRECOND_JACOBI && o->precond != PB_PRECOND_GMG)
    return pb_fail(PB_ERR_ARG, "bad precond");
  if (!(o->rel_tol > 0) || o->max_iter < 0) return pb_fail(PB_ERR_ARG, "bad tolerance or max_iter");
  if (o->precision == PB_PREC_F32_REFINE && (!(o->inner_tol > 0) || o->max_outer < 1))
    return pb_fail(PB_ERR_ARG, "refinement needs inner_tol > 0 and max_outer >= 1");
  return PB_OK;
}

Batch pb_single_batch(pb_grid *g) {
  Batch B;
  B.inst = g->dinst;
  B.st_items = g->st_items;
  B.ch_items = g->ch_items;
  B.n_items = g->counts;
  B.work = (unsigned *)(g->counts + 4);
  B.resid_pending = g->counts + 2;
  B.resid_list = g->counts + 10;  // holds 0, the grid's only instance
  B.rs_part = g->rs_part;
  B.st_part = g->st_part;
  B.ch_part = g->ch_part;
  B.error = g->err;
  return B;
}

// A single grid's update pass runs over row chunks, reading the Ap its
// stencil pass stored.  The tile update pass (Ap formed again from p, 34 B
// per node and iteration instead of 38; 1 here) is the faster form for a
// server batch, but not on one grid: on 257^3 it measured 0.43-0.47 of
// measured HBM against 0.64 for the row chunks, and the whole iteration
// 156 us against 146 us.
#ifndef PB_GRID_TILE_UPDATE
#define PB_GRID_TILE_UPDATE 0
#endif
static bool grid_tile_update(const pb_grid *g, int mode, int coef) {
  return PB_GRID_TILE_UPDATE && !g->d.periodic && mode != MODE_F64 && coef == COEF_PACKED;
}
static KernelGrid single_kernel_grid(const pb_grid *g, int mode, int coef) {
  KernelGrid kg = kernel_grid(mode, coef, g->ctx->num_sms, true);
  kg.stencil_blocks = std::min(kg.stencil_blocks, g->n_st);
  kg.update_blocks = std::min(kg.update_blocks, g->n_ch);
  kg.fast = !g->d.periodic;
  if (grid_tile_update(g, mode, coef)) {
    kg.tile_update = 1;
    kg.update_tile_blocks = std::min(kg.update_tile_blocks, g->n_st);
    kg.update_fast_blocks = std::min(kg.update_fast_blocks, g->n_st);
  }
  return kg;
}

static int auto_ticks(const pb_grid *g) {
  // enough work per host check that the poll is cheap, few enough that a
  // converged solve does not idle long
  const double n = (double)g->n_pad;
  if (n >= 4e6) return 8;
  if (n >= 5e5) return 16;
  return 32;
}

pb_status pb_run_ticks(pb_grid *g, int mode, int coef, int ticks) {
  cudaStream_t s = g->ctx->stream;
  if (!g->graph || g->graph_mode != mode || g->graph_coef != coef || g->graph_ticks != ticks) {
    if (g->graph) {
      cudaGraphExecDestroy(g->graph);
      g->graph = nullptr;
    }
    const KernelGrid kg = single_kernel_grid(g, mode, coef);
    Batch B = pb_single_batch(g);
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int t = 0; t < ticks; t++) {
      cudaError_t e = launch_tick(B, mode, coef, kg, s);
      if (e != cudaSuccess) {
        cudaStreamEndCapture(s, &graph);
        return pb_fail(PB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
      }
    }
    CK(cudaStreamEndCapture(s, &graph));
    cudaError_t e = cudaGraphInstantiate(&g->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return pb_fail(PB_ERR_CUDA, std::string("graph: ") + cudaGetErrorString(e));
    g->graph_mode = mode;
    g->graph_coef = coef;
    g->graph_ticks = ticks;
  }
  CK(cudaGraphLaunch(g->graph, s));
  g->ctx->stats->launches += 3ull * ticks;
  return PB_OK;
}

// Measurement mode: every kernel launched on its own between CUDA events,
// with a synchronisation after each so that its work kind is known.
static pb_status profiled_loop(pb_grid *g, int mode, int coef, long max_ticks, pb_solve_info *info) {
  cudaStream_t s = g->ctx->stream;
  const KernelGrid kg = single_kernel_grid(g, mode, coef);
  Batch B = pb_single_batch(g);
  Scal *hs = g->ctx->host_scal;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  pb_solve_info acc;
  memset(&acc, 0, sizeof(acc));
  int phase = PH_RESID;
  pb_status st = PB_OK;
  for (long t = 0; t < 3 * max_ticks; t++) {
    const int which = t % 3 == 0 ? 4 : t % 3 == 1 ? 1 : 2;
    cudaError_t e = cudaEventRecord(e0, s);
    if (!e) e = launch_phase(B, mode, coef, kg, which, s);
    if (!e) e = cudaEventRecord(e1, s);
    if (!e) e = cudaMemcpyAsync(hs, g->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    float ms = 0;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e) {
      st = pb_fail(PB_ERR_CUDA, std::string("profiled launch: ") + cudaGetErrorString(e));
      break;
    }
    g->ctx->stats->launches += 1;
    g->ctx->stats->d2h += sizeof(Scal);
    if (which == 4) {
      if (phase == PH_RESID) { acc.ms_resid += ms; acc.n_resid++; }
    } else if (which == 1) {
      if (phase == PH_START || phase == PH_INNER) { acc.ms_stencil += ms; acc.n_stencil++; }
    } else if (phase == PH_INNER) {
      acc.ms_update += ms;
      acc.n_update++;
    }
    phase = hs->phase;
    if (phase == PH_DONE) break;
  }
  if (phase != PH_DONE && !st) hs->status = PB_ERR_TIMEOUT;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->ms_stencil = acc.ms_stencil; info->n_stencil = acc.n_stencil;
    info->ms_update = acc.ms_update; info->n_update = acc.n_update;
    info->ms_resid = acc.ms_resid; info->n_resid = acc.n_resid;
  }
  return st;
}

// ---------------------------------------------------------------------------
// Tile-plan autotuner: time the stencil pass of candidate plans on the grid.

static pb_status realloc_work_lists(pb_grid *g, int mode) {
  void *lists[] = {g->st_items, g->ch_items, g->st_part, g->ch_part, g->rs_part};
  for (void *p : lists)
    if (p) cudaFree(p);
  g->st_items = g->ch_items = nullptr;
  g->st_part = g->ch_part = g->rs_part = nullptr;
  if (g->graph) {  // captured over the old lists
    cudaGraphExecDestroy(g->graph);
    g->graph = nullptr;
  }
  return pb_ensure_workspace(g, mode);
}

extern "C" pb_status pb_grid_autotune(pb_grid *g, int precision, pb_tune_info *info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!g) return pb_fail(PB_ERR_ARG, "pb_grid_autotune: NULL grid");
  if (precision < PB_PREC_F64 || precision > PB_PREC_F32_REFINE)
    return pb_fail(PB_ERR_ARG, "pb_grid_autotune: bad precision");
  if (g->batch) return pb_fail(PB_ERR_ARG, "pb_grid_autotune: a server's grid");
  CK(cudaSetDevice(g->ctx->device));
  const int mode = precision == PB_PREC_F64 ? MODE_F64
                   : precision == PB_PREC_F32 ? MODE_F32 : MODE_F32_REFINE;
  const int coef = pb_inner_coef(g, mode);
  pb_status st;
  if ((st = pb_ensure_workspace(g, mode))) return st;
  cudaStream_t s = g->ctx->stream;
  const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz, sms = g->ctx->num_sms;
  const KernelGrid kplan = kernel_grid(MODE_F32, COEF_PACKED, sms, true);  // as at creation
  struct Plan { int tx, h, zc; };
  std::vector<Plan> cand{{g->tiles_x, g->H, g->tiles_z}};  // the analytic default first
  const int tx_min = (nx + WMAX - 1) / WMAX;
  const int resident = std::min(kplan.stencil_blocks, 2 * sms);
  for (int tx = tx_min; tx <= tx_min + 1; tx++) {
    const int W = round_up((nx + tx - 1) / tx, NV);
    if (tx > tx_min && W < 32) continue;  // narrower tiles lose to their halos
    const int hmax = std::min(HMAX, TILE_NODES / W);
    for (int hf : {hmax, (3 * hmax) / 4, hmax / 2}) {
      if (hf < 4) continue;
      const int ty = (ny + hf - 1) / hf, h = (ny + ty - 1) / ty;
      const int z0 = std::min(std::max(1, resident / (tx * ty)), std::max(1, nz / 4));
      for (int zc : {z0, 2 * z0}) {
        if (zc > std::max(1, nz / 2)) continue;
        bool dup = false;
        for (const Plan &p : cand) dup |= p.tx == tx && p.h == h && p.zc == zc;
        if (!dup) cand.push_back(Plan{tx, h, zc});
      }
    }
  }
  pb_solve_opts o;
  memset(&o, 0, sizeof(o));
  o.precond = PB_PRECOND_JACOBI;
  o.precision = precision;
  o.rel_tol = 1e-6;
  o.max_iter = 1;
  o.inner_tol = 1e-3;
  o.max_outer = 1;
  // each timed launch starts from the same scalars: an INNER iteration, alpha
  // = beta = 0 (x and p stay as they are; the values are scratch)
  Scal S0 = pb_initial_scal(1.0);
  S0.phase = PH_INNER;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_plan = [&](double &us) -> pb_status {
    Inst I;
    pb_status r;
    if ((r = pb_make_inst(g, &o, mode, coef, I))) return r;
    if (grid_tile_update(g, mode, coef)) I.ap = nullptr;  // as in the solves
    CK(cudaMemcpyAsync(g->dinst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
    const KernelGrid kg = single_kernel_grid(g, mode, coef);
    const Batch B = pb_single_batch(g);
    std::vector<float> t;
    for (int rep = 0; rep < 4; rep++) {
      CK(cudaMemcpyAsync(g->scal, &S0, sizeof(Scal), cudaMemcpyHostToDevice, s));
      CK(cudaEventRecord(e0, s));
      CK(launch_phase(B, mode, coef, kg, 1, s));
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0) t.push_back(ms);  // the first run warms the plan's descriptors
    }
    g->ctx->stats->launches += 4;
    std::sort(t.begin(), t.end());
    us = 1e3 * t[t.size() / 2];
    return PB_OK;
  };
  int best = 0;
  double best_us = 0, default_us = 0;
  for (size_t k = 0; k < cand.size() && !st; k++) {
    pb_apply_plan(g, kplan, false, cand[k].tx, cand[k].h, cand[k].zc);
    double us = 0;
    if ((st = realloc_work_lists(g, mode)) || (st = time_plan(us))) break;
    if (k == 0) default_us = us;
    if (k == 0 || us < best_us) {
      best_us = us;
      best = (int)k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pb_apply_plan(g, kplan, false, cand[best].tx, cand[best].h, cand[best].zc);
  const pb_status st2 = realloc_work_lists(g, mode);
  if (st) return st;
  if (st2) return st2;
  if (info) {
    info->W = g->W;
    info->H = g->H;
    info->tz = g->tz;
    info->n_tiles = g->n_st;
    info->candidates = (int)cand.size();
    info->us_default = default_us;
    info->us_best = best_us;
  }
  return PB_OK;
}

extern "C" pb_status pb_pcg_solve(pb_grid *g, const pb_solve_opts *o, double *phi,
                                  pb_solve_info *info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!g || !phi) return pb_fail(PB_ERR_ARG, "pb_pcg_solve: NULL grid or phi");
  pb_status st = check_opts(o);
  if (st) return st;
  CK(cudaSetDevice(g->ctx->device));
  if (o->precond == PB_PRECOND_GMG) {
    if (g->d.periodic) return pb_fail(PB_ERR_ARG, "the multigrid preconditioner is for the free-space boundary");
    return pb_gmg_solve(g, o, phi, info);
  }
  cudaStream_t s = g->ctx->stream;
  const size_t n = (size_t)g->d.nx * g->d.ny * g->d.nz;
  if (g->bnorm == 0.0) {  // A phi = 0 has the solution phi = 0
    CK(cudaMemsetAsync(phi, 0, n * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    if (info) info->status = PB_OK;
    return PB_OK;
  }
  const int mode = o->precision == PB_PREC_F64 ? MODE_F64
                   : o->precision == PB_PREC_F32 ? MODE_F32 : MODE_F32_REFINE;
  const int coef = pb_inner_coef(g, mode);
  if ((st = pb_ensure_workspace(g, mode))) return st;
  pb_solve_opts oo = *o;
  if (mode != MODE_F32_REFINE) oo.max_outer = 1;
  Inst I;
  if ((st = pb_make_inst(g, &oo, mode, coef, I))) return st;
  if (grid_tile_update(g, mode, coef)) I.ap = nullptr;  // the update pass forms Ap again
  Scal S0 = pb_initial_scal(g->bnorm);
  CK(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, s));
  CK(cudaMemcpyAsync(g->dinst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g->scal, &S0, sizeof(Scal), cudaMemcpyHostToDevice, s));
  static const int one_pending = 1;  // the solve opens with a residual pass
  CK(cudaMemcpyAsync(g->counts + 2, &one_pending, sizeof(int), cudaMemcpyHostToDevice, s));
  g->ctx->stats->h2d += sizeof(Inst) + sizeof(Scal) + sizeof(int);
  if (o->warm_start) {
    CK(launch_pack(phi, g->x64, g->d.nx, g->d.ny, g->d.nz, g->g.px, s));
    g->ctx->stats->launches += 1;
  } else {
    CK(cudaMemsetAsync(g->x64, 0, g->n_pad * sizeof(double), s));
  }
  const int ticks = o->poll_every > 0 ? o->poll_every : auto_ticks(g);
  // every tick advances at least one phase step; bound the host loop
  const long max_ticks = (long)oo.max_iter + 2L * (oo.max_outer + 2) + 4L * ticks;
  Scal *hs = g->ctx->host_scal;
  long done_ticks = 0;
  if (o->profile) {
    if ((st = profiled_loop(g, mode, coef, max_ticks, info))) return st;
  } else {
    int *herr_poll = (int *)(hs + 1);  // pinned slot after the scalars
    for (;;) {
      if ((st = pb_run_ticks(g, mode, coef, ticks))) return st;
      done_ticks += ticks;
      CK(cudaMemcpyAsync(hs, g->scal, sizeof(Scal), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(herr_poll, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
      g->ctx->stats->d2h += sizeof(Scal) + sizeof(int);
      CK(cudaStreamSynchronize(s));
      if (hs->phase == PH_DONE) break;
      if (*herr_poll & 2) break;  // a pipeline wait gave up: the solve cannot finish
      if (done_ticks > max_ticks) {
        hs->status = PB_ERR_TIMEOUT;
        break;
      }
    }
  }
  Scal S = *hs;
  {
    int *herr = (int *)(hs + 1);  // pinned slot after the scalars
    CK(cudaMemcpyAsync(herr, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (*herr & 2) S.status = PB_ERR_TIMEOUT;  // a device pipeline wait gave up
  }
  CK(launch_unpack(S.xbuf ? g->x64b : g->x64, phi, g->d.nx, g->d.ny, g->d.nz, g->g.px, s));
  g->ctx->stats->launches += 1;
  CK(cudaStreamSynchronize(s));
  if (info) {
    info->status = S.status;
    info->iterations = S.total_iter;
    info->outer_steps = S.outer;
    info->relres = S.relres;
    info->relres_true = S.relres_true;
  }
  if (S.status != PB_OK) {
    const char *why = S.status == PB_ERR_NOT_CONVERGED ? "iteration cap reached"
                      : S.status == PB_ERR_BREAKDOWN   ? "CG breakdown (p.Ap <= 0 or non-finite)"
                      : S.status == PB_ERR_TIMEOUT     ? "solve did not finish (device wait timed out)"
                                                       : "solve did not finish";
    return pb_fail(S.status, why);
  }
  return PB_OK;
}

extern "C" pb_status pb_energy(pb_grid *g, const double *phi, double *energy) {
  if (!g || !phi || !energy) return pb_fail(PB_ERR_ARG, "pb_energy: NULL argument");
  CK(cudaSetDevice(g->ctx->device));
  cudaStream_t s = g->ctx->stream;
  CK(launch_energy(g->xyzq, g->n_atoms, g->d.nx, g->d.ny, g->d.nz, g->d.nx, g->d.periodic, g->d.h,
                   g->d.origin[0], g->d.origin[1], g->d.origin[2], phi,
                   g->scratch + SCR_ENERGY_PART, g->scratch + SCR_ENERGY, s));
  CK(cudaMemcpyAsync(energy, g->scratch + SCR_ENERGY, sizeof(double), cudaMemcpyDeviceToHost, s));
  g->ctx->stats->launches += g->n_atoms > 0 ? 2 : 1;
  g->ctx->stats->d2h += sizeof(double);
  CK(cudaStreamSynchronize(s));
  return PB_OK;
}

// Solvation energy (Sec. 3.1): the solved system, then the reference system
// (eps_out -> eps_in, no salt), one grid at a time.
extern "C" pb_status pb_solvation_energy(pb_ctx *ctx, const pb_grid_desc *desc, int n_atoms,
                                         const double *xyz, const double *q, const double *radius,
                                         const pb_solve_opts *opts, double *phi, pb_solvation *out) {
  if (!ctx || !desc || !opts || !phi || !out)
    return pb_fail(PB_ERR_ARG, "pb_solvation_energy: NULL argument");
  memset(out, 0, sizeof(*out));
  pb_status st = pb_check_desc(desc);
  if (st) return st;
  if ((st = check_opts(opts))) return st;
  if (desc->periodic)
    return pb_fail(PB_ERR_ARG, "pb_solvation_energy: the reference system of a periodic grid "
                               "has no salt, and its operator is singular");
  CK(cudaSetDevice(ctx->device));
  const size_t n = (size_t)desc->nx * desc->ny * desc->nz;
  pb_status first = PB_OK;
  auto solve_one = [&](const pb_grid_desc *d, const pb_solve_opts *o, double *x, double *e,
                       pb_solve_info *info) -> pb_status {
    pb_grid *g = nullptr;
    pb_status s = pb_setup_grid(ctx, d, n_atoms, xyz, q, radius, &g);
    if (s) return s;
    s = pb_pcg_solve(g, o, x, info);
    if (s == PB_OK || s == PB_ERR_NOT_CONVERGED || s == PB_ERR_BREAKDOWN) {
      if (s && !first) first = s;
      s = pb_energy(g, x, e);
    }
    pb_free_grid(g);
    return s;
  };
  if ((st = solve_one(desc, opts, phi, &out->e_solv, &out->solv))) return st;
  pb_grid_desc d0 = *desc;
  d0.eps_out = desc->eps_in;
  d0.ionic_strength = 0.0;
  pb_solve_opts o0 = *opts;
  o0.warm_start = 0;
  double *x0 = nullptr;
  if ((st = pb_dalloc((void **)&x0, n * sizeof(double)))) return st;
  st = solve_one(&d0, &o0, x0, &out->e_ref, &out->ref);
  cudaFree(x0);
  if (st) return st;
  out->dG = out->e_solv - out->e_ref;
  return first;
}

extern "C" pb_status pb_grid_export(pb_grid *g, int what, void *dst, size_t bytes) {
  if (!g || !dst) return pb_fail(PB_ERR_ARG, "pb_grid_export: NULL argument");
  CK(cudaSetDevice(g->ctx->device));
  cudaStream_t s = g->ctx->stream;
  const size_t nx = g->d.nx, ny = g->d.ny, nz = g->d.nz, px = g->g.px;
  auto need = [&](size_t b) { return bytes == b; };
  if (what == PB_EXPORT_B) {
    if (!need(nx * ny * nz * 8)) return pb_fail(PB_ERR_ARG, "export: size mismatch");
    CK(cudaMemcpy2DAsync(dst, nx * 8, g->b, px * 8, nx * 8, ny * nz, cudaMemcpyDeviceToHost, s));
  } else if (what == PB_EXPORT_GHOST) {
    if (!need(g->n_ghost * 8)) return pb_fail(PB_ERR_ARG, "export: size mismatch");
    CK(cudaMemcpyAsync(dst, g->ghost, g->n_ghost * 8, cudaMemcpyDeviceToHost, s));
  } else if (what == PB_EXPORT_LAMBDA) {
    if (!need(nx * ny * nz)) return pb_fail(PB_ERR_ARG, "export: size mismatch");
    uint8_t *tmp = nullptr;
    pb_status st = pb_dalloc((void **)&tmp, nx * ny * nz);
    if (st) return st;
    cudaError_t e = launch_export_lambda(g->code, g->g, tmp, s);
    if (!e) e = cudaMemcpyAsync(dst, tmp, nx * ny * nz, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e) return pb_fail(PB_ERR_CUDA, cudaGetErrorString(e));
  } else if (what >= PB_EXPORT_EPS_X && what <= PB_EXPORT_EPS_Z) {
    const size_t nc = px * (ny + 1) * (nz + 1);
    size_t width, height;
    if (what == PB_EXPORT_EPS_X) { width = nx + 1; height = ny * nz; }
    else if (what == PB_EXPORT_EPS_Y) { width = nx; height = (ny + 1) * nz; }
    else { width = nx; height = ny * (nz + 1); }
    if (!need(width * height * 8)) return pb_fail(PB_ERR_ARG, "export: size mismatch");
    if (g->d.eps_model == PB_EPS_HARMONIC) {  // the FP64 edge arrays themselves
      const void *src = what == PB_EXPORT_EPS_X ? g->ex64 : what == PB_EXPORT_EPS_Y ? g->ey64 : g->ez64;
      CK(cudaMemcpy2DAsync(dst, width * 8, src, px * 8, width * 8, height, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return PB_OK;
    }
    double *ex = nullptr, *ey = nullptr, *ez = nullptr;
    pb_status st;
    if ((st = pb_dalloc((void **)&ex, nc * 8))) return st;
    if ((st = pb_dalloc((void **)&ey, nc * 8))) { cudaFree(ex); return st; }
    if ((st = pb_dalloc((void **)&ez, nc * 8))) { cudaFree(ex); cudaFree(ey); return st; }
    cudaError_t e = launch_expand(g->code, g->g, g->d.eps_in, g->d.eps_out, g->kbh2, COEF_F64, ex,
                                  ey, ez, nullptr, s);
    const double *src = what == PB_EXPORT_EPS_X ? ex : what == PB_EXPORT_EPS_Y ? ey : ez;
    if (!e) e = cudaMemcpy2DAsync(dst, width * 8, src, px * 8, width * 8, height,
                                  cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    cudaFree(ex); cudaFree(ey); cudaFree(ez);
    if (e) return pb_fail(PB_ERR_CUDA, cudaGetErrorString(e));
  } else {
    return pb_fail(PB_ERR_ARG, "export: unknown array");
  }
  CK(cudaStreamSynchronize(s));
  return PB_OK;
}
