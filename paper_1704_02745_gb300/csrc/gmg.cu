// gmg.cu -- geometric-multigrid preconditioned CG (pb_pcg_solve with
// PB_PRECOND_GMG).  The paper lists geometric multigrid among the classical PB
// solvers (Sec. 2) and names multigrid solvers tailored to the PB problem as
// the way to further gains (Sec. 4); the scheme below is the one the oracle
// (oracle/gmg.py) states:
//
//   levels     vertex-centred: coarse node I sits on fine node 2I, coarse size
//              (n + 1) / 2 per axis, down to 3 nodes on the shortest axis;
//   operator   the h^2-scaled seven-point operator rediscretised at spacing
//              2h: a coarse edge's eps is the series combination
//              2 / (1/e_a + 1/e_b) of the two fine edges it spans on the fine
//              line through the coarse nodes, lambda the fine node's, and
//              kbar^2 (2h)^2 replaces kbar^2 h^2;
//   transfer   trilinear prolongation P (coarse ghosts zero), restriction
//              P^T r / 2;
//   V-cycle    NU damped-Jacobi sweeps (weight OMEGA) from zero, coarse
//              correction, NU sweeps; COARSE_SWEEPS sweeps on the coarsest
//              level: a symmetric positive definite preconditioner;
//   outer      preconditioned CG (Sec. 2.2) in FP64 with z = V(r); the V-cycle
//              runs in FP32 on FP32 copies of each level's operator.
//
// Vectors and coefficient arrays of the hierarchy are dense (no row pitch):
// ex (nz, ny, nx+1), ey (nz, ny+1, nx), ez (nz+1, ny, nx), nodes (nz, ny, nx),
// edge entry e of a line being the edge between nodes e-1 and e.
#include <cmath>
#include <string>
#include <vector>

#include "pb.h"
#include "pb_host.h"
#include "pb_internal.cuh"
#include "solve.cuh"

namespace pb {

constexpr float MG_OMEGA = 0.8f;
constexpr int MG_NU = 2, MG_COARSEST = 3, MG_COARSE_SWEEPS = 20, MG_NT = 256;

struct MgDims {
  int nx, ny, nz;
  __host__ __device__ size_t nodes() const { return (size_t)nx * ny * nz; }
  __host__ __device__ size_t nex() const { return (size_t)(nx + 1) * ny * nz; }
  __host__ __device__ size_t ney() const { return (size_t)nx * (ny + 1) * nz; }
  __host__ __device__ size_t nez() const { return (size_t)nx * ny * (nz + 1); }
};

static int mg_blocks(size_t n) {
  const size_t b = (n + MG_NT - 1) / MG_NT;
  return (int)(b < 152 * 32 ? (b ? b : 1) : 152 * 32);
}
#define MG_LOOP(t, n) \
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (n); t += (size_t)gridDim.x * blockDim.x)

// Level 0 FP64 edges and lambda from the grid: its FP64 edge arrays (row
// pitch px) when it has them, else the code bits.
__global__ void k_mg_level0(MgDims d, int px, const uint8_t *code, const double *ex64, const double *ey64,
                            const double *ez64, double ein, double eout, double *ex, double *ey,
                            double *ez, uint8_t *lam) {
  MG_LOOP(t, d.nex()) {  // x-edges: entry i of row (j, k) is the edge (i-1, i)
    const size_t i = t % (d.nx + 1), row = t / (d.nx + 1);
    if (ex64) {
      ex[t] = ex64[row * px + i];
    } else {
      const bool first = i == 0;
      const uint8_t c = code[row * px + (first ? 0 : i - 1)];
      ex[t] = (first ? (c & 1u) : (c & 2u)) ? ein : eout;
    }
  }
  MG_LOOP(t, d.ney()) {  // y-edges: row j of plane k is the edge (j-1, j)
    const size_t i = t % d.nx, j = (t / d.nx) % (d.ny + 1), k = t / ((size_t)d.nx * (d.ny + 1));
    if (ey64) {
      ey[t] = ey64[(k * (d.ny + 1) + j) * px + i];
    } else {
      const bool first = j == 0;
      const uint8_t c = code[(k * d.ny + (first ? 0 : j - 1)) * px + i];
      ey[t] = (first ? (c & 4u) : (c & 8u)) ? ein : eout;
    }
  }
  MG_LOOP(t, d.nez()) {  // z-edges: plane k is the edge (k-1, k)
    const size_t i = t % d.nx, j = (t / d.nx) % d.ny, k = t / ((size_t)d.nx * d.ny);
    if (ez64) {
      ez[t] = ez64[(k * d.ny + j) * px + i];
    } else {
      const bool first = k == 0;
      const uint8_t c = code[((first ? 0 : k - 1) * d.ny + j) * px + i];
      ez[t] = (first ? (c & 16u) : (c & 32u)) ? ein : eout;
    }
  }
  MG_LOOP(t, d.nodes()) {
    const size_t i = t % d.nx, row = t / d.nx;
    lam[t] = (code[row * px + i] & 64u) ? 0 : 1;
  }
}

__device__ __forceinline__ double mg_series(double a, double b) {
  return __ddiv_rn(2.0, __dadd_rn(__ddiv_rn(1.0, a), __ddiv_rn(1.0, b)));
}

// Coarse FP64 edges and lambda of level l+1 from level l.
__global__ void k_mg_coarsen(MgDims f, MgDims c, const double *fex, const double *fey, const double *fez,
                             const uint8_t *flam, double *cex, double *cey, double *cez, uint8_t *clam) {
  MG_LOOP(t, c.nex()) {
    const size_t I = t % (c.nx + 1), J = (t / (c.nx + 1)) % c.ny, K = t / ((size_t)(c.nx + 1) * c.ny);
    const size_t row = ((2 * K) * f.ny + 2 * J) * (f.nx + 1);
    const long a = min(max(2 * (long)I - 1, 0L), (long)f.nx), b = min(2 * (long)I, (long)f.nx);
    cex[t] = mg_series(fex[row + a], fex[row + b]);
  }
  MG_LOOP(t, c.ney()) {
    const size_t I = t % c.nx, J = (t / c.nx) % (c.ny + 1), K = t / ((size_t)c.nx * (c.ny + 1));
    const long a = min(max(2 * (long)J - 1, 0L), (long)f.ny), b = min(2 * (long)J, (long)f.ny);
    const size_t base = (2 * K) * (f.ny + 1) * (size_t)f.nx + 2 * I;
    cey[t] = mg_series(fey[base + a * f.nx], fey[base + b * f.nx]);
  }
  MG_LOOP(t, c.nez()) {
    const size_t I = t % c.nx, J = (t / c.nx) % c.ny, K = t / ((size_t)c.nx * c.ny);
    const long a = min(max(2 * (long)K - 1, 0L), (long)f.nz), b = min(2 * (long)K, (long)f.nz);
    const size_t base = (2 * J) * (size_t)f.nx + 2 * I, pl = (size_t)f.nx * f.ny;
    cez[t] = mg_series(fez[a * pl + base], fez[b * pl + base]);
  }
  MG_LOOP(t, c.nodes()) {
    const size_t I = t % c.nx, J = (t / c.nx) % c.ny, K = t / ((size_t)c.nx * c.ny);
    clam[t] = flam[((2 * K) * f.ny + 2 * J) * f.nx + 2 * I];
  }
}

// FP32 copies of a level's edges and its diagonal (six edges in the order
// x-, x+, y-, y+, z-, z+, then + kbh2 lambda, summed in FP64).
__global__ void k_mg_finish(MgDims d, double kbh2, const double *ex, const double *ey, const double *ez,
                            const uint8_t *lam, float *fex, float *fey, float *fez, float *fdiag) {
  MG_LOOP(t, d.nex()) fex[t] = (float)ex[t];
  MG_LOOP(t, d.ney()) fey[t] = (float)ey[t];
  MG_LOOP(t, d.nez()) fez[t] = (float)ez[t];
  MG_LOOP(t, d.nodes()) {
    const size_t i = t % d.nx, j = (t / d.nx) % d.ny, k = t / ((size_t)d.nx * d.ny);
    const size_t xr = (k * d.ny + j) * (d.nx + 1) + i, yr = (k * (d.ny + 1) + j) * d.nx + i;
    const size_t zr = (k * d.ny + j) * d.nx + i, pl = (size_t)d.nx * d.ny;
    double s = __dadd_rn(ex[xr], ex[xr + 1]);
    s = __dadd_rn(s, ey[yr]);
    s = __dadd_rn(s, ey[yr + d.nx]);
    s = __dadd_rn(s, ez[zr]);
    s = __dadd_rn(s, ez[zr + pl]);
    s = __dadd_rn(s, __dmul_rn(kbh2, (double)lam[t]));
    fdiag[t] = (float)s;
  }
}

struct MgOp {  // FP32 operator of one level (device pointers)
  MgDims d;
  const float *ex, *ey, *ez, *diag;
};

// Node indices in 32 bits (a grid has at most 2e9 nodes, checked when it is
// created): 32-bit division costs a fraction of 64-bit division per node.
__device__ __forceinline__ void mg_ijk(const MgDims &d, size_t t, uint32_t &i, uint32_t &j, uint32_t &k) {
  const uint32_t tt = (uint32_t)t, row = tt / (uint32_t)d.nx;
  i = tt - row * (uint32_t)d.nx;
  k = row / (uint32_t)d.ny;
  j = row - k * (uint32_t)d.ny;
}

__device__ __forceinline__ float mg_apply(const MgOp &A, const float *u, size_t t) {
  const int nx = A.d.nx, ny = A.d.ny, nz = A.d.nz;
  uint32_t i32, j32, k32;
  mg_ijk(A.d, t, i32, j32, k32);
  const size_t i = i32, j = j32, k = k32;
  const size_t xr = (k * ny + j) * (nx + 1) + i, yr = (k * (ny + 1) + j) * nx + i, pl = (size_t)nx * ny;
  float s = 0.f;
  if (i > 0) s += A.ex[xr] * u[t - 1];
  if (i + 1 < (size_t)nx) s += A.ex[xr + 1] * u[t + 1];
  if (j > 0) s += A.ey[yr] * u[t - nx];
  if (j + 1 < (size_t)ny) s += A.ey[yr + nx] * u[t + nx];
  if (k > 0) s += A.ez[t] * u[t - pl];
  if (k + 1 < (size_t)nz) s += A.ez[t + pl] * u[t + pl];
  return A.diag[t] * u[t] - s;
}

// One damped-Jacobi sweep: out = in + omega (r - A in) / diag (in = NULL: zero).
__global__ void k_mg_jacobi(MgOp A, const float *in, const float *r, float *out) {
  MG_LOOP(t, A.d.nodes()) {
    const float res = in ? r[t] - mg_apply(A, in, t) : r[t];
    out[t] = (in ? in[t] : 0.f) + MG_OMEGA * res / A.diag[t];
  }
}

// res = r - A z, then the coarse right-hand side P^T res / 2 (gathered:
// coarse node I takes fine nodes 2I and 2I +- 1 with weights 1 and 1/2 per
// axis) in a second kernel.
__global__ void k_mg_residual(MgOp A, const float *z, const float *r, float *res) {
  MG_LOOP(t, A.d.nodes()) res[t] = r[t] - mg_apply(A, z, t);
}
__global__ void k_mg_restrict(MgDims f, MgDims c, const float *res, float *rc) {
  MG_LOOP(t, c.nodes()) {
    uint32_t I32, J32, K32;
    mg_ijk(c, t, I32, J32, K32);
    const long I = I32, J = J32, K = K32;
    float s = 0.f;
    for (int dk = -1; dk <= 1; dk++) {
      const long k = 2 * K + dk;
      if (k < 0 || k >= f.nz) continue;
      for (int dj = -1; dj <= 1; dj++) {
        const long j = 2 * J + dj;
        if (j < 0 || j >= f.ny) continue;
        for (int di = -1; di <= 1; di++) {
          const long i = 2 * I + di;
          if (i < 0 || i >= f.nx) continue;
          const float w = (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * (dk ? 0.5f : 1.f);
          s += w * res[(k * f.ny + j) * f.nx + i];
        }
      }
    }
    rc[t] = 0.5f * s;
  }
}
// z += P e: fine node i takes coarse i/2 (even) or the mean of (i-1)/2 and
// (i+1)/2 (odd), per axis; coarse indices past the end are the zero ghost.
__global__ void k_mg_prolong_add(MgDims f, MgDims c, const float *e, float *z) {
  MG_LOOP(t, f.nodes()) {
    uint32_t i32, j32, k32;
    mg_ijk(f, t, i32, j32, k32);
    const long i = i32, j = j32, k = k32;
    float s = 0.f;
    for (int ck = 0; ck < 2; ck++) {
      const long K = ck ? (k + 1) / 2 : k / 2;
      const float wk = (k % 2 == 0) ? (ck ? 0.f : 1.f) : 0.5f;
      if (wk == 0.f || K >= c.nz) continue;
      for (int cj = 0; cj < 2; cj++) {
        const long J = cj ? (j + 1) / 2 : j / 2;
        const float wj = (j % 2 == 0) ? (cj ? 0.f : 1.f) : 0.5f;
        if (wj == 0.f || J >= c.ny) continue;
        for (int ci = 0; ci < 2; ci++) {
          const long I = ci ? (i + 1) / 2 : i / 2;
          const float wi = (i % 2 == 0) ? (ci ? 0.f : 1.f) : 0.5f;
          if (wi == 0.f || I >= c.nx) continue;
          s += wk * wj * wi * e[(K * c.ny + J) * c.nx + I];
        }
      }
    }
    z[t] += s;
  }
}

// Outer FP64 loop: r (FP64) to the V-cycle's FP32 right-hand side and back.
__global__ void k_mg_to_f32(size_t n, const double *a, float *b) { MG_LOOP(t, n) b[t] = (float)a[t]; }
__global__ void k_mg_to_f64(size_t n, const float *a, double *b) { MG_LOOP(t, n) b[t] = (double)a[t]; }

// Deterministic dot product: per-CTA partials in a fixed order, then one CTA.
constexpr int MG_DOT_CTAS = 256;
__global__ void k_mg_dot_partial(size_t n, const double *a, const double *b, double *part) {
  __shared__ double red[MG_NT];
  double s = 0.0;
  const size_t per = (n + MG_DOT_CTAS - 1) / MG_DOT_CTAS, lo = blockIdx.x * per;
  const size_t hi = lo + per < n ? lo + per : n;
  for (size_t t = lo + threadIdx.x; t < hi; t += MG_NT) s = fma(a[t], b[t], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = MG_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_mg_dot_final(const double *part, double *out) {
  __shared__ double red[MG_NT];
  double s = 0.0;
  for (int t = threadIdx.x; t < MG_DOT_CTAS; t += MG_NT) s += part[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = MG_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
// Scalars of the outer CG on the device, so that a graph of several
// iterations runs without host round trips: rz = r.z, pap = p.Ap, rr = r.r,
// rz_new = the next r.z; done stops the updates (convergence when rr <
// stop2 = (tol ||b||)^2, the iteration cap, or breakdown), it counts the
// iterations taken.
struct MgScal {
  double rz, pap, rr, rz_new, alpha, beta, stop2;
  int it, done, status, max_iter;
};
__global__ void k_mg_alpha(MgScal *S) {  // alpha = r.z / p.Ap, or breakdown
  if (S->done) return;
  const double a = S->rz / S->pap;
  if (!(S->pap > 0.0) || !isfinite(a)) {
    S->status = PB_ERR_BREAKDOWN;
    S->done = 1;
    S->alpha = 0.0;
  } else {
    S->alpha = a;
  }
}
__global__ void k_mg_check(MgScal *S) {  // after x, r are updated and r.r formed
  if (S->done) return;
  S->it++;
  if (S->rr < S->stop2) {
    S->status = PB_OK;
    S->done = 1;
  } else if (S->it >= S->max_iter) {
    S->done = 1;
  }
}
__global__ void k_mg_beta(MgScal *S) {  // beta = r.z (new) / r.z
  if (S->done) return;
  S->beta = S->rz_new / S->rz;
  S->rz = S->rz_new;
}
// x += alpha p; r -= alpha Ap (alpha from the device scalars)
__global__ void k_mg_update_dev(size_t n, const MgScal *S, const double *p, const double *ap, double *x,
                                double *r) {
  if (S->done) return;
  const double alpha = S->alpha;
  MG_LOOP(t, n) {
    x[t] = fma(alpha, p[t], x[t]);
    r[t] = fma(-alpha, ap[t], r[t]);
  }
}
// p = z + beta p (beta from the device scalars)
__global__ void k_mg_direction_dev(size_t n, const MgScal *S, const double *z, double *p) {
  if (S->done) return;
  const double beta = S->beta;
  MG_LOOP(t, n) p[t] = fma(beta, p[t], z[t]);
}
// r = b - r (the Ap of x0 in r): b read from the padded layout
__global__ void k_mg_initial_residual(MgDims d, int px, const double *b, double *r) {
  MG_LOOP(t, d.nodes()) {
    const size_t i = t % d.nx, row = t / d.nx;
    r[t] = b[row * px + i] - r[t];
  }
}

}  // namespace pb

using namespace pb;

// ---------------------------------------------------------------------------
// Host side: the hierarchy of a grid, built on the first GMG solve.

struct pb_mg {
  struct Level {
    MgDims d;
    double kbh2;
    double *ex64 = nullptr, *ey64 = nullptr, *ez64 = nullptr;
    uint8_t *lam = nullptr;
    float *ex = nullptr, *ey = nullptr, *ez = nullptr, *diag = nullptr;
    float *z0 = nullptr, *z1 = nullptr, *r = nullptr, *res = nullptr;
  };
  std::vector<Level> lv;
  double *x = nullptr, *r = nullptr, *p = nullptr, *ap = nullptr, *z = nullptr, *part = nullptr;
  MgScal *S = nullptr;     // device scalars of the outer CG
  MgScal *hS = nullptr;    // pinned host copy
  // graph of MG_GRAPH_ITERS outer iterations (captured on the first solve)
  cudaGraphExec_t graph = nullptr;
  int graph_coef = -1;
  unsigned long long graph_launches = 0;  // kernels per graph launch
  std::vector<void *> owned;
};

static pb_status mg_alloc(pb_mg *m, void **p, size_t bytes) {
  pb_status st = pb_dalloc(p, bytes);
  if (!st) m->owned.push_back(*p);
  return st;
}

void pb_mg_release(pb_mg *m) {
  if (!m) return;
  if (m->graph) cudaGraphExecDestroy(m->graph);
  if (m->hS) cudaFreeHost(m->hS);
  for (void *p : m->owned) cudaFree(p);
  delete m;
}

static pb_status mg_build(pb_grid *g, pb_mg **out) {
  cudaStream_t s = g->ctx->stream;
  pb_mg *m = new pb_mg();
  auto fail = [&](pb_status st) {
    pb_mg_release(m);
    return st;
  };
  MgDims d{g->d.nx, g->d.ny, g->d.nz};
  double kbh2 = g->kbh2;
  pb_status st;
  while (true) {
    pb_mg::Level L;
    L.d = d;
    L.kbh2 = kbh2;
    if ((st = mg_alloc(m, (void **)&L.ex64, d.nex() * 8)) || (st = mg_alloc(m, (void **)&L.ey64, d.ney() * 8)) ||
        (st = mg_alloc(m, (void **)&L.ez64, d.nez() * 8)) || (st = mg_alloc(m, (void **)&L.lam, d.nodes())) ||
        (st = mg_alloc(m, (void **)&L.ex, d.nex() * 4)) || (st = mg_alloc(m, (void **)&L.ey, d.ney() * 4)) ||
        (st = mg_alloc(m, (void **)&L.ez, d.nez() * 4)) || (st = mg_alloc(m, (void **)&L.diag, d.nodes() * 4)) ||
        (st = mg_alloc(m, (void **)&L.z0, d.nodes() * 4)) || (st = mg_alloc(m, (void **)&L.z1, d.nodes() * 4)) ||
        (st = mg_alloc(m, (void **)&L.r, d.nodes() * 4)) || (st = mg_alloc(m, (void **)&L.res, d.nodes() * 4)))
      return fail(st);
    m->lv.push_back(L);
    if (std::min(d.nx, std::min(d.ny, d.nz)) <= MG_COARSEST) break;
    d = MgDims{(d.nx + 1) / 2, (d.ny + 1) / 2, (d.nz + 1) / 2};
    kbh2 *= 4.0;  // kbar^2 (2h)^2
  }
  const size_t n = m->lv[0].d.nodes();
  if ((st = mg_alloc(m, (void **)&m->x, n * 8)) || (st = mg_alloc(m, (void **)&m->r, n * 8)) ||
      (st = mg_alloc(m, (void **)&m->p, n * 8)) || (st = mg_alloc(m, (void **)&m->ap, n * 8)) ||
      (st = mg_alloc(m, (void **)&m->z, n * 8)) || (st = mg_alloc(m, (void **)&m->part, MG_DOT_CTAS * 8)) ||
      (st = mg_alloc(m, (void **)&m->S, sizeof(MgScal))))
    return fail(st);
  if (cudaMallocHost((void **)&m->hS, sizeof(MgScal)) != cudaSuccess) {
    cudaGetLastError();
    m->hS = nullptr;
    return fail(pb_fail(PB_ERR_OOM, "multigrid: pinned scalars"));
  }
  // level 0 from the grid, then coarsen
  const pb_mg::Level &L0 = m->lv[0];
  k_mg_level0<<<mg_blocks(L0.d.nex()), MG_NT, 0, s>>>(
      L0.d, g->g.px, g->code, (const double *)g->ex64, (const double *)g->ey64, (const double *)g->ez64,
      g->d.eps_in, g->d.eps_out, L0.ex64, L0.ey64, L0.ez64, L0.lam);
  for (size_t l = 0; l + 1 < m->lv.size(); l++) {
    const pb_mg::Level &F = m->lv[l], &C = m->lv[l + 1];
    k_mg_coarsen<<<mg_blocks(C.d.nex()), MG_NT, 0, s>>>(F.d, C.d, F.ex64, F.ey64, F.ez64, F.lam, C.ex64,
                                                        C.ey64, C.ez64, C.lam);
  }
  for (const pb_mg::Level &L : m->lv)
    k_mg_finish<<<mg_blocks(L.d.nex()), MG_NT, 0, s>>>(L.d, L.kbh2, L.ex64, L.ey64, L.ez64, L.lam, L.ex, L.ey,
                                                       L.ez, L.diag);
  g->ctx->stats->launches += 1 + 2 * m->lv.size() - 1;
  if (cudaGetLastError() != cudaSuccess) return fail(pb_fail(PB_ERR_CUDA, "multigrid setup kernels"));
  *out = m;
  return PB_OK;
}

static MgOp op_of(const pb_mg::Level &L) { return MgOp{L.d, L.ex, L.ey, L.ez, L.diag}; }

// z_l = V(r_l) on level l (result in L.z1 after the post-smoothing).
static void vcycle(pb_mg *m, size_t l, cudaStream_t s, unsigned long long &launches) {
  pb_mg::Level &L = m->lv[l];
  const MgOp A = op_of(L);
  const int nb = mg_blocks(L.d.nodes());
  if (l + 1 == m->lv.size()) {  // coarsest: sweeps from zero, ending in z1
    float *a = L.z0, *b = L.z1;
    k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, nullptr, L.r, MG_COARSE_SWEEPS % 2 ? b : a);
    float *cur = MG_COARSE_SWEEPS % 2 ? b : a;
    for (int t = 1; t < MG_COARSE_SWEEPS; t++) {
      float *nxt = cur == a ? b : a;
      k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, cur, L.r, nxt);
      cur = nxt;
    }
    launches += MG_COARSE_SWEEPS;
    return;
  }
  // pre-smoothing: z0 = S(0), z1 = S(z0)
  k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, nullptr, L.r, L.z0);
  k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, L.z0, L.r, L.z1);
  pb_mg::Level &C = m->lv[l + 1];
  k_mg_residual<<<nb, MG_NT, 0, s>>>(A, L.z1, L.r, L.res);
  k_mg_restrict<<<mg_blocks(C.d.nodes()), MG_NT, 0, s>>>(L.d, C.d, L.res, C.r);
  launches += 4;
  vcycle(m, l + 1, s, launches);
  k_mg_prolong_add<<<nb, MG_NT, 0, s>>>(L.d, C.d, C.z1, L.z1);
  // post-smoothing: z0 = S(z1), z1 = S(z0)
  k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, L.z1, L.r, L.z0);
  k_mg_jacobi<<<nb, MG_NT, 0, s>>>(A, L.z0, L.r, L.z1);
  launches += 3;
}

// The preconditioned CG of Sec. 2.2 with z = V(r), in FP64.  Its scalars
// stay on the device (MgScal): after the first direction, the host launches a
// CUDA graph of MG_GRAPH_ITERS iterations (the operator, three dot products,
// the updates and a V-cycle each: about 80 kernels) and reads the scalars
// once per graph; iterations after convergence leave x and r as they are.
// Called by pb_pcg_solve for PB_PRECOND_GMG.
#ifndef MG_GRAPH_ITERS
#define MG_GRAPH_ITERS 3
#endif
pb_status pb_gmg_solve(pb_grid *g, const pb_solve_opts *o, double *phi, pb_solve_info *info) {
  cudaStream_t s = g->ctx->stream;
  if (!g->mg) {
    pb_status st = mg_build(g, &g->mg);
    if (st) return st;
  }
  pb_mg *m = g->mg;
  const pb_mg::Level &L0 = m->lv[0];
  const size_t n = L0.d.nodes();
  const int nb = mg_blocks(n);
  unsigned long long launches = 0, n_reads = 0;
  Inst I;
  pb_solve_opts oo = *o;
  pb_status st;
  if ((st = pb_ensure_workspace(g, MODE_F64))) return st;
  const int coef = pb_inner_coef(g, MODE_F64);
  if ((st = pb_make_inst(g, &oo, MODE_F64, coef, I))) return st;
  CK(cudaMemcpyAsync(g->dinst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
  MgScal *S = m->S, *hS = m->hS;
  auto dot = [&](const double *a, const double *b, double *out) {
    k_mg_dot_partial<<<MG_DOT_CTAS, MG_NT, 0, s>>>(n, a, b, m->part);
    k_mg_dot_final<<<1, MG_NT, 0, s>>>(m->part, out);
    launches += 2;
  };
  auto read_scal = [&]() -> pb_status {  // *hS = *S
    CK(cudaMemcpyAsync(hS, S, sizeof(MgScal), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    n_reads++;
    return PB_OK;
  };
  auto apply = [&](const double *u, double *au) -> cudaError_t {
    launches += 1;
    return launch_apply(I, g->dinst, u, au, 0, s);
  };
  auto precondition = [&]() {  // m->z = V(m->r)
    k_mg_to_f32<<<nb, MG_NT, 0, s>>>(n, m->r, m->lv[0].r);
    vcycle(m, 0, s, launches);
    k_mg_to_f64<<<nb, MG_NT, 0, s>>>(n, m->lv[0].z1, m->z);
    launches += 2;
  };
  // One outer iteration, from p, r, z and rz: alpha, x and r, the stop test,
  // z = V(r), beta, p.
  auto iteration = [&]() -> cudaError_t {
    cudaError_t e = apply(m->p, m->ap);
    dot(m->p, m->ap, &S->pap);
    k_mg_alpha<<<1, 1, 0, s>>>(S);
    k_mg_update_dev<<<nb, MG_NT, 0, s>>>(n, S, m->p, m->ap, m->x, m->r);
    dot(m->r, m->r, &S->rr);
    k_mg_check<<<1, 1, 0, s>>>(S);
    precondition();
    dot(m->r, m->z, &S->rz_new);
    k_mg_beta<<<1, 1, 0, s>>>(S);
    k_mg_direction_dev<<<nb, MG_NT, 0, s>>>(n, S, m->z, m->p);
    launches += 5;
    return e != cudaSuccess ? e : cudaGetLastError();
  };
  // x0 = phi (warm start) or 0; r = b - A x0
  if (o->warm_start) CK(cudaMemcpyAsync(m->x, phi, n * 8, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(m->x, 0, n * 8, s));
  CK(apply(m->x, m->r));
  k_mg_initial_residual<<<nb, MG_NT, 0, s>>>(L0.d, g->g.px, g->b, m->r);
  launches += 1;
  const double bnorm = g->bnorm;
  MgScal h0;
  memset(&h0, 0, sizeof(h0));
  h0.stop2 = (o->rel_tol * bnorm) * (o->rel_tol * bnorm);
  h0.max_iter = o->max_iter;
  h0.status = PB_ERR_NOT_CONVERGED;
  *hS = h0;
  CK(cudaMemcpyAsync(S, hS, sizeof(MgScal), cudaMemcpyHostToDevice, s));
  dot(m->r, m->r, &S->rr);
  if ((st = read_scal())) return st;
  double rel = bnorm > 0 ? std::sqrt(hS->rr) / bnorm : 0.0;
  int it = 0, status = PB_OK;
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(m->x, 0, n * 8, s));
    rel = 0.0;
  } else if (!(rel < o->rel_tol) && o->max_iter > 0) {
    precondition();
    CK(cudaMemcpyAsync(m->p, m->z, n * 8, cudaMemcpyDeviceToDevice, s));
    dot(m->r, m->z, &S->rz);
    if (!m->graph || m->graph_coef != coef) {  // capture MG_GRAPH_ITERS iterations
      if (m->graph) cudaGraphExecDestroy(m->graph);
      m->graph = nullptr;
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      const unsigned long long before = launches;
      for (int k = 0; k < MG_GRAPH_ITERS && e == cudaSuccess; k++) e = iteration();
      m->graph_launches = launches - before;
      launches = before;  // counted when the graph runs
      const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return pb_fail(PB_ERR_CUDA, std::string("multigrid graph capture: ") +
                                        cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      const cudaError_t e3 = cudaGraphInstantiate(&m->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) {
        m->graph = nullptr;
        return pb_fail(PB_ERR_CUDA, std::string("multigrid graph: ") + cudaGetErrorString(e3));
      }
      m->graph_coef = coef;
    }
    while (true) {
      CK(cudaGraphLaunch(m->graph, s));
      launches += m->graph_launches;
      if ((st = read_scal())) return st;
      if (hS->done) break;
    }
    it = hS->it;
    status = hS->status;
    rel = std::sqrt(hS->rr) / bnorm;
  } else if (!(rel < o->rel_tol)) {
    status = PB_ERR_NOT_CONVERGED;
  }
  // true residual of the result, then phi = x
  CK(apply(m->x, m->ap));
  CK(cudaMemcpyAsync(m->z, m->ap, n * 8, cudaMemcpyDeviceToDevice, s));
  k_mg_initial_residual<<<nb, MG_NT, 0, s>>>(L0.d, g->g.px, g->b, m->z);
  launches += 1;
  dot(m->z, m->z, &S->rr);
  CK(cudaMemcpyAsync(phi, m->x, n * 8, cudaMemcpyDeviceToDevice, s));
  if ((st = read_scal())) return st;
  const double rr_true = hS->rr;
  g->ctx->stats->launches += launches;
  g->ctx->stats->h2d += sizeof(Inst) + sizeof(MgScal);
  g->ctx->stats->d2h += sizeof(MgScal) * n_reads + 8;
  if (info) {
    info->status = status;
    info->iterations = it;
    info->outer_steps = 1;
    info->relres = rel;
    info->relres_true = bnorm > 0 ? std::sqrt(rr_true) / bnorm : 0.0;
  }
  return status == PB_OK ? PB_OK : pb_fail(status, status == PB_ERR_BREAKDOWN ? "CG breakdown" : "not converged");
}
