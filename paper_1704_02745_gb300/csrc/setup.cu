// setup.cu -- grid setup kernels (dielectric map, lambda, charges, Debye-Hueckel
// boundary, right-hand side) of the linear FDPB method, arXiv:1704.02745
// Sec. 2.1 (Eq. 3-4) and Sec. 2.7 (eps 1 / 80, free-space boundary).
//
// Coordinates are evaluated exactly as: node  o + i*h,  edge midpoint
// o + (i + 0.5)*h, and the inside test |m - x_a|^2 < r_a^2 as
// (dx*dx + dy*dy) + dz*dz, each operation rounded on its own (__d*_rn), so
// the dielectric map is the same bit pattern whatever the evaluation order.
#include <cmath>

#include "pb_internal.cuh"
#include "setup.cuh"

namespace pb {

// ---------------------------------------------------------------------------
// Index i modulo n in [0, n).
__device__ __forceinline__ long wrap_index(long i, long n) {
  const long r = i % n;
  return r < 0 ? r + n : r;
}

// Packed codes start at 0: every edge outside (eps_out), every node outside.
__global__ void k_init_code(uint8_t *code, size_t n_pad) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; e < n_pad; e += (size_t)gridDim.x * blockDim.x) code[e] = 0;
}

__device__ __forceinline__ bool inside_sphere(double mx, double my, double mz, double ax, double ay,
                                              double az, double r2) {
  double dx = __dsub_rn(mx, ax), dy = __dsub_rn(my, ay), dz = __dsub_rn(mz, az);
  double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  return d2 < r2;
}

__device__ __forceinline__ double node_coord(double o, long i, double h) {
  return __dadd_rn(o, __dmul_rn((double)i, h));
}
__device__ __forceinline__ double mid_coord(double o, long i, double h) {
  return __dadd_rn(o, __dmul_rn(__dadd_rn((double)i, 0.5), h));
}

// One CTA per atom, one thread per node of the atom's bounding box (one
// spacing of margin): the node and the midpoints of its six edges are tested
// against the sphere, and the result is OR-ed into the node's code byte with
// one atomic (bits 0-5: edges x-, x+, y-, y+, z-, z+ inside; bit 6: node
// inside).  Each edge is tested by both of its nodes with the same exact rule,
// so the two copies of its bit agree.  The test runs in FP32 with a wide
// margin; points within the margin of the sphere surface are decided by the
// exact FP64 test, so the map is the one the FP64 definition gives.
//
// Periodic grids: the box is not clipped; a node visited at unwrapped index i
// tests its points at their unwrapped coordinates o + i*h and ORs into the
// node at i modulo n, so each edge or node is inside when some periodic image
// of it is (its two end nodes test the same unwrapped midpoints).
constexpr float INSIDE_MARGIN = 1e-3f;  // relative to r^2 + 1; the FP32 error of d^2 is < 1e-5 A^2
__global__ void k_eps_scatter(const dbl4 *atoms, int n_atoms, Geom g, uint32_t *code32,
                              int kappa_mask) {
  const int a = blockIdx.x;
  if (a >= n_atoms) return;
  const dbl4 A = atoms[a];  // x, y, z, radius
  const double r2 = __dmul_rn(A.w, A.w);
  const float r2f = (float)r2, margin = INSIDE_MARGIN * (r2f + 1.0f);
  long i0 = (long)floor(__ddiv_rn(A.x - A.w - g.ox, g.h)) - 1;
  long i1 = (long)ceil(__ddiv_rn(A.x + A.w - g.ox, g.h)) + 1;
  long j0 = (long)floor(__ddiv_rn(A.y - A.w - g.oy, g.h)) - 1;
  long j1 = (long)ceil(__ddiv_rn(A.y + A.w - g.oy, g.h)) + 1;
  long k0 = (long)floor(__ddiv_rn(A.z - A.w - g.oz, g.h)) - 1;
  long k1 = (long)ceil(__ddiv_rn(A.z + A.w - g.oz, g.h)) + 1;
  if (!g.periodic) {
    i0 = max(i0, 0L); i1 = min(i1, (long)g.nx - 1);
    j0 = max(j0, 0L); j1 = min(j1, (long)g.ny - 1);
    k0 = max(k0, 0L); k1 = min(k1, (long)g.nz - 1);
  }
  if (i0 > i1 || j0 > j1 || k0 > k1) return;
  // box extents are a few dozen nodes: 32-bit index arithmetic
  const int ni = (int)(i1 - i0 + 1), nj = (int)(j1 - j0 + 1), cnt = ni * nj * (int)(k1 - k0 + 1);
  // FP32 offsets from the atom of the box's first node (exact up to one FP32
  // rounding), then steps of h: a few hundred ulp of a few A at most
  const float bx = (float)(node_coord(g.ox, i0, g.h) - A.x);
  const float by = (float)(node_coord(g.oy, j0, g.h) - A.y);
  const float bz = (float)(node_coord(g.oz, k0, g.h) - A.z);
  const float hf = (float)g.h;
  const size_t rowp = (size_t)g.px, plane = (size_t)g.px * g.ny;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int tj = t / ni, tk = tj / nj;
    const long i = i0 + (t - tj * ni), j = j0 + (tj - tk * nj), k = k0 + tk;
    const float dx = bx + (float)(i - i0) * hf, dy = by + (float)(j - j0) * hf;
    const float dz = bz + (float)(k - k0) * hf;
    const float hh = 0.5f * hf;
    // squared distances of the 7 test points: node, x-, x+, y-, y+, z-, z+ midpoints
    const float yz = dy * dy + dz * dz, xz = dx * dx + dz * dz, xy = dx * dx + dy * dy;
    float d2[7];
    d2[0] = dx * dx + yz;
    d2[1] = (dx - hh) * (dx - hh) + yz;
    d2[2] = (dx + hh) * (dx + hh) + yz;
    d2[3] = (dy - hh) * (dy - hh) + xz;
    d2[4] = (dy + hh) * (dy + hh) + xz;
    d2[5] = (dz - hh) * (dz - hh) + xy;
    d2[6] = (dz + hh) * (dz + hh) + xy;
    uint32_t bits = 0;
#pragma unroll
    for (int p = 0; p < 7; p++) {
      bool in;
      if (d2[p] < r2f - margin) in = true;
      else if (d2[p] > r2f + margin) in = false;
      else {  // close to the surface: the exact FP64 test of the definition
        const long ii = p == 1 ? i - 1 : i, jj = p == 3 ? j - 1 : j, kk = p == 5 ? k - 1 : k;
        const double mx = (p == 1 || p == 2) ? mid_coord(g.ox, ii, g.h) : node_coord(g.ox, i, g.h);
        const double my = (p == 3 || p == 4) ? mid_coord(g.oy, jj, g.h) : node_coord(g.oy, j, g.h);
        const double mz = (p == 5 || p == 6) ? mid_coord(g.oz, kk, g.h) : node_coord(g.oz, k, g.h);
        in = inside_sphere(mx, my, mz, A.x, A.y, A.z, r2);
      }
      if (in) bits |= p == 0 ? (kappa_mask ? 64u : 0u) : (1u << (p - 1));
    }
    if (bits) {
      const long iw = g.periodic ? wrap_index(i, g.nx) : i, jw = g.periodic ? wrap_index(j, g.ny) : j;
      const long kw = g.periodic ? wrap_index(k, g.nz) : k;
      const size_t e = kw * plane + jw * rowp + iw;
      atomicOr(code32 + (e >> 2), bits << ((e & 3) * 8));
    }
  }
}

// Trilinear charge spreading: f = (x - o)/h, i0 = floor(f), w = f - i0; the
// 8 corner weights per axis are w or 1 - w, the contribution ((q*wx)*wy)*wz.
// Contributions are accumulated as 64-bit fixed point (rounded to a multiple
// of 1/scale, scale a power of two with sum|q| * scale <= 2^62): integer
// addition is associative, so the grid charges do not depend on the order in
// which the atomics land.  An atom whose cell leaves the grid sets *err; on a
// periodic grid the corners wrap modulo n instead.
__global__ void k_spread(const dbl4 *xyzq, int n_atoms, Geom g, double scale,
                         unsigned long long *qn, int *err) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const dbl4 A = xyzq[a];  // x, y, z, q
  double f[3] = {__ddiv_rn(__dsub_rn(A.x, g.ox), g.h), __ddiv_rn(__dsub_rn(A.y, g.oy), g.h),
                 __ddiv_rn(__dsub_rn(A.z, g.oz), g.h)};
  const int n[3] = {g.nx, g.ny, g.nz};
  double w[3][2];
  long c0[3];
  for (int d = 0; d < 3; d++) {
    double fl = floor(f[d]);
    if (g.periodic ? !isfinite(fl) : !(fl >= 0.0 && fl + 1.0 <= (double)(n[d] - 1))) {
      atomicOr(err, 1);
      return;
    }
    c0[d] = (long)fl;
    w[d][1] = __dsub_rn(f[d], fl);
    w[d][0] = __dsub_rn(1.0, w[d][1]);
  }
  for (int dk = 0; dk < 2; dk++)
    for (int dj = 0; dj < 2; dj++)
      for (int di = 0; di < 2; di++) {
        double c = __dmul_rn(__dmul_rn(__dmul_rn(A.w, w[0][di]), w[1][dj]), w[2][dk]);
        long ci = c0[0] + di, cj = c0[1] + dj, ck = c0[2] + dk;
        if (g.periodic) {
          ci = wrap_index(ci, g.nx);
          cj = wrap_index(cj, g.ny);
          ck = wrap_index(ck, g.nz);
        }
        size_t e = ((size_t)ck * g.ny + cj) * g.px + ci;
        atomicAdd(qn + e, (unsigned long long)__double2ll_rn(__dmul_rn(c, scale)));
      }
}

// Ghost node t in the face order x-, x+, y-, y+, z-, z+ (dense faces).
__device__ __forceinline__ void ghost_pos(const Geom &g, long t, double &px, double &py,
                                          double &pz) {
  const long fx = (long)g.ny * g.nz, fy = (long)g.nx * g.nz;
  long i, j, k;
  if (t < 2 * fx) {
    int side = t >= fx; long u = t - side * fx;
    i = side ? g.nx : -1; j = u % g.ny; k = u / g.ny;
  } else if (t < 2 * fx + 2 * fy) {
    long v = t - 2 * fx; int side = v >= fy; long u = v - side * fy;
    j = side ? g.ny : -1; i = u % g.nx; k = u / g.nx;
  } else {
    long fz = (long)g.nx * g.ny, v = t - 2 * fx - 2 * fy; int side = v >= fz; long u = v - side * fz;
    k = side ? g.nz : -1; i = u % g.nx; j = u / g.nx;
  }
  px = node_coord(g.ox, i, g.h);
  py = node_coord(g.oy, j, g.h);
  pz = node_coord(g.oz, k, g.h);
}

constexpr int DH_NT = 128;

// Debye-Hueckel potential at each ghost node, FP64:
//   phi_g = sum_a q_a exp(-kappa r) / (eps_out r), atoms in input order.
__global__ void __launch_bounds__(DH_NT) k_dh_f64(const dbl4 *xyzq, int n_atoms, Geom g,
                                                  double kappa, double eps_out, double *ghost,
                                                  long n_ghost) {
  __shared__ dbl4 sa[DH_NT];
  const long t = blockIdx.x * (long)DH_NT + threadIdx.x;
  double px = 0, py = 0, pz = 0;
  if (t < n_ghost) ghost_pos(g, t, px, py, pz);
  double s = 0.0;
  for (int base = 0; base < n_atoms; base += DH_NT) {
    __syncthreads();
    if (base + threadIdx.x < n_atoms) sa[threadIdx.x] = xyzq[base + threadIdx.x];
    __syncthreads();
    const int m = min(DH_NT, n_atoms - base);
    for (int u = 0; u < m; u++) {
      const dbl4 A = sa[u];
      double dx = __dsub_rn(px, A.x), dy = __dsub_rn(py, A.y), dz = __dsub_rn(pz, A.z);
      double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
      double r = sqrt(d2);
      double tq = __dmul_rn(A.w, exp(-__dmul_rn(kappa, r)));
      s = __dadd_rn(s, __ddiv_rn(tq, __dmul_rn(eps_out, r)));
    }
  }
  if (t < n_ghost) ghost[t] = s;
}

// Same sum in FP32 arithmetic: hardware reciprocal square root and base-2
// exponential (rsqrt.approx, ex2.approx: a few ulp), FP32 partial sums over
// blocks of DH_NT atoms added into an FP64 accumulator.  The ghost value is
// stored as FP64.
__device__ __forceinline__ float fast_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__global__ void __launch_bounds__(DH_NT) k_dh_f32(const dbl4 *xyzq, int n_atoms, Geom g,
                                                  double kappa, double eps_out, double *ghost,
                                                  long n_ghost) {
  __shared__ float4 sa[DH_NT];
  const long t = blockIdx.x * (long)DH_NT + threadIdx.x;
  double px = 0, py = 0, pz = 0;
  if (t < n_ghost) ghost_pos(g, t, px, py, pz);
  // positions relative to the grid origin keep FP32 rounding small
  const float fx = (float)(px - g.ox), fy = (float)(py - g.oy), fz = (float)(pz - g.oz);
  const float k2 = (float)(kappa * 1.4426950408889634);  // kappa / ln 2
  const float inv_eps = (float)(1.0 / eps_out);
  double s = 0.0;
  for (int base = 0; base < n_atoms; base += DH_NT) {
    __syncthreads();
    if (base + threadIdx.x < n_atoms) {
      const dbl4 A = xyzq[base + threadIdx.x];
      sa[threadIdx.x] = make_float4((float)(A.x - g.ox), (float)(A.y - g.oy), (float)(A.z - g.oz),
                                    (float)A.w * inv_eps);
    }
    __syncthreads();
    const int m = min(DH_NT, n_atoms - base);
    float part = 0.f;
    for (int u = 0; u < m; u++) {
      const float4 A = sa[u];
      const float dx = fx - A.x, dy = fy - A.y, dz = fz - A.z;
      const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const float rinv = fast_rsqrt(d2);
      part = fmaf(A.w * rinv, fast_exp2(-k2 * (d2 * rinv)), part);
    }
    s += (double)part;
  }
  if (t < n_ghost) ghost[t] = s;
}

// b = (4 pi / h) q_node, then every boundary row adds eps_edge * phi_ghost for
// its ghost neighbours in the face order x-, x+, y-, y+, z-, z+; and the
// partial sums of b^2 (one per CTA over its rows, in a fixed order).  A warp
// takes one row (y, z) at a time, its lanes the x positions.  qn (fixed
// point) and b may alias: each element is read before it is written.
// scale = 4 pi / h / (fixed-point scale): the latter is a power of two, so
// qn * scale rounds as (qn / fixed-point scale) * (4 pi / h) does.
// ex64/ey64/ez64 (harmonic-average grids, else NULL): the ghost edges' eps;
// otherwise eps_in or eps_out from the code bits.
constexpr int FOLD_CTAS = PB_FOLD_CTAS, FOLD_NT = 256;
__global__ void __launch_bounds__(FOLD_NT) k_fold_rhs(const long long *qn, const uint8_t *code,
                                                      const double *ghost, Geom g, double scale,
                                                      double ein, double eout, const double *ex64,
                                                      const double *ey64, const double *ez64,
                                                      double *b, double *part) {
  __shared__ double red[FOLD_NT];
  const int rows = g.ny * g.nz, per = (rows + FOLD_CTAS - 1) / FOLD_CTAS;
  const int r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const long fx = (long)g.ny * g.nz, fy = (long)g.nx * g.nz, fz = (long)g.nx * g.ny;
  double s = 0.0;
  for (int row = r0 + warp; row < r1; row += FOLD_NT / 32) {
    const int j = row % g.ny, k = row / g.ny;
    const size_t base = (size_t)row * g.px;
    for (int i = lane; i < g.px; i += 32) {
      const size_t e = base + i;
      if (i >= g.nx) {
        b[e] = 0.0;
        continue;
      }
      double v = __dmul_rn((double)qn[e], scale);
      const uint32_t c = code[e];
      // eps of the six ghost edges (read only on boundary nodes)
      auto eps = [&](int bit, size_t idx, const double *arr) {
        return arr ? arr[idx] : ((c & bit) ? ein : eout);
      };
      const size_t pxs = g.px, nys = g.ny;
      if (i == 0)
        v = __dadd_rn(v, __dmul_rn(eps(1, e, ex64), ghost[(long)k * g.ny + j]));
      if (i == g.nx - 1)
        v = __dadd_rn(v, __dmul_rn(eps(2, e + 1, ex64), ghost[fx + (long)k * g.ny + j]));
      if (j == 0)
        v = __dadd_rn(v, __dmul_rn(eps(4, ((size_t)k * (nys + 1)) * pxs + i, ey64),
                                   ghost[2 * fx + (long)k * g.nx + i]));
      if (j == g.ny - 1)
        v = __dadd_rn(v, __dmul_rn(eps(8, ((size_t)k * (nys + 1) + nys) * pxs + i, ey64),
                                   ghost[2 * fx + fy + (long)k * g.nx + i]));
      if (k == 0)
        v = __dadd_rn(v, __dmul_rn(eps(16, (size_t)j * pxs + i, ez64),
                                   ghost[2 * fx + 2 * fy + (long)j * g.nx + i]));
      if (k == g.nz - 1)
        v = __dadd_rn(v, __dmul_rn(eps(32, ((size_t)g.nz * nys + j) * pxs + i, ez64),
                                   ghost[2 * fx + 2 * fy + fz + (long)j * g.nx + i]));
      b[e] = v;
      s = fma(v, v, s);
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = FOLD_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Explicit coefficient arrays from the packed codes (pitch px; see the layout
// in pb_internal.cuh).  Pads hold 1 so that every diagonal is positive.
template <typename C, typename D>
__global__ void k_expand_coef(const uint8_t *code, Geom g, double ein, double eout, double kbh2,
                              C *ex, C *ey, C *ez, D *diag) {
  const size_t px = g.px, ny = g.ny, nz = g.nz, nx = g.nx;
  const size_t n_ex = px * ny * nz, n_ey = px * (ny + 1) * nz, n_ez = px * ny * (nz + 1);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t n_all = n_ey > n_ez ? n_ey : n_ez;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n_all; e += stride) {
    const size_t i = e % px, row = e / px;
    if (e < n_ex) {
      double v = 1.0;
      if (i < nx) v = (code[row * px + i] & 1u) ? ein : eout;
      else if (i == nx) v = (code[row * px + nx - 1] & 2u) ? ein : eout;
      ex[e] = (C)v;
    }
    if (e < n_ey) {  // ey: row = k*(ny+1) + j
      const size_t j = row % (ny + 1), k = row / (ny + 1);
      double v = 1.0;
      if (i < nx) {
        if (j < ny) v = (code[(k * ny + j) * px + i] & 4u) ? ein : eout;
        else v = (code[(k * ny + ny - 1) * px + i] & 8u) ? ein : eout;
      }
      ey[e] = (C)v;
    }
    if (e < n_ez) {  // ez: row = k*ny + j
      const size_t j = row % ny, k = row / ny;
      double v = 1.0;
      if (i < nx) {
        if (k < nz) v = (code[(k * ny + j) * px + i] & 16u) ? ein : eout;
        else v = (code[((nz - 1) * ny + j) * px + i] & 32u) ? ein : eout;
      }
      ez[e] = (C)v;
    }
    if (e < n_ex && diag) {
      D dv = (D)1;
      if (i < nx) {
        const uint32_t c = code[e];
        D s = (D)((c & 1u) ? ein : eout);
        s = s + (D)((c & 2u) ? ein : eout);
        s = s + (D)((c & 4u) ? ein : eout);
        s = s + (D)((c & 8u) ? ein : eout);
        s = s + (D)((c & 16u) ? ein : eout);
        s = s + (D)((c & 32u) ? ein : eout);
        s = s + (D)kbh2 * (D)(((c >> 6) & 1u) ^ 1u);
        dv = s;
      }
      diag[e] = dv;
    }
  }
}

// Dense lambda from the codes (for export).
__global__ void k_export_lambda(const uint8_t *code, Geom g, uint8_t *lam) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t % g.nx, row = t / g.nx;
    lam[t] = ((code[row * g.px + i] >> 6) & 1u) ^ 1u;
  }
}

// Sum of squares of b, deterministic: per-CTA partials then one CTA in order.
__global__ void k_sum_final(const double *part, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------------------
// Weighted harmonic-average boundary dielectric (Sec. 2.7).  Every edge takes
// 1 / (w/eps_in + (1-w)/eps_out), w the fraction of the edge (the segment
// between its two nodes, coordinates o + i*h) strictly inside the union of
// the atom spheres; w = 0 and w = 1 give eps_out and eps_in exactly.  Each
// atom whose sphere meets the segment contributes the parameter interval
//   s = r*r - (du*du + dv*dv),  q = sqrt(s),
//   t0 = ((c - q) - p) / h,  t1 = ((c + q) - p) / h,  clipped to [0, 1],
// (u, v the other two axes, every operation rounded on its own); the
// intervals are sorted by start, then end, merged (touching ones joined) and
// their lengths summed in order.  Candidate atoms come from a cell list; an
// FP32 test with a wide margin discards atoms that cannot meet the segment.

// Cell of coordinate v on one axis: cubes of side cs from c0.
__device__ __forceinline__ int cell_index(double v, double c0, double cs, int n) {
  const int i = (int)floor((v - c0) / cs);
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}
struct Cells {
  double x0, y0, z0, cs;
  int ncx, ncy, ncz;
};
__device__ __forceinline__ int atom_cell(const Cells &c, const dbl4 &a) {
  return (cell_index(a.z, c.z0, c.cs, c.ncz) * c.ncy + cell_index(a.y, c.y0, c.cs, c.ncy)) * c.ncx +
         cell_index(a.x, c.x0, c.cs, c.ncx);
}
__global__ void k_cell_count(const dbl4 *atoms, int n_atoms, Cells c, int *count) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n_atoms) atomicAdd(count + atom_cell(c, atoms[a]), 1);
}
// Exclusive prefix sum of n counts into start[0..n] (one CTA of 1024 threads,
// each a contiguous chunk), and the fill cursors.
__global__ void __launch_bounds__(1024) k_cell_scan(const int *count, int n, int *start, int *cursor) {
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024, lo = threadIdx.x * per, hi = min(n, lo + per);
  int s = 0;
  for (int t = lo; t < hi; t++) s += count[t];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan of the chunk sums
    const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int t = lo; t < hi; t++) {
    start[t] = run;
    cursor[t] = run;
    run += count[t];
  }
  if (threadIdx.x == 1023) start[n] = part[1023];
}
// list[slot]: the atom; rel[slot]: its position relative to the grid origin
// and its radius in FP32 (for the pre-test).
__global__ void k_cell_fill(const dbl4 *atoms, int n_atoms, Cells c, Geom g, int *cursor, int *list,
                            float4 *rel) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_atoms) return;
  const dbl4 A = atoms[a];
  const int slot = atomicAdd(cursor + atom_cell(c, A), 1);
  list[slot] = a;
  rel[slot] = make_float4((float)(A.x - g.ox), (float)(A.y - g.oy), (float)(A.z - g.oz), (float)A.w);
}
__global__ void k_fill_one(double *a, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    a[e] = 1.0;
}

constexpr int HARMONIC_MAX_IV = 48;  // intervals one edge may collect
constexpr int HARMONIC_NT = 128;
__global__ void __launch_bounds__(HARMONIC_NT)
    k_harmonic_eps(const dbl4 *atoms, const int *start, const int *list, const float4 *rel, Cells c,
                   Geom g, double r_max, double ein, double eout, double *ex, double *ey, double *ez,
                   int *err) {
  const long nxe = (long)(g.nx + 1) * g.ny * g.nz, nye = (long)g.nx * (g.ny + 1) * g.nz;
  const long nze = (long)g.nx * g.ny * (g.nz + 1);
  long t = blockIdx.x * (long)HARMONIC_NT + threadIdx.x;
  if (t >= nxe + nye + nze) return;
  int ax;
  long i, j, k;  // start node of the edge (-1 on the edge axis is the ghost layer)
  double *out;
  if (t < nxe) {
    ax = 0;
    i = t % (g.nx + 1) - 1; j = (t / (g.nx + 1)) % g.ny; k = t / ((long)(g.nx + 1) * g.ny);
    out = ex + ((size_t)k * g.ny + j) * g.px + (i + 1);
  } else if ((t -= nxe) < nye) {
    ax = 1;
    i = t % g.nx; j = (t / g.nx) % (g.ny + 1) - 1; k = t / ((long)g.nx * (g.ny + 1));
    out = ey + ((size_t)k * (g.ny + 1) + (j + 1)) * g.px + i;
  } else {
    t -= nye;
    ax = 2;
    i = t % g.nx; j = (t / g.nx) % g.ny; k = t / ((long)g.nx * g.ny) - 1;
    out = ez + ((size_t)(k + 1) * g.ny + j) * g.px + i;
  }
  const double p[3] = {__dadd_rn(g.ox, __dmul_rn((double)i, g.h)),
                       __dadd_rn(g.oy, __dmul_rn((double)j, g.h)),
                       __dadd_rn(g.oz, __dmul_rn((double)k, g.h))};
  const double c0[3] = {c.x0, c.y0, c.z0};
  const int nc[3] = {c.ncx, c.ncy, c.ncz};
  int lo_c[3], hi_c[3];
  for (int d = 0; d < 3; d++) {
    lo_c[d] = cell_index(p[d] - r_max, c0[d], c.cs, nc[d]);
    hi_c[d] = cell_index(p[d] + (d == ax ? g.h : 0.0) + r_max, c0[d], c.cs, nc[d]);
  }
  const int u = (ax + 1) % 3, v = (ax + 2) % 3;
  // FP32 pre-test relative to the grid origin: the perpendicular distance and
  // the extent along the axis, with a margin far above their FP32 error
  const float hf = (float)g.h, MARGIN = 1e-3f;
  const float pf[3] = {(float)i * hf, (float)j * hf, (float)k * hf};
  double lo_iv[HARMONIC_MAX_IV], hi_iv[HARMONIC_MAX_IV];
  int n_iv = 0;
  bool full = false, overflow = false;
  for (int cz = lo_c[2]; cz <= hi_c[2] && !full; cz++)
    for (int cy = lo_c[1]; cy <= hi_c[1] && !full; cy++)
      for (int cx = lo_c[0]; cx <= hi_c[0] && !full; cx++) {
        const int cell = (cz * c.ncy + cy) * c.ncx + cx;
        for (int s = start[cell]; s < start[cell + 1]; s++) {
          const float4 R = rel[s];
          const float rc[3] = {R.x, R.y, R.z};
          const float fu = pf[u] - rc[u], fv = pf[v] - rc[v], fa = rc[ax] - pf[ax];
          if (fu * fu + fv * fv > R.w * R.w + MARGIN) continue;
          if (fa + R.w < -MARGIN || fa - R.w > hf + MARGIN) continue;
          // exact FP64 interval
          const dbl4 A = atoms[list[s]];
          const double cc[3] = {A.x, A.y, A.z};
          const double du = __dsub_rn(p[u], cc[u]), dv = __dsub_rn(p[v], cc[v]);
          const double d2 = __dadd_rn(__dmul_rn(du, du), __dmul_rn(dv, dv));
          const double sq = __dsub_rn(__dmul_rn(A.w, A.w), d2);
          if (!(sq > 0.0)) continue;
          const double q = __dsqrt_rn(sq);
          const double t0 = __ddiv_rn(__dsub_rn(__dsub_rn(cc[ax], q), p[ax]), g.h);
          const double t1 = __ddiv_rn(__dsub_rn(__dadd_rn(cc[ax], q), p[ax]), g.h);
          const double lo = t0 > 0.0 ? t0 : 0.0, hi = t1 < 1.0 ? t1 : 1.0;
          if (!(lo < hi)) continue;
          if (lo == 0.0 && hi == 1.0) {  // one sphere covers the whole edge: w = 1
            full = true;
            break;
          }
          if (n_iv == HARMONIC_MAX_IV) {
            overflow = true;
            continue;
          }
          // insertion in (lo, hi) order
          int at = n_iv++;
          while (at > 0 && (lo_iv[at - 1] > lo || (lo_iv[at - 1] == lo && hi_iv[at - 1] > hi))) {
            lo_iv[at] = lo_iv[at - 1];
            hi_iv[at] = hi_iv[at - 1];
            at--;
          }
          lo_iv[at] = lo;
          hi_iv[at] = hi;
        }
      }
  if (overflow && !full) atomicOr(err, 4);
  double w;
  if (full) {
    w = 1.0;
  } else if (n_iv == 0) {
    w = 0.0;
  } else {
    w = 0.0;
    double lo = lo_iv[0], hi = hi_iv[0];
    for (int q = 1; q < n_iv; q++) {
      if (lo_iv[q] <= hi) {
        if (hi_iv[q] > hi) hi = hi_iv[q];
      } else {
        w = __dadd_rn(w, __dsub_rn(hi, lo));
        lo = lo_iv[q];
        hi = hi_iv[q];
      }
    }
    w = __dadd_rn(w, __dsub_rn(hi, lo));
  }
  *out = w == 0.0 ? eout
         : w == 1.0 ? ein
                    : __ddiv_rn(1.0, __dadd_rn(__ddiv_rn(w, ein), __ddiv_rn(__dsub_rn(1.0, w), eout)));
}

// diag64 (six edges in the order x-, x+, y-, y+, z-, z+, then + kbh2 lambda)
// and the inner solve's rounded copies; pads hold 1.
template <typename C>
__global__ void k_harmonic_finish(const uint8_t *code, Geom g, double kbh2, const double *ex64,
                                  const double *ey64, const double *ez64, double *diag64, C *ex,
                                  C *ey, C *ez, float *diag) {
  const size_t px = g.px, ny = g.ny, nz = g.nz, nx = g.nx;
  const size_t n_ex = px * ny * nz, n_ey = px * (ny + 1) * nz, n_ez = px * ny * (nz + 1);
  const size_t n_all = n_ey > n_ez ? n_ey : n_ez;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n_all;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < n_ex) {
      const size_t i = e % px, row = e / px;
      const size_t j = row % ny, k = row / ny;
      double d = 1.0;
      if (i < nx) {
        d = ex64[e];
        d = __dadd_rn(d, ex64[e + 1]);
        d = __dadd_rn(d, ey64[(k * (ny + 1) + j) * px + i]);
        d = __dadd_rn(d, ey64[(k * (ny + 1) + j + 1) * px + i]);
        d = __dadd_rn(d, ez64[(k * ny + j) * px + i]);
        d = __dadd_rn(d, ez64[((k + 1) * ny + j) * px + i]);
        d = __dadd_rn(d, __dmul_rn(kbh2, (code[e] & 64u) ? 0.0 : 1.0));
      }
      diag64[e] = d;
      if (diag) diag[e] = (float)d;
      if (ex) ex[e] = (C)ex64[e];
    }
    if (ex && e < n_ey) ey[e] = (C)ey64[e];
    if (ex && e < n_ez) ez[e] = (C)ez64[e];
  }
}

// ---------------------------------------------------------------------------
// Host launchers

static int grid_for(size_t n, int nt) {
  size_t b = (n + nt - 1) / nt;
  return (int)(b < 152 * 64 ? (b ? b : 1) : 152 * 64);
}

CellPlan cell_plan(const Geom &g, double r_max) {
  CellPlan p;
  p.size = r_max + g.h;
  p.ncx = (int)std::ceil((g.nx + 1) * g.h / p.size) + 3;
  p.ncy = (int)std::ceil((g.ny + 1) * g.h / p.size) + 3;
  p.ncz = (int)std::ceil((g.nz + 1) * g.h / p.size) + 3;
  return p;
}
size_t cell_buffer_bytes(const CellPlan &p, int n_atoms) {
  return sizeof(int) * (3 * (size_t)p.n() + 1 + (size_t)n_atoms) + 16 + sizeof(float4) * (size_t)n_atoms;
}

cudaError_t launch_setup(const SetupArgs &a, cudaStream_t st) {
  const Geom &g = a.g;
  const size_t n_pad = (size_t)g.px * g.ny * g.nz;
  k_init_code<<<grid_for(n_pad, 256), 256, 0, st>>>(a.code, n_pad);
  if (a.n_atoms > 0) {
#ifndef PB_EPS_NT
#define PB_EPS_NT 64  // 128 measured 20% slower on the serving stream's grids
#endif
    k_eps_scatter<<<a.n_atoms, PB_EPS_NT, 0, st>>>(a.atoms_xyzr, a.n_atoms, g, (uint32_t *)a.code,
                                             a.kappa_mask);
    k_spread<<<(a.n_atoms + 127) / 128, 128, 0, st>>>(a.atoms_xyzq, a.n_atoms, g, a.q_scale,
                                                      (unsigned long long *)a.b, a.err);
  }
  const long n_ghost = 2L * ((long)g.ny * g.nz + (long)g.nx * g.nz + (long)g.nx * g.ny);
  if (a.n_atoms > 0 && !g.periodic) {  // a periodic grid has no boundary
    const int blocks = (int)((n_ghost + DH_NT - 1) / DH_NT);
    if (a.dh_f32)
      k_dh_f32<<<blocks, DH_NT, 0, st>>>(a.atoms_xyzq, a.n_atoms, g, a.kappa, a.eout, a.ghost,
                                         n_ghost);
    else
      k_dh_f64<<<blocks, DH_NT, 0, st>>>(a.atoms_xyzq, a.n_atoms, g, a.kappa, a.eout, a.ghost,
                                         n_ghost);
  } else {
    cudaMemsetAsync(a.ghost, 0, sizeof(double) * n_ghost, st);
  }
  if (a.ex64) {  // harmonic-average dielectric: the FP64 edge arrays, needed by the fold
    const CellPlan cp = cell_plan(g, a.r_max);
    const Cells c{g.ox - g.h - cp.size, g.oy - g.h - cp.size, g.oz - g.h - cp.size, cp.size,
                  cp.ncx, cp.ncy, cp.ncz};
    const long ncell = cp.n();
    int *count = (int *)a.cell_buf, *start = count + ncell, *cursor = start + ncell + 1;
    int *list = cursor + ncell;
    float4 *rel = (float4 *)(((uintptr_t)(list + a.n_atoms) + 15) & ~(uintptr_t)15);
    const size_t n_ex = (size_t)g.px * g.ny * g.nz, n_c = (size_t)g.px * (g.ny + 1) * (g.nz + 1);
    k_fill_one<<<grid_for(n_ex, 256), 256, 0, st>>>(a.ex64, n_ex);
    k_fill_one<<<grid_for(n_c, 256), 256, 0, st>>>(a.ey64, n_c);
    k_fill_one<<<grid_for(n_c, 256), 256, 0, st>>>(a.ez64, n_c);
    cudaMemsetAsync(count, 0, sizeof(int) * ncell, st);
    if (a.n_atoms > 0) {
      k_cell_count<<<(a.n_atoms + 255) / 256, 256, 0, st>>>(a.atoms_xyzr, a.n_atoms, c, count);
      k_cell_scan<<<1, 1024, 0, st>>>(count, (int)ncell, start, cursor);
      k_cell_fill<<<(a.n_atoms + 255) / 256, 256, 0, st>>>(a.atoms_xyzr, a.n_atoms, c, g, cursor,
                                                           list, rel);
    } else {
      cudaMemsetAsync(start, 0, sizeof(int) * (ncell + 1), st);
    }
    const long n_edges = (long)(g.nx + 1) * g.ny * g.nz + (long)g.nx * (g.ny + 1) * g.nz +
                         (long)g.nx * g.ny * (g.nz + 1);
    k_harmonic_eps<<<(unsigned)((n_edges + HARMONIC_NT - 1) / HARMONIC_NT), HARMONIC_NT, 0, st>>>(
        a.atoms_xyzr, start, list, rel, c, g, a.r_max, a.ein, a.eout, a.ex64, a.ey64, a.ez64, a.err);
  }
  k_fold_rhs<<<FOLD_CTAS, FOLD_NT, 0, st>>>((const long long *)a.b, a.code, a.ghost, g,
                                            a.c4pi_h / a.q_scale, a.ein, a.eout, a.ex64, a.ey64,
                                            a.ez64, a.b, a.scratch);
  k_sum_final<<<1, 256, 0, st>>>(a.scratch, FOLD_CTAS, a.bnorm2);
  return cudaGetLastError();
}

cudaError_t launch_expand(const uint8_t *code, const Geom &g, double ein, double eout, double kbh2,
                          int coef, void *ex, void *ey, void *ez, void *diag, cudaStream_t st) {
  const size_t n = (size_t)g.px * (g.ny + 1) * (g.nz + 1);
  const int blocks = grid_for(n, 256);
  if (coef == COEF_F32)
    k_expand_coef<float, float><<<blocks, 256, 0, st>>>(code, g, ein, eout, kbh2, (float *)ex,
                                                        (float *)ey, (float *)ez, (float *)diag);
  else if (coef == COEF_BF16)
    k_expand_coef<__nv_bfloat16, float><<<blocks, 256, 0, st>>>(
        code, g, ein, eout, kbh2, (__nv_bfloat16 *)ex, (__nv_bfloat16 *)ey, (__nv_bfloat16 *)ez,
        (float *)diag);
  else
    k_expand_coef<double, double><<<blocks, 256, 0, st>>>(code, g, ein, eout, kbh2, (double *)ex,
                                                          (double *)ey, (double *)ez,
                                                          (double *)diag);
  return cudaGetLastError();
}

cudaError_t launch_harmonic_finish(const uint8_t *code, const Geom &g, double kbh2, const double *ex64,
                                   const double *ey64, const double *ez64, double *diag64, int coef,
                                   void *ex, void *ey, void *ez, void *diag, cudaStream_t st) {
  const size_t n = (size_t)g.px * (g.ny + 1) * (g.nz + 1);
  const int blocks = grid_for(n, 256);
  if (coef == COEF_BF16)
    k_harmonic_finish<__nv_bfloat16><<<blocks, 256, 0, st>>>(
        code, g, kbh2, ex64, ey64, ez64, diag64, (__nv_bfloat16 *)ex, (__nv_bfloat16 *)ey,
        (__nv_bfloat16 *)ez, (float *)diag);
  else
    k_harmonic_finish<float><<<blocks, 256, 0, st>>>(code, g, kbh2, ex64, ey64, ez64, diag64,
                                                      (float *)ex, (float *)ey, (float *)ez,
                                                      (float *)diag);
  return cudaGetLastError();
}

cudaError_t launch_export_lambda(const uint8_t *code, const Geom &g, uint8_t *lam, cudaStream_t st) {
  k_export_lambda<<<grid_for((size_t)g.nx * g.ny * g.nz, 256), 256, 0, st>>>(code, g, lam);
  return cudaGetLastError();
}

}  // namespace pb
