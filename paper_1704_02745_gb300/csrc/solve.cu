// solve.cu -- phase kernels of the batched Jacobi-PCG solve of the linear
// FDPB system A phi = b (arXiv:1704.02745 Sec. 2.2 preconditioned CG, Sec. 2.4
// Jacobi preconditioner M = diag A, operator of Eq. 3-4).
//
// One CG iteration is two passes over HBM:
//   stencil pass (k_stencil, INNER phase), iteration l:
//       p_{l-1} = z_{l-1} + beta_{l-1} p_{l-2}      (z = M^-1 r, rebuilt on the fly,
//                                                    halos recomputed in shared memory)
//       Ap_{l-1}, partial p.Ap                      (seven-point stencil)
//       x_{l-1} = x_{l-2} + alpha_{l-1} p_{l-2}     (the previous step's x update,
//                                                    deferred to this pass)
//     finaliser: alpha_l = (r.z) / (p.Ap)
//   update pass (k_update):
//       r_l = r_{l-1} - alpha_l Ap_{l-1}; z_l = M^-1 r_l; partial r.z, r.r
//     finaliser: beta_l = (r.z)_l / (r.z)_{l-1}; ||r_l|| / ||rhs|| < tol -> stop
// The same stencil kernel runs the RESID phase, FP64 throughout:
//       x_new = x64 + d + alpha p   (the last deferred update folded in)
//       r64 = b - A x_new; inner rhs r = (T) r64; partial ||r64||^2, r.z
//     finaliser: FP64 true residual test, then DONE or a new inner solve
//     (iterative refinement, FP32 inner / FP64 outer).
// alpha, beta and the stop test are formed on the device by the last CTA to
// finish an instance's tiles, summing the per-tile partials in tile order, so
// results are bitwise reproducible and independent of the other instances in
// a batch.  Every kernel loops persistently over a work list of (instance,
// tile) items and skips instances in another phase (convergence masks).
#include <cuda_bf16.h>

#include <type_traits>

#include "coef.cuh"
#include "pb_internal.cuh"
#include "solve.cuh"

namespace pb {

// Halo bookkeeping: threads 0..2*TY+2*TX-1 each own one halo cell of a plane.
struct Halo {
  int hi, hj, sx, sy;
  bool role;
};
__device__ __forceinline__ Halo halo_of(int x0, int y0) {
  Halo h{-1, -1, 0, 0, false};
  const int t = threadIdx.x;
  if (t < TY) { h.hi = x0 - 1; h.hj = y0 + t; h.sx = 0; h.sy = t + 1; h.role = true; }
  else if (t < 2 * TY) { h.hi = x0 + TX; h.hj = y0 + t - TY; h.sx = TX + 1; h.sy = t - TY + 1; h.role = true; }
  else if (t < 2 * TY + TX) { h.hi = x0 + t - 2 * TY; h.hj = y0 - 1; h.sx = t - 2 * TY + 1; h.sy = 0; h.role = true; }
  else if (t < 2 * TY + 2 * TX) { h.hi = x0 + t - 2 * TY - TX; h.hj = y0 + TY; h.sx = t - 2 * TY - TX + 1; h.sy = TY + 1; h.role = true; }
  return h;
}

struct TileGeo {
  int i, j, z0, z1, x0, y0;
  bool valid;
};
__device__ __forceinline__ TileGeo tile_geo(const Inst &I, int tile) {
  TileGeo g;
  const int bx = tile % I.tiles_x, rest = tile / I.tiles_x;
  const int by = rest % I.tiles_y, bz = rest / I.tiles_y;
  g.x0 = bx * TX; g.y0 = by * TY;
  g.z0 = bz * I.tz; g.z1 = min(g.z0 + I.tz, I.nz);
  g.i = g.x0 + (int)(threadIdx.x % TX);
  g.j = g.y0 + (int)(threadIdx.x / TX);
  g.valid = g.i < I.nx && g.j < I.ny;
  return g;
}

// ---------------------------------------------------------------------------
// INNER phase, stencil pass of one tile.  Returns this thread's p.Ap.
template <typename T, int CM>
__device__ __forceinline__ double cg_tile(const Inst &I, const Scal &S, int tile,
                                          T (*sp)[TY + 2][TX + 2]) {
  constexpr bool SEP = sizeof(T) == 4;  // FP32 inner solves accumulate into d
  const TileGeo G = tile_geo(I, tile);
  const Halo H = halo_of(G.x0, G.y0);
  const bool hvalid = H.role && H.hi >= 0 && H.hi < I.nx && H.hj >= 0 && H.hj < I.ny;
  const size_t px = I.px, plane = (size_t)I.px * I.ny;
  const size_t ec0 = (size_t)G.j * px + G.i, eh0 = (size_t)H.hj * px + H.hi;
  const bool first = S.phase == PH_START;
  const T beta = (T)S.beta, alpha = (T)S.alpha;
  const T *__restrict__ r = (const T *)I.r;
  const T *__restrict__ pold = (const T *)(S.pbuf ? I.p1 : I.p0);
  T *__restrict__ pnew = (T *)(S.pbuf ? I.p0 : I.p1);
  T *__restrict__ ap = (T *)I.ap;
  T *__restrict__ x = SEP ? (T *)I.d : (T *)(S.xbuf ? I.x64b : I.x64);

  auto pn = [&](size_t e, T &po) -> T {
    po = pold[e];
    const T z = zval<T, CM>(I, e, r[e]);
    return first ? z : z + beta * po;
  };

  T pm = 0, pc = 0, poc = 0, dummy;
  if (G.valid && G.z0 > 0) pm = pn((size_t)(G.z0 - 1) * plane + ec0, dummy);
  if (G.valid) pc = pn((size_t)G.z0 * plane + ec0, poc);
  sp[0][threadIdx.x / TX + 1][threadIdx.x % TX + 1] = pc;
  if (H.role) sp[0][H.sy][H.sx] = hvalid ? pn((size_t)G.z0 * plane + eh0, dummy) : (T)0;
  const int tx = threadIdx.x % TX + 1, ty = threadIdx.x / TX + 1;
  int cur = 0;
  T acc = 0;
  for (int k = G.z0; k < G.z1; ++k) {
    const int nxt = cur == 2 ? 0 : cur + 1;
    T pnx = 0, ponx = 0;
    if (k + 1 < I.nz) {
      if (G.valid) pnx = pn((size_t)(k + 1) * plane + ec0, ponx);
      if (H.role) sp[nxt][H.sy][H.sx] = hvalid ? pn((size_t)(k + 1) * plane + eh0, dummy) : (T)0;
    } else if (H.role) {
      sp[nxt][H.sy][H.sx] = 0;
    }
    sp[nxt][ty][tx] = pnx;
    __syncthreads();
    if (G.valid) {
      const size_t e = (size_t)k * plane + ec0;
      const NodeCoef<T> c = node_coef<T, CM>(I, e, k);
      T s = c.exm * sp[cur][ty][tx - 1];
      s += c.exp * sp[cur][ty][tx + 1];
      s += c.eym * sp[cur][ty - 1][tx];
      s += c.eyp * sp[cur][ty + 1][tx];
      s += c.ezm * pm;
      s += c.ezp * pnx;
      const T a = c.diag * pc - s;
      pnew[e] = pc;
      ap[e] = a;
      if (SEP) x[e] = first ? (T)0 : x[e] + alpha * poc;
      else if (!first) x[e] = x[e] + alpha * poc;
      acc += pc * a;
    }
    pm = pc; pc = pnx; poc = ponx; cur = nxt;
  }
  return (double)acc;
}

// RESID phase (FP64): fold the deferred update, true residual, new inner rhs.
template <typename T, int CM>
__device__ __forceinline__ void resid_tile(const Inst &I, const Scal &S, int tile,
                                           double (*sq)[TY + 2][TX + 2], double &rr64,
                                           double &rz) {
  constexpr bool SEP = sizeof(T) == 4;
  const TileGeo G = tile_geo(I, tile);
  const Halo H = halo_of(G.x0, G.y0);
  const bool hvalid = H.role && H.hi >= 0 && H.hi < I.nx && H.hj >= 0 && H.hj < I.ny;
  const size_t px = I.px, plane = (size_t)I.px * I.ny;
  const size_t ec0 = (size_t)G.j * px + G.i, eh0 = (size_t)H.hj * px + H.hi;
  const double alpha = S.alpha;
  const double *__restrict__ xin = S.xbuf ? I.x64b : I.x64;
  double *__restrict__ xout = S.xbuf ? I.x64 : I.x64b;
  const T *__restrict__ d = (const T *)I.d;
  const T *__restrict__ p = (const T *)(S.pbuf ? I.p1 : I.p0);
  T *__restrict__ r = (T *)I.r;

  // Before the first inner solve there is nothing to fold (d and p unset).
  const bool fold = S.outer > 0;
  auto xn = [&](size_t e) -> double {
    double v = xin[e];
    if (!fold) return v;
    if (SEP) v += (double)d[e];
    return v + alpha * (double)p[e];
  };

  double xm = 0, xc = 0;
  if (G.valid && G.z0 > 0) xm = xn((size_t)(G.z0 - 1) * plane + ec0);
  if (G.valid) xc = xn((size_t)G.z0 * plane + ec0);
  const int tx = threadIdx.x % TX + 1, ty = threadIdx.x / TX + 1;
  sq[0][ty][tx] = xc;
  if (H.role) sq[0][H.sy][H.sx] = hvalid ? xn((size_t)G.z0 * plane + eh0) : 0.0;
  int cur = 0;
  rr64 = 0.0; rz = 0.0;
  for (int k = G.z0; k < G.z1; ++k) {
    const int nxt = cur == 2 ? 0 : cur + 1;
    double xnx = 0;
    if (k + 1 < I.nz) {
      if (G.valid) xnx = xn((size_t)(k + 1) * plane + ec0);
      if (H.role) sq[nxt][H.sy][H.sx] = hvalid ? xn((size_t)(k + 1) * plane + eh0) : 0.0;
    } else if (H.role) {
      sq[nxt][H.sy][H.sx] = 0.0;
    }
    sq[nxt][ty][tx] = xnx;
    __syncthreads();
    if (G.valid) {
      const size_t e = (size_t)k * plane + ec0;
      const NodeCoef<double> c = node_coef64<CM>(I, e, k);
      double s = c.exm * sq[cur][ty][tx - 1];
      s += c.exp * sq[cur][ty][tx + 1];
      s += c.eym * sq[cur][ty - 1][tx];
      s += c.eyp * sq[cur][ty + 1][tx];
      s += c.ezm * xm;
      s += c.ezp * xnx;
      const double res = I.b[e] - (c.diag * xc - s);
      xout[e] = xc;
      const T rt = (T)res;
      r[e] = rt;
      rr64 += res * res;
      rz += (double)(rt * zval<T, CM>(I, e, rt));
    }
    xm = xc; xc = xnx; cur = nxt;
  }
}

// ---------------------------------------------------------------------------
// Deterministic block reductions.

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum two values over the CTA; thread 0 gets the result.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int u = 0; u < NT / 32; u++) { sa += red[2 * u]; sb += red[2 * u + 1]; }
    a = sa; b = sb;
  }
  __syncthreads();
}

// Sum column c of n partials (stride 2) with the whole CTA in a fixed order.
__device__ __forceinline__ void sum_partials(const double *part, int n, double &s0, double &s1,
                                             double *red) {
  double a = 0, b = 0;
  for (int t = threadIdx.x; t < n; t += NT) {
    a += __ldcg(part + 2 * t);
    b += __ldcg(part + 2 * t + 1);
  }
  block_sum2(a, b, red);
  s0 = a; s1 = b;
}

// ---------------------------------------------------------------------------
// Finalisers (run by the last CTA of an instance; thread 0 writes).

__device__ void fin_cg(const Inst &I, Scal *S, double pap) {
  S->cnt2 = 0;
  const double alpha = S->rz_old / pap;
  if (!(pap > 0.0) || !isfinite(alpha)) {
    S->status = 6;  // PB_ERR_BREAKDOWN
    S->phase = PH_DONE;
    return;
  }
  S->alpha = alpha;
  S->pbuf ^= 1;
  S->phase = PH_INNER;
}

__device__ void fin_update(const Inst &I, Scal *S, double rz, double rr) {
  S->cnt3 = 0;
  if (!isfinite(rz) || !isfinite(rr)) {
    S->status = 6;
    S->phase = PH_DONE;
    return;
  }
  S->beta = rz / S->rz_old;
  S->rz_old = rz;
  S->iter += 1;
  S->total_iter += 1;
  S->relres = sqrt(rr) / S->ref_norm;
  const double tol = I.mode == MODE_F32_REFINE ? I.inner_tol : I.tol;
  if (S->relres < tol) {
    S->phase = PH_RESID;
  } else if (S->total_iter >= I.max_iter) {
    S->status = 5;  // PB_ERR_NOT_CONVERGED
    S->phase = PH_RESID;
  }
}

__device__ void fin_resid(const Inst &I, Scal *S, double rr64, double rz) {
  S->cnt2 = 0;
  S->xbuf ^= 1;  // the new solution now sits in the other x buffer
  const double rel = sqrt(rr64) / I.bnorm;
  S->relres_true = rel;
  if (!isfinite(rel)) {
    S->status = 6;
    S->phase = PH_DONE;
    return;
  }
  if (rel < I.tol) {
    if (S->outer == 0) S->relres = rel;
    S->status = 0;
    S->phase = PH_DONE;
    return;
  }
  if (S->outer >= 1) {
    const bool refine = I.mode == MODE_F32_REFINE;
    if (!refine || S->status != 0 || S->outer >= I.max_outer || S->total_iter >= I.max_iter) {
      if (refine && S->status == 0) S->status = 5;
      S->phase = PH_DONE;
      return;
    }
  }
  S->outer += 1;
  S->iter = 0;
  S->alpha = 0.0;
  S->beta = 0.0;
  S->rz_old = rz;
  S->ref_norm = I.mode == MODE_F32_REFINE ? sqrt(rr64) : I.bnorm;
  S->relres = I.mode == MODE_F32_REFINE ? 1.0 : rel;
  S->phase = PH_START;
}

// ---------------------------------------------------------------------------
// Phase kernels.

template <typename T, int CM>
__global__ void __launch_bounds__(NT) k_stencil(Batch B) {
  __shared__ __align__(16) double smem[3][TY + 2][TX + 2];
  __shared__ double red[2 * (NT / 32)];
  __shared__ int s_phase, s_last;
  for (int it = blockIdx.x; it < B.n_st_items; it += gridDim.x) {
    const Item item = B.st_items[it];
    const Inst &I = B.inst[item.inst];
    Scal *Sp = I.s;
    if (threadIdx.x == 0) s_phase = *(volatile int *)&Sp->phase;
    __syncthreads();
    const int ph = s_phase;
    if (ph == PH_INNER || ph == PH_START || ph == PH_RESID) {
      const Scal S = *Sp;
      double v0 = 0, v1 = 0;
      if (ph != PH_RESID) v0 = cg_tile<T, CM>(I, S, item.tile, (T(*)[TY + 2][TX + 2])smem);
      else resid_tile<T, CM>(I, S, item.tile, smem, v0, v1);
      block_sum2(v0, v1, red);
      if (threadIdx.x == 0) {
        double *part = B.st_part + 2 * (size_t)(I.st_base + item.tile);
        part[0] = v0;
        part[1] = v1;
        __threadfence();
        const unsigned prev = atomicAdd(&Sp->cnt2, 1u);
        s_last = prev == (unsigned)(I.n_st - 1);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        double s0, s1;
        sum_partials(B.st_part + 2 * (size_t)I.st_base, I.n_st, s0, s1, red);
        if (threadIdx.x == 0) {
          if (ph == PH_RESID) fin_resid(I, Sp, s0, s1);
          else fin_cg(I, Sp, s0);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int CM>
__global__ void __launch_bounds__(NT) k_update(Batch B) {
  constexpr int V = 16 / sizeof(T);
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type VT;
  __shared__ double red[2 * (NT / 32)];
  __shared__ int s_phase, s_last;
  for (int it = blockIdx.x; it < B.n_ch_items; it += gridDim.x) {
    const Item item = B.ch_items[it];
    const Inst &I = B.inst[item.inst];
    Scal *Sp = I.s;
    if (threadIdx.x == 0) s_phase = *(volatile int *)&Sp->phase;
    __syncthreads();
    if (s_phase == PH_INNER) {
      const T alpha = (T)Sp->alpha;
      const size_t lo = (size_t)item.tile * CH;
      const size_t hi = min(lo + (size_t)CH, I.n_pad);
      T *__restrict__ r = (T *)I.r;
      const T *__restrict__ ap = (const T *)I.ap;
      T rz = 0, rr = 0;
      for (size_t e = lo + (size_t)threadIdx.x * V; e < hi; e += (size_t)NT * V) {
        VT rv = *(const VT *)(r + e);
        const VT av = *(const VT *)(ap + e);
        T *rp = (T *)&rv;
        const T *apv = (const T *)&av;
#pragma unroll
        for (int u = 0; u < V; u++) {
          rp[u] = rp[u] - alpha * apv[u];
          const T z = zval<T, CM>(I, e + u, rp[u]);
          rz += rp[u] * z;
          rr += rp[u] * rp[u];
        }
        *(VT *)(r + e) = rv;
      }
      double a = (double)rz, b = (double)rr;
      block_sum2(a, b, red);
      if (threadIdx.x == 0) {
        double *part = B.ch_part + 2 * (size_t)(I.ch_base + item.tile);
        part[0] = a;
        part[1] = b;
        __threadfence();
        const unsigned prev = atomicAdd(&Sp->cnt3, 1u);
        s_last = prev == (unsigned)(I.n_ch - 1);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        double s0, s1;
        sum_partials(B.ch_part + 2 * (size_t)I.ch_base, I.n_ch, s0, s1, red);
        if (threadIdx.x == 0) fin_update(I, Sp, s0, s1);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side

template <typename T, int CM>
static cudaError_t phase_impl(const Batch &B, const KernelGrid &kg, int which, cudaStream_t st) {
  if (which & 1) k_stencil<T, CM><<<kg.stencil_blocks, NT, 0, st>>>(B);
  if (which & 2) k_update<T, CM><<<kg.update_blocks, NT, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_phase(const Batch &B, int mode, int coef, const KernelGrid &kg, int which,
                         cudaStream_t st) {
  if (mode == MODE_F64) {
    if (coef == COEF_F64) return phase_impl<double, COEF_F64>(B, kg, which, st);
    return phase_impl<double, COEF_PACKED>(B, kg, which, st);
  }
  if (coef == COEF_F32) return phase_impl<float, COEF_F32>(B, kg, which, st);
  if (coef == COEF_BF16) return phase_impl<float, COEF_BF16>(B, kg, which, st);
  return phase_impl<float, COEF_PACKED>(B, kg, which, st);
}

cudaError_t launch_tick(const Batch &B, int mode, int coef, const KernelGrid &kg, cudaStream_t st) {
  return launch_phase(B, mode, coef, kg, 3, st);
}

template <typename T, int CM>
static void occ(int &s, int &u) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s, k_stencil<T, CM>, NT, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&u, k_update<T, CM>, NT, 0);
}

KernelGrid kernel_grid(int mode, int coef, int num_sms) {
  int s = 1, u = 1;
  if (mode == MODE_F64) {
    if (coef == COEF_F64) occ<double, COEF_F64>(s, u);
    else occ<double, COEF_PACKED>(s, u);
  } else if (coef == COEF_F32) occ<float, COEF_F32>(s, u);
  else if (coef == COEF_BF16) occ<float, COEF_BF16>(s, u);
  else occ<float, COEF_PACKED>(s, u);
  KernelGrid kg;
  kg.stencil_blocks = num_sms * (s > 0 ? s : 1);
  kg.update_blocks = num_sms * (u > 0 ? u : 1);
  return kg;
}

}  // namespace pb
