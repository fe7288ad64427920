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
//   update pass (k_update over row chunks, reading the Ap the stencil pass
//   stored; or k_update_tile over the stencil tiles, forming Ap again):
//       r_l = r_{l-1} - alpha_l Ap_{l-1}; z_l = M^-1 r_l; partial r.z, r.r
//     finaliser: beta_l = (r.z)_l / (r.z)_{l-1}; ||r_l|| / ||rhs|| < tol -> stop
// The residual pass (k_resid, RESID phase, the x and b - A x arithmetic FP64):
//       x_new = x64 + d + alpha p   (the last deferred update folded in)
//       r64 = b - A x_new; inner rhs r = (T) r64; partial ||r64||^2, r.z
//     finaliser: FP64 true residual test, then DONE or a new inner solve
//     (iterative refinement, FP32 inner / FP64 outer).
// alpha, beta and the stop test are formed on the device by the last CTA to
// finish an instance's tiles, summing the per-tile partials in tile order, so
// results are bitwise reproducible and independent of the other instances in
// a batch.  Every kernel loops persistently over a work list of (instance,
// tile) items and skips instances in another phase (convergence masks).
//
// Stencil-pass data movement: a CTA owns a W x H column tile and marches over
// its z range.  One thread issues TMA tile loads (cp.async.bulk.tensor) of z,
// p_old (tile + one-node halo, x widened to the 16-byte rule), the code bytes
// and the centre tile of x, NSTAGE planes ahead of the plane being computed,
// each stage completing on its own mbarrier.  The grid boundary needs no test:
// TMA fills out-of-range elements with zeros, which is exactly the zero ghost
// of the operator.  New directions p are built in a ring of three shared
// planes with halo, from which the stencil reads the in-plane neighbours;
// each thread keeps its own group's p on the planes z-1, z, z+1 in registers.
#include <cuda_bf16.h>

#include <type_traits>

#include "coef.cuh"
#include "pb_internal.cuh"
#include "solve.cuh"

// Explicit coefficient storage: a group's coefficients are requested before
// the stage wait and CTA barrier of the iteration that uses them (FP32
// arrays: the 257^3 stencil pass 153 -> 134 us), or just before use (FP64).
// BF16 arrays are requested early as raw words and widened after the wait
// (PB_BF16_EARLY; widening them where they are requested makes the thread
// wait for the loads there, and measured slower: 141 -> 150 us).
// PB_COEF_EARLY = 0 keeps every storage on the late form.
#ifndef PB_COEF_EARLY
#define PB_COEF_EARLY 1
#endif
#ifndef PB_BF16_EARLY
#define PB_BF16_EARLY 1
#endif
#ifndef PB_BF16_AHEAD
#define PB_BF16_AHEAD 1
#endif
namespace pb {
template <int CM> struct CoefEarly { static constexpr bool value = PB_COEF_EARLY && CM == COEF_F32; };
template <int CM> struct RawEarly {
  static constexpr bool value = PB_COEF_EARLY && PB_BF16_EARLY && CM == COEF_BF16;
};


// ---------------------------------------------------------------------------
// TMA / mbarrier primitives (inline PTX).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
#ifdef PB_WAIT_HINT
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(PB_WAIT_HINT)
      : "memory");
#else
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
#endif
  return ok != 0;
}
// Wait for phase `parity` of a barrier, giving up after 1e8 SM cycles (~50 ms
// at 2 GHz; a TMA tile load lands in microseconds).  A wait that gives up sets
// the launch's error word, and the host reports PB_ERR_TIMEOUT.
#ifndef PB_WAIT_CYCLES
#define PB_WAIT_CYCLES 100000000LL
#endif
constexpr long long WAIT_CYCLES = PB_WAIT_CYCLES;
constexpr int CG_RING_PLANES = 3;  // p planes with halo held by a CG stencil pass
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
#ifdef PB_WAIT_SLEEP_NS
    __nanosleep(PB_WAIT_SLEEP_NS);
#endif
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

#ifdef PB_FAULT_TEST
// Test builds only (compiled with -DPB_FAULT_TEST, never into the product
// library): while this count is positive, the first stage wait of a tile, in
// the thread that issues the tile's copies, gives up at once, as a wait that
// ran out of time would.  The copies themselves are issued and land as usual;
// the exit path must wait for every one of them.
__device__ int g_fault_abandon_waits;
__device__ __forceinline__ bool fault_abandon_wait() {
  return *(volatile int *)&g_fault_abandon_waits > 0 && atomicAdd(&g_fault_abandon_waits, -1) > 0;
}
#endif
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Programmatic dependent launch: let the next kernel in the stream start
// launching now, and wait until the previous kernel's results are visible.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Tile geometry.  A CTA owns a W x H column tile; thread t owns NV consecutive
// x columns (a "group"), so all shared and global accesses of the centre
// nodes are 16-byte vectors.

struct TileG {
  int x0, y0, z0, z1, tx, ty;  // tile origin and z range; group origin in the tile
  bool in_tile;                // thread owns a group of the tile
  bool row_ok;                 // ... whose row is inside the grid
  uint32_t vmask;              // bit u: node tx+u is inside the grid
};
// tz: z planes per tile (I.tz for the CG passes, I.rtz for the residual pass)
__device__ __forceinline__ TileG tile_g(const Inst &I, int tile, int tz) {
  TileG g;
  const int bx = tile % I.tiles_x, rest = tile / I.tiles_x;
  const int by = rest % I.tiles_y, bz = rest / I.tiles_y;
  const int gw = I.W / NV;
  g.x0 = bx * I.W;
  g.y0 = by * I.H;
  g.z0 = bz * tz;
  g.z1 = min(g.z0 + tz, I.nz);
  g.tx = (threadIdx.x % gw) * NV;
  g.ty = threadIdx.x / gw;
  g.in_tile = (int)threadIdx.x < gw * I.H;
  g.row_ok = g.in_tile && g.y0 + g.ty < I.ny;
  g.vmask = 0;
  if (g.row_ok)
    for (int u = 0; u < NV; u++)
      if (g.x0 + g.tx + u < I.nx) g.vmask |= 1u << u;
  return g;
}

// Halo cell owned by this thread: cell h = lane * (NT/32) + warp, so every warp
// gets the same share; cells are the left and right columns, then the bottom
// and top rows.
struct HaloG {
  int hx, hy;  // tile-relative position, -1 .. W / -1 .. H
  bool role;
};
__device__ __forceinline__ HaloG halo_g(const Inst &I) {
  HaloG h{0, 0, false};
  const int t = (threadIdx.x % 32) * (NT / 32) + threadIdx.x / 32, W = I.W, H = I.H;
  if (t < H) { h.hx = -1; h.hy = t; h.role = true; }
  else if (t < 2 * H) { h.hx = W; h.hy = t - H; h.role = true; }
  else if (t < 2 * H + W) { h.hx = t - 2 * H; h.hy = -1; h.role = true; }
  else if (t < 2 * H + 2 * W) { h.hx = t - 2 * H - W; h.hy = H; h.role = true; }
  return h;
}

// NV-element vectors in 16-byte pieces.
template <typename T> struct Vec { T v[NV]; };
template <typename T>
__device__ __forceinline__ Vec<T> ldv(const T *p) {
  Vec<T> r;
  if (sizeof(T) == 4) {
    const float4 a = *(const float4 *)p;
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
  } else {
    const double2 a = ((const double2 *)p)[0], b = ((const double2 *)p)[1];
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = b.x; r.v[3] = b.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ void stv(T *p, const Vec<T> &r) {
  if (sizeof(T) == 4) {
    *(float4 *)p = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    ((double2 *)p)[0] = make_double2(r.v[0], r.v[1]);
    ((double2 *)p)[1] = make_double2(r.v[2], r.v[3]);
  }
}

// The scalars a tile reads (a copy of the full Scal would hold ~20 registers).
struct TileScal {
  double alpha, beta;
  int phase, pbuf, xbuf, outer;
};
__device__ __forceinline__ TileScal tile_scal(const Scal *S) {
  TileScal t;
  t.alpha = S->alpha;
  t.beta = S->beta;
  t.phase = S->phase;
  t.pbuf = S->pbuf;
  t.xbuf = S->xbuf;
  t.outer = S->outer;
  return t;
}

template <typename T> struct Pair { T d, i; };

// Stage ring of the TMA pipeline: stage index and the phase parity of every
// stage, advanced one plane at a time.
struct StageRing {
  uint32_t st;     // stage of the next plane to consume
  uint32_t phase;  // bit s: parity of the next completion of stage s
};

// ---------------------------------------------------------------------------
// INNER phase, one tile of either pass of a CG iteration (TMA pipeline, a
// ring of p planes in shared memory for the in-plane neighbours, the z
// neighbours in registers):
//
//   PASS 0 (direction): p = z + beta p_old (one fused multiply-add per node,
//     halo included, since the stored vector is z = M^-1 r), Ap, this
//     thread's p.Ap in v0; stores p and the deferred x update, and Ap when
//     I.ap is set (for the row-chunk update pass).
//   PASS 1 (update, batches): loads the p just stored, forms Ap again -- the
//     same operations in the same order, so bit for bit the Ap of pass 0 --
//     then r = M z - alpha Ap, z = M^-1 r; stores z; r.z in v0, r.r in v1.
//
// Recomputing Ap costs the p read of pass 1 (4 B per node) and saves the Ap
// write of pass 0 and read of pass 1 (8 B), but a tile pass runs at a nearly
// fixed time per plane and tile, whatever its bytes: it pays where many
// grids fill every SM with tiles (a server batch, and no Ap array resident),
// not on one grid, where the row-chunk update pass streams faster.  dtab: the
// operator's diagonal, mtab: {diag A, M^-1}, by code byte, in shared memory
// per item.  Sets `abort` if a pipeline wait timed out.
//
// Periodic grids: the z planes before and after the grid are the last and
// the first (the TMA loads wrap the plane index), and every ring cell that
// lies outside the grid in x or y -- halo cells and the overhanging lanes and
// rows of the last tiles -- takes the wrapped node's value from global memory.
template <typename T, int CM, int NS, int PASS>
__device__ __forceinline__ void cg_tile(const Inst &I, const TileScal &S, int tile, uint8_t *stages,
                                        T *ring, const T *dtab, const Pair<T> *mtab, uint64_t *full,
                                        StageRing &SR, bool &abort, double &v0, double &v1) {
  constexpr bool SEP = sizeof(T) == 4;  // FP32 inner solves accumulate into d
  constexpr bool UPD = PASS == 1;
  const TileG G = tile_g(I, tile, I.tz);
  const HaloG Hh = halo_g(I);
  const int W = I.W, H = I.H, RW = W + 2 * NV, CW = I.cw, RGW = W + 2 * NV;
  const int ring_plane = RGW * (H + 2);
  // descriptor fields used in the plane loop, held in registers (the asm
  // statements of the pipeline clobber memory, which would force reloads)
  const uint32_t stage_bytes = UPD ? I.stage_bytes_upd : I.stage_bytes, off_p = I.off_p,
                 off_c = UPD ? I.off_c_upd : I.off_c, off_x = UPD ? I.off_x_upd : I.off_x;
  const uint32_t tma_bytes = UPD ? I.tma_bytes_upd : I.tma_bytes;
  const int cx0 = ((G.x0 - 1) >> 4) << 4;  // code box start: 16-byte aligned, <= x0 - 1
  const int Q = (G.z1 - G.z0) + 2;         // planes z0-1 .. z1
  const bool first = S.phase == PH_START;
  const T beta = first ? (T)0 : (T)S.beta, alpha = (T)S.alpha;
  const T ei = e_in<T>(I), eo = e_out<T>(I);
  // pass 0: p_old; pass 1: the p pass 0 stored (its finaliser flipped pbuf)
  const CUtensorMap *m_pold = S.pbuf ? &I.tm_p1 : &I.tm_p0;
  const CUtensorMap *m_x = SEP ? &I.tm_x0 : (S.xbuf ? &I.tm_x1 : &I.tm_x0);
  const size_t plane = (size_t)I.px * I.ny;
  const size_t ec0 = (size_t)(G.y0 + G.ty) * I.px + (G.x0 + G.tx);
  // output pointers walk plane by plane (first written plane: z0)
  T *pnew = (T *)(S.pbuf ? I.p0 : I.p1) + (size_t)G.z0 * plane + ec0;
  T *zout = (T *)I.z + (size_t)G.z0 * plane + ec0;
  const bool store_ap = !UPD && I.ap != nullptr;  // the row-chunk update pass reads Ap
  T *ap = store_ap ? (T *)I.ap + (size_t)G.z0 * plane + ec0 : pnew;
  T *x = (SEP ? (T *)I.d : (T *)(S.xbuf ? I.x64b : I.x64)) + (size_t)G.z0 * plane + ec0;
  const bool per = I.periodic != 0;
  const int nzg = I.nz;
  auto zwrap = [&](int z) { return !per ? z : z < 0 ? z + nzg : z >= nzg ? z - nzg : z; };
  // new direction at a node outside the grid (periodic): that of its image
  auto wrapped_p = [&](int gx, int gy, int zt) -> T {
    const int xw = gx % I.nx, yw = gy < 0 ? gy + I.ny : gy % I.ny;
    const size_t e = (size_t)zt * plane + (size_t)yw * I.px + xw;
    const T pv = ((const T *)(S.pbuf ? I.p1 : I.p0))[e];
    if (UPD) return pv;
    const T zv = ((const T *)I.z)[e];
    return first ? zv : zv + beta * pv;
  };

  // thread 0 issues plane z0-1+q into stage st
  auto issue = [&](int q, uint32_t st) {
    uint8_t *sb = stages + st * stage_bytes;
    const int z = zwrap(G.z0 - 1 + q);
    mbar_expect_tx(&full[st], tma_bytes);
    if (UPD) {  // p (halo box) in the first slot, the z centre box in the x slot
      tma_load_3d(sb, m_pold, &full[st], G.x0 - NV, G.y0 - 1, z);
      tma_load_3d(sb + off_c, &I.tm_code, &full[st], cx0, G.y0 - 1, z);
      tma_load_3d(sb + off_x, &I.tm_zc, &full[st], G.x0, G.y0, z);
    } else {
      tma_load_3d(sb, &I.tm_z, &full[st], G.x0 - NV, G.y0 - 1, z);
      tma_load_3d(sb + off_p, m_pold, &full[st], G.x0 - NV, G.y0 - 1, z);
      tma_load_3d(sb + off_c, &I.tm_code, &full[st], cx0, G.y0 - 1, z);
      tma_load_3d(sb + off_x, m_x, &full[st], G.x0, G.y0, z);
    }
  };
  if (threadIdx.x == 0) {
    uint32_t st = SR.st;
    for (int q = 0; q < min(NS, Q); ++q) {
      issue(q, st);
      st = st + 1 == NS ? 0 : st + 1;
    }
  }

  // this thread's group and halo cell in the stage boxes and the ring
  const int cr = (G.ty + 1) * RW + NV + G.tx;
  const int cc = (G.ty + 1) * CW + (G.x0 + G.tx - cx0);
  const int cg = (G.ty + 1) * RGW + NV + G.tx;
  const int cx = G.ty * W + G.tx;
  const int hr = (Hh.hy + 1) * RW + NV + Hh.hx;
  const int hg = (Hh.hy + 1) * RGW + NV + Hh.hx;

  // loop-invariant tests, hoisted
  const bool wrap_lanes = per && G.in_tile && (G.x0 + G.tx + NV > I.nx || G.y0 + G.ty >= I.ny);
  const int hgx = G.x0 + Hh.hx, hgy = G.y0 + Hh.hy;
  const bool halo_wrap = per && Hh.role && (hgx < 0 || hgx >= I.nx || hgy < 0 || hgy >= I.ny);
  const bool full_group = G.vmask == (1u << NV) - 1u;
  const T m_unit = (T)1;
  // Pass 1 on a grid without wrap reads the in-plane neighbours of plane q-1
  // straight from that plane's stage (the stored p with its halo, zero
  // outside the grid: what the ring would hold), so it writes no ring.  The
  // stage of plane q-1 is then in use until the barrier of iteration q+1:
  // iteration q refills the stage of plane q-2, one plane later than the
  // ring form refills that of plane q.
  const bool box_nb = UPD && !per;
  const T *sz_prev = nullptr;  // stage box of plane q-1 (box_nb)

  uint32_t code_prev = 0;
  T acc = 0, rz = 0, rr = 0;
  Vec<T> z_prev = {};          // pass 1: z of the plane whose Ap is formed next
  Vec<T> pc = {}, pm = {};     // this group's p on planes q-1 and q-2
  // ring slot of plane q; a thread writes slot q while a slower one, still
  // in its pass q-1, may read slot q-2: three slots, one barrier a plane.
  int rq = 0;
  uint32_t st_issue = SR.st;
  for (int u = 0; u < min(NS, Q); ++u) st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
  GroupRaw16 craw_next;  // BF16 words of the plane computed in the next iteration
  for (int q = 0; q < Q; ++q) {
    const int z = G.z0 - 1 + q;
    // explicit storage: the coefficients of plane z-1 (computed in this
    // iteration) are requested before the stage wait and the CTA barrier, so
    // their latency overlaps both
    GroupCoef<T> cpre;
    GroupRaw16 craw;
    if constexpr (CoefEarly<CM>::value) {
      if (q >= 2 && G.vmask)
        cpre = group_coef<T, CM>(I, (size_t)(z - 1) * plane + ec0, z - 1, (G.vmask >> (NV - 1)) & 1u);
    } else if constexpr (RawEarly<CM>::value) {
#if PB_BF16_AHEAD
      // a plane further ahead: plane z-1's words were requested in the
      // previous iteration, plane z's are requested now
      craw = craw_next;
      if (q >= 1 && z < G.z1 && G.vmask)
        craw_next = group_raw16(I, (size_t)z * plane + ec0, z, (G.vmask >> (NV - 1)) & 1u);
#else
      if (q >= 2 && G.vmask)
        craw = group_raw16(I, (size_t)(z - 1) * plane + ec0, z - 1, (G.vmask >> (NV - 1)) & 1u);
#endif
    }
    const uint32_t st = SR.st;
#ifdef PB_FAULT_TEST
    const bool ok = (q == 0 && threadIdx.x == 0 && fault_abandon_wait())
                        ? false : mbar_wait(&full[st], (SR.phase >> st) & 1u);
#else
    const bool ok = mbar_wait(&full[st], (SR.phase >> st) & 1u);
#endif
    SR.phase ^= 1u << st;
    SR.st = st + 1 == NS ? 0 : st + 1;
    const uint8_t *sb = stages + st * stage_bytes;
    const T *sz = (const T *)sb;
    const T *sp = (const T *)(sb + off_p);
    const uint8_t *sc = sb + off_c;
    const T *sx = (const T *)(sb + off_x);
    T *rg = ring + rq * ring_plane;
    const int rq1 = rq == 0 ? CG_RING_PLANES - 1 : rq - 1;
    Vec<T> pn = {}, zc = {};
    uint32_t codes = 0;
    // z and p_old are zero outside the grid (TMA fill, zero pads), and so is
    // p; the first direction is z itself, whatever p_old holds
    if (ok && G.in_tile) {
      pn = ldv(sz + cr);  // pass 1: p itself
      const Vec<T> po = UPD ? Vec<T>{} : ldv(sp + cr);
      codes = *(const uint32_t *)(sc + cc);
      if (UPD) zc = ldv(sx + cx);
      if (!UPD && !first) {
#pragma unroll
        for (int u = 0; u < NV; u++) pn.v[u] += beta * po.v[u];
      }
      if (wrap_lanes) {
#pragma unroll
        for (int u = 0; u < NV; u++)
          if (G.x0 + G.tx + u >= I.nx || G.y0 + G.ty >= I.ny)
            pn.v[u] = wrapped_p(G.x0 + G.tx + u, G.y0 + G.ty, zwrap(z));
      }
      if (!box_nb) stv(rg + cg, pn);
      // deferred update of the previous iteration: x += alpha p_old (the
      // first inner iteration starts the FP32 increment d from zero)
      if (!UPD && G.vmask && q >= 1 && q < Q - 1) {
        Vec<T> xn = {};
        if (!first) {
          xn = ldv(sx + cx);
#pragma unroll
          for (int u = 0; u < NV; u++) xn.v[u] += alpha * po.v[u];
        }
        if (SEP || !first) stv(x, xn);
      }
    }
    if (!UPD && q >= 1 && q < Q - 1) x += plane;
    if (ok && Hh.role && !box_nb) {
      if (halo_wrap)
        rg[hg] = wrapped_p(hgx < 0 ? hgx + I.nx : hgx, hgy, zwrap(z));
      else
        rg[hg] = UPD || first ? sz[hr] : sz[hr] + beta * sp[hr];
    }
    if (__syncthreads_or(!ok)) {
      // A wait gave up: let the copies already issued land -- those of this
      // plane q, whose wait gave up, and of every later plane issued -- each
      // for a bounded time, before the CTA leaves.
      if (threadIdx.x == 0) {
        uint32_t s2 = st, ph = SR.phase ^ (1u << st);  // plane q's stage and parity
        const int last = box_nb ? max(NS - 1, q + NS - 3) : q + NS - 1;  // last plane issued
        for (int u = q; u <= min(Q - 1, last); ++u) {
          mbar_wait(&full[s2], (ph >> s2) & 1u);
          ph ^= 1u << s2;
          s2 = s2 + 1 == NS ? 0 : s2 + 1;
        }
        SR.phase = ph;
        SR.st = s2;
      }
      abort = true;
      v0 = v1 = 0.0;
      return;
    }
    if (threadIdx.x == 0) {
      const int qi = box_nb ? q - 2 + NS : q + NS;  // refills the stage of plane q-2 or q
      if ((!box_nb || q >= 2) && qi < Q) {
        issue(qi, st_issue);
        st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
      }
    }
    if (q >= 2) {
      // groups with no node inside the grid store nothing: past the last
      // tile's valid columns they may lie beyond the row pitch (a group with
      // any valid node ends within it: pitch and group starts are multiples
      // of NV)
      if (G.vmask) {
        // plane q-1: in-plane neighbours from the ring (or its stage box:
        // the same layout), z neighbours and the centre from this thread's
        // registers
        const T *rm = box_nb ? sz_prev : ring + rq1 * ring_plane;
        const Vec<T> ym = ldv(rm + cg - RGW), yp = ldv(rm + cg + RGW);
        const T xl = rm[cg - 1], xr = rm[cg + NV];
        Vec<T> a, dgs, mis;  // packed: diag A (and M^-1, pass 1) by node
        if (CM == COEF_PACKED) {
#pragma unroll
          for (int u = 0; u < NV; u++) {
            const uint32_t b = (code_prev >> (8 * u)) & 127u;
            if (UPD) {
              const Pair<T> t = mtab[b];
              dgs.v[u] = t.d;
              mis.v[u] = t.i;
            } else {
              dgs.v[u] = dtab[b];
            }
          }
          // Eq. (3) with the six edge coefficients of the code byte.  A node
          // whose edges all lie on one side of the surface takes a single
          // coefficient times the neighbour sum; so does a whole group of
          // such nodes on the same side (all but the groups at the surface),
          // with no test per node.
          const uint32_t m6 = code_prev & 0x3F3F3F3Fu;
          if (m6 == 0u || m6 == 0x3F3F3F3Fu) {
            const T e = m6 ? ei : eo;
#pragma unroll
            for (int u = 0; u < NV; u++) {
              const T pl = u == 0 ? xl : pc.v[u - 1], pr = u == NV - 1 ? xr : pc.v[u + 1];
              const T s6 = ((pl + pr) + (ym.v[u] + yp.v[u])) + (pm.v[u] + pn.v[u]);
              a.v[u] = dgs.v[u] * pc.v[u] - e * s6;
            }
          } else {
#pragma unroll
            for (int u = 0; u < NV; u++) {
              const T pl = u == 0 ? xl : pc.v[u - 1], pr = u == NV - 1 ? xr : pc.v[u + 1];
              const uint32_t b = (code_prev >> (8 * u)) & 0xffu, e6 = b & 63u;
              if (e6 == 0u || e6 == 63u) {
                const T s6 = ((pl + pr) + (ym.v[u] + yp.v[u])) + (pm.v[u] + pn.v[u]);
                a.v[u] = dgs.v[u] * pc.v[u] - (e6 ? ei : eo) * s6;
              } else {
                T s = ((b & 1u) ? ei : eo) * pl;
                s += ((b & 2u) ? ei : eo) * pr;
                s += ((b & 4u) ? ei : eo) * ym.v[u];
                s += ((b & 8u) ? ei : eo) * yp.v[u];
                s += ((b & 16u) ? ei : eo) * pm.v[u];
                s += ((b & 32u) ? ei : eo) * pn.v[u];
                a.v[u] = dgs.v[u] * pc.v[u] - s;
              }
            }
          }
        } else {
          // explicit storage: the group's coefficients, requested at the top
          // of the iteration by vector loads (pad lanes read the arrays' pads,
          // and their Ap is zeroed below)
          if constexpr (RawEarly<CM>::value)
            cpre = group_expand(craw);
          else if constexpr (!CoefEarly<CM>::value)
            cpre = group_coef<T, CM>(I, (size_t)(z - 1) * plane + ec0, z - 1, (G.vmask >> (NV - 1)) & 1u);
          const GroupCoef<T> &c = cpre;
#pragma unroll
          for (int u = 0; u < NV; u++) {
            const T pl = u == 0 ? xl : pc.v[u - 1], pr = u == NV - 1 ? xr : pc.v[u + 1];
            T s = c.ex[u] * pl;
            s += c.ex[u + 1] * pr;
            s += c.eym[u] * ym.v[u];
            s += c.eyp[u] * yp.v[u];
            s += c.ezm[u] * pm.v[u];
            s += c.ezp[u] * pn.v[u];
            a.v[u] = c.diag[u] * pc.v[u] - s;
          }
        }
        if (!full_group) {  // pad columns keep Ap = 0
#pragma unroll
          for (int u = 0; u < NV; u++)
            if (!((G.vmask >> u) & 1u)) a.v[u] = 0;
        }
        if (UPD) {
          // r = M z - alpha Ap, z = M^-1 r (pads: z = Ap = 0 stay 0); with
          // the packed code, mtab holds {diag A, M^-1} by code byte
          Vec<T> zn;
#pragma unroll
          for (int u = 0; u < NV; u++) {
            T m, mi = m_unit;
            if (CM == COEF_PACKED) {
              m = I.precond ? dgs.v[u] : m_unit;
              mi = mis.v[u];
            } else {
              m = I.precond && ((G.vmask >> u) & 1u) ? cpre.diag[u] : m_unit;  // loaded with the group
            }
            const T r = m * z_prev.v[u] - alpha * a.v[u];
            zn.v[u] = CM == COEF_PACKED ? r * mi : r / m;
            rz += r * zn.v[u];
            rr += r * r;
          }
          stv(zout, zn);
        } else {
#pragma unroll
          for (int u = 0; u < NV; u++) acc += pc.v[u] * a.v[u];
          if (per && !full_group) {  // pad lanes hold wrapped values; p keeps zero pads
            Vec<T> pst = pc;
#pragma unroll
            for (int u = 0; u < NV; u++)
              if (!((G.vmask >> u) & 1u)) pst.v[u] = 0;
            stv(pnew, pst);
          } else {
            stv(pnew, pc);
          }
          if (store_ap) stv(ap, a);
        }
      }
      if (UPD) {
        zout += plane;
      } else {
        pnew += plane;
        ap += plane;
      }
    }
    pm = pc;
    pc = pn;
    sz_prev = sz;
    z_prev = zc;
    code_prev = codes;
    rq = rq + 1 == CG_RING_PLANES ? 0 : rq + 1;
  }
  v0 = UPD ? (double)rz : (double)acc;
  v1 = UPD ? (double)rr : 0.0;
}

}  // namespace pb

#include "fastpath.cuh"

namespace pb {

// RESID phase (FP64, plain loads): fold the deferred update, true residual,
// new inner right-hand side.  Same groups of NV nodes per thread, z pieces of
// I.rtz planes.  GB300 runs FP64 arithmetic at a small fraction of its FP32
// rate, so only x and b - A x are FP64: the last inner step d + alpha p is
// formed in the inner precision (as the next stencil pass would), and the
// sums r.r and r.z over a thread's nodes too.
template <typename T, int CM>
__device__ __forceinline__ void resid_tile(const Inst &I, const TileScal &S, int tile, double *ring,
                                           double &rr64, double &rz) {
  constexpr bool SEP = sizeof(T) == 4;
  const TileG G = tile_g(I, tile, I.rtz);
  const HaloG Hh = halo_g(I);
  const int RGW = I.W + 2 * NV, H = I.H;
  const bool per = I.periodic != 0;
  // periodic: positions outside the grid read their images
  auto wx = [&](int i) { return !per ? i : i < 0 ? i + I.nx : i % I.nx; };
  auto wy = [&](int j) { return !per ? j : j < 0 ? j + I.ny : j % I.ny; };
  auto wz = [&](int k) { return !per ? k : k < 0 ? k + I.nz : k % I.nz; };
  const int hi = wx(G.x0 + Hh.hx), hj = wy(G.y0 + Hh.hy);
  const bool hvalid = Hh.role && hi >= 0 && hi < I.nx && hj >= 0 && hj < I.ny;
  const size_t px = I.px, plane = (size_t)I.px * I.ny;
  const size_t ec0 = (size_t)(G.y0 + G.ty) * px + (G.x0 + G.tx);
  const size_t eh0 = hvalid ? (size_t)hj * px + hi : 0;
  const int cg = (G.ty + 1) * RGW + NV + G.tx, hg = (Hh.hy + 1) * RGW + NV + Hh.hx;
  const double alpha = S.alpha;
  const T alpha_t = (T)S.alpha;
  const double *__restrict__ xin = S.xbuf ? I.x64b : I.x64;
  double *__restrict__ xout = S.xbuf ? I.x64 : I.x64b;
  const T *__restrict__ d = (const T *)I.d;
  const T *__restrict__ p = (const T *)(S.pbuf ? I.p1 : I.p0);
  T *__restrict__ zo = (T *)I.z;
  // Before the first inner solve there is nothing to fold (d and p unset).
  const bool fold = S.outer > 0;
  auto xn = [&](size_t e) -> double {
    const double v = xin[e];
    if (!fold) return v;
    if (SEP) return v + (double)(d[e] + alpha_t * p[e]);
    return v + alpha * (double)p[e];
  };
  auto group = [&](int k, double *out) {  // x_new of this thread's nodes in plane k
    if (per) {  // lanes and rows past the grid hold their images
      const int kw = wz(k), jw = wy(G.y0 + G.ty);
#pragma unroll
      for (int u = 0; u < NV; u++)
        out[u] = G.in_tile ? xn((size_t)kw * plane + (size_t)jw * px + wx(G.x0 + G.tx + u)) : 0.0;
      return;
    }
#pragma unroll
    for (int u = 0; u < NV; u++)
      out[u] = ((G.vmask >> u) & 1u) && k >= 0 && k < I.nz ? xn((size_t)k * plane + ec0 + u) : 0.0;
  };
  double xm[NV], xc[NV], xnx[NV];
  group(G.z0 - 1, xm);
  group(G.z0, xc);
  const int rsz = RGW * (H + 2);
  if (G.in_tile)
    for (int u = 0; u < NV; u++) ring[cg + u] = xc[u];
  if (Hh.role) ring[hg] = hvalid ? xn((size_t)wz(G.z0) * plane + eh0) : 0.0;
  int cur = 0;
  T rr_t = 0, rz_t = 0;
  for (int k = G.z0; k < G.z1; ++k) {
    const int nxt = cur == 2 ? 0 : cur + 1;
    double *rn = ring + (size_t)nxt * rsz;
    group(k + 1, xnx);
    if (G.in_tile)
      for (int u = 0; u < NV; u++) rn[cg + u] = xnx[u];
    if (Hh.role) rn[hg] = hvalid && (per || k + 1 < I.nz) ? xn((size_t)wz(k + 1) * plane + eh0) : 0.0;
    __syncthreads();
    const double *rc = ring + (size_t)cur * rsz;
#pragma unroll
    for (int u = 0; u < NV; u++) {
      if (!((G.vmask >> u) & 1u)) continue;
      const size_t e = (size_t)k * plane + ec0 + u;
      const NodeCoef<double> c = node_coef64<CM>(I, e, k);
      double s = c.exm * rc[cg + u - 1];
      s += c.exp * rc[cg + u + 1];
      s += c.eym * rc[cg + u - RGW];
      s += c.eyp * rc[cg + u + RGW];
      s += c.ezm * xm[u];
      s += c.ezp * xnx[u];
      const double res = I.b[e] - (c.diag * xc[u] - s);
      xout[e] = xc[u];
      const T rt = (T)res, zt = zval<T, CM>(I, e, rt);
      zo[e] = zt;
      rr_t += rt * rt;
      rz_t += rt * zt;
    }
#pragma unroll
    for (int u = 0; u < NV; u++) { xm[u] = xc[u]; xc[u] = xnx[u]; }
    cur = nxt;
  }
  rr64 = (double)rr_t;
  rz = (double)rz_t;
}

// ---------------------------------------------------------------------------
// Deterministic block reductions.

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum two values over the CTA of NTH threads; thread 0 gets the result.
template <int NTH>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int u = 0; u < NTH / 32; u++) { sa += red[2 * u]; sb += red[2 * u + 1]; }
    a = sa; b = sb;
  }
  __syncthreads();
}

// Sum the two columns of n partials with the whole CTA in a fixed order.
template <int NTH>
__device__ __forceinline__ void sum_partials(const double *part, int n, double &s0, double &s1,
                                             double *red) {
  double a = 0, b = 0;
  for (int t = threadIdx.x; t < n; t += NTH) {
    a += __ldcg(part + 2 * t);
    b += __ldcg(part + 2 * t + 1);
  }
  block_sum2<NTH>(a, b, red);
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

// inst: the instance's index in the batch, listed for a residual pass when
// its inner solve ends.
__device__ void fin_update(const Inst &I, Scal *S, double rz, double rr, int inst,
                           int *resid_pending, int *resid_list) {
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
  const double tol = I.mode == MODE_F32_REFINE ? S->itol : I.tol;
  const bool end = S->relres < tol || S->total_iter >= I.max_iter;
  if (S->relres >= tol && end) S->status = 5;  // PB_ERR_NOT_CONVERGED
  if (end) {
    S->phase = PH_RESID;
    resid_list[atomicAdd(resid_pending, 1)] = inst;
  }
}

__device__ void fin_resid(const Inst &I, Scal *S, double rr64, double rz) {
  S->cnt2 = 0;
  S->xbuf ^= 1;  // the new solution now sits in the other x buffer
  const double rel = sqrt(rr64) / S->bnorm;
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
  S->ref_norm = I.mode == MODE_F32_REFINE ? sqrt(rr64) : S->bnorm;
  S->relres = I.mode == MODE_F32_REFINE ? 1.0 : rel;
  // an inner solve reduces its residual by no more than the outer tolerance
  // still needs (with a factor 2 of margin), and by at least inner_tol
  S->itol = fmax(I.inner_tol, 0.5 * I.tol / rel);
  S->phase = PH_START;
}

// ---------------------------------------------------------------------------
// Phase kernels.

// Ring of three planes with halo, sized for the largest tile in FP64 (the
// RESID pass).
constexpr int RING_CELLS = max_ring_cells();
__host__ __device__ constexpr size_t ring_bytes(size_t es, int planes = 3) {
  return ((size_t)planes * RING_CELLS * es + 127) / 128 * 128;
}
// The fast tile passes (fastpath.cuh) for FP32 packed grids without wrap, in
// kernels of their own (FAST = true) that the host launches when no grid of
// the launch needs wrap; 0 keeps every launch on the general cg_tile.
#ifndef PB_FASTPATH
#define PB_FASTPATH 1
#endif
// Stencil pass configurations: TMA pipeline depth in z planes, and resident
// CTAs per SM the register budget targets.  The FP32 packed-code pass (the one
// of served and refined solves) runs three CTAs of 256 threads per SM over a
// server batch (G = 0: many tiles, the largest first, so the SMs stay evenly
// loaded).  On a single grid (G = 1: about two tiles per SM) it runs two CTAs
// per SM at most (its shared memory is padded so that a third does not fit):
// with room for three, the CTA scheduler may stack three tiles on one SM
// while another holds one, and the stacked SM sets the pace.  Four stages
// were slower than three.  The passes that also read coefficient arrays need
// more registers; the FP64 pass is held to one CTA per SM by its shared
// memory.
#ifndef PB_STAGES_F32
#define PB_STAGES_F32 3
#endif
#ifndef PB_MINB_F32
#define PB_MINB_F32 3
#endif
#ifndef PB_STAGES_GRID
#define PB_STAGES_GRID 3
#endif
#ifndef PB_MINB_GRID
#define PB_MINB_GRID 2
#endif
template <typename T, int CM, int G> struct StencilCfg {
  static constexpr bool lean = sizeof(T) == 4 && CM == COEF_PACKED;
  static constexpr int stages = lean ? (G ? PB_STAGES_GRID : PB_STAGES_F32) : sizeof(T) == 4 ? 4 : 3;
  static constexpr int minb = lean ? (G ? PB_MINB_GRID : PB_MINB_F32) : sizeof(T) == 4 ? 2 : 1;
};
// The tile update pass (server batches): a smaller stage (one halo box).
#ifndef PB_STAGES_UPD
#define PB_STAGES_UPD 4
#endif
#ifndef PB_MINB_UPD
#define PB_MINB_UPD 3
#endif
template <typename T, int CM> struct UpdCfg {
  static constexpr bool lean = sizeof(T) == 4 && CM == COEF_PACKED;
  static constexpr int stages = lean ? PB_STAGES_UPD : StencilCfg<T, CM, 0>::stages;
  static constexpr int minb = lean ? PB_MINB_UPD : StencilCfg<T, CM, 0>::minb;
};
// The fast update pass holds no ring: six stages (four planes ahead of the
// one it forms) in the shared memory of three CTAs per SM; four measured 3%
// slower.
#ifndef PB_STAGES_UPD_FAST
#define PB_STAGES_UPD_FAST 6
#endif

// Diagonal of the operator of precision T by code byte (shared memory).
template <typename T>
__device__ __forceinline__ void build_dtab(const Inst &I, T *dtab) {
  if (threadIdx.x < 128) dtab[threadIdx.x] = tab_d<T>(I, dtab_index(threadIdx.x));
}

// The operator's diagonal and the Jacobi preconditioner's inverse by code
// byte: {diag A, M^-1} = {diag, 1/diag}, or {diag, 1} without preconditioner
// (then M = 1).  Shared memory.
template <typename T>
__device__ __forceinline__ void build_mtab(const Inst &I, Pair<T> *mtab) {
  if (threadIdx.x < 128) {
    const int k = dtab_index(threadIdx.x);
    mtab[threadIdx.x].d = tab_d<T>(I, k);
    mtab[threadIdx.x].i = I.precond ? tab_i<T>(I, k) : (T)1;
  }
}

// Dynamic item scheduling: a CTA takes the next item of the list from a
// counter in device memory when it finishes one, so items of unequal cost
// balance across the SMs.  The last CTA to leave puts the counters back to
// zero for the next launch (which reads them only after this grid completed).
__device__ __forceinline__ int take_item(unsigned *next) { return (int)atomicAdd(next, 1u); }
__device__ __forceinline__ void leave_items(unsigned *next, unsigned *done) {
  if (atomicAdd(done, 1u) == gridDim.x - 1) {
    atomicExch(next, 0u);
    atomicExch(done, 0u);
  }
}

// One pass of a CG iteration over the stencil tiles of every instance in the
// batch (PASS 0: direction, p.Ap, then alpha; PASS 1: update, r.z and r.r,
// then beta and the stop test).  Work counters 0/1 (pass 0) or 2/3 (pass 1);
// the tile partials of both passes share st_part (pass 1 starts after pass 0
// has finished with them).
template <typename T, int CM, int PASS, int G, bool FAST>
__device__ __forceinline__ void cg_pass(const Batch &B) {
  constexpr int NS = PASS == 1 ? (FAST ? PB_STAGES_UPD_FAST : UpdCfg<T, CM>::stages)
                               : StencilCfg<T, CM, G>::stages;
  constexpr bool UPD = PASS == 1;
  extern __shared__ __align__(128) uint8_t dyn[];
  __shared__ __align__(8) uint64_t full[NS];
  __shared__ double red[2 * (NT / 32)];
  __shared__ T dtab[128];
  __shared__ Pair<T> mtab[UPD ? 128 : 1];
  __shared__ int s_phase, s_last, s_inst, s_item;
  unsigned *next = &B.work[UPD ? 2 : 0], *done = &B.work[UPD ? 3 : 1];
  // TMA destinations must be 16-byte aligned; align the whole region to 128:
  // the ring of p planes, then the stages.
  uint8_t *base = (uint8_t *)(((uintptr_t)dyn + 127) & ~(uintptr_t)127);
  T *ring = (T *)base;
  uint8_t *stages = FAST && UPD ? base : base + ring_bytes(sizeof(T), CG_RING_PLANES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; s++) mbar_init(&full[s], 1);
    mbar_fence_init();
    s_inst = -1;
  }
  pdl_launch_dependents();
  pdl_wait();
  if (threadIdx.x == 0) s_item = take_item(next);
  __syncthreads();
  StageRing SR{0u, 0u};
  bool abort = false;
  const int n_items = B.n_items[0];
  for (int it = s_item; it < n_items; it = s_item) {
    const Item item = B.st_items[it];
    const Inst &I = B.inst[item.inst];
    Scal *Sp = I.s;
    const bool new_inst = s_inst != item.inst;
    __syncthreads();  // everyone has read s_inst
    if (threadIdx.x == 0) {
      s_phase = *(volatile int *)&Sp->phase;
      s_inst = item.inst;
    }
    if (new_inst) {
      build_dtab<T>(I, dtab);
      if (UPD) build_mtab<T>(I, mtab);
    }
    __syncthreads();
    const int ph = s_phase;
    if (ph == PH_INNER || (!UPD && ph == PH_START)) {
      const TileScal S = tile_scal(Sp);
      double v0 = 0.0, v1 = 0.0;
      if constexpr (FAST) {  // FP32, packed codes, no wrap (checked by the host)
        if constexpr (UPD) {
          fast_update<NS>(I, S, item.tile, stages, (const Pair<float> *)mtab, full, SR, abort, v0, v1);
        } else if (S.phase == PH_START) {
          fast_stencil<NS, true>(I, S, item.tile, stages, (float *)ring, (const float *)dtab, full, SR,
                                 abort, v0);
        } else {
          fast_stencil<NS, false>(I, S, item.tile, stages, (float *)ring, (const float *)dtab, full,
                                  SR, abort, v0);
        }
      } else {
        cg_tile<T, CM, NS, PASS>(I, S, item.tile, stages, ring, dtab, mtab, full, SR, abort, v0, v1);
      }
      if (abort) {
        if (threadIdx.x == 0) atomicOr(B.error, 2);  // a pipeline wait timed out
        break;
      }
      if (threadIdx.x == 0) s_item = take_item(next);
      block_sum2<NT>(v0, v1, red);
      if (threadIdx.x == 0) {
        double *part = B.st_part + 2 * (size_t)(I.st_base + item.tile);
        part[0] = v0;
        part[1] = v1;
        __threadfence();
        const unsigned prev = atomicAdd(UPD ? &Sp->cnt3 : &Sp->cnt2, 1u);
        s_last = prev == (unsigned)(I.n_st - 1);
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        double s0, s1;
        sum_partials<NT>(B.st_part + 2 * (size_t)I.st_base, I.n_st, s0, s1, red);
        if (threadIdx.x == 0) {
          if (UPD) fin_update(I, Sp, s0, s1, item.inst, B.resid_pending, B.resid_list);
          else fin_cg(I, Sp, s0);
        }
      }
    } else if (threadIdx.x == 0) {
      s_item = take_item(next);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) leave_items(next, done);
}

template <typename T, int CM, int G, bool FAST = false>
__global__ void __launch_bounds__(NT, StencilCfg<T, CM, G>::minb) k_stencil(Batch B) {
  cg_pass<T, CM, 0, G, FAST>(B);
}
template <typename T, int CM, bool FAST = false>
__global__ void __launch_bounds__(NT, UpdCfg<T, CM>::minb) k_update_tile(Batch B) {
  cg_pass<T, CM, 1, 0, FAST>(B);
}

// RESID pass of the instances that asked for one (FP64, plain loads).  Its
// items are the listed instances' z pieces, numbered instance after instance
// (a CTA maps an item to its instance with a prefix sum of the piece counts
// in shared memory).  A launch with none pending returns at once.  The last
// CTA to leave clears the pending count: every later request comes from a
// kernel that runs after this one.
constexpr int RESID_LIST_MAX = 1024;  // instances per batch at most
template <typename T, int CM>
__global__ void __launch_bounds__(NT) k_resid(Batch B) {
  extern __shared__ __align__(128) uint8_t dyn[];
  __shared__ double red[2 * (NT / 32)];
  __shared__ int s_cum[RESID_LIST_MAX + 1], s_inst[RESID_LIST_MAX];
  __shared__ int s_last, s_item;
  double *ring = (double *)(((uintptr_t)dyn + 127) & ~(uintptr_t)127);
  pdl_launch_dependents();
  pdl_wait();
  const int n_list = min(*(volatile int *)B.resid_pending, RESID_LIST_MAX);
  if (n_list == 0) return;
  for (int t = threadIdx.x; t < n_list; t += NT) {
    const int j = B.resid_list[t];
    s_inst[t] = j;
    s_cum[t + 1] = B.inst[j].n_rs;
  }
  if (threadIdx.x == 0) s_item = take_item(&B.work[4]);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_cum[0] = 0;
    for (int t = 0; t < n_list; t++) s_cum[t + 1] += s_cum[t];
  }
  __syncthreads();
  const int n_items = s_cum[n_list];
  for (int it = s_item; it < n_items; it = s_item) {
    int lo = 0, hi = n_list - 1;  // the entry t with s_cum[t] <= it < s_cum[t + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (s_cum[mid] <= it) lo = mid;
      else hi = mid - 1;
    }
    const int tile = it - s_cum[lo];
    const Inst &I = B.inst[s_inst[lo]];
    Scal *Sp = I.s;
    const TileScal S = tile_scal(Sp);
    __syncthreads();  // everyone has read s_item
    if (S.phase != PH_RESID) {
      // an instance stopped by the host between launches (a cancelled
      // request) while it waited for this pass: nothing to do
      if (threadIdx.x == 0) s_item = take_item(&B.work[4]);
      __syncthreads();
      continue;
    }
    double v0 = 0, v1 = 0;
    resid_tile<T, CM>(I, S, tile, ring, v0, v1);
    if (threadIdx.x == 0) s_item = take_item(&B.work[4]);
    block_sum2<NT>(v0, v1, red);
    if (threadIdx.x == 0) {
      double *part = B.rs_part + 2 * (size_t)(I.rs_base + tile);
      part[0] = v0;
      part[1] = v1;
      __threadfence();
      const unsigned prev = atomicAdd(&Sp->cnt2, 1u);
      s_last = prev == (unsigned)(I.n_rs - 1);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double s0, s1;
      sum_partials<NT>(B.rs_part + 2 * (size_t)I.rs_base, I.n_rs, s0, s1, red);
      if (threadIdx.x == 0) fin_resid(I, Sp, s0, s1);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && atomicAdd(&B.work[5], 1u) == gridDim.x - 1) {
    atomicExch(&B.work[4], 0u);
    atomicExch(&B.work[5], 0u);
    atomicExch(B.resid_pending, 0);
  }
}

// Update pass over row chunks (the form for a single grid, whose stencil pass
// stored Ap): r = M z - alpha Ap, z = M^-1 r, partial r.z and r.r per chunk.
template <typename T, int CM>
__global__ void __launch_bounds__(NT_UPD) k_update(Batch B) {
  constexpr int V = 16 / sizeof(T);
#ifndef PB_UPD_UNROLL
#define PB_UPD_UNROLL 4
#endif
  constexpr int U = PB_UPD_UNROLL;  // vectors loaded before any is stored (loads in flight per thread)
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type VT;
  __shared__ double red[2 * (NT_UPD / 32)];
  __shared__ Pair<T> mtab[128];
  __shared__ int s_phase, s_last, s_inst, s_item;
  if (threadIdx.x == 0) s_inst = -1;
  pdl_launch_dependents();
  pdl_wait();
  if (threadIdx.x == 0) s_item = take_item(&B.work[2]);
  __syncthreads();
  const int n_items = B.n_items[1];
  for (int it = s_item; it < n_items; it = s_item) {
    const Item item = B.ch_items[it];
    const Inst &I = B.inst[item.inst];
    Scal *Sp = I.s;
    const bool new_inst = s_inst != item.inst;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_phase = *(volatile int *)&Sp->phase;
      s_inst = item.inst;
    }
    if (new_inst) build_mtab<T>(I, mtab);
    __syncthreads();
    if (s_phase == PH_INNER) {
      const T alpha = (T)Sp->alpha;
      const uint32_t vx = (uint32_t)(I.nx + V - 1) / V;  // vectors per row; pads are zero
      const uint32_t magic = I.vx_magic;                  // ceil(2^32 / vx): row = f * magic >> 32
      const int row0 = item.tile * I.rows_per_chunk;
      const uint32_t nrows = (uint32_t)min(I.rows_per_chunk, I.ny * I.nz - row0);
      const uint32_t nvec = nrows * vx;
      T *__restrict__ zp = (T *)I.z + (size_t)row0 * I.px;
      const T *__restrict__ ap = (const T *)I.ap + (size_t)row0 * I.px;
      const uint8_t *__restrict__ code = I.code + (size_t)row0 * I.px;
      const uint32_t px = I.px;
      T rz = 0, rr = 0;
      for (uint32_t f0 = threadIdx.x; f0 < nvec; f0 += U * NT_UPD) {
        uint32_t e[U];
        VT zv[U], av[U];
        uint32_t codes[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
          const uint32_t f = f0 + k * NT_UPD;
          const uint32_t row = vx == 1 ? f : __umulhi(f, magic);
          e[k] = row * px + (f - row * vx) * V;
          if (f < nvec) {
            zv[k] = *(const VT *)(zp + e[k]);
            av[k] = __ldcs((const VT *)(ap + e[k]));
            codes[k] = V == 4 ? *(const uint32_t *)(code + e[k]) : *(const uint16_t *)(code + e[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < U; k++) {
          if (f0 + k * NT_UPD >= nvec) break;
          T *zk = (T *)&zv[k];
          const T *apv = (const T *)&av[k];
#pragma unroll
          for (int u = 0; u < V; u++) {
            // r = M z - alpha A p, then z = M^-1 r (pads: z = Ap = 0 stay 0)
            T m, mi = (T)1;
            if (CM == COEF_PACKED) {
              const Pair<T> t = mtab[(codes[k] >> (8 * u)) & 127u];
              m = I.precond ? t.d : (T)1;
              mi = t.i;
            } else {
              m = I.precond ? ((const T *)I.diag)[(size_t)row0 * px + e[k] + u] : (T)1;
            }
            const T r = m * zk[u] - alpha * apv[u];
            // explicit FP32 storage: times the correctly rounded reciprocal
            // (within an ulp of r / m, without a division per node)
            if constexpr (CM == COEF_PACKED) zk[u] = r * mi;
            else if constexpr (sizeof(T) == 4) zk[u] = r * __frcp_rn(m);
            else zk[u] = r / m;
            rz += r * zk[u];
            rr += r * r;
          }
          *(VT *)(zp + e[k]) = zv[k];
        }
      }
      double a = (double)rz, b = (double)rr;
      if (threadIdx.x == 0) s_item = take_item(&B.work[2]);
      block_sum2<NT_UPD>(a, b, red);
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
        sum_partials<NT_UPD>(B.ch_part + 2 * (size_t)I.ch_base, I.n_ch, s0, s1, red);
        if (threadIdx.x == 0) fin_update(I, Sp, s0, s1, item.inst, B.resid_pending, B.resid_list);
      }
    } else if (threadIdx.x == 0) {
      s_item = take_item(&B.work[2]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) leave_items(&B.work[2], &B.work[3]);
}

// ---------------------------------------------------------------------------
// Start a solve on each listed instance from the state its setup left on the
// device (no host round trip): an atom outside the grid ends the solve with
// PB_ERR_ARG; b = 0 ends it at once (the solution is phi = 0); otherwise
// the FP64 residual pass comes next, from the instance's current x (warm
// start) or from zero.
__global__ void k_start(const Inst *inst, const int *list, int n, int *resid_pending,
                        int *resid_list) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const Inst &I = inst[list[t]];
  Scal *S = I.s;
  const int xbuf = S->xbuf;
  Scal z = {};
  z.xbuf = xbuf;
  z.ref_norm = 1.0;
  z.rz_old = 1.0;
  z.bnorm = sqrt(*I.bnorm2);
  if (*I.err) {
    z.status = 1;  // PB_ERR_ARG
    z.phase = PH_DONE;
  } else if (z.bnorm == 0.0) {
    z.phase = PH_DONE;
    z.outer = -1;  // marks "phi = 0"
  } else {
    z.phase = PH_RESID;
    resid_list[atomicAdd(resid_pending, 1)] = list[t];
  }
  *S = z;
}

cudaError_t launch_start(const Inst *inst, const int *list, int n, int *resid_pending,
                         int *resid_list, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_start<<<(n + 127) / 128, 128, 0, st>>>(inst, list, n, resid_pending, resid_list);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host side

// Shared memory of the single-grid stencil build at least this (80 KB: two
// CTAs per SM at most).  On one 257^3 grid with the row-chunk update (the
// stencil pass also stores Ap) two CTAs per SM ran the pass in 95 us, three
// in 105 us; without the Ap store three would win (87 us), but the tile
// update pass that this needs loses more on one grid than that.
#ifndef PB_GRID_SMEM_MIN
#define PB_GRID_SMEM_MIN (80 * 1024)
#endif
constexpr size_t SMEM_TWO_PER_SM = PB_GRID_SMEM_MIN;  // > 228 KB / 3: two CTAs per SM at most
template <typename T, int CM, int G>
static size_t stencil_smem() {  // ring + stages, + alignment slack
  const size_t b = 128 + ring_bytes(sizeof(T), CG_RING_PLANES) +
                   (size_t)StencilCfg<T, CM, G>::stages * max_stage_bytes(sizeof(T));
  return G && b < SMEM_TWO_PER_SM ? SMEM_TWO_PER_SM : b;
}
template <typename T, int CM>
static size_t update_smem() {  // ring + compact stages of the tile update pass
  return 128 + ring_bytes(sizeof(T), CG_RING_PLANES) +
         (size_t)UpdCfg<T, CM>::stages * max_stage_bytes_upd(sizeof(T));
}
static size_t update_smem_fast() {  // the fast update pass: stages only
  return 128 + (size_t)PB_STAGES_UPD_FAST * max_stage_bytes_upd(sizeof(float));
}
static size_t resid_smem() { return 128 + ring_bytes(sizeof(double)); }


// Launch with the programmatic-stream-serialization attribute, so a kernel
// may be scheduled while its predecessor drains (each waits with
// griddepcontrol.wait before touching the predecessor's results).
template <typename... Args>
static cudaError_t launch_pdl(void (*k)(Args...), int blocks, int threads, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename T, int CM>
static cudaError_t phase_impl(const Batch &B, const KernelGrid &kg, int which, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (which & 4) e = launch_pdl(k_resid<T, CM>, kg.resid_blocks, NT, resid_smem(), st, B);
  constexpr bool can_fast = PB_FASTPATH && StencilCfg<T, CM, 0>::lean;
  const bool fast = can_fast && kg.fast;
  if (e == cudaSuccess && (which & 1)) {
    if constexpr (can_fast) {
      if (kg.single)
        e = fast ? launch_pdl(k_stencil<T, CM, 1, true>, kg.stencil_blocks, NT, stencil_smem<T, CM, 1>(), st, B)
                 : launch_pdl(k_stencil<T, CM, 1>, kg.stencil_blocks, NT, stencil_smem<T, CM, 1>(), st, B);
      else
        e = fast ? launch_pdl(k_stencil<T, CM, 0, true>, kg.stencil_blocks, NT, stencil_smem<T, CM, 0>(), st, B)
                 : launch_pdl(k_stencil<T, CM, 0>, kg.stencil_blocks, NT, stencil_smem<T, CM, 0>(), st, B);
    } else {
      e = launch_pdl(k_stencil<T, CM, 0>, kg.stencil_blocks, NT, stencil_smem<T, CM, 0>(), st, B);
    }
  }
  if (e == cudaSuccess && (which & 2)) {
    if (!kg.tile_update) {
      e = launch_pdl(k_update<T, CM>, kg.update_blocks, NT_UPD, 0, st, B);
    } else {
      if constexpr (can_fast)
        e = fast ? launch_pdl(k_update_tile<T, CM, true>, kg.update_fast_blocks, NT, update_smem_fast(), st, B)
                 : launch_pdl(k_update_tile<T, CM>, kg.update_tile_blocks, NT, update_smem<T, CM>(), st, B);
      else
        e = launch_pdl(k_update_tile<T, CM>, kg.update_tile_blocks, NT, update_smem<T, CM>(), st, B);
    }
  }
  return e != cudaSuccess ? e : cudaGetLastError();
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
  return launch_phase(B, mode, coef, kg, 7, st);
}

template <typename T, int CM>
static void occ(int &s, int &u, int &r, int &ut, int &uf, bool single) {
  const size_t sm = stencil_smem<T, CM, 0>(), rm = resid_smem();
  cudaFuncSetAttribute(k_stencil<T, CM, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_update_tile<T, CM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)update_smem<T, CM>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ut, k_update_tile<T, CM>, NT, update_smem<T, CM>());
  cudaFuncSetAttribute(k_resid<T, CM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rm);
  if constexpr (StencilCfg<T, CM, 0>::lean) {
    const size_t sm1 = stencil_smem<T, CM, 1>();
    cudaFuncSetAttribute(k_stencil<T, CM, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if constexpr (PB_FASTPATH) {  // the fast builds: the same launch bounds and shared memory
      cudaFuncSetAttribute(k_stencil<T, CM, 0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaFuncSetAttribute(k_stencil<T, CM, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
      cudaFuncSetAttribute(k_update_tile<T, CM, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)update_smem_fast());
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&uf, k_update_tile<T, CM, true>, NT, update_smem_fast());
    }
    if (single) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s, k_stencil<T, CM, 1>, NT, sm1);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s, k_stencil<T, CM, 0>, NT, sm);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s, k_stencil<T, CM, 0>, NT, sm);
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&u, k_update<T, CM>, NT_UPD, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_resid<T, CM>, NT, rm);
}

KernelGrid kernel_grid(int mode, int coef, int num_sms, bool single) {
  int s = 1, u = 1, r = 1, ut = 1, uf = 1;
  if (mode == MODE_F64) {
    if (coef == COEF_F64) occ<double, COEF_F64>(s, u, r, ut, uf, single);
    else occ<double, COEF_PACKED>(s, u, r, ut, uf, single);
  } else if (coef == COEF_F32) occ<float, COEF_F32>(s, u, r, ut, uf, single);
  else if (coef == COEF_BF16) occ<float, COEF_BF16>(s, u, r, ut, uf, single);
  else occ<float, COEF_PACKED>(s, u, r, ut, uf, single);
  KernelGrid kg;
  kg.stencil_per_sm = s > 0 ? s : 1;
  kg.update_per_sm = u > 0 ? u : 1;
  kg.stencil_blocks = num_sms * kg.stencil_per_sm;
  kg.update_blocks = num_sms * kg.update_per_sm;
  kg.resid_blocks = num_sms * (r > 0 ? r : 1);
  kg.update_tile_blocks = num_sms * (ut > 0 ? ut : 1);
  kg.update_fast_blocks = num_sms * (uf > 0 ? uf : 1);
  kg.tile_update = 0;
  kg.single = single ? 1 : 0;
  kg.fast = 0;
  return kg;
}

}  // namespace pb

#ifdef PB_FAULT_TEST
// Test builds only: make the next `count` first-plane stage waits give up at
// once (see g_fault_abandon_waits).  Returns 0, or PB_ERR_CUDA.
extern "C" int pb_test_abandon_waits(int count) {
  return cudaMemcpyToSymbol(pb::g_fault_abandon_waits, &count, sizeof(int)) == cudaSuccess ? 0 : 3;
}
#endif
