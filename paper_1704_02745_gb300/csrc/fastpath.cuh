// fastpath.cuh -- the two tile passes of a CG iteration (Sec. 2.2 preconditioned
// CG, Sec. 2.4 Jacobi, operator of Eq. 3) specialised to the case served
// batches run: FP32 inner solve, packed one-byte coefficients, free-space
// boundary (no wrap).  They compute what cg_tile computes for that case, with
// the same operations in the same order; only the bookkeeping is leaner (the general kernel's address arithmetic
// and per-plane case tests were most of its instructions):
//   - every shared-memory access uses a 32-bit shared address computed from a
//     per-tile base plus a per-thread offset fixed for the whole tile;
//   - every descriptor field and scalar the plane loop needs is read once
//     per tile into a register;
//   - the plane loop has no wrap, halo-patch or coefficient-storage cases;
//   - a group of four nodes with one code byte takes one table lookup.
// Included by solve.cu after its TMA / mbarrier primitives and tile geometry;
// the phase kernels built with FAST = true run these for every item.
#pragma once

#define PB_PRAGMA(x) _Pragma(#x)
#define PB_UNROLL(n) PB_PRAGMA(unroll n)

namespace pb {

__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ float lds1(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ldsu(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts4(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void sts1(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ float at(const float4 &v, int u) {
  return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w;
}

// Ap of a group of four nodes (Eq. 3, h^2-scaled) from the packed code bytes
// of the group (one byte per node), their diagonals d, the group's p on the
// planes below / at / above (pm, pc, pn), the rows below and above (ym, yp)
// and the x neighbours left of the first and right of the last node.
__device__ __forceinline__ float4 fast_ap(uint32_t codes, const float4 &d, const float4 &pm,
                                          const float4 &pc, const float4 &pn, const float4 &ym,
                                          const float4 &yp, float xl, float xr, float ei, float eo) {
  const float pl[4] = {xl, pc.x, pc.y, pc.z}, pr[4] = {pc.y, pc.z, pc.w, xr};
  const float c[4] = {pc.x, pc.y, pc.z, pc.w}, dd[4] = {d.x, d.y, d.z, d.w};
  const float m_[4] = {pm.x, pm.y, pm.z, pm.w}, n_[4] = {pn.x, pn.y, pn.z, pn.w};
  const float ya[4] = {ym.x, ym.y, ym.z, ym.w}, yb[4] = {yp.x, yp.y, yp.z, yp.w};
  float a[4];
  const uint32_t m6 = codes & 0x3F3F3F3Fu;
  if (m6 == 0u || m6 == 0x3F3F3F3Fu) {
    // every edge of the group on one side of the surface: one coefficient
    const float e = m6 ? ei : eo;
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const float s6 = ((pl[u] + pr[u]) + (ya[u] + yb[u])) + (m_[u] + n_[u]);
      a[u] = dd[u] * c[u] - e * s6;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t b = (codes >> (8 * u)) & 0xffu, e6 = b & 63u;
      if (e6 == 0u || e6 == 63u) {
        const float s6 = ((pl[u] + pr[u]) + (ya[u] + yb[u])) + (m_[u] + n_[u]);
        a[u] = dd[u] * c[u] - (e6 ? ei : eo) * s6;
      } else {
        float s = ((b & 1u) ? ei : eo) * pl[u];
        s += ((b & 2u) ? ei : eo) * pr[u];
        s += ((b & 4u) ? ei : eo) * ya[u];
        s += ((b & 8u) ? ei : eo) * yb[u];
        s += ((b & 16u) ? ei : eo) * m_[u];
        s += ((b & 32u) ? ei : eo) * n_[u];
        a[u] = dd[u] * c[u] - s;
      }
    }
  }
  return f4(a[0], a[1], a[2], a[3]);
}

// Thread 0's copies of one plane into one stage: the stencil pass's z box,
// p_old box, code box and x centre box, or (m1 == nullptr) the update pass's
// p box, code box and z centre box.  (Out of line it measured slower: the
// call spilled registers of the stencil pass.)
__device__ __forceinline__ void fast_issue(uint8_t *sb, uint64_t *bar, uint32_t bytes,
                                         const CUtensorMap *m0, const CUtensorMap *m1,
                                         const CUtensorMap *mc, const CUtensorMap *mx,
                                         uint32_t off1, uint32_t off_c, uint32_t off_x, int x0,
                                         int y0, int cx0, int z) {
  mbar_expect_tx(bar, bytes);
  tma_load_3d(sb, m0, bar, x0 - NV, y0 - 1, z);
  if (m1) tma_load_3d(sb + off1, m1, bar, x0 - NV, y0 - 1, z);
  tma_load_3d(sb + off_c, mc, bar, cx0, y0 - 1, z);
  tma_load_3d(sb + off_x, mx, bar, x0, y0, z);
}

// Drain after a stage wait gave up at plane q: thread 0 waits (bounded) for
// the copies of plane q and of every later plane issued, so none lands after
// the CTA leaves.  `last` is the last plane issued.
template <int NS>
__device__ __forceinline__ void fast_drain(uint64_t *full, StageRing &SR, uint32_t st, int q,
                                           int last) {
  if (threadIdx.x == 0) {
    uint32_t s2 = st, ph = SR.phase ^ (1u << st);
    for (int u = q; u <= last; ++u) {
      mbar_wait(&full[s2], (ph >> s2) & 1u);
      ph ^= 1u << s2;
      s2 = s2 + 1 == NS ? 0 : s2 + 1;
    }
    SR.phase = ph;
    SR.st = s2;
  }
}

// Stencil pass (PASS 0 of cg_tile) for one tile: p = z + beta p_old with the
// halo into a ring of three planes, Ap, this thread's p.Ap in v0; stores p,
// the deferred x update (d += alpha p_old) and, on a single grid, Ap.
template <int NS, bool FIRST>
__device__ __forceinline__ void fast_stencil(const Inst &I, const TileScal &S, int tile,
                                             uint8_t *stages, float *ring, const float *dtab,
                                             uint64_t *full, StageRing &SR, bool &abort,
                                             double &v0) {
  const TileG G = tile_g(I, tile, I.tz);
  const HaloG Hh = halo_g(I);
  const int W = I.W, H = I.H, RW = W + 2 * NV, CW = I.cw;
  const uint32_t stage_bytes = I.stage_bytes, off_p = I.off_p, off_c = I.off_c, off_x = I.off_x;
  const uint32_t tma_bytes = I.tma_bytes;
  const int cx0 = ((G.x0 - 1) >> 4) << 4;
  const int Q = (G.z1 - G.z0) + 2;
  const float beta = FIRST ? 0.f : (float)S.beta, alpha = (float)S.alpha;
  const float ei = I.ein32, eo = I.eout32;
  const CUtensorMap *m_z = &I.tm_z, *m_pold = S.pbuf ? &I.tm_p1 : &I.tm_p0, *m_code = &I.tm_code,
                    *m_x = &I.tm_x0;
  const size_t plane = (size_t)I.px * I.ny;
  const size_t ec0 = (size_t)(G.y0 + G.ty) * I.px + (G.x0 + G.tx);
  float *pnew = (float *)(S.pbuf ? I.p0 : I.p1) + (size_t)G.z0 * plane + ec0;
  float *xo = (float *)I.d + (size_t)G.z0 * plane + ec0;
  float *apo = (float *)I.ap;
  const bool store_ap = apo != nullptr;
  if (store_ap) apo += (size_t)G.z0 * plane + ec0;
  const int x0 = G.x0, y0 = G.y0, zb = G.z0 - 1;
  auto issue = [&](int q, uint32_t st) {
    fast_issue(stages + st * stage_bytes, &full[st], tma_bytes, m_z, m_pold, m_code, m_x, off_p, off_c,
               off_x, x0, y0, cx0, zb + q);
  };
  const int n0 = min(NS, Q);
  uint32_t st_issue = SR.st;
  if (threadIdx.x == 0)
    for (int q = 0; q < n0; ++q) {
      issue(q, st_issue);
      st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
    }
  else
    for (int q = 0; q < n0; ++q) st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;

  const uint32_t sbase = smem_u32(stages), rbase = smem_u32(ring);
  const uint32_t ring_plane_b = (uint32_t)(RW * (H + 2)) * 4u;
  const bool in_tile = G.in_tile, has = G.vmask != 0u;
  const uint32_t lane_mask = G.vmask;
  const uint32_t o_r = (uint32_t)((G.ty + 1) * RW + NV + G.tx) * 4u;  // centre: boxes and ring
  const uint32_t o_c = off_c + (uint32_t)((G.ty + 1) * CW + (G.x0 + G.tx - cx0));
  const uint32_t o_x = off_x + (uint32_t)(G.ty * W + G.tx) * 4u;  // x centre box
  const uint32_t o_h = (uint32_t)((Hh.hy + 1) * RW + NV + Hh.hx) * 4u;  // this thread's halo cell
  const bool role = Hh.role;
  const uint32_t row_b = (uint32_t)RW * 4u;

  float4 pm = f4(0, 0, 0, 0), pc = pm, pn = pm;
  uint32_t cprev = 0, ccur = 0;
  float acc = 0.f;
  uint32_t rq = 0;  // ring slot of plane q
#ifdef PB_FAST_UNROLL
  PB_UNROLL(PB_FAST_UNROLL)
#endif
  for (int q = 0; q < Q; ++q) {
    const uint32_t st = SR.st;
#ifdef PB_FAULT_TEST
    const bool ok = (q == 0 && threadIdx.x == 0 && fault_abandon_wait())
                        ? false : mbar_wait(&full[st], (SR.phase >> st) & 1u);
#else
    const bool ok = mbar_wait(&full[st], (SR.phase >> st) & 1u);
#endif
    SR.phase ^= 1u << st;
    SR.st = st + 1 == NS ? 0 : st + 1;
    const uint32_t sb = sbase + st * stage_bytes;
    const uint32_t rg = rbase + rq * ring_plane_b;
    // z and p_old are zero outside the grid (TMA fill, zero pads), so is p
    if (ok && in_tile) {
      const float4 zv = lds4(sb + o_r);
      const float4 po = lds4(sb + off_p + o_r);
      ccur = ldsu(sb + o_c);
      pn = FIRST ? zv
                 : f4(zv.x + beta * po.x, zv.y + beta * po.y, zv.z + beta * po.z, zv.w + beta * po.w);
      sts4(rg + o_r, pn);
      // deferred update of the previous iteration: d += alpha p_old (the first
      // inner iteration starts d from zero)
      if (has && q >= 1 && q < Q - 1) {
        float4 xn = f4(0, 0, 0, 0);
        if (!FIRST) {
          const float4 xv = lds4(sb + o_x);
          xn = f4(xv.x + alpha * po.x, xv.y + alpha * po.y, xv.z + alpha * po.z, xv.w + alpha * po.w);
        }
        *(float4 *)xo = xn;
      }
    }
    if (q >= 1 && q < Q - 1) xo += plane;
    if (ok && role) {
      const float hz = lds1(sb + o_h);
      sts1(rg + o_h, FIRST ? hz : hz + beta * lds1(sb + off_p + o_h));
    }
    if (__syncthreads_or(!ok)) {
      fast_drain<NS>(full, SR, st, q, min(Q - 1, q + NS - 1));
      abort = true;
      v0 = 0.0;
      return;
    }
    if (threadIdx.x == 0 && q + NS < Q) issue(q + NS, st_issue);
    st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
    if (q >= 2) {
      // plane q-1: in-plane neighbours from the ring, z neighbours and the
      // centre from this thread's registers
      if (has) {
        const uint32_t rm = rbase + (rq == 0 ? 2u : rq - 1u) * ring_plane_b + o_r;
        const float4 ym = lds4(rm - row_b), yp = lds4(rm + row_b);
        const float xl = lds1(rm - 4u), xr = lds1(rm + 16u);
        float4 d;
        if (cprev == (cprev & 0xffu) * 0x01010101u) {  // one code byte for the group
          const float t = dtab[cprev & 127u];
          d = f4(t, t, t, t);
        } else {
          d = f4(dtab[cprev & 127u], dtab[(cprev >> 8) & 127u], dtab[(cprev >> 16) & 127u],
                 dtab[(cprev >> 24) & 127u]);
        }
        float4 a = fast_ap(cprev, d, pm, pc, pn, ym, yp, xl, xr, ei, eo);
        if (lane_mask != 0xFu) {  // pad columns keep Ap = 0
          if (!(lane_mask & 1u)) a.x = 0.f;
          if (!(lane_mask & 2u)) a.y = 0.f;
          if (!(lane_mask & 4u)) a.z = 0.f;
          if (!(lane_mask & 8u)) a.w = 0.f;
        }
        acc += pc.x * a.x;
        acc += pc.y * a.y;
        acc += pc.z * a.z;
        acc += pc.w * a.w;
        *(float4 *)pnew = pc;
        if (store_ap) *(float4 *)apo = a;
      }
      pnew += plane;
      if (store_ap) apo += plane;
    }
    pm = pc;
    pc = pn;
    cprev = ccur;
    rq = rq == 2u ? 0u : rq + 1u;
  }
  v0 = (double)acc;
}

// Update pass (PASS 1 of cg_tile, the server batch's form): Ap formed again
// from the stored p, r = M z - alpha Ap, z = M^-1 r, this thread's r.z and
// r.r in v0, v1.  The in-plane neighbours of plane q-1 are read from that
// plane's stage (the stored p with its halo, zero outside the grid), so the
// stage of plane q-2 is refilled at iteration q.  (A form without the CTA
// barrier per plane -- each warp releasing stages through a shared count,
// the last one refilling -- measured 4% slower: the pass is bound by its
// instruction issue, not by warps waiting for each other.)
template <int NS>
__device__ __forceinline__ void fast_update(const Inst &I, const TileScal &S, int tile,
                                            uint8_t *stages, const Pair<float> *mtab,
                                            uint64_t *full, StageRing &SR, bool &abort,
                                            double &v0, double &v1) {
  const TileG G = tile_g(I, tile, I.tz);
  const int W = I.W, RW = W + 2 * NV, CW = I.cw;
  const uint32_t stage_bytes = I.stage_bytes_upd, off_c = I.off_c_upd, off_x = I.off_x_upd;
  const uint32_t tma_bytes = I.tma_bytes_upd;
  const int cx0 = ((G.x0 - 1) >> 4) << 4;
  const int Q = (G.z1 - G.z0) + 2;
  const float alpha = (float)S.alpha;
  const float ei = I.ein32, eo = I.eout32;
  const bool prec = I.precond != 0;
  const CUtensorMap *m_p = S.pbuf ? &I.tm_p1 : &I.tm_p0, *m_code = &I.tm_code, *m_zc = &I.tm_zc;
  const size_t plane = (size_t)I.px * I.ny;
  float *zout = (float *)I.z + (size_t)G.z0 * plane + (size_t)(G.y0 + G.ty) * I.px + (G.x0 + G.tx);
  const int x0 = G.x0, y0 = G.y0, zb = G.z0 - 1;
  auto issue = [&](int q, uint32_t st) {
    fast_issue(stages + st * stage_bytes, &full[st], tma_bytes, m_p, nullptr, m_code, m_zc, 0u, off_c,
               off_x, x0, y0, cx0, zb + q);
  };
  const int n0 = min(NS, Q);
  uint32_t st_issue = SR.st;
  if (threadIdx.x == 0)
    for (int q = 0; q < n0; ++q) {
      issue(q, st_issue);
      st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
    }
  else
    for (int q = 0; q < n0; ++q) st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;

  const uint32_t sbase = smem_u32(stages);
  const bool in_tile = G.in_tile, has = G.vmask != 0u;
  const uint32_t lane_mask = G.vmask;
  const uint32_t o_p = (uint32_t)((G.ty + 1) * RW + NV + G.tx) * 4u;
  const uint32_t o_c = off_c + (uint32_t)((G.ty + 1) * CW + (G.x0 + G.tx - cx0));
  const uint32_t o_z = off_x + (uint32_t)(G.ty * W + G.tx) * 4u;
  const uint32_t row_b = (uint32_t)RW * 4u;

  float4 pm = f4(0, 0, 0, 0), pc = pm, pn = pm;
  uint32_t sbp = sbase;
  float rz = 0.f, rr = 0.f;
#ifdef PB_FAST_UNROLL
  PB_UNROLL(PB_FAST_UNROLL)
#endif
  for (int q = 0; q < Q; ++q) {
    const uint32_t st = SR.st;
#ifdef PB_FAULT_TEST
    const bool ok = (q == 0 && threadIdx.x == 0 && fault_abandon_wait())
                        ? false : mbar_wait(&full[st], (SR.phase >> st) & 1u);
#else
    const bool ok = mbar_wait(&full[st], (SR.phase >> st) & 1u);
#endif
    SR.phase ^= 1u << st;
    SR.st = st + 1 == NS ? 0 : st + 1;
    const uint32_t sb = sbase + st * stage_bytes;
    if (ok && in_tile) pn = lds4(sb + o_p);
    if (__syncthreads_or(!ok)) {
      fast_drain<NS>(full, SR, st, q, min(Q - 1, max(NS - 1, q + NS - 3)));
      abort = true;
      v0 = v1 = 0.0;
      return;
    }
    if (q >= 2) {
      if (threadIdx.x == 0 && q - 2 + NS < Q) issue(q - 2 + NS, st_issue);
      st_issue = st_issue + 1 == NS ? 0 : st_issue + 1;
      if (has) {
        // plane q-1 from its stage (resident until iteration q+1 refills it):
        // in-plane neighbours of the stored p, z and the code bytes
        const uint32_t rm = sbp + o_p;
        const float4 ym = lds4(rm - row_b), yp = lds4(rm + row_b);
        const float xl = lds1(rm - 4u), xr = lds1(rm + 16u);
        const uint32_t cprev = ldsu(sbp + o_c);
        const bool one_code = cprev == (cprev & 0xffu) * 0x01010101u;
        float4 d;
        if (one_code) {  // one code byte for the group: one lookup
          const float t = mtab[cprev & 127u].d;
          d = f4(t, t, t, t);
        } else {
          d = f4(mtab[cprev & 127u].d, mtab[(cprev >> 8) & 127u].d, mtab[(cprev >> 16) & 127u].d,
                 mtab[(cprev >> 24) & 127u].d);
        }
        float4 a = fast_ap(cprev, d, pm, pc, pn, ym, yp, xl, xr, ei, eo);
        if (lane_mask != 0xFu) {
          if (!(lane_mask & 1u)) a.x = 0.f;
          if (!(lane_mask & 2u)) a.y = 0.f;
          if (!(lane_mask & 4u)) a.z = 0.f;
          if (!(lane_mask & 8u)) a.w = 0.f;
        }
        float4 mi;
        if (one_code) {
          const float t = mtab[cprev & 127u].i;
          mi = f4(t, t, t, t);
        } else {
          mi = f4(mtab[cprev & 127u].i, mtab[(cprev >> 8) & 127u].i, mtab[(cprev >> 16) & 127u].i,
                  mtab[(cprev >> 24) & 127u].i);
        }
        const float4 zprev = lds4(sbp + o_z);
        // r = M z - alpha Ap, z = M^-1 r (pads: z = Ap = 0 stay 0)
        const float4 m = prec ? d : f4(1.f, 1.f, 1.f, 1.f);
        const float r0 = m.x * zprev.x - alpha * a.x, r1 = m.y * zprev.y - alpha * a.y;
        const float r2 = m.z * zprev.z - alpha * a.z, r3 = m.w * zprev.w - alpha * a.w;
        const float4 zn = f4(r0 * mi.x, r1 * mi.y, r2 * mi.z, r3 * mi.w);
        rz += r0 * zn.x;
        rr += r0 * r0;
        rz += r1 * zn.y;
        rr += r1 * r1;
        rz += r2 * zn.z;
        rr += r2 * r2;
        rz += r3 * zn.w;
        rr += r3 * r3;
        *(float4 *)zout = zn;
      }
      zout += plane;
    }
    pm = pc;
    pc = pn;
    sbp = sb;
  }
  v0 = (double)rz;
  v1 = (double)rr;
}

}  // namespace pb
