// coef.cuh -- decoding of the operator coefficients of Eq. (3) (h^2-scaled)
// for one node, shared by the phase kernels and the helper kernels.
#pragma once
#include <cuda_bf16.h>

#include "pb_internal.cuh"

namespace pb {

template <typename T> __device__ __forceinline__ T tab_d(const Inst &I, int k);
template <> __device__ __forceinline__ float tab_d<float>(const Inst &I, int k) { return I.dtab32[k]; }
template <> __device__ __forceinline__ double tab_d<double>(const Inst &I, int k) { return I.dtab[k]; }
template <typename T> __device__ __forceinline__ T tab_i(const Inst &I, int k);
template <> __device__ __forceinline__ float tab_i<float>(const Inst &I, int k) { return I.idtab32[k]; }
template <> __device__ __forceinline__ double tab_i<double>(const Inst &I, int k) { return I.idtab[k]; }
template <typename T> __device__ __forceinline__ T e_in(const Inst &I);
template <> __device__ __forceinline__ float e_in<float>(const Inst &I) { return I.ein32; }
template <> __device__ __forceinline__ double e_in<double>(const Inst &I) { return I.ein; }
template <typename T> __device__ __forceinline__ T e_out(const Inst &I);
template <> __device__ __forceinline__ float e_out<float>(const Inst &I) { return I.eout32; }
template <> __device__ __forceinline__ double e_out<double>(const Inst &I) { return I.eout; }

template <int CM> struct Store;  // storage type of explicit edge coefficients
template <> struct Store<COEF_PACKED> { typedef float type; };
template <> struct Store<COEF_F32> { typedef float type; };
template <> struct Store<COEF_BF16> { typedef __nv_bfloat16 type; };
template <> struct Store<COEF_F64> { typedef double type; };

__device__ __forceinline__ float cvt(float v) { return v; }
__device__ __forceinline__ double cvt(double v) { return v; }
__device__ __forceinline__ float cvt(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> struct NodeCoef { T exm, exp, eym, eyp, ezm, ezp, diag; };

// Coefficients of node e = (k*ny + j)*px + i for the operator of precision T.
template <typename T, int CM>
__device__ __forceinline__ NodeCoef<T> node_coef(const Inst &I, size_t e, int k) {
  NodeCoef<T> c;
  if (CM == COEF_PACKED) {
    const uint32_t b = I.code[e];
    const T ei = e_in<T>(I), eo = e_out<T>(I);
    c.exm = (b & 1u) ? ei : eo; c.exp = (b & 2u) ? ei : eo;
    c.eym = (b & 4u) ? ei : eo; c.eyp = (b & 8u) ? ei : eo;
    c.ezm = (b & 16u) ? ei : eo; c.ezp = (b & 32u) ? ei : eo;
    c.diag = tab_d<T>(I, dtab_index(b));
  } else {
    typedef typename Store<CM>::type C;
    const C *ex = (const C *)I.ex, *ey = (const C *)I.ey, *ez = (const C *)I.ez;
    const size_t px = I.px, ey0 = e + (size_t)k * px, plane = px * I.ny;
    c.exm = (T)cvt(ex[e]); c.exp = (T)cvt(ex[e + 1]);
    c.eym = (T)cvt(ey[ey0]); c.eyp = (T)cvt(ey[ey0 + px]);
    c.ezm = (T)cvt(ez[e]); c.ezp = (T)cvt(ez[e + plane]);
    c.diag = ((const T *)I.diag)[e];
  }
  return c;
}

// Coefficients of a group of NV nodes e0 .. e0+NV-1 (e0 a multiple of NV, one
// row) from explicit storage, by vector loads.  The x-edge after the last
// node is read only when that node is in the grid (last_ok): otherwise it
// may lie past the row, and past the array on its last row.
template <typename T> struct GroupCoef { T ex[NV + 1], eym[NV], eyp[NV], ezm[NV], ezp[NV], diag[NV]; };
template <typename C, typename T>
__device__ __forceinline__ void load_group(const C *p, T *out) {
  if constexpr (sizeof(C) == 2) {  // four bf16 in 8 bytes
    const uint2 v = *(const uint2 *)p;
    const __nv_bfloat162 a = *(const __nv_bfloat162 *)&v.x, b = *(const __nv_bfloat162 *)&v.y;
    out[0] = (T)__low2float(a); out[1] = (T)__high2float(a);
    out[2] = (T)__low2float(b); out[3] = (T)__high2float(b);
  } else if constexpr (sizeof(C) == 4) {
    const float4 v = *(const float4 *)p;
    out[0] = (T)v.x; out[1] = (T)v.y; out[2] = (T)v.z; out[3] = (T)v.w;
  } else {
    const double2 v0 = ((const double2 *)p)[0], v1 = ((const double2 *)p)[1];
    out[0] = (T)v0.x; out[1] = (T)v0.y; out[2] = (T)v1.x; out[3] = (T)v1.y;
  }
}
template <typename T, int CM>
__device__ __forceinline__ GroupCoef<T> group_coef(const Inst &I, size_t e0, int k, bool last_ok) {
  typedef typename Store<CM>::type C;
  static_assert(NV == 4, "group loads are four-wide");
  const C *ex = (const C *)I.ex, *ey = (const C *)I.ey, *ez = (const C *)I.ez;
  const size_t px = I.px, ey0 = e0 + (size_t)k * px, plane = px * I.ny;
  GroupCoef<T> g;
  load_group<C, T>(ex + e0, g.ex);
  g.ex[NV] = last_ok ? (T)cvt(ex[e0 + NV]) : (T)0;
  load_group<C, T>(ey + ey0, g.eym);
  load_group<C, T>(ey + ey0 + px, g.eyp);
  load_group<C, T>(ez + e0, g.ezm);
  load_group<C, T>(ez + e0 + plane, g.ezp);
  load_group<T, T>((const T *)I.diag + e0, g.diag);
  return g;
}

// The same group's coefficients as the words loaded (BF16 storage): the
// loads are issued here and their results first used by group_expand, so a
// request made early does not wait for its data where it is made.
struct GroupRaw16 {
  uint2 ex, eym, eyp, ezm, ezp;
  unsigned short exl;
  float4 diag;
};
__device__ __forceinline__ GroupRaw16 group_raw16(const Inst &I, size_t e0, int k, bool last_ok) {
  const __nv_bfloat16 *ex = (const __nv_bfloat16 *)I.ex, *ey = (const __nv_bfloat16 *)I.ey;
  const __nv_bfloat16 *ez = (const __nv_bfloat16 *)I.ez;
  const size_t px = I.px, ey0 = e0 + (size_t)k * px, plane = px * I.ny;
  GroupRaw16 r;
  r.ex = *(const uint2 *)(ex + e0);
  r.exl = last_ok ? *(const unsigned short *)(ex + e0 + NV) : (unsigned short)0;  // bf16 +0
  r.eym = *(const uint2 *)(ey + ey0);
  r.eyp = *(const uint2 *)(ey + ey0 + px);
  r.ezm = *(const uint2 *)(ez + e0);
  r.ezp = *(const uint2 *)(ez + e0 + plane);
  r.diag = *(const float4 *)((const float *)I.diag + e0);
  return r;
}
__device__ __forceinline__ void bf16x4(uint2 v, float *out) {
  const __nv_bfloat162 a = *(const __nv_bfloat162 *)&v.x, b = *(const __nv_bfloat162 *)&v.y;
  out[0] = __low2float(a); out[1] = __high2float(a);
  out[2] = __low2float(b); out[3] = __high2float(b);
}
__device__ __forceinline__ GroupCoef<float> group_expand(const GroupRaw16 &r) {
  static_assert(NV == 4, "group loads are four-wide");
  GroupCoef<float> g;
  bf16x4(r.ex, g.ex);
  g.ex[NV] = __uint_as_float((uint32_t)r.exl << 16);  // bf16 -> fp32 is exact: the high half
  bf16x4(r.eym, g.eym);
  bf16x4(r.eyp, g.eyp);
  bf16x4(r.ezm, g.ezm);
  bf16x4(r.ezp, g.ezp);
  g.diag[0] = r.diag.x; g.diag[1] = r.diag.y; g.diag[2] = r.diag.z; g.diag[3] = r.diag.w;
  return g;
}

// z = M^-1 r at node e (Jacobi), or z = r without preconditioner.
template <typename T, int CM>
__device__ __forceinline__ T zval(const Inst &I, size_t e, T r) {
  if (!I.precond) return r;
  if (CM == COEF_PACKED) return r * tab_i<T>(I, dtab_index(I.code[e]));
  return r / ((const T *)I.diag)[e];
}

// Exact FP64 operator coefficients (from the codes, or the FP64 arrays).
template <int CM>
__device__ __forceinline__ NodeCoef<double> node_coef64(const Inst &I, size_t e, int k) {
  if (CM == COEF_F64) return node_coef<double, COEF_F64>(I, e, k);
  if (CM != COEF_PACKED && I.rx) {  // FP64 edges behind rounded inner copies
    NodeCoef<double> c;
    const size_t px = I.px, ey0 = e + (size_t)k * px, plane = px * I.ny;
    c.exm = I.rx[e]; c.exp = I.rx[e + 1];
    c.eym = I.ry[ey0]; c.eyp = I.ry[ey0 + px];
    c.ezm = I.rz[e]; c.ezp = I.rz[e + plane];
    c.diag = I.rdiag[e];
    return c;
  }
  return node_coef<double, COEF_PACKED>(I, e, k);
}

}  // namespace pb
