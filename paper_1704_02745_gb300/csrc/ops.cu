// ops.cu -- helper kernels of libpb: dense <-> padded copies, the operator
// applied to a dense vector (Eq. 3-4), and the electrostatic energy.
#include "coef.cuh"
#include "pb_internal.cuh"
#include "solve.cuh"

namespace pb {

static int blocks_for(size_t n, int nt) {
  size_t b = (n + nt - 1) / nt;
  return (int)(b < 152 * 32 ? (b ? b : 1) : 152 * 32);
}

// Node indices split in 32-bit arithmetic: a grid has at most 2e9 nodes
// (checked when it is created), and 32-bit division costs a fraction of
// 64-bit division per node.
__device__ __forceinline__ size_t padded_of(size_t t, int nx, int px) {
  const uint32_t tt = (uint32_t)t, row = tt / (uint32_t)nx;
  return (size_t)row * px + (tt - row * (uint32_t)nx);
}
__global__ void k_pack(const double *dense, double *padded, int nx, int ny, int nz, int px) {
  const size_t n = (size_t)nx * ny * nz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    padded[padded_of(t, nx, px)] = dense[t];
}
__global__ void k_unpack(const double *padded, double *dense, int nx, int ny, int nz, int px) {
  const size_t n = (size_t)nx * ny * nz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dense[t] = padded[padded_of(t, nx, px)];
}

cudaError_t launch_pack(const double *dense, double *padded, int nx, int ny, int nz, int px,
                        cudaStream_t st) {
  k_pack<<<blocks_for((size_t)nx * ny * nz, 256), 256, 0, st>>>(dense, padded, nx, ny, nz, px);
  return cudaGetLastError();
}
cudaError_t launch_unpack(const double *padded, double *dense, int nx, int ny, int nz, int px,
                          cudaStream_t st) {
  k_unpack<<<blocks_for((size_t)nx * ny * nz, 256), 256, 0, st>>>(padded, dense, nx, ny, nz, px);
  return cudaGetLastError();
}

// (A u)_c = diag_c u_c - sum_nb eps_edge u_nb, ghosts zero; dense u and Au.
template <typename T, int CM>
__global__ void k_apply(const Inst *dI, const T *u, T *au) {
  const Inst &I = *dI;
  const int nx = I.nx, ny = I.ny, nz = I.nz;
  const size_t n = (size_t)nx * ny * nz;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const uint32_t tt = (uint32_t)t, row32 = tt / (uint32_t)nx, k32 = row32 / (uint32_t)ny;
    const int i = (int)(tt - row32 * (uint32_t)nx);
    const int j = (int)(row32 - k32 * (uint32_t)ny), k = (int)k32;
    const size_t row = row32;
    const size_t e = row * I.px + i;
    const NodeCoef<T> c = node_coef<T, CM>(I, e, k);
    T s = 0;
    if (I.periodic) {  // neighbours modulo n
      const size_t rowb = t - i, pl = (size_t)nx * ny, plb = t - (size_t)k * pl;
      s += c.exm * u[rowb + (i > 0 ? i - 1 : nx - 1)];
      s += c.exp * u[rowb + (i < nx - 1 ? i + 1 : 0)];
      s += c.eym * u[t - (size_t)j * nx + (size_t)(j > 0 ? j - 1 : ny - 1) * nx];
      s += c.eyp * u[t - (size_t)j * nx + (size_t)(j < ny - 1 ? j + 1 : 0) * nx];
      s += c.ezm * u[plb + (size_t)(k > 0 ? k - 1 : nz - 1) * pl];
      s += c.ezp * u[plb + (size_t)(k < nz - 1 ? k + 1 : 0) * pl];
    } else {
      if (i > 0) s += c.exm * u[t - 1];
      if (i < nx - 1) s += c.exp * u[t + 1];
      if (j > 0) s += c.eym * u[t - nx];
      if (j < ny - 1) s += c.eyp * u[t + nx];
      if (k > 0) s += c.ezm * u[t - (size_t)nx * ny];
      if (k < nz - 1) s += c.ezp * u[t + (size_t)nx * ny];
    }
    au[t] = c.diag * u[t] - s;
  }
}

cudaError_t launch_apply(const Inst &I, const Inst *dI, const void *u, void *au, int dtype,
                         cudaStream_t st) {
  const int blocks = blocks_for((size_t)I.nx * I.ny * I.nz, 256);
  if (dtype == 0) {  // FP64: exact coefficients
    if (I.coef == COEF_F64)
      k_apply<double, COEF_F64><<<blocks, 256, 0, st>>>(dI, (const double *)u, (double *)au);
    else
      k_apply<double, COEF_PACKED><<<blocks, 256, 0, st>>>(dI, (const double *)u, (double *)au);
  } else {
    if (I.coef == COEF_F32)
      k_apply<float, COEF_F32><<<blocks, 256, 0, st>>>(dI, (const float *)u, (float *)au);
    else if (I.coef == COEF_BF16)
      k_apply<float, COEF_BF16><<<blocks, 256, 0, st>>>(dI, (const float *)u, (float *)au);
    else
      k_apply<float, COEF_PACKED><<<blocks, 256, 0, st>>>(dI, (const float *)u, (float *)au);
  }
  return cudaGetLastError();
}

// Energy: 1/2 * 332.0637 * sum_a q_a * (trilinear interpolation of phi at x_a)
// with the weights of the charge spreading, so it equals 1/2 * 332.0637 *
// sum_nodes q_node phi_node up to rounding order.  Per-CTA partials, then one
// CTA sums them in order (deterministic).
constexpr int EN_NT = 256;
// px: row pitch of phi in elements (nx for a dense array).  An atom whose
// trilinear cell leaves the grid reads nothing and makes the energy NaN; on a
// periodic grid the cell's corners wrap modulo n.
__global__ void k_energy_partial(const dbl4 *xyzq, int n_atoms, int nx, int ny, int nz, int px,
                                 int periodic, double h, double ox, double oy, double oz,
                                 const double *phi, double *part) {
  __shared__ double red[EN_NT];
  double acc = 0.0;
  const int a = blockIdx.x * EN_NT + threadIdx.x;
  if (a < n_atoms) {
    const dbl4 A = xyzq[a];
    const double f[3] = {__ddiv_rn(__dsub_rn(A.x, ox), h), __ddiv_rn(__dsub_rn(A.y, oy), h),
                         __ddiv_rn(__dsub_rn(A.z, oz), h)};
    double w[3][2];
    long c0[3];
    const long n[3] = {nx, ny, nz};
    bool inside = true;
    for (int d = 0; d < 3; d++) {
      const double fl = floor(f[d]);
      c0[d] = (long)fl;
      w[d][1] = __dsub_rn(f[d], fl);
      w[d][0] = __dsub_rn(1.0, w[d][1]);
      // the cell's upper corner may be the last node only when its weight is 0
      if (periodic) inside = inside && isfinite(fl);
      else inside = inside && fl >= 0.0 && (c0[d] + 1 < n[d] || (c0[d] + 1 == n[d] && w[d][1] == 0.0));
    }
    if (!inside) {
      acc = __longlong_as_double(0x7ff8000000000000LL);  // NaN
    } else {
      for (int dk = 0; dk < 2; dk++)
        for (int dj = 0; dj < 2; dj++)
          for (int di = 0; di < 2; di++) {
            const double c = __dmul_rn(__dmul_rn(__dmul_rn(A.w, w[0][di]), w[1][dj]), w[2][dk]);
            long ci = c0[0] + di, cj = c0[1] + dj, ck = c0[2] + dk;
            if (periodic) {
              ci = ((ci % nx) + nx) % nx;
              cj = ((cj % ny) + ny) % ny;
              ck = ((ck % nz) + nz) % nz;
            } else if (ci >= nx || cj >= ny || ck >= nz) {
              continue;  // weight 0
            }
            const size_t t = ((size_t)ck * ny + cj) * px + ci;
            acc += c * phi[t];
          }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = EN_NT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_energy_final(const double *part, int n, double *out) {
  __shared__ double red[EN_NT];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += EN_NT) s += part[t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = EN_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * 332.0637 * red[0];
}

cudaError_t launch_energy(const dbl4 *xyzq, int n_atoms, int nx, int ny, int nz, int px,
                          int periodic, double h, double ox, double oy, double oz,
                          const double *phi, double *scratch, double *out, cudaStream_t st) {
  const int blocks = n_atoms > 0 ? (n_atoms + EN_NT - 1) / EN_NT : 0;
  if (blocks > 0)
    k_energy_partial<<<blocks, EN_NT, 0, st>>>(xyzq, n_atoms, nx, ny, nz, px, periodic, h, ox, oy,
                                               oz, phi, scratch);
  k_energy_final<<<1, EN_NT, 0, st>>>(scratch, blocks, out);
  return cudaGetLastError();
}

}  // namespace pb
