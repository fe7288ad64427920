// probe.cu -- pb_measure_alu: the device's measured FP64 and FP32 FMA rates.
//
// The paper has no counterpart (its solver ran in FP32 only).  The rate is
// the roofline of the kernels whose FP64 arithmetic, not their bytes, sets
// their time on this GPU: the FP64 true residual of the refinement and the
// plain FP64 solves.  The probe is a pure arithmetic loop: every thread runs
// eight independent FMA chains, so the FMA pipes, not the dependency latency,
// bound it; its only memory traffic is one store per thread.
#include <string>

#include "pb.h"
#include "pb_host.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_probe(T *out, int iters, T a, T c) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) x[i] = (T)(threadIdx.x % 32) * (T)1e-3 + (T)i;
  for (int k = 0; k < iters; k++) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) x[i] = fma(x[i], a, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

// FMAs per second of k_fma_probe<T> (best of three timed launches after one
// untimed launch).
template <typename T>
pb_status rate(pb_ctx *ctx, T *out, int blocks, int iters, double *fma_per_s) {
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 0;
  pb_status st = PB_OK;
  for (int rep = 0; rep < 4 && st == PB_OK; rep++) {
    cudaEventRecord(e0, s);
    // a = 1 - 2^-20, c = 2^-20: every chain stays near 1, never denormal or infinite
    k_fma_probe<T><<<blocks, PROBE_THREADS, 0, s>>>(out, iters, (T)(1.0 - 0x1p-20), (T)0x1p-20);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      st = pb_fail(PB_ERR_CUDA, std::string("pb_measure_alu: ") + cudaGetErrorString(e));
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0 || ms < best)) best = ms;
  }
  ctx->stats->launches += 4;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == PB_OK)
    *fma_per_s = (double)blocks * PROBE_THREADS * PROBE_CHAINS * (double)iters / (best * 1e-3);
  return st;
}

}  // namespace

extern "C" pb_status pb_measure_alu(pb_ctx *ctx, pb_alu_rates *out) {
  if (!ctx || !out) return pb_fail(PB_ERR_ARG, "pb_measure_alu: NULL argument");
  memset(out, 0, sizeof(*out));
  CK(cudaSetDevice(ctx->device));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<double>, PROBE_THREADS, 0));
  const int blocks = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
  double *buf = nullptr;
  pb_status st = pb_dalloc((void **)&buf, (size_t)blocks * PROBE_THREADS * sizeof(double));
  if (st) return st;
  // ~1e10 FP64 FMAs (tens of ms at GB300's FP64 rate); 32x as many in FP32
  st = rate<double>(ctx, buf, blocks, 4096, &out->fp64_fma_per_s);
  if (!st) st = rate<float>(ctx, (float *)buf, blocks, 4096 * 32, &out->fp32_fma_per_s);
  cudaFree(buf);
  out->sms = ctx->num_sms;
  int khz = 0;
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device) == cudaSuccess)
    out->sm_max_mhz = khz / 1000.0;
  else
    cudaGetLastError();
  return st;
}
