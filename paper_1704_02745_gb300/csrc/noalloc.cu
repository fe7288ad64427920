// noalloc.cu -- pb_energy_noalloc: the electrostatic energy of a potential
// computed without any device allocation.
//
// Some callers cannot allocate device memory at all: a molecular-dynamics
// engine whose memory manager owns every device byte, or a time-critical loop
// where a cudaMalloc / cudaFree (which synchronise the device) is not
// allowed.  This entry point takes only the caller's device arrays; the
// per-CTA partial sums of the reduction live in a fixed array of this
// library's own device memory, reserved when the library is loaded.
#include <mutex>

#include "pb.h"
#include "pb_host.h"
#include "pb_internal.cuh"
#include "solve.cuh"

using namespace pb;

namespace {

// Partial sums of the energy reduction: one per CTA of 256 atoms.  Every GPU
// that loads this library holds this array until the process exits.
constexpr int NOALLOC_PARTIALS = 4096;
constexpr int NOALLOC_MAX_ATOMS = NOALLOC_PARTIALS * 256;
static __device__ __align__(256) double g_energy_partials[NOALLOC_PARTIALS];

// Device address of g_energy_partials on each device, taken once per device
// with that device current (the host-side name of the array is only a
// stand-in, not a device address).  The cache is keyed by device index and
// kept for the life of the process, so it assumes one CUDA context per device
// (the runtime's primary context): after cudaDeviceReset, or under another
// context made current on the device, the cached address would be stale.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_scratch[MAX_DEVICES] = {};

}  // namespace

extern "C" pb_status pb_energy_noalloc(int n_atoms, const double *xyzq, int nx, int ny, int nz,
                                       double h, const double *origin, const double *phi,
                                       double *energy, void *cuda_stream) {
  if (n_atoms < 0 || n_atoms > NOALLOC_MAX_ATOMS)
    return pb_fail(PB_ERR_ARG, "pb_energy_noalloc: n_atoms must be in [0, " +
                                   std::to_string(NOALLOC_MAX_ATOMS) + "]");
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0) || !origin || !energy ||
      (n_atoms > 0 && (!xyzq || !phi)))
    return pb_fail(PB_ERR_ARG, "pb_energy_noalloc: bad grid or NULL pointer");
  if (((uintptr_t)xyzq) % 32 != 0)
    return pb_fail(PB_ERR_ARG, "pb_energy_noalloc: xyzq must be 32-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pb_fail(PB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return pb_fail(PB_ERR_ARG, "pb_energy_noalloc: device index too large");
  double *scratch;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {  // set-up on the first call on this device
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_energy_partials);
      if (e != cudaSuccess)
        return pb_fail(PB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch[dev] = (double *)p;
    }
    scratch = g_scratch[dev];
  }
  // Every partial the final sum reads is written by this call first, so the
  // array needs no clearing; calls that overlap on the GPU share it and race.
  e = launch_energy((const dbl4 *)xyzq, n_atoms, nx, ny, nz, nx, 0, h, origin[0], origin[1], origin[2], phi,
                    scratch, energy, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return pb_fail(PB_ERR_CUDA, std::string("energy kernels: ") + cudaGetErrorString(e));
  return PB_OK;
}
