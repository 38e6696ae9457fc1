// ocp_linearize_noalloc: the linearisation with its scratch in a fixed,
// library-owned device array instead of the grid's own scratch buffer.
//
// Who needs it: code that must not allocate device memory at the moment it
// linearises -- a caller whose memory is owned by a host application or an
// embedding framework with its own allocator, or a real-time loop under a
// fixed memory budget that may not grow.  Such a caller still passes its
// inputs and outputs; this entry point itself calls no cudaMalloc, cudaFree
// or any allocating routine.
//
// The array holds kStaticScratchDoubles doubles (32 MiB).  Every GPU that
// loads the library holds it until the process exits.  The scratch needs 100
// doubles per cell, so grids of at most kStaticScratchDoubles / 100 = 41 943
// cells are accepted; larger grids are rejected with OCP_ERR_INVALID_ARG.
//
// In host code the array's name is only a host-side stand-in, not a device
// address: the device address is looked up with cudaGetSymbolAddress, once
// per device, with that device current, on the first call made on it.  That
// first call per device should therefore come before any stream capture.
//
// Every call shares the one array and leaves its contents behind.  Nothing
// in it has to start at zero: each entry a call reads was written earlier in
// the same call.  Calls that overlap on the GPU (on different streams, or on
// different grids at the same time) race on the array and must not be made.
#include <cmath>
#include <mutex>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace {

constexpr long long kStaticScratchDoubles = 4LL * 1024 * 1024;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" ocp_status ocp_linearize_noalloc(ocp_grid* g, const double* u_new, const int8_t* flag_new,
                                            const double* u_old, const int8_t* flag_old, double dt,
                                            double* residual, double* bsr_val, double* face_flux,
                                            void* stream) {
  if (!g) return ocp::report(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!u_new || !u_old || !residual || !bsr_val)
    return ocp::report(OCP_ERR_INVALID_ARG, "u_new, u_old, residual, bsr_val are required");
  if (g->prm.nb == 3 && (!flag_new || !flag_old))
    return ocp::report(OCP_ERR_INVALID_ARG, "flags are required with three phases");
  if (!(std::isfinite(dt) && dt > 0.0)) return ocp::report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  const long long need = ocp::linearize_scratch_doubles(g->prm.N);
  if (need > kStaticScratchDoubles)
    return ocp::report(OCP_ERR_INVALID_ARG,
                       "ocp_linearize_noalloc: grid has %lld cells but the static scratch holds at most %lld cells",
                       (long long)g->prm.N, kStaticScratchDoubles / (need / g->prm.N));
  if (g->device < 0 || g->device >= kMaxDevices)
    return ocp::report(OCP_ERR_UNSUPPORTED, "device ordinal %d out of the supported range", g->device);

  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != g->device) e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));

  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[g->device]) {
      // set-up, once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e == cudaSuccess && p) g_scratch_addr[g->device] = static_cast<double*>(p);
    }
    scratch = g_scratch_addr[g->device];
  }
  if (e == cudaSuccess && scratch)
    e = ocp::launch_linearize_scratch(g, scratch, u_new, flag_new, u_old, flag_old, dt, residual, bsr_val,
                                      face_flux, (cudaStream_t)stream);
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  if (e != cudaSuccess)
    return ocp::report(OCP_ERR_CUDA, "ocp_linearize_noalloc: %s", cudaGetErrorString(e));
  if (!scratch) return ocp::report(OCP_ERR_CUDA, "ocp_linearize_noalloc: no device address for the scratch");
  return OCP_OK;
}
