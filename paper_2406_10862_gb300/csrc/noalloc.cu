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
// The array holds kStaticScratchDoubles doubles (32 MiB).  The scratch needs
// 100 doubles per cell, so grids of at most kStaticScratchDoubles / 100 =
// 41 943 cells are accepted; larger grids are rejected with
// OCP_ERR_INVALID_ARG.
//
// When the array is reserved: with CUDA's lazy module loading (the default)
// the array and the kernels are only loaded onto a device when they are first
// used there, and loading them allocates device memory.  So ocp_grid_create,
// which allocates anyway, does that first use: on the grid's device it looks
// up the array's device address with cudaGetSymbolAddress (which loads the
// array, reserving its 32 MiB on that device until the process exits) and
// loads the linearisation kernels, and it keeps the address in the grid.  In
// host code the array's name is only a host-side stand-in, never a device
// address; device code could name it directly, host code uses the address.
// A device reset (cudaDeviceReset) invalidates every grid on that device, and
// with it the address.
//
// Every call shares the one array and leaves its contents behind.  Nothing
// in it has to start at zero: each entry a call reads was written earlier in
// the same call.  Calls that overlap on the GPU (on different streams, or on
// different grids at the same time) race on the array and must not be made.
#include <cmath>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace {

constexpr long long kStaticScratchDoubles = 4LL * 1024 * 1024;   // 32 MiB

static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

}  // namespace

namespace ocp {

// Device address of the array on the current device (loads it there).
cudaError_t static_scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  *out = (e == cudaSuccess) ? static_cast<double*>(p) : nullptr;
  if (e == cudaSuccess && !p) e = cudaErrorInvalidSymbol;
  return e;
}

}  // namespace ocp

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
  if (!g->d_static_scratch)
    return ocp::report(OCP_ERR_CUDA, "ocp_linearize_noalloc: no device address for the static scratch");

  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != g->device) e = cudaSetDevice(g->device);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  e = ocp::launch_linearize_scratch(g, g->d_static_scratch, u_new, flag_new, u_old, flag_old, dt, residual,
                                    bsr_val, face_flux, (cudaStream_t)stream);
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  if (e != cudaSuccess)
    return ocp::report(OCP_ERR_CUDA, "ocp_linearize_noalloc: %s", cudaGetErrorString(e));
  return OCP_OK;
}
