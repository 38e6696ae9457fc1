// Sustained FP64 FMA rate of a device (see include/ocp_probe.h).
#include "../../include/ocp_probe.h"
#include "kernels.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 4096;

// Two operand patterns, because the DFMA rate of GB300 depends on them:
// chains through the multiplicand with kernel-constant operands
// (v = v*a + b) run at about 505 G/s, accumulation chains with
// loop-invariant register multiplicands (v = x*y + v) at about 597 G/s.
// The probe reports the faster one: the highest FP64 FMA rate the device
// sustains.
template <int PATTERN>
__global__ void __launch_bounds__(256) dfma_probe_kernel(double* out, double a, double b) {
  double v[kChains], x[kChains], y[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) {
    v[q] = threadIdx.x * 1e-3 + q;
    x[q] = 1e-3 * (1 + ((threadIdx.x + q) & 7));
    y[q] = 1e-3 * (2 + ((threadIdx.x * 3 + q) & 7));
  }
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int q = 0; q < kChains; ++q) v[q] = PATTERN == 0 ? fma(v[q], a, b) : fma(x[q], y[q], v[q]);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += v[q];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" ocp_status ocp_probe_fp64(int device, int reps, double* dfma_per_s) {
  if (!dfma_per_s || reps < 1) return ocp::report(OCP_ERR_INVALID_ARG, "ocp_probe_fp64: bad arguments");
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8, threads = 256;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * blocks * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  for (int pattern = 0; pattern < 2; ++pattern)
    for (int r = 0; e == cudaSuccess && r < reps + 1; ++r) {
      cudaEventRecord(e0);
      if (pattern == 0) dfma_probe_kernel<0><<<blocks, threads>>>(out, 0.999999, 1e-7);
      else dfma_probe_kernel<1><<<blocks, threads>>>(out, 0.999999, 1e-7);
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const double rate = (double)blocks * threads * kIters * kChains / (ms * 1e-3);
      if (r > 0 && rate > best) best = rate;   // the first launch of each pattern is a warm-up
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_probe_fp64: %s", cudaGetErrorString(e));
  *dfma_per_s = best;
  return OCP_OK;
}
