// Sustained FP64 FMA rate of a device (see include/ocp_probe.h).
#include "../../include/ocp_probe.h"
#include "kernels.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) dfma_probe_kernel(double* out, double a, double b) {
  double v[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) v[q] = threadIdx.x * 1e-3 + q;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int q = 0; q < kChains; ++q) v[q] = fma(v[q], a, b);
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
  for (int r = 0; e == cudaSuccess && r < reps + 1; ++r) {
    cudaEventRecord(e0);
    dfma_probe_kernel<<<blocks, threads>>>(out, 0.999999, 1e-7);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double rate = (double)blocks * threads * kIters * kChains / (ms * 1e-3);
    if (r > 0 && rate > best) best = rate;   // the first launch is a warm-up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_probe_fp64: %s", cudaGetErrorString(e));
  *dfma_per_s = best;
  return OCP_OK;
}
