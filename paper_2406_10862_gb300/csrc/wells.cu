// Wells with their bottom-hole pressures as unknowns: the "w" rows and
// columns of the global Jacobian (Sec. 3.4.1) and the pressure monitoring of
// AllWells (Sec. 3.2.4).
//
//   well_rows_kernel  one warp per well: at every perforation the source
//                     q_e(u_cell, p_bh) with its derivatives; writes
//                     B = dR_cell/dp_bh per perforation, the well equation
//                     (pressure or surface-rate control) R_w, C = dR_w/du_cell
//                     per perforation and D = dR_w/dp_bh;
//   schur_kernel      one warp per well: the Schur complement of the well
//                     unknowns, applied matrix-free next to the block-CSR
//                     SpMV -- (A - B D^-1 C) x, the reduced right-hand side
//                     and the back-substitution for the well unknowns;
//   well_update_kernel  p_bh update and the switch of a rate-controlled well
//                     to pressure control at its limit;
//   cnv_kernel        scaled residual maxima for the Newton convergence test.
//
// Every perforation belongs to one well and every cell to at most one
// perforation, so each kernel writes disjoint rows; sums over a well's
// perforations are per-lane in order, then a fixed butterfly, then lane 0's
// value is broadcast: results are deterministic.
#include <cmath>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace ocp {
namespace {

constexpr int kWellThreads = 128;    // four wells per CTA

__device__ __forceinline__ double warp_sum(double t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return __shfl_sync(0xffffffffu, t, 0);
}

unsigned well_blocks(int nwell) { return (unsigned)((nwell * 32 + kWellThreads - 1) / kWellThreads); }

template <int NB>
__global__ void __launch_bounds__(kWellThreads) well_rows_kernel(
    Params P, const Table* __restrict__ gT, const double* __restrict__ u, const int8_t* __restrict__ flag,
    const double* __restrict__ phi, const Perf* __restrict__ perf, const int32_t* __restrict__ first, int nwell,
    const double* __restrict__ p_bh, const ocp_well_ctrl* __restrict__ ctrl, double* __restrict__ w_res,
    double* __restrict__ w_b, double* __restrict__ w_c, double* __restrict__ w_d, int* status) {
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nwell) return;                       // whole warps leave together
  const long long N = P.N;
  const ocp_well_ctrl cw = ctrl[w];
  const double pb = p_bh[w];
  const int k0 = first[w], k1 = first[w + 1];
  const bool rate = cw.mode == 1;
  const bool bad = (cw.mode != 0 && cw.mode != 1) || (rate && (cw.phase < 0 || cw.phase >= NB || k0 == k1));
  if (bad && lane == 0) atomicOr(status, kStatBadControl);
  const int ph = rate && !bad ? cw.phase : 0;
  double q_sum = 0.0, d_sum = 0.0;
  for (int k = k0 + lane; k < k1; k += 32) {
    Perf pf = perf[k];
    pf.p_bh = pb;
    const long long c = pf.cell;
    CellQ q{};
    CellAux a{};
    cell_quantities<NB, true>(P, *gT, u[c], u[N + c], (NB == 3) ? u[2 * N + c] : 0.0,
                              (NB == 3) ? (flag[c] & 1) : 0, phi[c], q, a);
    double src[3], ds[3][3];
    well_source<NB>(pf, q, a, src, ds);
    // d src / d p_bh of an open perforation: producers WI lambda_a (gas with
    // the dissolved part R_s WI lambda_o), injectors WI lambda_t b
    double dsp[3] = {0.0, 0.0, 0.0};
    if (pf.kind == 0) {
      if (positive(q.p - pb)) {
        dsp[0] = pf.wi * q.lw;
        dsp[1] = pf.wi * q.lo;
        if (NB == 3) dsp[2] = fma(q.rs, dsp[1], pf.wi * q.lg);
      }
    } else if (positive(pb - q.p)) {
      const int e = (pf.phase == 0) ? 0 : NB - 1;
      dsp[e] = pf.wi * a.mob * ((pf.phase == 0) ? a.bw : a.bg);
    }
#pragma unroll
    for (int e = 0; e < NB; ++e) w_b[(long long)k * NB + e] = neg(dsp[e]);
    const double sgn = pf.kind == 0 ? -1.0 : 1.0;
    if (rate && !bad) {
#pragma unroll
      for (int v = 0; v < NB; ++v) w_c[(long long)k * NB + v] = sgn * ds[ph][v];
      q_sum = fma(sgn, src[ph], q_sum);
      d_sum = fma(sgn, dsp[ph], d_sum);
    } else {
#pragma unroll
      for (int v = 0; v < NB; ++v) w_c[(long long)k * NB + v] = 0.0;
    }
  }
  q_sum = warp_sum(q_sum);
  d_sum = warp_sum(d_sum);
  if (lane == 0) {
    if (rate && !bad) {
      w_res[w] = q_sum - cw.target;
      w_d[w] = d_sum;
    } else {
      w_res[w] = pb - cw.target;
      w_d[w] = 1.0;
    }
  }
}

// MODE 0: out += alpha Bs (D^-1 (Cs . in));  MODE 1: out += alpha Bs (D^-1 bw);
// MODE 2: xw = D^-1 (bw - Cs . in).
template <int NB, int MODE>
__global__ void __launch_bounds__(kWellThreads) schur_kernel(const Perf* __restrict__ perf,
                                                             const int32_t* __restrict__ first, int nwell,
                                                             WellSchur ws, double alpha,
                                                             const double* __restrict__ in, double* out,
                                                             const double* __restrict__ bw, double* __restrict__ xw,
                                                             const double* __restrict__ skip) {
  const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= nwell || (skip != nullptr && *skip != 0.0)) return;
  const int k0 = first[w], k1 = first[w + 1];
  double t = 0.0;
  if (MODE != 1) {
    for (int k = k0 + lane; k < k1; k += 32) {
      const long long c = perf[k].cell;
#pragma unroll
      for (int v = 0; v < NB; ++v) t = fma(ws.cs[(long long)k * NB + v], in[c * NB + v], t);
    }
    t = warp_sum(t);
  }
  const double dw = ws.d[w];
  if (MODE == 2) {
    if (lane == 0) xw[w] = (bw[w] - t) / dw;
    return;
  }
  const double tw = alpha * ((MODE == 1 ? bw[w] : t) / dw);
  for (int k = k0 + lane; k < k1; k += 32) {
    const long long c = perf[k].cell;
#pragma unroll
    for (int e = 0; e < NB; ++e) out[c * NB + e] = fma(ws.bs[(long long)k * NB + e], tw, out[c * NB + e]);
  }
}

__global__ void well_update_kernel(int nwell, const Perf* __restrict__ perf, const int32_t* __restrict__ first,
                                   double* __restrict__ p_bh, const double* __restrict__ dp, double scale,
                                   ocp_well_ctrl* __restrict__ ctrl, unsigned long long* dp_max, int* nswitch) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwell) return;
  const double d = scale * dp[w];
  double p = p_bh[w] + d;
  atomicMax(dp_max, (unsigned long long)__double_as_longlong(fabs(d)));
  ocp_well_ctrl cw = ctrl[w];
  if (cw.mode == 1 && first[w] < first[w + 1]) {
    const int kind = perf[first[w]].kind;
    if ((kind == 0 && p < cw.limit) || (kind == 1 && p > cw.limit)) {
      cw.mode = 0;
      cw.target = cw.limit;
      ctrl[w] = cw;
      p = cw.limit;
      atomicAdd(nswitch, 1);
    }
  }
  p_bh[w] = p;
}

// out[e] = max_c |R[c NB + e]| / (phi_c V / dt), the bits of a non-negative
// double ordered as an unsigned integer (atomicMax is exact and
// order-independent; a NaN ranks above every number).
template <int NB>
__global__ void cnv_kernel(long long N, const double* __restrict__ phi, double scale, const double* __restrict__ r,
                           unsigned long long* out) {
  __shared__ unsigned long long sm[NB];
  if (threadIdx.x < NB) sm[threadIdx.x] = 0ull;
  __syncthreads();
  unsigned long long m[NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) m[e] = 0ull;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const double pv = phi[c] * scale;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(r[c * NB + e]) / pv);
      m[e] = b > m[e] ? b : m[e];
    }
  }
#pragma unroll
  for (int e = 0; e < NB; ++e) atomicMax(&sm[e], m[e]);
  __syncthreads();
  if (threadIdx.x < NB) atomicMax(&out[threadIdx.x], sm[threadIdx.x]);
}

__global__ void well_norm_kernel(int nwell, const double* __restrict__ w_res, const ocp_well_ctrl* __restrict__ ctrl,
                                 unsigned long long* out) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwell) return;
  const ocp_well_ctrl cw = ctrl[w];
  const double den = cw.mode == 1 ? fmax(fabs(cw.target), 1.0) : 1.0;
  atomicMax(out, (unsigned long long)__double_as_longlong(fabs(w_res[w]) / den));
}

struct Guard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit Guard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~Guard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

cudaError_t launch_well_schur(const ocp_grid* g, const WellSchur& ws, int mode, double alpha, const double* in,
                              double* out, const double* bw, double* xw, cudaStream_t s, const double* skip) {
  if (g->nwell == 0) return cudaSuccess;
  const unsigned nb = well_blocks(g->nwell);
  const bool three = g->prm.nb == 3;
#define OCP_SCHUR(NBV, M) \
  schur_kernel<NBV, M><<<nb, kWellThreads, 0, s>>>(g->d_perf, g->d_well_first, g->nwell, ws, alpha, in, out, bw, xw, \
                                                    skip)
  if (mode == 0) { if (three) OCP_SCHUR(3, 0); else OCP_SCHUR(2, 0); }
  else if (mode == 1) { if (three) OCP_SCHUR(3, 1); else OCP_SCHUR(2, 1); }
  else { if (three) OCP_SCHUR(3, 2); else OCP_SCHUR(2, 2); }
#undef OCP_SCHUR
  return cudaGetLastError();
}

}  // namespace ocp

extern "C" {

ocp_status ocp_linearize_wells(ocp_grid* g, const double* u_new, const int8_t* flag_new, const double* u_old,
                               const int8_t* flag_old, double dt, const double* p_bh, const ocp_well_ctrl* ctrl,
                               double* residual, double* bsr_val, double* face_flux, double* well_res,
                               double* well_b, double* well_c, double* well_d, void* stream) {
  using namespace ocp;
  if (!g) return report(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!u_new || !u_old || !residual || !bsr_val) return report(OCP_ERR_INVALID_ARG, "u_new, u_old, residual, bsr_val are required");
  if (g->prm.nb == 3 && (!flag_new || !flag_old)) return report(OCP_ERR_INVALID_ARG, "flags are required with three phases");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (g->nwell > 0 && (!p_bh || !ctrl || !well_res || !well_d || (g->nperf > 0 && (!well_b || !well_c))))
    return report(OCP_ERR_INVALID_ARG, "p_bh, ctrl, well_res, well_b, well_c and well_d are required with wells");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_linearize(g, u_new, flag_new, u_old, flag_old, dt, residual, bsr_val, face_flux, s,
                                   g->nwell > 0 ? p_bh : nullptr);
  if (e == cudaSuccess && g->nwell > 0) {
    const unsigned nb = well_blocks(g->nwell);
    if (g->prm.nb == 3)
      well_rows_kernel<3><<<nb, kWellThreads, 0, s>>>(g->prm, g->d_table, u_new, flag_new, g->d_phi, g->d_perf,
                                                      g->d_well_first, g->nwell, p_bh, ctrl, well_res, well_b,
                                                      well_c, well_d, g->d_status);
    else
      well_rows_kernel<2><<<nb, kWellThreads, 0, s>>>(g->prm, g->d_table, u_new, flag_new, g->d_phi, g->d_perf,
                                                      g->d_well_first, g->nwell, p_bh, ctrl, well_res, well_b,
                                                      well_c, well_d, g->d_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_linearize_wells: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_bicgstab_wells(ocp_grid* g, const double* val, const double* well_b, const double* well_c,
                              const double* well_d, const double* b, const double* b_w, double* x, double* x_w,
                              double rtol, int maxit, int transpose, double* work, int* iters, double* relres,
                              void* stream) {
  using namespace ocp;
  if (!g || !val || !b || !x || !work) return report(OCP_ERR_INVALID_ARG, "grid, val, b, x and work are required");
  if (g->nwell == 0) return ocp_bicgstab(g, val, b, x, rtol, maxit, transpose, work, iters, relres, stream);
  if (!well_d || !b_w || !x_w || (g->nperf > 0 && (!well_b || !well_c)))
    return report(OCP_ERR_INVALID_ARG, "well_b, well_c, well_d, b_w and x_w are required with wells");
  if (b == x) return report(OCP_ERR_INVALID_ARG, "b and x must not overlap");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = (long long)g->prm.nb * g->prm.N;
  // transposed system [A^T C^T; B^T D]: the same elimination with B and C exchanged
  WellSchur ws{transpose ? well_c : well_b, transpose ? well_b : well_c, well_d};
  double* bred = work + (solver_work_doubles(g) - n);
  cudaError_t e = cudaMemcpyAsync(bred, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  // b' = b - B D^-1 b_w
  if (e == cudaSuccess) e = launch_well_schur(g, ws, 1, -1.0, nullptr, bred, b_w, nullptr, s);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_bicgstab_wells: %s", cudaGetErrorString(e));
  ocp_status st = bicgstab_run(g, val, &ws, bred, x, rtol, maxit, transpose, work, iters, relres, s);
  // x_w = D^-1 (b_w - C x), also after a solve that stopped short
  e = launch_well_schur(g, ws, 2, 0.0, x, nullptr, b_w, x_w, s);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_bicgstab_wells: %s", cudaGetErrorString(e));
  return st;
}

ocp_status ocp_well_update(ocp_grid* g, double* p_bh, const double* dp, double scale, ocp_well_ctrl* ctrl,
                           double* dp_max, int* nswitch, void* stream) {
  using namespace ocp;
  if (!g || !dp_max || !nswitch) return report(OCP_ERR_INVALID_ARG, "grid, dp_max and nswitch are required");
  if (g->nwell > 0 && (!p_bh || !dp || !ctrl)) return report(OCP_ERR_INVALID_ARG, "p_bh, dp and ctrl are required");
  if (!std::isfinite(scale)) return report(OCP_ERR_INVALID_ARG, "scale must be finite");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dp_max, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(nswitch, 0, sizeof(int), s);
  if (e == cudaSuccess && g->nwell > 0) {
    well_update_kernel<<<(g->nwell + 127) / 128, 128, 0, s>>>(g->nwell, g->d_perf, g->d_well_first, p_bh, dp, scale,
                                                              ctrl, reinterpret_cast<unsigned long long*>(dp_max),
                                                              nswitch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_well_update: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_residual_norms(ocp_grid* g, const double* residual, double dt, const double* well_res,
                              const ocp_well_ctrl* ctrl, double* norms, void* stream) {
  using namespace ocp;
  if (!g || !residual || !norms) return report(OCP_ERR_INVALID_ARG, "grid, residual and norms are required");
  if (g->nwell > 0 && (!well_res || !ctrl)) return report(OCP_ERR_INVALID_ARG, "well_res and ctrl are required with wells");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* out = reinterpret_cast<unsigned long long*>(norms);
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 4, s);
  if (e == cudaSuccess) {
    const double scale = g->prm.vol_rb / dt;
    const unsigned blocks = (unsigned)(2 * g->sms);
    if (g->prm.nb == 3) cnv_kernel<3><<<blocks, 256, 0, s>>>(g->prm.N, g->d_phi, scale, residual, out);
    else cnv_kernel<2><<<blocks, 256, 0, s>>>(g->prm.N, g->d_phi, scale, residual, out);
    if (g->nwell > 0) well_norm_kernel<<<(g->nwell + 127) / 128, 128, 0, s>>>(g->nwell, well_res, ctrl, out + 3);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_residual_norms: %s", cudaGetErrorString(e));
  return OCP_OK;
}

}  // extern "C"
