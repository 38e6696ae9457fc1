// The equations in pressure and component amounts with the volume balance
// (Sec. 2.1, eq. 4): unknowns (P, N_w, N_o[, N_g]) per cell, amounts in
// surface volumes per bulk volume.
//
// The fluxes and well terms depend on the amounts only through the explicit
// black-oil phase split, which maps (P, N) to the natural variables
// (p, S_w[, X]) of the other path.  So the component rows of the (P, N)
// Jacobian are the natural-variable blocks times, per column cell, the
// derivative M = d(p, S_w, X)/d(P, N) of the split; the accumulation is
// (N - N_old) V / dt.  Eliminating N_w with the cell's volume-balance row
// r_v = phi(P) - V_f (Schur complement on the diagonal block) turns M into
// the 3x3 (2x2) matrix T = M E and a vector t = M e_w c_r per cell.
//
//   pn_split_kernel   per cell: phase split, natural state and flag, M, the
//                     volume-balance row, T, t and the elimination
//                     coefficients c = a / a_w, c_r = r_v / a_w;
//   (the tile kernels of the natural path, accumulation left out)
//   pn_reduce_kernel  per block row: B3 = B T_col, R3 = R + acc - sum B t_col
//                     - [water row] (V/dt) c_r, the accumulation's reduced
//                     derivative on the diagonal, and optionally the full
//                     system (component rows B M_col, volume row a);
//   pn_update_kernel  the Newton update of (P, N) with N_w recovered from
//                     the volume row.
#include <cmath>

#include "kernels.cuh"
#include "ocp_internal.cuh"
#include "pn_split.cuh"

namespace ocp {
namespace {

// per-cell data of the (P, N) path, variable-major blocks of N doubles
template <int NB>
struct PnLayout {
  static constexpr int kNat = 0;                       // natural state, NB
  static constexpr int kT = NB;                        // T, NB*NB (row-major)
  static constexpr int kt = NB + NB * NB;              // t, NB
  static constexpr int kM = 2 * NB + NB * NB;          // M, NB*(NB+1)
  static constexpr int kA = kM + NB * (NB + 1);        // volume row a, NB+1, then r_v
  static constexpr int kCount = kA + NB + 2;
};

template <int NB>
__global__ void pn_split_kernel(Params P, const Table* __restrict__ gT, const double* __restrict__ pn,
                                const double* __restrict__ phi_ref, double* __restrict__ d,
                                int8_t* __restrict__ flag, double* __restrict__ elim, int* status) {
  using Lo = PnLayout<NB>;
  constexpr int L = NB + 1;
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const Table& T = *gT;
  const double p = pn[c], nw = pn[N + c], no = pn[2 * N + c], ng = (NB == 3) ? pn[3 * N + c] : 0.0;
  if (!(finite(p) && finite(nw) && finite(no) && finite(ng))) atomicOr(status, kStatNonFinite);
  Split<NB> sp;
  phase_split<NB>(P, T, p, nw, no, ng, sp);
  const double Vf = sp.Vf;
  const double* dVf = sp.dVf;
  const double sw = sp.sw, x = sp.x;
  const int f = sp.flag;
  const auto& M = sp.M;
  // volume balance r_v = phi(p) - V_f and its row a
  const double phi = phi_ref[c] * fma(P.cr, p - P.p_ref, 1.0);
  const double rv = phi - Vf;
  double a[L];
  a[0] = phi_ref[c] * P.cr - dVf[0];
  for (int k = 1; k < L; ++k) a[k] = -dVf[k];
  // eliminate N_w: dN_w = -(c_P dP + c_o dN_o [+ c_g dN_g]) + c_r
  const double iaw = 1.0 / a[1];
  double cc[L];                         // c_P, (unused), c_o[, c_g]
  for (int k = 0; k < L; ++k) cc[k] = a[k] * iaw;
  const double cr = rv * iaw;
  // reduced columns: P, N_o[, N_g] = full columns 0, 2[, 3]
  double* __restrict__ dp = d;
  for (int i = 0; i < NB; ++i) {
    for (int j = 0; j < NB; ++j) {
      const int k = (j == 0) ? 0 : j + 1;
      dp[(Lo::kT + i * NB + j) * N + c] = fma(-M[i][1], cc[k], M[i][k]);
    }
    dp[(Lo::kt + i) * N + c] = M[i][1] * cr;
    for (int k = 0; k < L; ++k) dp[(Lo::kM + i * L + k) * N + c] = M[i][k];
  }
  for (int k = 0; k < L; ++k) dp[(Lo::kA + k) * N + c] = a[k];
  dp[(Lo::kA + L) * N + c] = rv;
  dp[(Lo::kNat + 0) * N + c] = p;
  dp[(Lo::kNat + 1) * N + c] = sw;
  if (NB == 3) dp[(Lo::kNat + 2) * N + c] = x;
  if (NB == 3) flag[c] = (int8_t)f;
  elim[c] = cc[0];
  elim[N + c] = cc[2];
  if (NB == 3) elim[2 * N + c] = cc[3];
  elim[NB * N + c] = cr;
}

// The row's blocks are walked on the grid's 7-point pattern (neighbour
// types -z, -y, -x, self, +x, +y, +z, the order of the stored columns), with
// the row start in closed form: no dependent index loads, so every block's
// gathers can be issued early, and the diagonal's extra terms are placed at
// compile time.
template <int NB>
__global__ void __launch_bounds__(128) pn_reduce_kernel(Params P, const double* __restrict__ d,
                                                        const double* __restrict__ elim,
                                                        const double* __restrict__ pn_new,
                                                        const double* __restrict__ pn_old, double scale,
                                                        double* __restrict__ res, double* __restrict__ val,
                                                        double* __restrict__ res4, double* __restrict__ val4) {
  using Lo = PnLayout<NB>;
  constexpr int L = NB + 1;
  const long long N = P.N;
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= N) return;
  int ri, rj, rk;
  cell_ijk(P, r, ri, rj, rk);
  const bool has[7] = {rk > 0, rj > 0, ri > 0, true, ri + 1 < P.nx, rj + 1 < P.ny, rk + 1 < P.nz};
  const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
  const long long s0 = row_start_ijk(P, r, ri, rj, rk);
  double rr[NB];
  for (int e = 0; e < NB; ++e) rr[e] = fma(pn_new[(e + 1) * N + r] - pn_old[(e + 1) * N + r], scale, res[r * NB + e]);
  if (res4) {
    for (int e = 0; e < NB; ++e) res4[r * L + e] = rr[e];
    res4[r * L + NB] = d[(Lo::kA + L) * N + r];
  }
  int slot = 0;
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    if (!has[t]) continue;
    const long long s = s0 + slot;
    ++slot;
    const long long c = r + off[t];
    double B[NB][NB];
    for (int e = 0; e < NB; ++e)
      for (int v = 0; v < NB; ++v) B[e][v] = val[(long long)s * NB * NB + e * NB + v];
    double Tc[NB][NB], tc[NB];
    for (int i = 0; i < NB; ++i) {
      tc[i] = d[(Lo::kt + i) * N + c];
      for (int j = 0; j < NB; ++j) Tc[i][j] = d[(Lo::kT + i * NB + j) * N + c];
    }
    if (val4) {
      double Mc[NB][L];
      for (int i = 0; i < NB; ++i)
        for (int k = 0; k < L; ++k) Mc[i][k] = d[(Lo::kM + i * L + k) * N + c];
      double* b4 = val4 + (long long)s * L * L;
      for (int e = 0; e < NB; ++e)
        for (int k = 0; k < L; ++k) {
          double acc = 0.0;
          for (int i = 0; i < NB; ++i) acc = fma(B[e][i], Mc[i][k], acc);
          b4[e * L + k] = (t == 3 && k == e + 1) ? acc + scale : acc;
        }
      for (int k = 0; k < L; ++k) b4[NB * L + k] = (t == 3) ? d[(Lo::kA + k) * N + r] : 0.0;
    }
    for (int e = 0; e < NB; ++e) {
      double corr = 0.0;
      for (int i = 0; i < NB; ++i) corr = fma(B[e][i], tc[i], corr);
      rr[e] -= corr;
      for (int j = 0; j < NB; ++j) {
        double acc = 0.0;
        for (int i = 0; i < NB; ++i) acc = fma(B[e][i], Tc[i][j], acc);
        if (t == 3) {
          // accumulation (N_e - N_e,old) V/dt: water row through the
          // eliminated N_w, the other rows on their own amounts
          if (e == 0) acc = fma(-elim[j * N + r], scale, acc);
          else if (j == e) acc += scale;
        }
        val[s * NB * NB + e * NB + j] = acc;
      }
    }
  }
  rr[0] = fma(-elim[NB * N + r], scale, rr[0]);
  for (int e = 0; e < NB; ++e) res[r * NB + e] = rr[e];
}

template <int NB>
__global__ void pn_update_kernel(long long N, double* __restrict__ pn, const double* __restrict__ dx, double sc,
                                 const double* __restrict__ elim, unsigned long long* dmax) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  double x[NB];
  for (int i = 0; i < NB; ++i) x[i] = dx[c * NB + i];
  // N_w component of the full solution from the volume row
  double xw = elim[NB * N + c];
  for (int i = 0; i < NB; ++i) xw = fma(-elim[i * N + c], x[i], xw);
  const double d0 = sc * x[0], dw = sc * xw;
  pn[c] += d0;
  pn[N + c] += dw;
  atomicMax(&dmax[0], (unsigned long long)__double_as_longlong(fabs(d0)));
  atomicMax(&dmax[1], (unsigned long long)__double_as_longlong(fabs(dw)));
  for (int i = 1; i < NB; ++i) {
    const double di = sc * x[i];
    pn[(i + 1) * N + c] += di;
    atomicMax(&dmax[i + 1], (unsigned long long)__double_as_longlong(fabs(di)));
  }
}

template <int NB>
__global__ void pn_norm_kernel(long long N, const double* __restrict__ phi, double scale,
                               const double* __restrict__ res4, unsigned long long* out) {
  constexpr int L = NB + 1;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const double pv = phi[c] * scale;
  for (int e = 0; e < NB; ++e)
    atomicMax(&out[e], (unsigned long long)__double_as_longlong(fabs(res4[c * L + e]) / pv));
  atomicMax(&out[3], (unsigned long long)__double_as_longlong(fabs(res4[c * L + NB])));
}

// (P, N) of a natural state: N = phi S b per bulk volume (eq. 4)
template <int NB>
__global__ void pn_from_natural_kernel(Params P, const Table* __restrict__ gT, const double* __restrict__ u,
                                       const int8_t* __restrict__ flag, const double* __restrict__ phi_ref,
                                       double* __restrict__ pn) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  double m[3];
  cell_masses<NB, false>(P, *gT, u[c], u[N + c], NB == 3 ? u[2 * N + c] : 0.0, NB == 3 ? (flag[c] & 1) : 0,
                         phi_ref[c], m);
  pn[c] = u[c];
  for (int e = 0; e < NB; ++e) pn[(e + 1) * N + c] = m[e];
}

unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

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
}  // namespace ocp

extern "C" {

ocp_status ocp_linearize_pn(ocp_grid* g, const double* pn_new, const double* pn_old, double dt, double* residual,
                            double* bsr_val, double* elim, double* residual_full, double* bsr_val_full,
                            int8_t* flag, void* stream) {
  using namespace ocp;
  if (!g || !pn_new || !pn_old || !residual || !bsr_val || !elim)
    return report(OCP_ERR_INVALID_ARG, "grid, pn_new, pn_old, residual, bsr_val and elim are required");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  const int nb = g->prm.nb;
  const long long N = g->prm.N;
  cudaError_t e = cudaSuccess;
  if (!g->d_pn) {
    const long long per = nb == 3 ? PnLayout<3>::kCount : PnLayout<2>::kCount;
    e = cudaMalloc((void**)&g->d_pn, sizeof(double) * per * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_pn_flag, (size_t)N);
    if (e == cudaSuccess) e = cudaMemset(g->d_pn_flag, 0, (size_t)N);
    if (e != cudaSuccess) {
      cudaFree(g->d_pn);
      cudaFree(g->d_pn_flag);
      g->d_pn = nullptr;
      g->d_pn_flag = nullptr;
      return report(OCP_ERR_OOM, "ocp_linearize_pn: %s", cudaGetErrorString(e));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const double scale = g->prm.vol_rb / dt;
  if (nb == 3)
    pn_split_kernel<3><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, pn_new, g->d_phi, g->d_pn, g->d_pn_flag, elim,
                                               g->d_status);
  else
    pn_split_kernel<2><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, pn_new, g->d_phi, g->d_pn, g->d_pn_flag, elim,
                                               g->d_status);
  e = cudaGetLastError();
  // the natural path on the split state, accumulation left out (the natural
  // state is its own old state: nothing is read from it)
  const double* unat = g->d_pn;
  if (e == cudaSuccess)
    e = launch_linearize(g, unat, g->d_pn_flag, unat, g->d_pn_flag, dt, residual, bsr_val, nullptr, s, nullptr, 1);
  if (e == cudaSuccess) {
    if (nb == 3)
      pn_reduce_kernel<3><<<nblk(N, 128), 128, 0, s>>>(g->prm, g->d_pn, elim, pn_new,
                                                       pn_old, scale, residual, bsr_val, residual_full, bsr_val_full);
    else
      pn_reduce_kernel<2><<<nblk(N, 128), 128, 0, s>>>(g->prm, g->d_pn, elim, pn_new,
                                                       pn_old, scale, residual, bsr_val, residual_full, bsr_val_full);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && flag) e = cudaMemcpyAsync(flag, g->d_pn_flag, (size_t)N, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_linearize_pn: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_pn_update(ocp_grid* g, double* pn, const double* dx, double scale, const double* elim, double* dx_max,
                         void* stream) {
  using namespace ocp;
  if (!g || !pn || !dx || !elim || !dx_max) return report(OCP_ERR_INVALID_ARG, "grid, pn, dx, elim, dx_max are required");
  if (!std::isfinite(scale)) return report(OCP_ERR_INVALID_ARG, "scale must be finite");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = g->prm.N;
  cudaError_t e = cudaMemsetAsync(dx_max, 0, sizeof(double) * (g->prm.nb + 1), s);
  if (e == cudaSuccess) {
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(dx_max);
    if (g->prm.nb == 3) pn_update_kernel<3><<<nblk(N), 256, 0, s>>>(N, pn, dx, scale, elim, dm);
    else pn_update_kernel<2><<<nblk(N), 256, 0, s>>>(N, pn, dx, scale, elim, dm);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_pn_update: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_pn_from_natural(ocp_grid* g, const double* u, const int8_t* flag, double* pn, void* stream) {
  using namespace ocp;
  if (!g || !u || !pn || (g->prm.nb == 3 && !flag)) return report(OCP_ERR_INVALID_ARG, "grid, u, flag and pn are required");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = g->prm.N;
  if (g->prm.nb == 3) pn_from_natural_kernel<3><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, pn);
  else pn_from_natural_kernel<2><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, pn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_pn_from_natural: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_pn_norms(ocp_grid* g, const double* residual_full, double dt, double* norms, void* stream) {
  using namespace ocp;
  if (!g || !residual_full || !norms) return report(OCP_ERR_INVALID_ARG, "grid, residual_full and norms are required");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = g->prm.N;
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 4, s);
  if (e == cudaSuccess) {
    unsigned long long* out = reinterpret_cast<unsigned long long*>(norms);
    const double scale = g->prm.vol_rb / dt;
    if (g->prm.nb == 3) pn_norm_kernel<3><<<nblk(N), 256, 0, s>>>(N, g->d_phi, scale, residual_full, out);
    else pn_norm_kernel<2><<<nblk(N), 256, 0, s>>>(N, g->d_phi, scale, residual_full, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_pn_norms: %s", cudaGetErrorString(e));
  return OCP_OK;
}

}  // extern "C"
