// IMPEC in pressure and component amounts: the pressure from the volume
// balance at the new level, linearised about the old one with mobilities,
// upwind directions, densities and capillary offsets frozen at the old level
// (a 7-point system with one unknown per cell), then the explicit
// conservative update of the amounts.
//
//   impec_cell_kernel    per cell: phase split and cell properties at the old
//                        level, the fluid volume's derivatives (V_f,P and
//                        w_i = dV_f/dN_i), kept in the grid's scratch;
//   impec_matrix_kernel  per cell row: for each face and phase the frozen
//                        coefficient T lambda_up and the old potential
//                        difference, weighted by w_i of the row cell; wells
//                        at the new cell pressure with old mobilities;
//   impec_update_kernel  per cell: the face fluxes and well terms at the new
//                        pressure and N^{n+1} = N^n + (Q - sum F) dt / V.
// A face's flux seen from its two cells is the exact negation of the same
// floating-point expression, so the update conserves every component to
// rounding.
#include <cmath>

#include "kernels.cuh"
#include "ocp_internal.cuh"
#include "pn_split.cuh"

namespace ocp {
namespace {

enum {
  kP = 0, kOffW, kOffG, kRhoW, kRhoO, kRhoG, kLamW, kLamO, kLamG, kRs, kWw, kWo, kWg, kDiag0, kE0, kMob, kBw, kBg,
  kImpecSlots
};

template <int NB>
__global__ void impec_cell_kernel(Params P, const Table* __restrict__ gT, const double* __restrict__ pn,
                                  const double* __restrict__ phi_ref, double scale, double* __restrict__ d,
                                  int* status) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const double p = pn[c], nw = pn[N + c], no = pn[2 * N + c], ng = (NB == 3) ? pn[3 * N + c] : 0.0;
  if (!(finite(p) && finite(nw) && finite(no) && finite(ng))) atomicOr(status, kStatNonFinite);
  Split<NB> sp;
  phase_split<NB>(P, *gT, p, nw, no, ng, sp);
  CellQ q{};
  CellAux a{};
  cell_quantities<NB, true>(P, *gT, p, sp.sw, sp.x, sp.flag, phi_ref[c], q, a, true);
  const double phi = phi_ref[c] * fma(P.cr, p - P.p_ref, 1.0);
  d[kP * N + c] = p;
  d[kOffW * N + c] = q.pw - p;
  d[kOffG * N + c] = (NB == 3) ? q.pg - p : 0.0;
  d[kRhoW * N + c] = q.rw;
  d[kRhoO * N + c] = q.ro;
  d[kRhoG * N + c] = (NB == 3) ? q.rg : 0.0;
  d[kLamW * N + c] = q.lw;
  d[kLamO * N + c] = q.lo;
  d[kLamG * N + c] = (NB == 3) ? q.lg : 0.0;
  d[kRs * N + c] = (NB == 3) ? q.rs : 0.0;
  d[kWw * N + c] = sp.dVf[1];
  d[kWo * N + c] = sp.dVf[2];
  d[kWg * N + c] = (NB == 3) ? sp.dVf[3] : 0.0;
  d[kDiag0 * N + c] = scale * (phi_ref[c] * P.cr - sp.dVf[0]);
  d[kE0 * N + c] = scale * (phi - sp.Vf);
  d[kMob * N + c] = a.mob;
  d[kBw * N + c] = a.bw;
  d[kBg * N + c] = (NB == 3) ? a.bg : 0.0;
}

// The cell's neighbours in column order (-z, -y, -x, +x, +y, +z) and the
// data of one face: per phase the frozen coefficient T lambda_up and the old
// potential difference (from the cell to the neighbour), and the oil's
// upwind R_s.
struct FaceCoef {
  double c[3], dphi[3], rs_up;
};

template <int NB>
__device__ __forceinline__ void face_coef(const Params& P, const double* __restrict__ d, long long c, long long n,
                                          double T, double hz, FaceCoef& f) {
  const long long N = P.N;
  const double pc = d[kP * N + c], pn_ = d[kP * N + n];
  const int offs[3] = {kOffW, -1, kOffG};
  const int rhos[3] = {kRhoW, kRhoO, kRhoG};
  const int lams[3] = {kLamW, kLamO, kLamG};
  for (int ph = 0; ph < NB; ++ph) {                // water, oil[, gas]
    const int al = ph;
    const double oc = offs[ph] >= 0 ? d[offs[ph] * N + c] : 0.0;
    const double on = offs[ph] >= 0 ? d[offs[ph] * N + n] : 0.0;
    double dphi = (pc + oc) - (pn_ + on);
    if (hz != 0.0) dphi = fma(-(d[rhos[ph] * N + c] + d[rhos[ph] * N + n]), hz, dphi);
    const bool up = nonneg(dphi);
    f.c[al] = T * (up ? d[lams[ph] * N + c] : d[lams[ph] * N + n]);
    f.dphi[al] = dphi;
    if (al == 1) f.rs_up = (NB == 3) ? (up ? d[kRs * N + c] : d[kRs * N + n]) : 0.0;
  }
}

// Neighbour t of c (t = 0..5: -z, -y, -x, +x, +y, +z): index, face axis and
// side, transmissibility and the gravity head factor.
__device__ __forceinline__ bool neighbour(const Params& P, const double* __restrict__ trans, long long c, int i, int j,
                                          int k, int t, long long& n, double& T, double& hz) {
  const int axis[6] = {2, 1, 0, 0, 1, 2};
  const bool plus = t >= 3;
  const int ax = axis[t];
  bool has;
  long long off;
  if (ax == 0) { has = plus ? (i + 1 < P.nx) : (i > 0); off = 1; }
  else if (ax == 1) { has = plus ? (j + 1 < P.ny) : (j > 0); off = P.nx; }
  else { has = plus ? (k + 1 < P.nz) : (k > 0); off = P.nxy; }
  if (!has) return false;
  n = plus ? c + off : c - off;
  T = trans[ax * P.N + (plus ? c : n)];
  hz = (ax == 2) ? (plus ? -P.grav_dz : P.grav_dz) : 0.0;
  return true;
}

// Component fluxes out of c through one face at a pressure change
// (dPc, dPn); K = the old-level part, C = the coefficient of (dPc - dPn).
template <int NB>
__device__ __forceinline__ void comp_flux(const FaceCoef& f, double* C, double* K) {
  C[0] = f.c[0];
  K[0] = f.c[0] * f.dphi[0];
  C[1] = f.c[1];
  K[1] = f.c[1] * f.dphi[1];
  if (NB == 3) {
    C[2] = fma(f.rs_up, f.c[1], f.c[2]);
    K[2] = fma(f.rs_up, K[1], f.c[2] * f.dphi[2]);
  }
}

// Well terms of the cell: Q_i(dP) = Q0_i + Qp_i dP (old mobilities, open
// state of the old level).
template <int NB>
__device__ __forceinline__ void well_terms(const Params& P, const double* __restrict__ d, long long c, const Perf& w,
                                           double* Q0, double* Qp) {
  const long long N = P.N;
  for (int e = 0; e < NB; ++e) Q0[e] = Qp[e] = 0.0;
  const double p = d[kP * N + c];
  if (w.kind == 0) {
    if (!positive(p - w.p_bh)) return;
    const double g = w.p_bh - p;
    const double lw = w.wi * d[kLamW * N + c], lo = w.wi * d[kLamO * N + c];
    Q0[0] = lw * g;
    Qp[0] = neg(lw);
    Q0[1] = lo * g;
    Qp[1] = neg(lo);
    if (NB == 3) {
      const double lg = w.wi * d[kLamG * N + c], rs = d[kRs * N + c];
      Q0[2] = fma(rs, Q0[1], lg * g);
      Qp[2] = neg(fma(rs, lo, lg));
    }
  } else {
    if (!positive(w.p_bh - p)) return;
    const int e = (w.phase == 0) ? 0 : NB - 1;
    const double coef = w.wi * d[kMob * N + c] * ((w.phase == 0) ? d[kBw * N + c] : d[kBg * N + c]);
    Q0[e] = coef * (w.p_bh - p);
    Qp[e] = neg(coef);
  }
}

template <int NB>
__global__ void impec_matrix_kernel(Params P, const double* __restrict__ trans, const int32_t* __restrict__ row_ptr,
                                    const int32_t* __restrict__ perf_of_cell, const Perf* __restrict__ perf,
                                    const double* __restrict__ d, double* __restrict__ val, double* __restrict__ rhs) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const double w[3] = {d[kWw * N + c], d[kWo * N + c], NB == 3 ? d[kWg * N + c] : 0.0};
  double diag = d[kDiag0 * N + c];
  double E = d[kE0 * N + c];
  int s = row_ptr[c];
  double lower[3];
  int nl = 0;
  double upper[3];
  int nu = 0;
  for (int t = 0; t < 6; ++t) {
    long long n;
    double T, hz;
    if (!neighbour(P, trans, c, i, j, k, t, n, T, hz)) continue;
    FaceCoef f;
    face_coef<NB>(P, d, c, n, T, hz, f);
    double C[3], K[3];
    comp_flux<NB>(f, C, K);
    double sc = 0.0, sk = 0.0;
    for (int e = 0; e < NB; ++e) {
      sc = fma(w[e], C[e], sc);
      sk = fma(w[e], K[e], sk);
    }
    E += sk;
    diag += sc;
    if (t < 3) lower[nl++] = neg(sc);
    else upper[nu++] = neg(sc);
  }
  const int ip = perf_of_cell[c];
  if (ip >= 0) {
    double Q0[3], Qp[3];
    well_terms<NB>(P, d, c, perf[ip], Q0, Qp);
    for (int e = 0; e < NB; ++e) {
      E = fma(-w[e], Q0[e], E);
      diag = fma(-w[e], Qp[e], diag);
    }
  }
  for (int q = 0; q < nl; ++q) val[s++] = lower[q];
  val[s++] = diag;
  for (int q = 0; q < nu; ++q) val[s++] = upper[q];
  rhs[c] = neg(E);
}

template <int NB>
__global__ void impec_update_kernel(Params P, const double* __restrict__ trans, const int32_t* __restrict__ perf_of_cell,
                                    const Perf* __restrict__ perf, const double* __restrict__ d,
                                    const double* __restrict__ pn_old, const double* __restrict__ dp, double inv_scale,
                                    double* __restrict__ pn_new) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const double dpc = dp[c];
  double out[3] = {0.0, 0.0, 0.0};
  for (int t = 0; t < 6; ++t) {
    long long n;
    double T, hz;
    if (!neighbour(P, trans, c, i, j, k, t, n, T, hz)) continue;
    FaceCoef f;
    face_coef<NB>(P, d, c, n, T, hz, f);
    const double dd = dpc - dp[n];
    // phase fluxes at the new pressure, then components (dissolved gas with the oil)
    double F[3];
    for (int al = 0; al < NB; ++al) F[al] = f.c[al] * (f.dphi[al] + dd);
    out[0] += F[0];
    out[1] += F[1];
    if (NB == 3) out[2] += fma(f.rs_up, F[1], F[2]);
  }
  double Q[3] = {0.0, 0.0, 0.0};
  const int ip = perf_of_cell[c];
  if (ip >= 0) {
    double Q0[3], Qp[3];
    well_terms<NB>(P, d, c, perf[ip], Q0, Qp);
    for (int e = 0; e < NB; ++e) Q[e] = fma(Qp[e], dpc, Q0[e]);
  }
  pn_new[c] = pn_old[c] + dpc;
  for (int e = 0; e < NB; ++e) pn_new[(e + 1) * N + c] = fma(Q[e] - out[e], inv_scale, pn_old[(e + 1) * N + c]);
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

ocp_status ocp_impec_pressure(ocp_grid* g, const double* pn, double dt, double* val, double* rhs, void* stream) {
  using namespace ocp;
  if (!g || !pn || !val || !rhs) return report(OCP_ERR_INVALID_ARG, "grid, pn, val and rhs are required");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  static_assert(kImpecSlots <= 100, "IMPEC data must fit the linearisation scratch");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = g->prm.N;
  const double scale = g->prm.vol_rb / dt;
  if (g->prm.nb == 3) {
    impec_cell_kernel<3><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, pn, g->d_phi, scale, g->d_scratch, g->d_status);
    impec_matrix_kernel<3><<<nblk(N), 256, 0, s>>>(g->prm, g->d_trans, g->d_row_ptr, g->d_perf_of_cell, g->d_perf,
                                                   g->d_scratch, val, rhs);
  } else {
    impec_cell_kernel<2><<<nblk(N), 256, 0, s>>>(g->prm, g->d_table, pn, g->d_phi, scale, g->d_scratch, g->d_status);
    impec_matrix_kernel<2><<<nblk(N), 256, 0, s>>>(g->prm, g->d_trans, g->d_row_ptr, g->d_perf_of_cell, g->d_perf,
                                                   g->d_scratch, val, rhs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_impec_pressure: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_impec_update(ocp_grid* g, const double* pn_old, const double* dp, double dt, double* pn_new,
                            void* stream) {
  using namespace ocp;
  if (!g || !pn_old || !dp || !pn_new) return report(OCP_ERR_INVALID_ARG, "grid, pn_old, dp and pn_new are required");
  if (pn_old == pn_new) return report(OCP_ERR_INVALID_ARG, "pn_old and pn_new must not overlap");
  if (!(std::isfinite(dt) && dt > 0.0)) return report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  cudaStream_t s = (cudaStream_t)stream;
  const long long N = g->prm.N;
  const double inv_scale = dt / g->prm.vol_rb;
  if (g->prm.nb == 3)
    impec_update_kernel<3><<<nblk(N), 256, 0, s>>>(g->prm, g->d_trans, g->d_perf_of_cell, g->d_perf, g->d_scratch,
                                                   pn_old, dp, inv_scale, pn_new);
  else
    impec_update_kernel<2><<<nblk(N), 256, 0, s>>>(g->prm, g->d_trans, g->d_perf_of_cell, g->d_perf, g->d_scratch,
                                                   pn_old, dp, inv_scale, pn_new);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_impec_update: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_bicgstab_scalar(ocp_grid* g, const double* val, const double* b, double* x, double rtol, int maxit,
                               double* work, int* iters, double* relres, void* stream) {
  using namespace ocp;
  if (!g || !val || !b || !x || !work) return report(OCP_ERR_INVALID_ARG, "grid, val, b, x and work are required");
  if (b == x) return report(OCP_ERR_INVALID_ARG, "b and x must not overlap");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  return bicgstab_run(g, val, nullptr, b, x, rtol, maxit, 0, work, iters, relres, (cudaStream_t)stream, 1);
}

}  // extern "C"
