// C interface of the library: argument checking, grid set-up and the
// launches.  See include/ocp.h for the contract of every entry point.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace {

thread_local char g_err[512] = "";

ocp_status fail(ocp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

ocp_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(OCP_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(OCP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the grid's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

void free_grid(ocp_grid* g) {
  if (!g) return;
  cudaFree(g->d_table);
  cudaFree(g->d_row_ptr);
  cudaFree(g->d_col_idx);
  cudaFree(g->d_trans);
  cudaFree(g->d_wlnk);
  cudaFree(g->d_phi);
  cudaFree(g->d_perf_of_cell);
  cudaFree(g->d_perf);
  cudaFree(g->d_well_first);
  cudaFree(g->d_status);
  cudaFree(g->d_scratch);
  cudaFree(g->d_sync);
  cudaFree(g->d_pn);
  if (g->solve_exec) cudaGraphExecDestroy(g->solve_exec);
  if (g->solve_cap) cudaStreamDestroy(g->solve_cap);
  cudaFree(g->d_pn_flag);
  delete g;
}

ocp_status validate(const ocp_grid_desc* d) {
  if (!d) return fail(OCP_ERR_INVALID_ARG, "descriptor is NULL");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(OCP_ERR_INVALID_ARG, "nx, ny, nz must be >= 1");
  const double N = (double)d->nx * d->ny * d->nz;
  if (7.0 * N >= 2147483647.0) return fail(OCP_ERR_INVALID_ARG, "grid too large for int32 block indices");
  if (!finite_pos(d->dx) || !finite_pos(d->dy) || !finite_pos(d->dz)) return fail(OCP_ERR_INVALID_ARG, "dx, dy, dz must be finite and > 0");
  if (!std::isfinite(d->top_depth)) return fail(OCP_ERR_INVALID_ARG, "top_depth must be finite");
  if (d->nphase != 2 && d->nphase != 3) return fail(OCP_ERR_INVALID_ARG, "nphase must be 2 or 3");
  if (!d->lnk || !d->phi) return fail(OCP_ERR_INVALID_ARG, "lnk and phi are required");
  const long long n = (long long)N;
  for (long long c = 0; c < n; ++c) {
    if (!std::isfinite(d->lnk[c])) return fail(OCP_ERR_INVALID_ARG, "lnk[%lld] is not finite", c);
    if (!finite_pos(d->phi[c])) return fail(OCP_ERR_INVALID_ARG, "phi[%lld] must be finite and > 0", c);
  }
  if (!finite_pos(d->kz_over_kx)) return fail(OCP_ERR_INVALID_ARG, "kz_over_kx must be > 0");
  if (!std::isfinite(d->cr) || !std::isfinite(d->p_ref) || !std::isfinite(d->cw) || !std::isfinite(d->co_under) ||
      !std::isfinite(d->cmu_under))
    return fail(OCP_ERR_INVALID_ARG, "compressibilities and p_ref must be finite");
  if (d->nrow < 2 || d->nrow > ocp::kMaxRows) return fail(OCP_ERR_INVALID_ARG, "nrow must be in [2, %d]", ocp::kMaxRows);
  if (!d->tab_p || !d->tab_Bo || !d->tab_muo || (d->nphase == 3 && (!d->tab_Bg || !d->tab_Rs || !d->tab_mug)))
    return fail(OCP_ERR_INVALID_ARG, "PVT table columns are missing");
  for (int k = 0; k < d->nrow; ++k) {
    if (!std::isfinite(d->tab_p[k]) || (k > 0 && !(d->tab_p[k] > d->tab_p[k - 1])))
      return fail(OCP_ERR_INVALID_ARG, "tab_p must be finite and strictly increasing");
    if (!finite_pos(d->tab_Bo[k]) || !finite_pos(d->tab_muo[k])) return fail(OCP_ERR_INVALID_ARG, "tab_Bo, tab_muo must be > 0");
    if (d->nphase == 3) {
      if (!finite_pos(d->tab_Bg[k]) || !finite_pos(d->tab_mug[k])) return fail(OCP_ERR_INVALID_ARG, "tab_Bg, tab_mug must be > 0");
      if (!std::isfinite(d->tab_Rs[k]) || (k > 0 && !(d->tab_Rs[k] > d->tab_Rs[k - 1])))
        return fail(OCP_ERR_INVALID_ARG, "tab_Rs must be finite and strictly increasing");
    }
  }
  if (!finite_pos(d->bw_ref) || !finite_pos(d->muw)) return fail(OCP_ERR_INVALID_ARG, "bw_ref and muw must be > 0");
  if (!std::isfinite(d->rho_osc) || !std::isfinite(d->rho_gsc) || !std::isfinite(d->rho_wsc))
    return fail(OCP_ERR_INVALID_ARG, "surface densities must be finite");
  const double ends[] = {d->swc, d->sorw, d->sorg, d->sgc};
  for (double e : ends)
    if (!(e >= 0.0 && e < 1.0)) return fail(OCP_ERR_INVALID_ARG, "saturation end points must be in [0, 1)");
  if (!(1.0 - d->swc - d->sorw > 0.0)) return fail(OCP_ERR_INVALID_ARG, "1 - swc - sorw must be > 0");
  if (d->nphase == 3 && (!(1.0 - d->swc - d->sgc - d->sorg > 0.0) || !(1.0 - d->swc - d->sorg > 0.0)))
    return fail(OCP_ERR_INVALID_ARG, "gas end points leave no mobile range");
  const double ex[] = {d->nw, d->now, d->ng, d->nog};
  for (double e : ex)
    if (!(e >= 1.0 && std::isfinite(e))) return fail(OCP_ERR_INVALID_ARG, "Corey exponents must be >= 1");
  if (!finite_pos(d->kro_cw) || !(d->krw_max >= 0.0) || !(d->krg_max >= 0.0) || !(d->pcow_max >= 0.0) ||
      !(d->pcgo_max >= 0.0))
    return fail(OCP_ERR_INVALID_ARG, "relative permeability / capillary maxima must be >= 0 (kro_cw > 0)");
  if (d->nwell < 0 || (d->nwell > 0 && !d->wells)) return fail(OCP_ERR_INVALID_ARG, "bad well list");
  for (int w = 0; w < d->nwell; ++w) {
    const ocp_well& W = d->wells[w];
    if (W.kind != 0 && W.kind != 1) return fail(OCP_ERR_INVALID_ARG, "well %d: kind must be 0 or 1", w);
    if (W.kind == 1 && !(W.phase == 0 || (W.phase == 2 && d->nphase == 3)))
      return fail(OCP_ERR_INVALID_ARG, "well %d: injected phase must be 0 (water) or 2 (gas, three-phase only)", w);
    if (!finite_pos(W.rw) || !std::isfinite(W.p_bh) || !std::isfinite(W.skin))
      return fail(OCP_ERR_INVALID_ARG, "well %d: rw > 0, finite p_bh and skin required", w);
    if (W.nperf < 0 || (W.nperf > 0 && !W.cells)) return fail(OCP_ERR_INVALID_ARG, "well %d: bad perforation list", w);
    const double r_o = 0.14 * std::sqrt(d->dx * d->dx + d->dy * d->dy);
    if (!(std::log(r_o / W.rw) + W.skin > 0.0)) return fail(OCP_ERR_INVALID_ARG, "well %d: ln(r_o/rw) + skin must be > 0", w);
    for (int k = 0; k < W.nperf; ++k)
      if (W.cells[k] < 0 || W.cells[k] >= n) return fail(OCP_ERR_INVALID_ARG, "well %d: perforation cell out of range", w);
  }
  return OCP_OK;
}

}  // namespace

namespace ocp {
// Records a formatted message as this thread's last error (for entry points
// defined in other translation units) and returns the status.
ocp_status report(ocp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}
}  // namespace ocp

extern "C" {

const char* ocp_last_error(void) { return g_err; }

ocp_status ocp_grid_create(const ocp_grid_desc* d, int device, ocp_grid** out) {
  if (!out) return fail(OCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ocp_status st = validate(d);
  if (st != OCP_OK) return st;

  const long long N = (long long)d->nx * d->ny * d->nz;
  const int nb = d->nphase;

  // wells: one perforation entry per perforated cell, each cell in one well
  std::vector<int32_t> perf_of_cell(N, -1);
  std::vector<ocp::Perf> perf;
  std::vector<int32_t> well_first(1, 0);
  const double r_o = 0.14 * std::sqrt(d->dx * d->dx + d->dy * d->dy);
  for (int w = 0; w < d->nwell; ++w) {
    const ocp_well& W = d->wells[w];
    const double geom = ocp::kDarcy * 2.0 * M_PI * d->dz / (std::log(r_o / W.rw) + W.skin);
    for (int k = 0; k < W.nperf; ++k) {
      const long long c = W.cells[k];
      if (perf_of_cell[c] >= 0) return fail(OCP_ERR_INVALID_ARG, "cell %lld is perforated twice", c);
      perf_of_cell[c] = (int32_t)perf.size();
      ocp::Perf p;
      p.cell = (int)c;
      p.well = w;
      p.kind = W.kind;
      p.phase = W.phase;
      p.geom = geom;
      p.wi = 0.0;   // k * geom, filled on the device below
      p.p_bh = W.p_bh;
      perf.push_back(p);
    }
    well_first.push_back((int32_t)perf.size());
  }

  DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  ocp_grid* g = new (std::nothrow) ocp_grid();
  if (!g) return fail(OCP_ERR_OOM, "host allocation failed");
  g->device = device;
  g->nwell = d->nwell;
  g->nperf = (int)perf.size();

  // table: reciprocal FVFs and viscosities, slopes, inverse R_s pieces
  ocp::Table& T = g->h_table;
  std::memset(&T, 0, sizeof(T));
  T.nrow = d->nrow;
  for (int k = 0; k < d->nrow; ++k) {
    T.p[k] = d->tab_p[k];
    T.y[0][k] = 1.0 / d->tab_Bo[k];
    T.y[1][k] = 1.0 / d->tab_muo[k];
    if (nb == 3) {
      T.y[2][k] = 1.0 / d->tab_Bg[k];
      T.y[3][k] = 1.0 / d->tab_mug[k];
      T.y[4][k] = d->tab_Rs[k];
      T.rs[k] = d->tab_Rs[k];
    }
    T.pkey[k] = ocp::dkey(T.p[k]);
    T.rskey[k] = ocp::dkey(T.rs[k]);
  }
  for (int k = 0; k + 1 < d->nrow; ++k) {
    const double hp = T.p[k + 1] - T.p[k];
    for (int col = 0; col < 5; ++col) T.s[col][k] = (T.y[col][k + 1] - T.y[col][k]) / hp;
    if (nb == 3) T.q[k] = (T.p[k + 1] - T.p[k]) / (T.rs[k + 1] - T.rs[k]);
  }

  ocp::Params& P = g->prm;
  std::memset(&P, 0, sizeof(P));
  P.nx = d->nx; P.ny = d->ny; P.nz = d->nz; P.nb = nb;
  P.N = N; P.nxy = (long long)d->nx * d->ny;
  ocp::div_magic((unsigned)d->nx, P.nx_m, P.nx_s);
  ocp::div_magic((unsigned)d->ny, P.ny_m, P.ny_s);
  P.dz = d->dz;
  P.p_ref = d->p_ref; P.cr = d->cr; P.bw_ref = d->bw_ref; P.cw = d->cw; P.imu_w = 1.0 / d->muw;
  P.rho_osc = d->rho_osc; P.rho_wsc = d->rho_wsc; P.cg = d->rho_gsc / ocp::kRbFt3;
  P.co = d->co_under; P.cmu = d->cmu_under;
  P.swc = d->swc; P.sorw = d->sorw; P.sorg = d->sorg; P.sgc = d->sgc;
  P.inv_w = 1.0 / (1.0 - d->swc - d->sorw);
  P.inv_g = (nb == 3) ? 1.0 / (1.0 - d->swc - d->sgc - d->sorg) : 0.0;
  P.inv_og = (nb == 3) ? 1.0 / (1.0 - d->swc - d->sorg) : 0.0;
  P.nw = d->nw; P.now = d->now; P.ng = d->ng; P.nog = d->nog;
  P.sq_w = d->nw == 2.0; P.sq_ow = d->now == 2.0; P.sq_g = d->ng == 2.0; P.sq_og = d->nog == 2.0;
  P.krw_max = d->krw_max; P.krg_max = d->krg_max; P.kc = d->kro_cw;
  P.pcow_max = d->pcow_max; P.pcgo_max = (nb == 3) ? d->pcgo_max : 0.0;
  P.grav_dz = 0.5 * ocp::kGrav * d->dz;
  P.pcow2 = 2.0 * d->pcow_max;
  P.pcgo2 = (nb == 3) ? 2.0 * d->pcgo_max : 0.0;
  P.bw_p = d->bw_ref * d->cw;
  P.rw_p = (d->bw_ref * d->cw) * d->rho_wsc;
  P.bw_p_imu = (d->bw_ref * d->cw) * P.imu_w;
  P.vol_rb = d->dx * d->dy * d->dz / ocp::kRbFt3;

  g->sms = 0;
  g->max_cluster = 0;
  g->dx = d->dx;
  g->dy = d->dy;
  g->kz_over_kx = d->kz_over_kx;
  g->nnzb = 7 * N - 2 * ((long long)d->ny * d->nz + (long long)d->nx * d->nz + (long long)d->nx * d->ny);
  g->scratch_doubles = ocp::linearize_scratch_doubles(N);

  cudaError_t e = cudaSuccess;
  double* d_lnk = nullptr;
#define OCP_ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 8)
  OCP_ALLOC(g->d_table, sizeof(ocp::Table));
  OCP_ALLOC(g->d_row_ptr, sizeof(int32_t) * (N + 1));
  OCP_ALLOC(g->d_col_idx, sizeof(int32_t) * g->nnzb);
  OCP_ALLOC(g->d_trans, sizeof(double) * 3 * N);
  OCP_ALLOC(g->d_wlnk, sizeof(double) * 6 * N);
  OCP_ALLOC(g->d_phi, sizeof(double) * N);
  OCP_ALLOC(g->d_perf_of_cell, sizeof(int32_t) * N);
  OCP_ALLOC(g->d_perf, sizeof(ocp::Perf) * perf.size());
  OCP_ALLOC(g->d_well_first, sizeof(int32_t) * well_first.size());
  OCP_ALLOC(g->d_status, sizeof(int));
  OCP_ALLOC(g->d_scratch, sizeof(double) * g->scratch_doubles);
  OCP_ALLOC(g->d_sync, sizeof(unsigned) * (1 + 2 * ((N + 31) / 32)));
  OCP_ALLOC(d_lnk, sizeof(double) * N);
#undef OCP_ALLOC
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, device);
  // default launch shape (ocp_grid_set_shape and the batch autotuner can
  // change it): one CTA per tile, tiles as large as the grid's size allows
  g->cfg = ocp::default_cfg(N, g->sms);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_table, &T, sizeof(T), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_phi, d->phi, sizeof(double) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_lnk, d->lnk, sizeof(double) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_perf_of_cell, perf_of_cell.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !perf.empty())
    e = cudaMemcpy(g->d_perf, perf.data(), sizeof(ocp::Perf) * perf.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->d_well_first, well_first.data(), sizeof(int32_t) * well_first.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = ocp::launch_setup(g, d_lnk, d->dx, d->dy, d->dz, d->kz_over_kx, 0);
  if (e == cudaSuccess) e = ocp::launch_perf_wi(g, d_lnk, 0);
  // the no-allocation entry point's array and kernels, loaded now (this call
  // allocates anyway) so that that entry point never triggers a lazy load
  if (e == cudaSuccess) e = ocp::static_scratch_address(&g->d_static_scratch);
  if (e == cudaSuccess) e = ocp::preload_linearize(nb);
  if (e == cudaSuccess) {           // small grids may run as one cluster launch
    g->max_cluster = ocp::cluster_max_tiles(nb);
    g->cfg = ocp::default_cfg(N, g->sms, g->max_cluster);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_lnk);
  if (e != cudaSuccess) {
    free_grid(g);
    return cuda_fail(e, "ocp_grid_create");
  }
  *out = g;
  return OCP_OK;
}

ocp_status ocp_grid_destroy(ocp_grid* g) {
  if (!g) return OCP_OK;
  DeviceGuard guard(g->device);
  free_grid(g);
  return OCP_OK;
}

ocp_status ocp_grid_info(const ocp_grid* g, int64_t* ncell, int* nb, int64_t* nnzb) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (ncell) *ncell = g->prm.N;
  if (nb) *nb = g->prm.nb;
  if (nnzb) *nnzb = g->nnzb;
  return OCP_OK;
}

ocp_status ocp_bsr_pattern(const ocp_grid* g, const int32_t** row_ptr, const int32_t** col_idx) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (row_ptr) *row_ptr = g->d_row_ptr;
  if (col_idx) *col_idx = g->d_col_idx;
  return OCP_OK;
}

ocp_status ocp_linearize(ocp_grid* g, const double* u_new, const int8_t* flag_new, const double* u_old,
                         const int8_t* flag_old, double dt, double* residual, double* bsr_val,
                         double* face_flux, void* stream) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!u_new || !u_old || !residual || !bsr_val) return fail(OCP_ERR_INVALID_ARG, "u_new, u_old, residual, bsr_val are required");
  if (g->prm.nb == 3 && (!flag_new || !flag_old)) return fail(OCP_ERR_INVALID_ARG, "flags are required with three phases");
  if (!(std::isfinite(dt) && dt > 0.0)) return fail(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  DeviceGuard guard(g->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaError_t e = ocp::launch_linearize(g, u_new, flag_new, u_old, flag_old, dt, residual, bsr_val, face_flux,
                                        (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ocp_linearize launch");
  return OCP_OK;
}

ocp_status ocp_bsr_spmv(const ocp_grid* g, const double* val, double alpha, const double* x, double beta,
                        double* y, int transpose, void* stream) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!val || !x || !y) return fail(OCP_ERR_INVALID_ARG, "val, x, y are required");
  if (x == y) return fail(OCP_ERR_INVALID_ARG, "x and y must not overlap");
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return fail(OCP_ERR_INVALID_ARG, "alpha and beta must be finite");
  DeviceGuard guard(g->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaError_t e = ocp::launch_spmv(g, val, alpha, x, beta, y, transpose, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ocp_bsr_spmv launch");
  return OCP_OK;
}

ocp_status ocp_adjoint_vjp(ocp_grid* g, const double* u_new, const int8_t* flag_new, const double* u_old,
                           const int8_t* flag_old, double dt, const double* bsr_val, const double* face_flux,
                           const double* lambda, double* g_unew, double* g_uold, double* g_lnk, double* g_phi,
                           void* stream) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!u_new || !u_old || !lambda) return fail(OCP_ERR_INVALID_ARG, "u_new, u_old, lambda are required");
  if (g->prm.nb == 3 && (!flag_new || !flag_old)) return fail(OCP_ERR_INVALID_ARG, "flags are required with three phases");
  if (g_unew && !bsr_val) return fail(OCP_ERR_INVALID_ARG, "g_unew needs bsr_val");
  if (g_lnk && !face_flux) return fail(OCP_ERR_INVALID_ARG, "g_lnk needs face_flux");
  if (!(std::isfinite(dt) && dt > 0.0)) return fail(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  DeviceGuard guard(g->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaError_t e = ocp::launch_vjp(g, u_new, flag_new, u_old, flag_old, dt, bsr_val, face_flux, lambda, g_unew,
                                  g_uold, g_lnk, g_phi, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ocp_adjoint_vjp launch");
  return OCP_OK;
}

ocp_status ocp_well_rates(ocp_grid* g, const double* u, const int8_t* flag, double* q, void* stream) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  if (!u || !q || (g->prm.nb == 3 && !flag)) return fail(OCP_ERR_INVALID_ARG, "u, flag and q are required");
  DeviceGuard guard(g->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaError_t e = ocp::launch_well_rates(g, u, flag, q, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ocp_well_rates launch");
  return OCP_OK;
}

ocp_status ocp_get_status(ocp_grid* g, void* stream) {
  if (!g) return fail(OCP_ERR_INVALID_ARG, "grid is NULL");
  DeviceGuard guard(g->device);
  if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int h = 0;
  e = cudaMemcpy(&h, g->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(g->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
  if (h & ocp::kStatNonFinite) return fail(OCP_ERR_NONFINITE, "a kernel met a non-finite value");
  if (h & ocp::kStatBadFlag) return fail(OCP_ERR_INVALID_ARG, "a phase-state flag was neither 0 nor 1");
  if (h & ocp::kStatTimeout) return fail(OCP_ERR_TIMEOUT, "a bounded device wait expired");
  if (h & ocp::kStatBadControl) return fail(OCP_ERR_INVALID_ARG, "a well control was invalid");
  return OCP_OK;
}

}  // extern "C"
