// Launchers shared between the translation units of the library.
#pragma once
#include "ocp_internal.cuh"

namespace ocp {

int64_t linearize_scratch_doubles(int64_t N);
cudaError_t launch_linearize(const ocp_grid* g, const double* u_new, const int8_t* f_new,
                             const double* u_old, const int8_t* f_old, double dt, double* res,
                             double* val, double* face_flux, cudaStream_t s, const double* p_bh = nullptr,
                             int no_acc = 0);
// The same launches with the per-cell scratch given explicitly (used by the
// entry point that must not allocate).
cudaError_t launch_linearize_scratch(const ocp_grid* g, double* scratch, const double* u_new,
                                     const int8_t* f_new, const double* u_old, const int8_t* f_old, double dt,
                                     double* res, double* val, double* face_flux, cudaStream_t s);
ocp_status report(ocp_status st, const char* fmt, ...);
// Device address of the no-allocation entry point's library array on the
// current device; the lookup loads the array there (reserving it).
cudaError_t static_scratch_address(double** out);
// Loads the linearisation kernels for nb x nb blocks onto the current device
// (under lazy module loading their first launch would otherwise load them).
cudaError_t preload_linearize(int nb);
cudaError_t launch_perf_wi(ocp_grid* g, const double* lnk, cudaStream_t s);
int64_t solver_work_doubles(const ocp_grid* g);

// Well terms of a Jacobian with bottom-hole-pressure unknowns, oriented for
// the system being solved: bs couples the wells into the cell rows, cs the
// cells into the well rows (nb values per perforation each), d the well
// diagonal (one per well).
struct WellSchur {
  const double* bs;
  const double* cs;
  const double* d;
};
// mode 0: out += alpha bs (d^-1 (cs . in)); 1: out += alpha bs (d^-1 bw);
// 2: xw = d^-1 (bw - cs . in)
// skip: when not null, the kernels return at once if *skip != 0 (a solver's
// done flag, so that the iterations left in a replayed graph cost nothing).
cudaError_t launch_well_schur(const ocp_grid* g, const WellSchur& ws, int mode, double alpha, const double* in,
                              double* out, const double* bw, double* xw, cudaStream_t s,
                              const double* skip = nullptr);
// Left block-Jacobi BiCGSTAB on A (ws == nullptr) or on the Schur complement
// A - bs d^-1 cs of the well unknowns.
// nbs: block size of the system (0: the grid's; 1: a scalar system on the
// grid's pattern).
ocp_status bicgstab_run(ocp_grid* g, const double* val, const WellSchur* ws, const double* b, double* x,
                        double rtol, int maxit, int transpose, double* work, int* iters, double* relres,
                        cudaStream_t s, int nbs = 0);
cudaError_t launch_tiles(int nb, const TileList* lists, const ModelArgs& single, const LaunchCfg& cfg,
                         int sms, cudaStream_t s);
// The ordered (persistent) launch; O.nitems holds the number of tiles.
cudaError_t launch_ordered(int nb, const TileList* lists, OrderedList O, const ModelArgs& single,
                           const LaunchCfg& cfg, int sms, cudaStream_t s);
// The one-cluster launch of a small grid (at most max_tiles 32-cell tiles):
// the first model of `models`, or `single` when models is null.
cudaError_t launch_cluster(int nb, const ModelArgs* models, const ModelArgs& single, long long N, int max_tiles,
                           cudaStream_t s);
int cluster_max_tiles(int nb);
ModelArgs model_args(const ocp_grid* g, double* scratch, const double* u_new, const int8_t* f_new,
                     const double* u_old, const int8_t* f_old, double dt, double* res, double* val,
                     double* face_flux);
cudaError_t launch_spmv(const ocp_grid* g, const double* val, double alpha, const double* x, double beta,
                        double* y, int transpose, cudaStream_t s, int nbs = 0, const double* skip = nullptr);
cudaError_t launch_vjp(const ocp_grid* g, const double* u_new, const int8_t* f_new, const double* u_old,
                       const int8_t* f_old, double dt, const double* val, const double* face_flux,
                       const double* lam, double* g_unew, double* g_uold, double* g_lnk, double* g_phi,
                       cudaStream_t s);
cudaError_t launch_well_rates(const ocp_grid* g, const double* u, const int8_t* flag, double* q,
                              cudaStream_t s);
cudaError_t launch_setup(ocp_grid* g, const double* d_lnk, double dx, double dy, double dz,
                         double kz_over_kx, cudaStream_t s);

}  // namespace ocp
