/*
 * ocp.h -- C interface of the GB300 black-oil FIM linearisation library.
 *
 * One fully implicit (FIM) Newton linearisation of the black-oil component
 * mass balances on a Cartesian grid with two-point fluxes, the block-CSR
 * matrix-vector product the linear solver iterates on, and the adjoint
 * vector-Jacobian product.  The equations are the component conservation law
 * (eq. 1) with Darcy velocities (eq. 2) and the component amounts of eq. 4,
 * in the black-oil closure where saturations, compositions and densities
 * follow explicitly from the primary variables (Sec. 2.1).  The work is split
 * the way the paper splits the reservoir: cell terms (Bulk: PVT, SAT, ROCK,
 * ACCU -- Sec. 3.2.3), connection terms (BulkConn) and well terms (AllWells --
 * Sec. 3.2.4), assembled into block rows of a block-CSR matrix (InternalMat of
 * the LinearSystem module, Sec. 3.3.3) for the Newton step of Sec. 3.2.5.
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: psi, ft, mD, cP, day; oil and water in stb, gas in scf.
 * Cells: N = nx*ny*nz in natural order c = i + nx*(j + ny*k); k grows
 *   downward (depth of layer k is top_depth + (k + 1/2) dz).
 * Unknowns per cell (nb of them): three-phase (p, S_w, X) with X = S_g where
 *   flag == 0 (saturated oil) and X = R_s where flag == 1 (undersaturated
 *   oil); two-phase oil-water (p, S_w).  p is the oil pressure.
 * State arrays u are variable-major: u[v*N + c].  Flags are int8[N].
 * Residual, SpMV and adjoint vectors are block-interleaved: r[nb*c + e] with
 *   equations ordered water, oil[, gas].
 * Jacobian: block-CSR with int32 row_ptr[N+1], col_idx[nnzb] (columns
 *   ascending: c-nx*ny, c-nx, c-1, c, c+1, c+nx, c+nx*ny where they exist),
 *   nnzb = 7N - 2(ny*nz + nx*nz + nx*ny), and
 *   val[(s*nb + e)*nb + v] = dR[row, e] / du[col_idx[s], v]  (row-major
 *   nb x nb blocks).
 * Pointers passed to the compute calls are DEVICE pointers to memory the
 *   caller owns (the library never frees them and keeps none after return),
 *   on the device the grid was created on, 8-byte aligned.
 * Compute calls are asynchronous on the given CUDA stream (NULL = the legacy
 *   default stream).  Argument errors are returned immediately and nothing is
 *   launched.  Errors found on the device (non-finite values, bad flags) are
 *   sticky in the grid's status word and reported by ocp_get_status().
 * There is no CPU fallback: every compute call runs CUDA kernels for sm_103a.
 * Only ocp_grid_create, ocp_batch_create, their destroy calls and the first
 *   ocp_linearize_pn on a grid (its phase-split data) allocate or free device
 *   memory; the first ocp_bicgstab* call on a grid creates a stream and a
 *   CUDA graph that the grid keeps.
 * ocp_last_error() returns a thread-local message describing the last failure.
 */
#ifndef OCP_H
#define OCP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OCP_OK = 0,
  OCP_ERR_INVALID_ARG = 1,  /* bad pointer, size, flag or descriptor field */
  OCP_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  OCP_ERR_OOM = 3,          /* device allocation failed */
  OCP_ERR_NONFINITE = 4,    /* a kernel met a NaN/Inf input or produced one */
  OCP_ERR_TIMEOUT = 5,      /* a bounded wait expired */
  OCP_ERR_UNSUPPORTED = 6   /* valid request the library does not implement */
} ocp_status;

/* A well controlled by bottom-hole pressure (AllWells, Sec. 3.2.4).  Each
 * perforated cell exchanges fluid with the well through Peaceman's index
 * WI = C 2 pi k dz / (ln(r_o / rw) + skin), r_o = 0.14 sqrt(dx^2 + dy^2).
 * A producer (kind 0) takes every phase where p > p_bh; an injector (kind 1)
 * pushes its one phase (0 water, 2 gas) where p_bh > p, with the cell's total
 * mobility.  A cell may be perforated by at most one well. */
typedef struct {
  int kind;               /* 0 producer, 1 injector */
  int phase;              /* injected phase of an injector: 0 water, 2 gas */
  double p_bh;            /* bottom-hole pressure, psi */
  double rw;              /* wellbore radius, ft (> 0) */
  double skin;
  int nperf;              /* number of perforated cells */
  const int64_t* cells;   /* HOST array [nperf] of natural cell indices */
} ocp_well;

/* Grid, rock, fluid and wells: the statement of the problem (Sec. 2.1 and the
 * Bulk sub-modules of Sec. 3.2.3).  All pointers are HOST pointers; the
 * library copies what it needs and keeps none of them. */
typedef struct {
  int nx, ny, nz;                 /* cells per direction, each >= 1 */
  double dx, dy, dz;              /* cell size, ft (> 0) */
  double top_depth;               /* depth of the top face, ft */
  int nphase;                     /* 3 (black oil, 3x3 blocks) or 2 (oil-water, 2x2) */
  const double* lnk;              /* [N] ln(k_x / mD); k_y = k_x, k_z = kz_over_kx k_x */
  const double* phi;              /* [N] porosity at p_ref (> 0) */
  double kz_over_kx, cr, p_ref;   /* rock: phi(p) = phi (1 + cr (p - p_ref)) */
  int nrow;                       /* PVT rows, 2..64, tab_p strictly increasing */
  const double *tab_p, *tab_Bo, *tab_Bg, *tab_Rs, *tab_muo, *tab_mug;
  /* water b_w = bw_ref (1 + cw (p - p_ref)), constant viscosity muw;
   * surface densities (lb/ft^3); undersaturated oil compressibility co_under
   * and viscosibility cmu_under (1/psi) */
  double bw_ref, cw, muw, rho_osc, rho_gsc, rho_wsc, co_under, cmu_under;
  /* Corey end points and exponents (>= 1), Stone II with kro_cw, and the
   * maximum oil-water and gas-oil capillary pressures (psi) */
  double swc, sorw, sorg, sgc, nw, now, ng, nog, krw_max, krg_max, kro_cw, pcow_max, pcgo_max;
  int nwell;
  const ocp_well* wells;          /* HOST array [nwell] */
} ocp_grid_desc;

typedef struct ocp_grid ocp_grid;     /* opaque, library-owned */

/* Set-up (Solver::Setup analogue, Sec. 3.3.1): validates the descriptor,
 * selects `device`, allocates the grid's device data (transmissibilities,
 * pore volumes, well indices, the block-CSR pattern, PVT constants) and
 * fills it.  Returns OCP_ERR_INVALID_ARG for an inconsistent descriptor,
 * OCP_ERR_OOM / OCP_ERR_CUDA on device failure (nothing leaks). */
ocp_status ocp_grid_create(const ocp_grid_desc* desc, int device, ocp_grid** out);
ocp_status ocp_grid_destroy(ocp_grid* grid);      /* NULL is accepted */

/* Sizes: number of cells, block size nb, number of stored blocks. */
ocp_status ocp_grid_info(const ocp_grid* grid, int64_t* ncell, int* nb, int64_t* nnzb);

/* Device pointers to the grid's block-CSR pattern (owned by the grid, valid
 * until ocp_grid_destroy). */
ocp_status ocp_bsr_pattern(const ocp_grid* grid, const int32_t** row_ptr, const int32_t** col_idx);

/* One FIM linearisation (Sec. 3.2.5 steps 1 and 3: property update and
 * Jacobian assembly).  Computes, for the backward-Euler step of length dt
 * (days, > 0) from (u_old, flag_old) to (u_new, flag_new):
 *   residual[nb*N]   R = (V/5.614583/dt)(m(u_new) - m(u_old)) + sum of
 *                    outgoing upwinded TPFA fluxes - well sources;
 *   bsr_val[nnzb*nb*nb]  J = dR/du_new in the layout above;
 *   face_flux[3*nb*N] (may be NULL) component fluxes across the +x, +y, +z
 *                    face of every cell: face_flux[(d*nb + e)*N + c], zero
 *                    where the face does not exist (input of the adjoint).
 * Device-detected NaN/Inf in the state, or a flag other than 0/1, sets the
 * sticky status OCP_ERR_NONFINITE / OCP_ERR_INVALID_ARG. */
ocp_status ocp_linearize(ocp_grid* grid, const double* u_new, const int8_t* flag_new,
                         const double* u_old, const int8_t* flag_old, double dt,
                         double* residual, double* bsr_val, double* face_flux, void* cuda_stream);

/* ocp_linearize without any device allocation behind it.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * when they linearise -- code whose device memory is owned by a host
 * application or framework with its own allocator, or a loop under a fixed
 * memory budget that may not grow.
 * Same arguments, outputs and errors as ocp_linearize, but its per-cell
 * scratch is a 32 MiB array owned by the library instead of the grid's
 * buffer, so it accepts grids of at most 41 943 cells and returns
 * OCP_ERR_INVALID_ARG for larger ones.  It calls no cudaMalloc, cudaFree or
 * other allocating routine, and triggers no lazy module load: the array is
 * reserved on a device, and the kernels loaded there, by the first
 * ocp_grid_create on that device (which allocates anyway); the array stays
 * reserved until the process exits, and the grid keeps its device address.
 * A device reset invalidates the grid and that address with it.  All calls
 * share the array and leave its contents behind (nothing in it needs to
 * start at zero): calls that overlap on the GPU race and must not be made. */
ocp_status ocp_linearize_noalloc(ocp_grid* grid, const double* u_new, const int8_t* flag_new,
                                 const double* u_old, const int8_t* flag_old, double dt,
                                 double* residual, double* bsr_val, double* face_flux, void* cuda_stream);

/* Block-CSR product of the linear solver (LinearSystem, Sec. 3.3.3):
 * y = alpha * A x + beta * y, or with transpose != 0, y = alpha * A^T x +
 * beta * y.  A is bsr_val on the grid's pattern; x and y are block-
 * interleaved [nb*N] device vectors and must not overlap.  beta == 0 does
 * not read y (so y may hold NaNs).  With 2x2 blocks and a 16-byte aligned
 * bsr_val the product stages the matrix through the copy engine; any other
 * alignment takes a register path with bit-identical results.  The staged
 * path's waits are bounded: one that expires leaves its rows unwritten and
 * makes ocp_get_status return OCP_ERR_TIMEOUT. */
ocp_status ocp_bsr_spmv(const ocp_grid* grid, const double* bsr_val, double alpha, const double* x,
                        double beta, double* y, int transpose, void* cuda_stream);

/* Adjoint vector-Jacobian products of the residual of ocp_linearize (the
 * derivative of eqs. 1, 2 and 4 with respect to the model parameters and the
 * states), for a block-interleaved multiplier lambda[nb*N]:
 *   g_unew[nb*N]  (J^T lambda), variable-major like u;
 *   g_uold[nb*N]  (dR/du_old)^T lambda, variable-major;
 *   g_lnk[N]      (dR/d ln k)^T lambda  (through T and WI);
 *   g_phi[N]      (dR/d phi)^T lambda   (through the pore volume).
 * bsr_val and face_flux must be the outputs of ocp_linearize at the same
 * states and dt.  Any g_* may be NULL (not computed).  Outputs are
 * overwritten, not accumulated. */
ocp_status ocp_adjoint_vjp(ocp_grid* grid, const double* u_new, const int8_t* flag_new,
                           const double* u_old, const int8_t* flag_old, double dt,
                           const double* bsr_val, const double* face_flux, const double* lambda,
                           double* g_unew, double* g_uold, double* g_lnk, double* g_phi,
                           void* cuda_stream);

/* Surface rates of every well at a state (AllWells, Sec. 3.2.4):
 * q[w*nb + e], component e of well w summed over its perforations,
 * positive into the reservoir (stb/day; scf/day for gas). */
ocp_status ocp_well_rates(ocp_grid* grid, const double* u, const int8_t* flag, double* q,
                          void* cuda_stream);

/* ---------------------------------------------------------------- batches
 * An ensemble of grids linearised together (the same arithmetic as calling
 * ocp_linearize on each grid, bit for bit).  The three stages of the
 * linearisation -- cell properties with accumulation and wells (Bulk and
 * AllWells, Secs. 3.2.3-3.2.4), faces (BulkConn), assembly (LinearSystem,
 * Sec. 3.3.3) -- each run as one launch over a tile list of every grid's
 * cells, largest grids first, so small grids no longer leave most of the GPU
 * idle.  The paper partitions one grid over MPI ranks instead; batching
 * independent models on one GPU has no counterpart in it. */
typedef struct ocp_batch ocp_batch;

/* Device pointers of one model's inputs and outputs, as for ocp_linearize. */
typedef struct {
  const double* u_new;
  const int8_t* flag_new;
  const double* u_old;
  const int8_t* flag_old;
  double* residual;
  double* bsr_val;
  double* face_flux;      /* may be NULL */
} ocp_batch_io;

/* Launch shape of the three stages (0 cell, 1 face, 2 assembly): cells per
 * tile (32, 64, 128 or 256; one thread per cell) and CTAs per SM of a persistent
 * launch (1..64), or 0 for one CTA per tile.
 * ordered = 0: three launches, one per stage.  ordered = 1: the cell stage as
 * above, then one persistent launch in which each CTA claims the face stage
 * of one tile after another from a device counter, in tile order, and
 * assembles the tile's rows once the tiles holding their - neighbours have
 * finished their faces (tile size cells_per_tile[1]; ctas_per_sm[1] CTAs per
 * SM, 0: as many as fit).  ordered = 2: one persistent launch of both the
 * cell and the face stages, each tile's cell stage claimed ahead of the face
 * stages that need it.  The waits on other tiles are bounded: one that
 * expires makes ocp_get_status return OCP_ERR_TIMEOUT.  ordered = 3: three
 * launches, the face stage with one warp per direction and the assembly with
 * one warp per equation over 32-cell tiles (cell stage as set), which
 * shortens each warp's chain of FP64 instructions for small grids.
 * ordered = 4: the stages of ordered = 3 (cell stage on 32-cell tiles) in
 * one launch of one thread-block cluster, one CTA per 32-cell tile, the
 * stages separated by cluster barriers instead of launch boundaries; only
 * for a single grid (or a batch of one) of at most ocp_grid_cluster_tiles
 * tiles, other shapes being rejected with OCP_ERR_INVALID_ARG when set.
 * The tile sizes and CTA counts are ignored in this mode.
 * Results do not depend on the shape, bit for bit. */
typedef struct {
  int cells_per_tile[3];
  int ctas_per_sm[3];
  int ordered;
} ocp_launch_shape;

/* Groups n >= 1 grids (same device, same number of phases; each grid may
 * appear once).  Allocates the argument table and tile lists.  The grids
 * must outlive the batch; ocp_linearize on a member grid while a batch call
 * on it is in flight races on the grid's scratch. */
ocp_status ocp_batch_create(ocp_grid* const* grids, int n, ocp_batch** out);
ocp_status ocp_batch_destroy(ocp_batch* batch);      /* NULL is accepted */

/* Sets every model's input/output device pointers (host array io[n]).
 * Synchronises the device. */
ocp_status ocp_batch_set_io(ocp_batch* batch, const ocp_batch_io* io);

/* Linearises every model for the step dt (three launches on the stream).
 * When dt differs from the previous call the argument table is re-uploaded,
 * which synchronises the stream. */
ocp_status ocp_batch_linearize(ocp_batch* batch, double dt, void* cuda_stream);

/* Same as ocp_batch_linearize, but the three launches are captured once (on
 * a private stream) into a CUDA graph that is replayed on cuda_stream. */
ocp_status ocp_batch_graph_launch(ocp_batch* batch, double dt, void* cuda_stream);

/* Autotuner: times every stage as a plain launch (ordered = 0) with 4 tile
 * sizes x 6 grid sizes (median of reps after a warm-up) and keeps the
 * fastest per stage, then times the whole pass so found against the split
 * stages (ordered = 3, and ordered = 4 when the batch is one grid that fits
 * one cluster) and the ordered launches (modes 1 and 2, 4 tile sizes, 4 grid
 * sizes) and keeps the fastest; returns it in *best (may be NULL).
 * Synchronises the stream many times. */
ocp_status ocp_batch_tune(ocp_batch* batch, double dt, int reps, ocp_launch_shape* best, void* cuda_stream);
ocp_status ocp_batch_set_shape(ocp_batch* batch, const ocp_launch_shape* shape);
ocp_status ocp_batch_get_shape(const ocp_batch* batch, ocp_launch_shape* shape);

/* Sticky device status of every member grid (see ocp_get_status). */
ocp_status ocp_batch_get_status(ocp_batch* batch, void* cuda_stream);

/* Launch shape of ocp_linearize on one grid (for example one found by
 * ocp_batch_tune on a batch of that grid alone).  A new grid starts with one
 * CTA per tile and the largest tiles (128 cells for the cell and face stages,
 * 256 for assembly) that still give every SM two CTAs, halving down to 32
 * cells for small grids; grids of fewer than 64 cells per SM start with
 * ordered = 3, and grids that fit one cluster (ocp_grid_cluster_tiles) with
 * ordered = 4. */
ocp_status ocp_grid_set_shape(ocp_grid* grid, const ocp_launch_shape* shape);
/* The launch shape ocp_linearize currently uses on the grid. */
ocp_status ocp_grid_get_shape(const ocp_grid* grid, ocp_launch_shape* shape);
/* *tiles = the largest grid, in 32-cell tiles, that ordered = 4 accepts on
 * the grid's device: the largest thread-block cluster of the one-cluster
 * kernel the device can run, at most 16 (0 if none).  No counterpart in
 * the paper: a property of the launch, not of the method. */
ocp_status ocp_grid_cluster_tiles(const ocp_grid* grid, int* tiles);

/* ---------------------------------------------------------------- Newton step
 * The rest of the FIM nonlinear iteration of Sec. 3.2.5 -- the linear solve
 * and update of step 2, the convergence data of step 4 -- and what the
 * multi-step adjoint needs around ocp_adjoint_vjp. */

/* Device workspace (doubles) that ocp_bicgstab needs for this grid. */
int64_t ocp_solver_work_doubles(const ocp_grid* grid);

/* Solves A x = b (A^T x = b with transpose != 0) for the grid's block-CSR
 * matrix bsr_val by BiCGSTAB with a block-Jacobi preconditioner D (exact
 * inverses of the diagonal blocks, left preconditioning) until
 * ||D^-1 (b - A x)|| <= rtol ||D^-1 b|| or maxit iterations -- a residual
 * scaled cell by cell into the units of the unknowns.  x holds the initial guess
 * on entry and the solution on return; b and x are block-interleaved [nb*N]
 * device vectors; work is a device buffer of ocp_solver_work_doubles().
 * The iterations run as replays of a CUDA graph of eight iterations with the
 * convergence test on the device; the stream is synchronised once per replay.
 * The graph is captured on the first call and kept on the grid while the
 * same bsr_val, x, work (and well terms) are passed; calls on one grid must
 * not overlap from several host threads.  The paper solves with
 * CPR-preconditioned FGMRES in PETSc/Hypre (Sec. 5.1); this plain Krylov
 * solver serves the Newton, adjoint and test drivers.  Returns
 * OCP_ERR_TIMEOUT when maxit is reached, OCP_ERR_NONFINITE on breakdown;
 * *iters and *relres (may be NULL) report the final state. */
ocp_status ocp_bicgstab(ocp_grid* grid, const double* bsr_val, const double* b, double* x, double rtol,
                        int maxit, int transpose, double* work, int* iters, double* relres, void* cuda_stream);

/* Newton update u += scale * du (du block-interleaved, u and flag as for
 * ocp_linearize; scale = -1 applies the solution of J x = R), with every
 * cell's saturation changes scaled down to at most
 * ds_max, then the phase switch of undersaturated oil: a saturated cell whose
 * S_g falls below zero becomes undersaturated with X = R_s,sat(p); an
 * undersaturated cell whose R_s exceeds R_s,sat(p) becomes saturated with
 * S_g = 0.  Writes the largest |du| applied per variable to du_max (device,
 * nb + 1 doubles: p, S_w, then S_g and R_s with three phases; the third is
 * zero with two) and the number of switched cells to *nswitch (device int). */
ocp_status ocp_newton_update(ocp_grid* grid, double* u, int8_t* flag, const double* du, double scale,
                             double ds_max, double* du_max, int* nswitch, void* cuda_stream);

/* Adjoint of ocp_well_rates: for device cotangents q_bar[nwell*nb], ADDS
 * sum q_bar dq/du into g_u (variable-major like u; may be NULL) and
 * sum q_bar dq/d ln k into g_lnk[N] (may be NULL). */
ocp_status ocp_well_rates_vjp(ocp_grid* grid, const double* u, const int8_t* flag, const double* q_bar,
                              double* g_u, double* g_lnk, void* cuda_stream);

/* Recomputes the transmissibilities, their ln k weights and the well indices
 * from a new permeability field lnk[N] (device), as ocp_grid_create did. */
ocp_status ocp_grid_update_perm(ocp_grid* grid, const double* lnk, void* cuda_stream);

/* ---------------------------------------------------------------- wells as unknowns
 * The global Jacobian of Sec. 3.4.1 has rows and columns for the wells: each
 * well's bottom-hole pressure p_bh is an unknown with one equation, set by the
 * well's control (AllWells monitors the well pressure, Sec. 3.2.4).  A control
 * is a device array of nwell ocp_well_ctrl:
 *   mode 0: pressure control, R_w = p_bh - target (psi);
 *   mode 1: surface-rate control of component `phase` (0 water, 1 oil,
 *           nb-1 gas incl. dissolved gas), R_w = s sum_perf q_phase - target
 *           with s = -1 for producers (production positive), +1 for injectors;
 *   limit:  the pressure a rate-controlled producer may not fall below, or an
 *           injector may not rise above (ocp_well_update).
 * Perforation-indexed arrays follow the wells in order and each well's
 * perforations in the order of ocp_well.cells (nperf = sum of nperf). */
typedef struct {
  int32_t mode;
  int32_t phase;
  double target;
  double limit;
} ocp_well_ctrl;

/* ocp_linearize with the perforation sources evaluated at p_bh[nwell]
 * (device) instead of each well's fixed ocp_well.p_bh, plus the well rows and
 * columns: well_res[nwell] = R_w, well_b[nperf*nb] = dR_cell/dp_bh (row e of
 * the perforated cell), well_c[nperf*nb] = dR_w/du_cell (variable v of the
 * perforated cell; zero under pressure control) and well_d[nwell] =
 * dR_w/dp_bh (1 under pressure control).  All device, caller-owned.  A
 * control with a mode other than 0 and 1, a phase outside [0, nb), or rate
 * control of a well without perforations sets the sticky status
 * OCP_ERR_INVALID_ARG and is treated as pressure control. */
ocp_status ocp_linearize_wells(ocp_grid* grid, const double* u_new, const int8_t* flag_new,
                               const double* u_old, const int8_t* flag_old, double dt, const double* p_bh,
                               const ocp_well_ctrl* ctrl, double* residual, double* bsr_val, double* face_flux,
                               double* well_res, double* well_b, double* well_c, double* well_d,
                               void* cuda_stream);

/* Solves the system with well unknowns, [A B; C D][x; x_w] = [b; b_w]
 * (transposed: [A^T C^T; B^T D]), by eliminating the well unknowns: BiCGSTAB
 * as in ocp_bicgstab on the Schur complement A - B D^-1 C, applied next to
 * the block-CSR product (its block-Jacobi blocks include the perforated
 * cells' rank-one terms), with b - B D^-1 b_w, then x_w = D^-1 (b_w - C x).
 * B, C, D as written by ocp_linearize_wells; b, x [nb*N] block-interleaved,
 * b_w, x_w [nwell]; x holds the initial guess.  work: ocp_solver_work_doubles().
 * Every D entry must be nonzero (a rate-controlled well needs an open
 * perforation).  Errors as ocp_bicgstab; x_w is written in every case. */
ocp_status ocp_bicgstab_wells(ocp_grid* grid, const double* bsr_val, const double* well_b,
                              const double* well_c, const double* well_d, const double* b, const double* b_w,
                              double* x, double* x_w, double rtol, int maxit, int transpose, double* work,
                              int* iters, double* relres, void* cuda_stream);

/* p_bh += scale * dp (device, nwell), then the pressure monitoring: a
 * rate-controlled producer whose p_bh fell below its limit, or injector whose
 * p_bh rose above it, changes to pressure control (ctrl is updated in place:
 * mode 0, target = limit) with p_bh = limit.  Writes max |scale dp| to
 * *dp_max and the number of switched wells to *nswitch (both device). */
ocp_status ocp_well_update(ocp_grid* grid, double* p_bh, const double* dp, double scale, ocp_well_ctrl* ctrl,
                           double* dp_max, int* nswitch, void* cuda_stream);

/* Convergence measures of a linearisation (Sec. 3.2.5, step 4): norms[e] =
 * max over cells of |R[c*nb+e]| / (phi_c V_c / dt), V in reservoir barrels,
 * for e < nb; norms[3] = max over wells of |R_w| / max(|target|, 1) for
 * rate control and |R_w| for pressure control (0 without wells).  norms is a
 * device array of 4 doubles; maxima of non-negative values are exact and
 * independent of the order of evaluation. */
ocp_status ocp_residual_norms(ocp_grid* grid, const double* residual, double dt, const double* well_res,
                              const ocp_well_ctrl* ctrl, double* norms, void* cuda_stream);

/* ---------------------------------------------------------------- pressure and amounts
 * The paper's own unknowns (Sec. 2.1, eq. 4): per cell the pressure P and the
 * component amounts N_w, N_o[, N_g] in surface volumes per bulk volume,
 * variable-major [(nb+1)*N] (P, then N_w, ...).  The black-oil phase split is
 * explicit: V_w = N_w / b_w; all gas dissolved (R_s = N_g / N_o,
 * undersaturated oil) when N_g <= R_s,sat(P) N_o, else R_s = R_s,sat(P) and
 * free gas V_g = (N_g - R_s N_o) / b_g; S_j = V_j / V_f.  Equations: the
 * component balances (accumulation (N - N_old) V / dt, fluxes and fixed-BHP
 * wells as ocp_linearize) and the volume balance r_v = phi(P) - V_f. */

/* Linearises in (P, N) and eliminates N_w with every cell's volume-balance
 * row (Schur complement on the diagonal block).  Writes the reduced system
 * over (P, N_o[, N_g]): residual [nb*N] and bsr_val [nnzb*nb*nb] (the grid's
 * pattern, block-interleaved as for ocp_linearize), and elim [(nb+1)*N]
 * variable-major (c_P, c_o[, c_g], c_r) with which the N_w part of the
 * solution x of the full system is x_Nw = c_r - c_P x_P - c_o x_No [- c_g x_Ng].
 * With residual_full [(nb+1)*N] and/or bsr_val_full [nnzb*(nb+1)^2] (each
 * may be NULL) also the full system, rows water, oil[, gas], volume and
 * columns P, N_w, N_o[, N_g].  flag (device int8 [N], may be NULL) receives the
 * split's state (1: undersaturated).  The first call on a grid allocates the
 * split's per-cell data (32 doubles and a byte per cell with three phases, 18
 * and a byte with two), so it must not be the call captured into a CUDA
 * graph; later calls allocate nothing.  A non-finite input sets the sticky status OCP_ERR_NONFINITE. */
ocp_status ocp_linearize_pn(ocp_grid* grid, const double* pn_new, const double* pn_old, double dt,
                            double* residual, double* bsr_val, double* elim, double* residual_full,
                            double* bsr_val_full, int8_t* flag, void* cuda_stream);

/* pn += scale * x_full, where x_full is the solution of the full system built
 * from the reduced solution dx [nb*N] (block-interleaved P, N_o[, N_g]) and
 * elim.  dx_max (device, nb+1 doubles) receives max |scale x_full| per
 * unknown (P, N_w, N_o[, N_g]). */
ocp_status ocp_pn_update(ocp_grid* grid, double* pn, const double* dx, double scale, const double* elim,
                         double* dx_max, void* cuda_stream);

/* (P, N) [(nb+1)*N] of a natural state u, flag (as for ocp_linearize):
 * P = p and N = phi(p) S b per bulk volume (eq. 4), on the volume-balance
 * manifold. */
ocp_status ocp_pn_from_natural(ocp_grid* grid, const double* u, const int8_t* flag, double* pn, void* cuda_stream);

/* Convergence measures of the full (P, N) residual: norms[e] = max over cells
 * of |R_e| / (phi V / dt) for the component rows e < nb, norms[3] = max |r_v|
 * (device, 4 doubles). */
ocp_status ocp_pn_norms(ocp_grid* grid, const double* residual_full, double dt, double* norms, void* cuda_stream);

/* ---------------------------------------------------------------- IMPEC
 * One IMPEC step (implicit pressure, explicit composition) in the (P, N)
 * unknowns above: the volume balance at the new level, linearised about the
 * old one and multiplied by V/dt,
 *   (V/dt)(phi - V_f) + (V/dt)(phi' - V_f,P) dP + sum_i w_i (sum_faces F_i - Q_i) = 0,
 * w_i = dV_f/dN_i, with every face's phase flux F = T lambda_up (Phi_i - Phi_j)
 * linear in the new pressure (mobility, upwind side, density and capillary
 * offset frozen at the old level; dissolved gas with the oil's upwind R_s) and
 * the wells at the new cell pressure with old mobilities and open state; then
 * N^{n+1} = N^n + (Q - sum F) dt / V at the new pressure. */

/* Builds the pressure system A dP = rhs for the state pn [(nb+1)*N]: val
 * [nnzb] one value per block of the grid's 7-point pattern (row order as
 * ocp_bsr_pattern), rhs [N].  The old-level data are kept in the grid's
 * linearisation scratch for ocp_impec_update: no other call that uses the
 * grid's scratch (ocp_linearize, ocp_linearize_wells, ocp_linearize_pn) may
 * come between the two on the grid. */
ocp_status ocp_impec_pressure(ocp_grid* grid, const double* pn, double dt, double* val, double* rhs,
                              void* cuda_stream);

/* The explicit update after ocp_impec_pressure(pn_old, dt) and a solve for
 * dp [N]: pn_new = (P + dp, N + (Q - sum F) dt / V).  pn_new must not
 * overlap pn_old. */
ocp_status ocp_impec_update(ocp_grid* grid, const double* pn_old, const double* dp, double dt, double* pn_new,
                            void* cuda_stream);

/* ocp_bicgstab for a scalar system on the grid's pattern (one value per
 * block, e.g. the IMPEC pressure matrix), Jacobi preconditioned; b, x [N]. */
ocp_status ocp_bicgstab_scalar(ocp_grid* grid, const double* val, const double* b, double* x, double rtol,
                               int maxit, double* work, int* iters, double* relres, void* cuda_stream);

/* ---------------------------------------------------------------- adaptive coupling
 * The adaptively coupled domain decomposition of Sec. 4 decides at the start
 * of each time step which subdomains to solve together: (1) mark the cells
 * whose phase saturation changed by more than `threshold` (the paper uses
 * 5e-3) between (u_old, flag_old) and (u_new, flag_new); (2) couple a
 * subdomain that holds a marked cell with every neighbouring subdomain, and a
 * subdomain that sees a marked cell as a ghost with the subdomain owning it;
 * (3) take the connected components of that graph.  Subdomains are the boxes
 * of a px x py x pz split of the grid (box b along x holds the cells i with
 * floor(i px / nx) == b, likewise along y and z).  labels[px*py*pz] (device)
 * receives the smallest subdomain index of each subdomain's component; work
 * is a device buffer of ocp_coupling_work_ints() ints; afterwards, with
 * S = px py pz, work[2S] holds the number of marked cells, work[2S+1] the
 * union-find retries and work[2S+2] an error flag (nonzero if a loop bound
 * was reached, which the algorithm's invariants rule out).  Asynchronous on
 * cuda_stream; labels and work are caller-owned; capturable in a CUDA graph.
 * Returns OCP_ERR_INVALID_ARG for null pointers, px, py, pz outside
 * [1, cells per direction] or a negative / non-finite threshold. */
int64_t ocp_coupling_work_ints(int px, int py, int pz);
ocp_status ocp_coupling_components(ocp_grid* grid, const double* u_new, const int8_t* flag_new,
                                   const double* u_old, const int8_t* flag_old, double threshold, int px,
                                   int py, int pz, int32_t* labels, int32_t* work, void* cuda_stream);

/* Synchronises the stream, then returns and clears the grid's sticky device
 * status (OCP_OK if no kernel reported a problem since the last call). */
ocp_status ocp_get_status(ocp_grid* grid, void* cuda_stream);

/* Thread-local description of the last error returned on this thread. */
const char* ocp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OCP_H */
