// Internal definitions of the GB300 black-oil FIM linearisation library.
//
// Everything here is FP64.  On GB300 (sm_103) the FP64 pipe issues about two
// DFMA per SM clock -- 1/74 of the FP32 rate -- and an FP64 compare costs as
// much as an FMA, so the device code below is written to spend as few FP64
// instructions as possible: branch decisions on doubles are taken on their
// bit patterns with integer instructions, every per-grid constant (reciprocal
// normalisations, table slopes, transmissibilities, well indices) is
// precomputed once at set-up, and horizontal faces skip the gravity term,
// whose depth difference is zero there.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ocp.h"

namespace ocp {

constexpr int kMaxRows = 64;           // PVT table rows
constexpr double kRbFt3 = 5.614583;    // ft^3 per reservoir barrel
constexpr double kDarcy = 0.001127;    // rb cP / (day psi mD ft)
constexpr double kGrav = 1.0 / 144.0;  // psi per (lb/ft^3 ft)

// Sticky device status bits (ocp_get_status maps them to ocp_status).
enum : int { kStatNonFinite = 1, kStatBadFlag = 2, kStatTimeout = 4, kStatBadControl = 8 };

// Preprocessed PVT table: knots and, per linear piece k, value and slope of
// b_o = 1/B_o, 1/mu_o, b_g = 1/B_g, 1/mu_g and R_s versus p, plus the inverse
// piece p(R_s) for undersaturated oil.  Filled on the host at set-up.
struct alignas(16) Table {    // 16-byte size and alignment: one bulk copy moves it
  int nrow;
  double p[kMaxRows];
  double rs[kMaxRows];
  double y[5][kMaxRows];       // 0 b_o, 1 imu_o, 2 b_g, 3 imu_g, 4 R_s at the knots
  double s[5][kMaxRows];       // slope of piece k
  double q[kMaxRows];          // dp/dR_s of piece k (inverse of R_s(p))
  long long pkey[kMaxRows];    // order-preserving integer keys of p and R_s knots
  long long rskey[kMaxRows];
};

// Per-grid scalar constants, passed to kernels by value.
struct Params {
  int nx, ny, nz, nb;
  long long N, nxy;
  double dz;
  double p_ref, cr, bw_ref, cw, imu_w;
  double rho_osc, rho_wsc, cg;            // cg = rho_gsc / 5.614583
  double co, cmu;
  double swc, sorw, sorg, sgc;
  double inv_w, inv_g, inv_og;            // 1/(1-swc-sorw), 1/(1-swc-sgc-sorg), 1/(1-swc-sorg)
  double nw, now, ng, nog;                // Corey exponents
  int sq_w, sq_ow, sq_g, sq_og;           // exponent == 2 (use a product, not pow)
  double krw_max, krg_max, kc;
  double pcow_max, pcgo_max;
  double grav_dz;                         // 0.5 * g * dz: half the potential head per unit density
  double vol_rb;                          // cell bulk volume in rb
  unsigned long long nx_m, ny_m;          // exact division by nx and ny: q = (c * m) >> (32 + s)
  int nx_s, ny_s;
  double pcow2, pcgo2;                    // 2 Pc_max (derivative factors)
  double bw_p;                            // d b_w / dp
  double rw_p, bw_p_imu;                  // d rho_w / dp, (d b_w / dp) / mu_w
};

// Well perforation data on the device (one entry per perforated cell).
struct Perf {
  int cell;
  int well;
  int kind;       // 0 producer, 1 injector
  int phase;      // injected phase (0 water, 2 gas)
  double wi;      // Peaceman index including k of the cell
  double p_bh;
  double geom;    // C 2 pi dz / (ln(r_o / r_w) + skin): wi = k geom
};

// Launch shape of the three linearisation stages (cell, face, assemble):
// cells per tile (one of kTileSizes; a CTA has one thread per cell of its
// tile) and CTAs per SM (0: one CTA per tile).
struct LaunchCfg {
  int tpb[3];
  int ctas_per_sm[3];
  int ordered;     // 0: three launches; 1: cell launch + ordered face/assembly launch
                   // (tile size tpb[1], grid ctas_per_sm[1]); 2: one ordered launch;
                   // 3: three launches, face and assembly split by direction / equation;
                   // 4: one launch of one thread-block cluster, stages as in 3
};
constexpr int kMaxClusterTiles = 16;   // the largest cluster the hardware offers (non-portable)
constexpr int kNumTileSizes = 4;
constexpr int kTileSizes[kNumTileSizes] = {32, 64, 128, 256};
inline int tile_index(int tpb) {
  for (int t = 0; t < kNumTileSizes; ++t)
    if (kTileSizes[t] == tpb) return t;
  return -1;
}
// Default launch shape of one grid of N cells on an SM count `sms`: the
// largest tiles (128 for the register-heavy cell and face stages, 256 for
// assembly) that still give every SM at least two CTAs, down to 32-cell
// tiles; a grid too small for that (fewer than 64 cells per SM) takes the
// face stage split by direction and the assembly by equation, since its
// time is its warps' FP64 instruction count, not the SMs' throughput, and a
// grid of at most `max_cluster` 32-cell tiles runs all three stages in one
// cluster launch.
inline LaunchCfg default_cfg(long long N, int sms, int max_cluster = 0) {
  LaunchCfg c;
  const long long S = sms > 0 ? sms : 1;
  for (int s = 0; s < 3; ++s) {
    int t = s < 2 ? 128 : 256;
    while (t > 32 && N < 2LL * t * S) t /= 2;
    c.tpb[s] = t;
    c.ctas_per_sm[s] = 0;
  }
  c.ordered = N < 2LL * 32 * S ? 3 : 0;
  if (N > 0 && (N + 31) / 32 <= max_cluster) c.ordered = 4;
  return c;
}

}  // namespace ocp

// The opaque handle of the C interface.
struct ocp_grid {
  int device;
  ocp::Params prm;
  ocp::Table* d_table;       // device copy of the table
  ocp::Table h_table;
  int64_t nnzb;
  int32_t* d_row_ptr;
  int32_t* d_col_idx;
  double* d_trans;           // [3][N] transmissibility of the +x,+y,+z face (0 outside)
  double* d_wlnk;            // [3][N] dlnT/dln k_i of the +face for its lower cell
  double* d_phi;             // [N] reference porosity
  int32_t* d_perf_of_cell;   // [N] perforation index or -1
  ocp::Perf* d_perf;         // [nperf]
  int nperf;
  int nwell;
  int32_t* d_well_first;     // [nwell+1] perforations of well w: well_first[w] .. well_first[w+1]
  int* d_status;             // sticky device status word
  double* d_scratch;         // per-cell scratch of the linearisation
  double* d_static_scratch;  // the no-allocation entry point's library array on this device
  unsigned* d_sync;          // ordered launch: item counter, then cell and face flags per 32-cell tile
  double* d_pn;              // per-cell data of the (P, N) path, allocated on its first use
  int8_t* d_pn_flag;
  cudaStream_t solve_cap;    // private stream on which the solver's iterations are captured
  cudaGraphExec_t solve_exec;  // a block of solver iterations, valid for the buffers in solve_key
  const void* solve_key[8];
  int64_t scratch_doubles;
  ocp::LaunchCfg cfg;        // launch shape of the linearisation
  int sms;                   // SM count of the device
  int max_cluster;           // largest one-cluster launch (32-cell tiles) the device runs, 0 if none
  double dx, dy, kz_over_kx; // geometry kept for permeability updates
};

namespace ocp {

// Everything one model's linearisation reads and writes (device pointers).
struct ModelArgs {
  Params P;
  const Table* table;
  const double* trans;
  const int32_t* row_ptr;
  const double* phi;
  const int32_t* perf_of_cell;
  const Perf* perf;
  int* status;
  double* scr;
  const double* u_new;
  const int8_t* f_new;
  const double* u_old;
  const int8_t* f_old;
  double* res;
  double* val;
  double* face_flux;
  double scale;              // bulk volume in rb / dt
  const double* p_bh;        // per-well bottom-hole pressures, or null for each perforation's own
  int no_acc;                // 1: leave the accumulation out (the (P, N) path adds its own)
};

// Tiles of `TPB` consecutive cells: with models == nullptr the single model
// passed by value, tile t starting at cell t * TPB; otherwise tiles[t] =
// (model, first cell).
struct TileList {
  const ModelArgs* models;
  const int2* tiles;
  int ntiles;
};

// The work list of the ordered (persistent) launch of the linearisation.
// With models == nullptr: the single model passed by value.  Otherwise the
// models in the order order[0..nmodels); tile_start[j] = tiles of the models
// before the j-th (so its tile flags start there, and its items at that
// number times the items per tile).
struct OrderedList {
  const ModelArgs* models;
  const int* order;
  const long long* tile_start;   // [nmodels + 1]
  int nmodels;
  long long nitems;
  unsigned* counter;             // next item (zero before the launch)
  int* flag_cell;                // per tile: cell stage done (zero before the launch)
  int* flag_face;                // per tile: face stage done (zero before the launch)
};

}  // namespace ocp

namespace ocp {

// ------------------------------------------------------------ cell indices
// Division of a non-negative 32-bit c by an invariant d as a multiply and a
// shift (the round-up method: m = floor(2^(32+s)/d) + 1, s = ceil(log2 d),
// exact for every 32-bit c).  Integer division is otherwise a long
// instruction sequence with a reciprocal; the cell index is split in every
// kernel, so this keeps the integer work off the FP64 kernels' critical path.
__host__ __device__ inline void div_magic(unsigned d, unsigned long long& m, int& s) {
  s = 0;
  while ((1ull << s) < d) ++s;
  m = ((1ull << (32 + s)) / d) + 1;
}
__device__ __forceinline__ int fdiv(int c, unsigned long long m, int s) {
  return (int)(((unsigned long long)(unsigned)c * m) >> (32 + s));
}
// (i, j, k) of cell c
__device__ __forceinline__ void cell_ijk(const Params& P, long long c, int& i, int& j, int& k) {
  const int ci = (int)c;
  const int q = fdiv(ci, P.nx_m, P.nx_s);
  i = ci - q * P.nx;
  k = fdiv(q, P.ny_m, P.ny_s);
  j = q - k * P.ny;
}
// Number of stored blocks in the rows before cell c = (i, j, k): 7 per
// earlier cell minus the missing neighbours of every earlier cell, in
// closed form.
__device__ __forceinline__ long long row_start_ijk(const Params& P, long long c, int i, int j, int k) {
  const long long nx = P.nx, nxy = P.nxy, N = P.N;
  const long long q = (long long)k * P.ny + j;            // c / nx
  const long long i0 = q + (i > 0);                        // earlier cells with i == 0
  const long long iL = q;                                  // ... with i == nx-1
  const long long rem = (long long)j * nx + i;             // c % nxy
  const long long j0 = k * nx + (rem < nx ? rem : nx);     // ... with j == 0
  const long long jL = k * nx + (rem > nxy - nx ? rem - (nxy - nx) : 0);
  const long long k0 = c < nxy ? c : nxy;                  // ... with k == 0
  const long long kL = c > N - nxy ? c - (N - nxy) : 0;    // ... with k == nz-1
  return 7 * c - (i0 + iL + j0 + jL + k0 + kL);
}

// ------------------------------------------------- programmatic launches
// The hot kernels are launched with programmatic stream serialisation
// (launch_pdl): the launch of one overlaps the end of the kernel before it on
// the stream.  Each begins with pdl_wait(), which returns once every grid it
// depends on has completed and its memory is visible, before it touches any
// global memory.  No kernel triggers its dependents early: measured on the
// 200 000-cell step, an early trigger made the SpMV slower (26.0 against
// 25.7 us), while the overlapped launch alone cut the serial end-to-end step
// from 1.85 to 1.70 ms and the 300-cell linearisation's stream launches from
// 31 to 25 us.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*kern)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

// ------------------------------------------------------- PVT table staging
// Polls an mbarrier's phase `parity` at most 2^20 times; false if it never
// completed.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 20); ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Copies the PVT table of a model into the CTA's shared memory with one
// bulk asynchronous copy (the TMA unit) that completes on the mbarrier
// `bar`; every thread of the CTA calls it and returns once the table has
// arrived.  `uses` counts the loads this CTA has made with `bar` (the
// mbarrier's phase).  The table is 16-byte aligned and sized (cudaMalloc'd,
// alignas(16)), as the copy requires.  The wait is bounded: a thread past
// its limit records kStatTimeout and waits once more for the copy in flight.
// Callers that reload the table must make sure no thread still reads the
// previous one (a barrier before the call).
// The two halves of load_table, for callers that issue other loads while the
// copy is in flight: table_copy_issue (thread 0 starts the copy; call it from
// every thread), then table_copy_wait (every thread).
__device__ __forceinline__ void table_copy_issue(Table& T, const Table* src, unsigned long long& bar, unsigned uses) {
  const unsigned ubar = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    if (uses == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ubar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ubar), "r"((unsigned)sizeof(Table))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (unsigned)__cvta_generic_to_shared(&T)),
                 "l"(src), "r"((unsigned)sizeof(Table)), "r"(ubar)
                 : "memory");
  }
}
__device__ __forceinline__ void table_copy_wait(unsigned long long& bar, unsigned& uses, int* status) {
  const unsigned ubar = (unsigned)__cvta_generic_to_shared(&bar);
  __syncthreads();                       // the mbarrier is initialised before anyone waits on it
  if (!mbar_wait(ubar, uses & 1u)) {
    atomicOr(status, kStatTimeout);
    mbar_wait(ubar, uses & 1u);
  }
  ++uses;
}
__device__ __forceinline__ void load_table(Table& T, const Table* src, unsigned long long& bar, unsigned& uses,
                                           int* status) {
  table_copy_issue(T, src, bar, uses);
  table_copy_wait(bar, uses, status);
}

// ---------------------------------------------------------------- bit tricks
// Order-preserving signed integer key of a double (total order on non-NaN).
__host__ __device__ inline long long dkey(double x) {
#ifdef __CUDA_ARCH__
  long long b = __double_as_longlong(x);
#else
  long long b;
  __builtin_memcpy(&b, &x, 8);
#endif
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// x >= 0 (true for +0 and -0), without an FP64 compare.
__device__ __forceinline__ bool nonneg(double x) { return dkey(x) >= dkey(-0.0); }
// x > 0 strictly.
__device__ __forceinline__ bool positive(double x) { return dkey(x) > 0; }
__device__ __forceinline__ bool finite(double x) {
  return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ double sel(bool c, double a, double b) { return c ? a : b; }

// Largest k <= nrow-2 with key[k] <= xk (binary search on integer keys).
__device__ __forceinline__ int segment(const long long* key, int nrow, long long xk) {
  int lo = 0, hi = nrow - 2;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (key[mid] <= xk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Power with a constant exponent >= 1 and its derivative; exponent 2 uses a
// product.  s is already clamped to [0, 1].
__device__ __forceinline__ void cpow(double s, double n, int sq, double& v, double& d) {
  if (sq) { v = s * s; d = s + s; }
  else { v = pow(s, n); d = n * pow(s, n - 1.0); }
}

// Clamp a normalised saturation to [0, 1]: outside, value clamped and slope 0.
__device__ __forceinline__ void clamp01(double& s, double& ds) {
  if (!nonneg(s)) { s = 0.0; ds = 0.0; }
  else if (dkey(s) > dkey(1.0)) { s = 1.0; ds = 0.0; }
}

// ------------------------------------------------------------ cell quantities
// Quantities of one cell that the face and well terms need, with derivatives
// with respect to the cell's own unknowns (p, S_w, X).  Two-phase cells use
// the water/oil entries only.
struct CellQ {
  double p, pw, pg;            // phase pressures (p_o = p)
  double dpw_sw, dpg_x;        // the only non-unit pressure derivatives
  double rw, rw_p;             // densities
  double ro, ro_p, ro_x;
  double rg, rg_p;
  double lw, lw_p, lw_sw;      // mobilities k_r b / mu
  double lo, lo_p, lo_sw, lo_x;
  double lg, lg_p, lg_x;
  double rs, rs_p, rs_x;       // dissolved gas-oil ratio
};

// Extra per-cell quantities for accumulation and injectors.
struct CellAux {
  double m[3], m_p[3], m_sw[3], m_x[3];    // phi S b per component, with derivatives
  double mob, mob_p, mob_sw, mob_x;         // total mobility sum k_r / mu
  double bw, bw_p, bg, bg_p;                // injected-phase b and its p-derivative
};

// Fluid (PVT module) quantities of one cell with their derivatives with
// respect to (p, X); saturated cells read the tables at p, undersaturated
// cells at the bubble point of their R_s (Sec. 3.2.3, PVT).  VISC also
// evaluates the reciprocal viscosities.
struct Pvt {
  double bw, bw_p;
  double bo, bo_p, bo_x, imo, imo_p, imo_x;
  double rs, rs_p, rs_x, sg, sg_x;
  double bg, bg_p, img, img_p;
};

template <int NB, bool VISC>
__device__ __forceinline__ void pvt(const Params& P, const Table& T, double p, double x, int flag, Pvt& f) {
  const double t = p - P.p_ref;
  f.bw = P.bw_ref * fma(P.cw, t, 1.0);
  f.bw_p = P.bw_p;
  const int kp = segment(T.pkey, T.nrow, dkey(p));
  const double dpk = p - T.p[kp];
  f.imo = f.imo_p = f.imo_x = 0.0;
  f.bg = f.bg_p = f.img = f.img_p = 0.0;
  if (NB == 3 && flag == 1) {
    const int kr = segment(T.rskey, T.nrow, dkey(x));
    const double pb = fma(x - T.rs[kr], T.q[kr], T.p[kr]);
    const double pb_x = T.q[kr];
    const double dpb = pb - T.p[kr];
    const double dp = p - pb;
    const double bsat = fma(dpb, T.s[0][kr], T.y[0][kr]);
    const double fb = fma(P.co, dp, 1.0);
    f.bo = bsat * fb;
    f.bo_p = bsat * P.co;
    f.bo_x = (T.s[0][kr] * fb - f.bo_p) * pb_x;
    if (VISC) {
      const double isat = fma(dpb, T.s[1][kr], T.y[1][kr]);
      const double fm = fma(-P.cmu, dp, 1.0);
      f.imo = isat * fm;
      f.imo_p = -isat * P.cmu;
      f.imo_x = (T.s[1][kr] * fm - f.imo_p) * pb_x;
    }
    f.rs = x; f.rs_p = 0.0; f.rs_x = 1.0;
    f.sg = 0.0; f.sg_x = 0.0;
  } else {
    f.bo = fma(dpk, T.s[0][kp], T.y[0][kp]);
    f.bo_p = T.s[0][kp]; f.bo_x = 0.0;
    if (VISC) {
      f.imo = fma(dpk, T.s[1][kp], T.y[1][kp]);
      f.imo_p = T.s[1][kp];
    }
    if (NB == 3) {
      f.rs = fma(dpk, T.s[4][kp], T.y[4][kp]);
      f.rs_p = T.s[4][kp];
      f.sg = x; f.sg_x = 1.0;
    } else {
      f.rs = 0.0; f.rs_p = 0.0;
      f.sg = 0.0; f.sg_x = 0.0;
    }
    f.rs_x = 0.0;
  }
  if (NB == 3) {
    f.bg = fma(dpk, T.s[2][kp], T.y[2][kp]);
    f.bg_p = T.s[2][kp];
    if (VISC) {
      f.img = fma(dpk, T.s[3][kp], T.y[3][kp]);
      f.img_p = T.s[3][kp];
    }
  }
}

// Component amounts per bulk volume, phi S b (eq. 4 in black-oil form), and
// with DERIV their derivatives with respect to (p, S_w, X).  Used for both
// time levels, so that an unchanged state gives an exactly zero accumulation.
// PART 2 computes every component, PART 0 only water and oil, PART 1 only
// gas (so that the components can be split between warps).
template <int NB, bool DERIV, int PART = 2>
__device__ __forceinline__ void masses(const Params& P, const Pvt& f, double p, double sw, double phi_ref,
                                       double* m, double* m_p, double* m_sw, double* m_x) {
  const double phi = phi_ref * fma(P.cr, p - P.p_ref, 1.0);
  const double so = (NB == 3) ? (1.0 - sw - f.sg) : (1.0 - sw);
  const double sob = so * f.bo;
  if (PART != 1) {
    m[0] = phi * sw * f.bw;
    m[1] = phi * sob;
  }
  if (PART != 0 && NB == 3) m[2] = phi * fma(f.sg, f.bg, f.rs * sob);
  if (DERIV) {
    const double phi_p = phi_ref * P.cr;
    const double so_x = -f.sg_x;
    if (PART != 1) {
      m_p[0] = fma(phi_p * sw, f.bw, phi * sw * f.bw_p);
      m_sw[0] = phi * f.bw;
      m_x[0] = 0.0;
      m_p[1] = fma(phi_p, sob, phi * so * f.bo_p);
      m_sw[1] = -phi * f.bo;
      m_x[1] = phi * fma(so_x, f.bo, so * f.bo_x);
    }
    if (PART != 0 && NB == 3) {
      const double G = fma(f.sg, f.bg, f.rs * sob);
      const double G_p = fma(f.sg, f.bg_p, fma(f.rs_p, sob, f.rs * so * f.bo_p));
      const double G_x = fma(f.sg_x, f.bg, fma(f.rs_x, sob, f.rs * fma(so_x, f.bo, so * f.bo_x)));
      m_p[2] = fma(phi_p, G, phi * G_p);
      m_sw[2] = -phi * f.rs * f.bo;
      m_x[2] = phi * G_x;
    }
  }
}

// Relative permeabilities of one cell (Corey; Stone II for oil with three
// phases, SAT module of Sec. 3.2.3) with their derivatives in (S_w, X), and
// the clamped normalised saturations the capillary pressures use.  `sg` is
// the cell's gas saturation: X in saturated three-phase cells, else 0.
struct Kr {
  double krw, krw_sw, kro, kro_sw, kro_x, krg, krg_x;
  double s_w, s_w_d, s_g, s_g_d;
  bool gx;                     // X is S_g (sg_x is 1 there and 0 otherwise)
};

// The water side (S_w, the oil-water curve) and the gas side (S_g, the
// oil-gas curve) of the relative permeabilities are independent; rel_perm
// combines them (so that the two sides can also run in different warps).
struct KrSide {
  double s, s_d;               // clamped normalised S_w or S_g and its slope
  double so_d;                 // slope of the normalised oil saturation of the curve
  double po, dpo;              // (s_ow or s_og)^n and its derivative
  double kr, kr_d;             // k_rw or k_rg and its derivative in S_w or S_g
};
__device__ __forceinline__ void rel_perm_w(const Params& P, double sw, KrSide& w) {
  double s_w = (sw - P.swc) * P.inv_w, s_w_d = P.inv_w;
  clamp01(s_w, s_w_d);
  double s_ow = (1.0 - sw - P.sorw) * P.inv_w, s_ow_d = -P.inv_w;
  clamp01(s_ow, s_ow_d);
  double pw_, dw_, pow_, dow_;
  cpow(s_w, P.nw, P.sq_w, pw_, dw_);
  cpow(s_ow, P.now, P.sq_ow, pow_, dow_);
  w.s = s_w;
  w.s_d = s_w_d;
  w.so_d = s_ow_d;
  w.po = pow_;
  w.dpo = dow_;
  w.kr = P.krw_max * pw_;
  w.kr_d = P.krw_max * dw_ * s_w_d;
}
__device__ __forceinline__ void rel_perm_g(const Params& P, double sg, KrSide& g) {
  double s_g = (sg - P.sgc) * P.inv_g, s_g_d = P.inv_g;
  clamp01(s_g, s_g_d);
  double s_og = (1.0 - sg - P.swc - P.sorg) * P.inv_og, s_og_d = -P.inv_og;
  clamp01(s_og, s_og_d);
  double pg_, dg_, pog_, dog_;
  cpow(s_g, P.ng, P.sq_g, pg_, dg_);
  cpow(s_og, P.nog, P.sq_og, pog_, dog_);
  g.s = s_g;
  g.s_d = s_g_d;
  g.so_d = s_og_d;
  g.po = pog_;
  g.dpo = dog_;
  g.kr = P.krg_max * pg_;
  g.kr_d = P.krg_max * dg_ * s_g_d;
}
// k_ro (Stone II with three phases, the oil-water curve with two) from the
// two sides; the sums are explicitly rounded so that they never take in a
// product from the side computations, wherever those ran.
template <int NB>
__device__ __forceinline__ void rel_perm_combine(const Params& P, const KrSide& w, const KrSide& g, int flag,
                                                 Kr& k) {
  double kro, kro_sw, kro_sg = 0.0, krg = 0.0, krg_sg = 0.0, s_g = 0.0, s_g_d = 0.0;
  if (NB == 3) {
    krg = g.kr;
    krg_sg = g.kr_d;
    s_g = g.s;
    s_g_d = g.s_d;
    // k_ro = kc [(k_row/kc + k_rw)(k_rog/kc + k_rg) - (k_rw + k_rg)], k_row/kc = s_ow^n
    const double A = __dadd_rn(w.po, w.kr);
    const double A_sw = fma(w.dpo, w.so_d, w.kr_d);
    const double B = __dadd_rn(g.po, krg);
    const double B_sg = fma(g.dpo, g.so_d, krg_sg);
    kro = P.kc * fma(A, B, -__dadd_rn(w.kr, krg));
    kro_sw = P.kc * fma(A_sw, B, -w.kr_d);
    kro_sg = P.kc * fma(A, B_sg, -krg_sg);
    if (!nonneg(kro)) { kro = 0.0; kro_sw = 0.0; kro_sg = 0.0; }
  } else {
    kro = P.kc * w.po;
    kro_sw = P.kc * w.dpo * w.so_d;
  }
  const bool gx = (NB == 3) && (flag == 0);
  k.krw = w.kr;
  k.krw_sw = w.kr_d;
  k.kro = kro;
  k.kro_sw = kro_sw;
  k.kro_x = gx ? kro_sg : 0.0;
  k.krg = krg;
  k.krg_x = gx ? krg_sg : 0.0;
  k.s_w = w.s;
  k.s_w_d = w.s_d;
  k.s_g = s_g;
  k.s_g_d = s_g_d;
  k.gx = gx;
}

template <int NB>
__device__ __forceinline__ void rel_perm(const Params& P, double sw, double sg, int flag, Kr& k) {
  KrSide w, g{};
  rel_perm_w(P, sw, w);
  if (NB == 3) rel_perm_g(P, sg, g);
  rel_perm_combine<NB>(P, w, g, flag, k);
}

// Capillary pressures: p_w = p - Pc_ow(S_w), p_g = p + Pc_go(S_g).
template <int NB>
__device__ __forceinline__ void cap_pressure(const Params& P, double p, const Kr& k, CellQ& q) {
  const double omw = 1.0 - k.s_w;
  q.p = p;
  q.pw = p - P.pcow_max * (omw * omw);
  q.dpw_sw = P.pcow2 * omw * k.s_w_d;
  if (NB == 3) {
    q.pg = p + P.pcgo_max * (k.s_g * k.s_g);
    q.dpg_x = k.gx ? P.pcgo2 * k.s_g * k.s_g_d : 0.0;
  }
}

// Phase densities and mobilities lambda = k_r b / mu with their derivatives:
// water and gas (WG), oil (O), or all.
template <int NB, bool WG = true, bool O = true>
__device__ __forceinline__ void dens_mob(const Params& P, const Pvt& f, const Kr& k, CellQ& q) {
  if (WG) {
    q.rw = f.bw * P.rho_wsc;
    q.rw_p = P.rw_p;
    if (NB == 3) {
      q.rg = f.bg * P.cg;
      q.rg_p = f.bg_p * P.cg;
    }
    const double bmw = f.bw * P.imu_w;
    q.lw = k.krw * bmw;
    q.lw_p = k.krw * P.bw_p_imu;
    q.lw_sw = k.krw_sw * bmw;
    if (NB == 3) {
      const double bmg = f.bg * f.img;
      q.lg = k.krg * bmg;
      q.lg_p = k.krg * fma(f.bg_p, f.img, f.bg * f.img_p);
      q.lg_x = k.krg_x * bmg;
      q.rs = f.rs; q.rs_p = f.rs_p; q.rs_x = f.rs_x;
    }
  }
  if (!O) return;
  const double ro0 = fma(f.rs, P.cg, P.rho_osc);
  q.ro = ro0 * f.bo;
  q.ro_p = fma(P.cg * f.rs_p, f.bo, ro0 * f.bo_p);
  q.ro_x = fma(P.cg * f.rs_x, f.bo, ro0 * f.bo_x);
  const double bmo = f.bo * f.imo;
  const double bmo_p = fma(f.bo_p, f.imo, f.bo * f.imo_p);
  const double bmo_x = fma(f.bo_x, f.imo, f.bo * f.imo_x);
  q.lo = k.kro * bmo;
  q.lo_p = k.kro * bmo_p;
  q.lo_sw = k.kro_sw * bmo;
  q.lo_x = fma(k.kro_x, bmo, k.kro * bmo_x);
}

// Total mobility sum k_r / mu and the injected phases' b (injector cells;
// zero elsewhere).
template <int NB>
__device__ __forceinline__ void total_mob(const Params& P, const Pvt& f, const Kr& k, bool injector,
                                          CellAux& a) {
  a.mob = a.mob_p = a.mob_sw = a.mob_x = 0.0;
  if (!injector) {
  } else if (NB == 3) {
    a.mob = fma(k.krw, P.imu_w, fma(k.kro, f.imo, k.krg * f.img));
    a.mob_p = fma(k.kro, f.imo_p, k.krg * f.img_p);
    a.mob_sw = fma(k.krw_sw, P.imu_w, k.kro_sw * f.imo);
    a.mob_x = fma(k.kro_x, f.imo, fma(k.kro, f.imo_x, k.krg_x * f.img));
    a.bg = f.bg; a.bg_p = f.bg_p;
  } else {
    a.mob = fma(k.krw, P.imu_w, k.kro * f.imo);
    a.mob_p = k.kro * f.imo_p;
    a.mob_sw = fma(k.krw_sw, P.imu_w, k.kro_sw * f.imo);
    a.mob_x = 0.0;
  }
  a.bw = f.bw; a.bw_p = f.bw_p;
}

// PVT, rock, Corey / Stone II, capillary pressure, densities and mobilities
// of one cell (Bulk: PVT, SAT, ROCK modules, Sec. 3.2.3); with AUX also the
// component amounts and (for injector cells) the total mobility.  The
// amounts are phi_ref S b scaled by whatever factor phi_ref carries.
template <int NB, bool AUX>
__device__ __forceinline__ void cell_quantities(const Params& P, const Table& T, double p, double sw,
                                                double x, int flag, double phi_ref, CellQ& q,
                                                CellAux& a, bool injector = true) {
  Pvt f;
  pvt<NB, true>(P, T, p, x, flag, f);
  Kr k;
  rel_perm<NB>(P, sw, f.sg, flag, k);
  cap_pressure<NB>(P, p, k, q);
  dens_mob<NB>(P, f, k, q);
  if (AUX) {
    masses<NB, true>(P, f, p, sw, phi_ref, a.m, a.m_p, a.m_sw, a.m_x);
    total_mob<NB>(P, f, k, injector, a);
  }
}

// Component amounts only (values, or values and derivatives), for the old
// time level and for the adjoint; no saturation functions are needed there.
template <int NB, bool DERIV>
__device__ __forceinline__ void cell_masses(const Params& P, const Table& T, double p, double sw,
                                            double x, int flag, double phi_ref, double* m,
                                            double* m_p = nullptr, double* m_sw = nullptr,
                                            double* m_x = nullptr) {
  Pvt f;
  pvt<NB, false>(P, T, p, x, flag, f);
  masses<NB, DERIV>(P, f, p, sw, phi_ref, m, m_p, m_sw, m_x);
}

// ---------------------------------------------------------------- face flux
// Sign flip without an FP64 instruction.
__device__ __forceinline__ double neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// One phase across one face: F = T lambda_up dphi with dphi = (pa_i - pa_j)
// - gbar (z_i - z_j), gbar = g (rho_i + rho_j) / 2, and its derivatives in
// the unknowns (p, S_w, X) of both cells.  `hz` = g (z_i - z_j) / 2; on
// horizontal faces (GRAV false) it is zero and the gravity arithmetic is not
// emitted.  The flags say which dependencies exist, so structural zeros cost
// no FP64 instruction:
//   PSW  the phase pressure depends on S_w (water, through Pc_ow), d = dpa;
//   PX   the phase pressure depends on X (gas, through Pc_go), d = dpa;
//   RX   the density depends on X (oil, through R_s);
//   LSW, LX  the mobility depends on S_w, X.
template <bool GRAV, bool PSW, bool PX, bool RX, bool LSW, bool LX>
__device__ __forceinline__ void phase_flux(double T, double hz, double pa_i, double pa_j, double dpa_i,
                                           double dpa_j, double rho_i, double rho_j, double rho_p_i,
                                           double rho_p_j, double rho_x_i, double rho_x_j, double l_i,
                                           double l_j, double l_p_i, double l_p_j, double l_sw_i,
                                           double l_sw_j, double l_x_i, double l_x_j, double& F,
                                           double (&di)[3], double (&dj)[3], bool& up) {
  double dphi = pa_i - pa_j;
  if (GRAV) dphi = fma(-(rho_i + rho_j), hz, dphi);
  up = nonneg(dphi);
  const double Tl = T * sel(up, l_i, l_j);
  const double Td = T * dphi;
  F = Tl * dphi;
  const double ulp = Td * sel(up, l_p_i, l_p_j);
  if (GRAV) {
    di[0] = fma(Tl, fma(-rho_p_i, hz, 1.0), sel(up, ulp, 0.0));
    dj[0] = fma(Tl, fma(-rho_p_j, hz, -1.0), sel(up, 0.0, ulp));
  } else {
    di[0] = Tl + sel(up, ulp, 0.0);
    dj[0] = sel(up, 0.0, ulp) - Tl;
  }
  double usw = 0.0;
  if (LSW) usw = Td * sel(up, l_sw_i, l_sw_j);
  if (PSW) {
    di[1] = fma(Tl, dpa_i, sel(up, usw, 0.0));
    dj[1] = fma(neg(Tl), dpa_j, sel(up, 0.0, usw));
  } else {
    di[1] = sel(up, usw, 0.0);
    dj[1] = sel(up, 0.0, usw);
  }
  double ux = 0.0;
  if (LX) ux = Td * sel(up, l_x_i, l_x_j);
  constexpr bool CX = PX || (GRAV && RX);   // dphi depends on X
  if (CX) {
    double cx_i, cx_j;
    if (PX) {
      cx_i = dpa_i;
      cx_j = neg(dpa_j);
    } else {
      cx_i = neg(rho_x_i * hz);
      cx_j = neg(rho_x_j * hz);
    }
    di[2] = fma(Tl, cx_i, sel(up, ux, 0.0));
    dj[2] = fma(Tl, cx_j, sel(up, 0.0, ux));
  } else {
    di[2] = sel(up, ux, 0.0);
    dj[2] = sel(up, 0.0, ux);
  }
}

// Flux of every component across one face (i -> j, j the + neighbour) and
// its derivatives with respect to both cells' unknowns (BulkConn, Sec. 3.2.4;
// Darcy's law eq. 2 in two-point form, phase-upwinded).
template <int NB>
struct FaceOut {
  double F[NB];
  double di[NB][3];   // dF_e / du_i[v]
  double dj[NB][3];   // dF_e / du_j[v]
};

// The three phases across one face (water, oil, gas) as separate calls, so
// that a face can also be computed one phase per warp; face_terms chains
// them.  a is cell i, b its + neighbour j.
template <int NB, bool GRAV>
__device__ __forceinline__ void water_flux(double T, double hz, const CellQ& a, const CellQ& b, double& F,
                                           double (&di)[3], double (&dj)[3], bool& up) {
  // water: p_w = p - Pc_ow(S_w); rho_w and lambda_w depend on p and S_w
  phase_flux<GRAV, true, false, false, true, false>(T, hz, a.pw, b.pw, a.dpw_sw, b.dpw_sw, a.rw, b.rw, a.rw_p,
                                                     b.rw_p, 0.0, 0.0, a.lw, b.lw, a.lw_p, b.lw_p, a.lw_sw,
                                                     b.lw_sw, 0.0, 0.0, F, di, dj, up);
}
template <int NB, bool GRAV>
__device__ __forceinline__ void oil_flux(double T, double hz, const CellQ& a, const CellQ& b, double& F,
                                         double (&di)[3], double (&dj)[3], bool& up) {
  // oil: p_o = p; rho_o and lambda_o depend on X only with three phases
  phase_flux<GRAV, false, false, NB == 3, true, NB == 3>(T, hz, a.p, b.p, 0.0, 0.0, a.ro, b.ro, a.ro_p, b.ro_p,
                                                          a.ro_x, b.ro_x, a.lo, b.lo, a.lo_p, b.lo_p, a.lo_sw,
                                                          b.lo_sw, a.lo_x, b.lo_x, F, di, dj, up);
}
template <int NB, bool GRAV>
__device__ __forceinline__ void gas_flux(double T, double hz, const CellQ& a, const CellQ& b, double& F,
                                         double (&di)[3], double (&dj)[3], bool& up) {
  // gas: p_g = p + Pc_go(S_g); rho_g depends on p, lambda_g on p and X
  phase_flux<GRAV, false, true, false, false, true>(T, hz, a.pg, b.pg, a.dpg_x, b.dpg_x, a.rg, b.rg, a.rg_p,
                                                     b.rg_p, 0.0, 0.0, a.lg, b.lg, a.lg_p, b.lg_p, 0.0, 0.0,
                                                     a.lg_x, b.lg_x, F, di, dj, up);
}
// The gas component: free gas plus the gas dissolved in the upstream oil
// (Fo, di_o, dj_o, up_o the oil phase; Fg, dg_i, dg_j the gas phase).
__device__ __forceinline__ void gas_component(const CellQ& a, const CellQ& b, bool up_o, double Fo,
                                              const double (&di_o)[3], const double (&dj_o)[3], double Fg,
                                              const double (&dg_i)[3], const double (&dg_j)[3], double& F,
                                              double (&di)[3], double (&dj)[3]) {
  const double rsu = sel(up_o, a.rs, b.rs);
  F = fma(rsu, Fo, Fg);
  const double frp = Fo * sel(up_o, a.rs_p, b.rs_p);
  const double frx = Fo * sel(up_o, a.rs_x, b.rs_x);
  di[0] = fma(rsu, di_o[0], dg_i[0]) + sel(up_o, frp, 0.0);
  dj[0] = fma(rsu, dj_o[0], dg_j[0]) + sel(up_o, 0.0, frp);
  di[1] = rsu * di_o[1];
  dj[1] = rsu * dj_o[1];
  di[2] = fma(rsu, di_o[2], dg_i[2]) + sel(up_o, frx, 0.0);
  dj[2] = fma(rsu, dj_o[2], dg_j[2]) + sel(up_o, 0.0, frx);
}

template <int NB, bool GRAV>
__device__ __forceinline__ void face_terms(double T, double hz, const CellQ& a, const CellQ& b,
                                           FaceOut<NB>& o) {
  bool up_w, up_o;
  water_flux<NB, GRAV>(T, hz, a, b, o.F[0], o.di[0], o.dj[0], up_w);
  oil_flux<NB, GRAV>(T, hz, a, b, o.F[1], o.di[1], o.dj[1], up_o);
  if (NB == 3) {
    double Fg, dg_i[3], dg_j[3];
    bool up_g;
    gas_flux<NB, GRAV>(T, hz, a, b, Fg, dg_i, dg_j, up_g);
    gas_component(a, b, up_o, o.F[1], o.di[1], o.dj[1], Fg, dg_i, dg_j, o.F[NB - 1], o.di[NB - 1],
                  o.dj[NB - 1]);
  }
}

// ---------------------------------------------------------------- wells
// Producer terms q_a = WI lambda_a (p_bh - p) by phase (g = p_bh - p < 0):
// well_source chains them; they can also run in different warps.
__device__ __forceinline__ void well_prod_water(const Perf& w, const CellQ& q, double g, double& src,
                                                double (&d)[3]) {
  src = w.wi * q.lw * g;
  d[0] = w.wi * fma(q.lw_p, g, -q.lw);
  d[1] = w.wi * q.lw_sw * g;
}
__device__ __forceinline__ void well_prod_oil(const Perf& w, const CellQ& q, double g, double& src,
                                              double (&d)[3]) {
  src = w.wi * q.lo * g;
  d[0] = w.wi * fma(q.lo_p, g, -q.lo);
  d[1] = w.wi * q.lo_sw * g;
  d[2] = w.wi * q.lo_x * g;
}
// The free-gas rate and its p and X derivatives.
__device__ __forceinline__ void well_prod_gas_free(const Perf& w, const CellQ& q, double g, double (&qg)[3]) {
  qg[0] = w.wi * q.lg * g;
  qg[1] = w.wi * fma(q.lg_p, g, -q.lg);
  qg[2] = w.wi * q.lg_x * g;
}
// The gas component: the free gas plus the gas dissolved in the produced oil
// (src_o, d_o the oil row).
__device__ __forceinline__ void well_prod_gas(const CellQ& q, double src_o, const double (&d_o)[3],
                                              const double (&qg)[3], double& src, double (&d)[3]) {
  src = fma(q.rs, src_o, qg[0]);
  d[0] = fma(q.rs, d_o[0], fma(q.rs_p, src_o, qg[1]));
  d[1] = q.rs * d_o[1];
  d[2] = fma(q.rs, d_o[2], fma(q.rs_x, src_o, qg[2]));
}

// Source of every component at a perforated cell (positive into the
// reservoir) and its derivatives (AllWells, Sec. 3.2.4).
template <int NB>
__device__ __forceinline__ void well_source(const Perf& w, const CellQ& q, const CellAux& a,
                                            double* src, double (*d)[3]) {
  for (int e = 0; e < NB; ++e) {
    src[e] = 0.0;
    d[e][0] = d[e][1] = d[e][2] = 0.0;
  }
  if (w.kind == 0) {
    const double drive = q.p - w.p_bh;
    if (!positive(drive)) return;
    const double g = w.p_bh - q.p;   // negative
    well_prod_water(w, q, g, src[0], d[0]);
    well_prod_oil(w, q, g, src[1], d[1]);
    if (NB == 3) {
      double qg[3];
      well_prod_gas_free(w, q, g, qg);
      well_prod_gas(q, src[1], d[1], qg, src[2], d[2]);
    }
  } else {
    const double drive = w.p_bh - q.p;
    if (!positive(drive)) return;
    const int e = (w.phase == 0) ? 0 : NB - 1;
    const double b = (w.phase == 0) ? a.bw : a.bg;
    const double b_p = (w.phase == 0) ? a.bw_p : a.bg_p;
    const double wmb = w.wi * a.mob * b;
    src[e] = wmb * drive;
    d[e][0] = w.wi * fma(fma(a.mob_p, b, a.mob * b_p), drive, -a.mob * b);
    d[e][1] = w.wi * a.mob_sw * b * drive;
    d[e][2] = w.wi * a.mob_x * b * drive;
  }
}

}  // namespace ocp
