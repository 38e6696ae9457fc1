// Block-CSR products and the adjoint vector-Jacobian product.
//
// spmv_grid_kernel  y = alpha A x + beta y on the grid's 7-point block pattern
//                   (the kernel the linear solver iterates on, Sec. 3.3.3);
// spmv_grid_t_kernel the transposed product: every output row gathers the
//                   blocks (n, c) of its column, located in closed form, so
//                   that it is owned by one thread and no atomics are needed;
// spmv_bulk_kernel  y = alpha A x + beta y for 2x2 and 1x1 blocks with the
//                   matrix slices staged by bulk asynchronous copies;
// vjp_kernel        lambda^T dR/d(u_new, u_old, ln k, phi) of the residual of
//                   eqs. 1, 2 and 4: J^T lambda with the column's blocks found in closed form, the
//                   transmissibility and well-index terms from the stored face
//                   fluxes (T and WI are linear in the fluxes), and the
//                   accumulation terms recomputed from the two states.
// setup_kernel      per-grid geometry: transmissibilities, their ln k weights
//                   and the block-CSR pattern.
// well_rate_kernel  surface rates of each well (one thread per well, its
//                   perforations summed in order).
#include "ocp_internal.cuh"
#include "kernels.cuh"

namespace ocp {

namespace {

// ------------------------------------------------------------------ pattern
// Neighbour types in column order: -z, -y, -x, self, +x, +y, +z.
__device__ __forceinline__ void neighbours(const Params& P, long long c, bool* has) {
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  has[0] = k > 0; has[1] = j > 0; has[2] = i > 0; has[3] = true;
  has[4] = i + 1 < P.nx; has[5] = j + 1 < P.ny; has[6] = k + 1 < P.nz;
}

// Number of stored blocks in the rows before c.
__device__ __forceinline__ long long row_start(const Params& P, long long c) {
  if (c >= P.N) return 7 * P.N - 2 * ((long long)P.ny * P.nz + (long long)P.nx * P.nz + P.nxy);
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  return row_start_ijk(P, c, i, j, k);
}

__global__ void setup_kernel(Params P, const double* __restrict__ lnk, double dx, double dy, double dz,
                             double kzr, double* __restrict__ trans, double* __restrict__ wlnk,
                             int32_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
  bool has[7];
  neighbours(P, c, has);
  // transmissibility of the +x, +y, +z face: harmonic combination of the two
  // half-cell conductances C A / (h/(2 k_c) + h/(2 k_n))
  const double h[3] = {dx, dy, dz};
  const double area[3] = {dy * dz, dx * dz, dx * dy};
  const double kc = exp(lnk[c]);
  for (int d = 0; d < 3; ++d) {
    double T = 0.0, wi = 0.0, wj = 0.0;
    if (has[4 + d]) {
      const double kn = exp(lnk[c + off[4 + d]]);
      const double fz = (d == 2) ? kzr : 1.0;
      const double ki_ = kc * fz, kj_ = kn * fz;
      T = (kDarcy * area[d]) / ((0.5 * h[d]) / ki_ + (0.5 * h[d]) / kj_);
      wi = kn / (kc + kn);   // d ln T / d ln k_c
      wj = kc / (kc + kn);   // d ln T / d ln k_n
    }
    trans[d * N + c] = T;
    wlnk[d * N + c] = wi;
    wlnk[(3 + d) * N + c] = wj;
  }
  const long long start = row_start(P, c);
  row_ptr[c] = (int32_t)start;
  if (c == N - 1) row_ptr[N] = (int32_t)row_start(P, N);
  int s = 0;
  for (int t = 0; t < 7; ++t) {
    if (!has[t]) continue;
    const long long n = c + off[t];
    col_idx[start + s] = (int32_t)n;
    ++s;
  }
}

// ------------------------------------------------------------------ SpMV
// mode 0: y = A x;  1: y = alpha A x;  2: y = alpha A x + beta y
// Product on the grid's own pattern, one thread per block row.  The FP64
// FMAs (NB*NB per block) are the binding resource on GB300, so the kernel
// is arranged to keep them fed: the columns come from the 7-point structure
// and the row's first block from the closed form of the row pointer (no
// dependent index loads), all x entries of the row are loaded first, then
// each block is loaded and consumed.  Rows with missing neighbours read x
// at their own cell instead and skip those blocks.  One-warp CTAs with a
// budget of 80 registers (24 warps per SM) measured fastest at 200 000 rows:
// 25.3 us against 25.8 us for 128-thread CTAs at 64 registers (32 warps),
// 25.4 for 64-thread CTAs at 80; 96 registers (20 warps) 26.5 us.
constexpr int kSpmvThreads = 32;
constexpr int kSpmvMinBlocks = 24;

template <int NB>
__global__ void __launch_bounds__(kSpmvThreads, kSpmvMinBlocks) spmv_grid_kernel(Params P, const int32_t* __restrict__ row_ptr,
                                                        const double* __restrict__ val, double alpha,
                                                        const double* __restrict__ x, double beta,
                                                        double* __restrict__ y, int mode,
                                                        const double* __restrict__ skip) {
  constexpr int B2 = NB * NB;
  pdl_wait();
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= P.N || (skip != nullptr && *skip != 0.0)) return;
  int ci, cj, ck;
  cell_ijk(P, c, ci, cj, ck);
  const bool has[7] = {ck > 0, cj > 0, ci > 0, true, ci + 1 < P.nx, cj + 1 < P.ny, ck + 1 < P.nz};
  const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
  int slot[7];
  int s = 0;
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    slot[t] = s;
    s += has[t];
  }
  double xv[7][NB];
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const long long n = has[t] ? c + off[t] : c;
#pragma unroll
    for (int v = 0; v < NB; ++v) xv[t][v] = x[n * NB + v];
  }
  const double* row = val + row_start_ijk(P, c, ci, cj, ck) * B2;
  double acc[NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) acc[e] = 0.0;
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    if (!has[t]) continue;
    const double* blk = row + slot[t] * B2;
    double b[B2];
#pragma unroll
    for (int q = 0; q < B2; ++q) b[q] = __ldg(blk + q);
#pragma unroll
    for (int e = 0; e < NB; ++e)
#pragma unroll
      for (int v = 0; v < NB; ++v) acc[e] = fma(b[e * NB + v], xv[t][v], acc[e]);
  }
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    double o = acc[e];
    if (mode >= 1) o = alpha * o;
    if (mode == 2) o = fma(beta, y[c * NB + e], o);
    y[c * NB + e] = o;
  }
}

// Transposed product on the grid's pattern, one thread per output row c:
// y_c = sum over the stored blocks (n, c) of A(n, c)^T x_n, with the blocks
// visited in the order of row c's columns (neighbour types -z .. +z).  Block
// (n, c) lies in row n at the slot of the opposite type 6 - t: n's row start
// in closed form plus the number of n's neighbour types before 6 - t, so no
// index is loaded.  The FMAs run in the order of a gather of row c's
// columns: block by block, each block's rows in turn.
template <int NB>
__global__ void __launch_bounds__(kSpmvThreads) spmv_grid_t_kernel(Params P, const double* __restrict__ val,
                                                                   double alpha, const double* __restrict__ x,
                                                                   double beta, double* __restrict__ y, int mode,
                                                                   const double* __restrict__ skip) {
  constexpr int B2 = NB * NB;
  pdl_wait();
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= P.N || (skip != nullptr && *skip != 0.0)) return;
  int ci, cj, ck;
  cell_ijk(P, c, ci, cj, ck);
  const bool has[7] = {ck > 0, cj > 0, ci > 0, true, ci + 1 < P.nx, cj + 1 < P.ny, ck + 1 < P.nz};
  const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
  double acc[NB];
#pragma unroll
  for (int v = 0; v < NB; ++v) acc[v] = 0.0;
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    if (!has[t]) continue;
    const long long n = c + off[t];
    // (i, j, k) of n and the slot of type 6 - t in its row
    const int ni = ci + (t == 4) - (t == 2), nj = cj + (t == 5) - (t == 1), nk = ck + (t == 6) - (t == 0);
    const bool hn[6] = {nk > 0, nj > 0, ni > 0, true, ni + 1 < P.nx, nj + 1 < P.ny};
    int sn = 0;
#pragma unroll
    for (int u = 0; u < 6 - t; ++u) sn += hn[u];
    const double* blk = val + (row_start_ijk(P, n, ni, nj, nk) + sn) * B2;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      const double l = x[n * NB + e];
#pragma unroll
      for (int v = 0; v < NB; ++v) acc[v] = fma(__ldg(blk + e * NB + v), l, acc[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NB; ++v) {
    double o = acc[v];
    if (mode >= 1) o = alpha * o;
    if (mode == 2) o = fma(beta, y[c * NB + v], o);
    y[c * NB + v] = o;
  }
}

// Product for 2x2 and 1x1 blocks with the CTA's slice of the matrix staged
// in shared memory by one bulk asynchronous copy (the TMA unit), completing
// on an mbarrier while the CTA's threads gather their x entries.  Rows of a
// CTA are consecutive, so their blocks are one contiguous range of `val`.
// A 2x2 row is at most 7 x 32 bytes: 128-row tiles take 28.7 KB and leave
// the SM at full occupancy.  With 3x3 blocks (504 bytes a row) shared memory
// would cap residency near 14 warps per SM, and the register kernel above is
// faster there (measured 28.6 against 30.5 us at 200 000 rows, while 2x2 at
// 1.12 M rows took 60 against 74 us).  Same FMAs in the same order as
// spmv_grid_kernel, so the two give identical bits.
//
// Bounds: the CTA's blocks occupy bytes [b0 B, b1 B) of val (B = 8 NB^2).
// The copy takes [s, e) with s = b0 B rounded down to 16 and e the smaller
// of b1 B rounded up to 16 and the array size rounded down to 16, so source
// (val must be 16-byte aligned), destination and size are 16-byte multiples
// and the copy stays inside the array.  The one double an array of odd size
// can have past e is read from global memory.  The wait is bounded: a
// thread past its limit records kStatTimeout (reported by ocp_get_status as
// OCP_ERR_TIMEOUT), waits once more for the copy in flight and returns.
constexpr int kBulkRows = 128;
constexpr unsigned kBulkSpin = 1u << 20;

__device__ __forceinline__ bool bulk_wait(unsigned bar) {
  for (unsigned it = 0; it < kBulkSpin; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int NB>
constexpr int bulk_smem_bytes() { return kBulkRows * 7 * 8 * NB * NB + 16; }

template <int NB>
__global__ void __launch_bounds__(kBulkRows) spmv_bulk_kernel(Params P, const int32_t* __restrict__ row_ptr,
                                                              long long nnzb, const double* __restrict__ val,
                                                              double alpha, const double* __restrict__ x,
                                                              double beta, double* __restrict__ y, int mode,
                                                              int* __restrict__ status, const double* __restrict__ skip) {
  constexpr int B2 = NB * NB;
  constexpr long long BB = 8 * B2;
  pdl_wait();
  if (skip != nullptr && *skip != 0.0) return;     // the same for every thread: before any barrier
  extern __shared__ __align__(128) unsigned char sbuf[];
  __shared__ __align__(8) unsigned long long bar;
  const long long r0 = (long long)blockIdx.x * kBulkRows;
  const long long r1 = r0 + kBulkRows < P.N ? r0 + kBulkRows : P.N;
  const long long b0 = row_ptr[r0], b1 = row_ptr[r1];
  const long long s = (b0 * BB) & ~15ll;
  const long long end16 = (nnzb * BB) & ~15ll;
  long long e = (b1 * BB + 15) & ~15ll;
  if (e > end16) e = end16;
  const long long size = e > s ? e - s : 0;
  const unsigned ubar = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0 && size > 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ubar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ubar), "r"((unsigned)size)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (unsigned)__cvta_generic_to_shared(sbuf)),
        "l"(reinterpret_cast<const unsigned char*>(val) + s), "r"((unsigned)size), "r"(ubar)
        : "memory");
  }
  const long long c = r0 + threadIdx.x;
  const bool live = c < P.N;
  int ci = 0, cj = 0, ck = 0;
  bool has[7] = {false, false, false, false, false, false, false};
  double xv[7][NB];
  if (live) {
    cell_ijk(P, c, ci, cj, ck);
    has[0] = ck > 0; has[1] = cj > 0; has[2] = ci > 0; has[3] = true;
    has[4] = ci + 1 < P.nx; has[5] = cj + 1 < P.ny; has[6] = ck + 1 < P.nz;
    const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      const long long n = has[t] ? c + off[t] : c;
#pragma unroll
      for (int v = 0; v < NB; ++v) xv[t][v] = x[n * NB + v];
    }
  }
  __syncthreads();                       // the barrier is initialised before anyone waits on it
  if (size > 0 && !bulk_wait(ubar)) {
    atomicOr(status, kStatTimeout);      // every thread that gives up reports it: its rows stay unwritten
    bulk_wait(ubar);                     // the copy in flight gets one more bounded wait
    return;
  }
  if (!live) return;
  const double* sm = reinterpret_cast<const double*>(sbuf);
  const long long rs = row_start_ijk(P, c, ci, cj, ck);
  double acc[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) acc[q] = 0.0;
  int slot = 0;
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    if (!has[t]) continue;
    const long long q0 = (rs + slot) * B2;   // index of the block's first double in val
    ++slot;
    double b[B2];
#pragma unroll
    for (int q = 0; q < B2; ++q) {
      const long long gi = q0 + q;
      b[q] = gi * 8 < e ? sm[(gi * 8 - s) >> 3] : val[gi];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int v = 0; v < NB; ++v) acc[q] = fma(b[q * NB + v], xv[t][v], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    double o = acc[q];
    if (mode >= 1) o = alpha * o;
    if (mode == 2) o = fma(beta, y[c * NB + q], o);
    y[c * NB + q] = o;
  }
}

// ------------------------------------------------------------------ adjoint
// 128-thread CTAs: at 64 registers four 256-thread CTAs fit an SM and the
// 200 000-cell adjoint's 782 CTAs split 3 : 2 over the SMs; 1563 CTAs of 128
// spread evenly enough (79 against 84 us).
constexpr int kVjpThreads = 128;

template <int NB>
__global__ void __launch_bounds__(kVjpThreads) vjp_kernel(Params P, const Table* __restrict__ gT,
                                                  const double* __restrict__ u_new,
                                                  const int8_t* __restrict__ f_new,
                                                  const double* __restrict__ u_old,
                                                  const int8_t* __restrict__ f_old,
                                                  const double* __restrict__ phi,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ face_flux,
                                                  const double* __restrict__ wlnk,
                                                  const int32_t* __restrict__ perf_of_cell,
                                                  const Perf* __restrict__ perf, double scale,
                                                  const double* __restrict__ lam,
                                                  double* __restrict__ g_unew, double* __restrict__ g_uold,
                                                  double* __restrict__ g_lnk, double* __restrict__ g_phi,
                                                  int* __restrict__ status) {
  pdl_wait();
  __shared__ Table T;
  __shared__ unsigned long long bar;
  unsigned uses = 0;
  load_table(T, gT, bar, uses, status);
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  double lc[NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) lc[e] = lam[c * NB + e];

  if (g_unew) {
    // J^T lambda: the blocks (n, c) of column c, found in closed form as in
    // spmv_grid_t_kernel, in the order of row c's columns
    int ci, cj, ck;
    cell_ijk(P, c, ci, cj, ck);
    const bool hc[7] = {ck > 0, cj > 0, ci > 0, true, ci + 1 < P.nx, cj + 1 < P.ny, ck + 1 < P.nz};
    const long long off[7] = {-P.nxy, -P.nx, -1, 0, 1, P.nx, P.nxy};
    double acc[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) acc[v] = 0.0;
#pragma unroll
    for (int t = 0; t < 7; ++t) {
      if (!hc[t]) continue;
      const long long n = c + off[t];
      const int ni = ci + (t == 4) - (t == 2), nj = cj + (t == 5) - (t == 1), nk = ck + (t == 6) - (t == 0);
      const bool hn[6] = {nk > 0, nj > 0, ni > 0, true, ni + 1 < P.nx, nj + 1 < P.ny};
      int sn = 0;
#pragma unroll
      for (int u = 0; u < 6 - t; ++u) sn += hn[u];
      const double* blk = val + (row_start_ijk(P, n, ni, nj, nk) + sn) * NB * NB;
#pragma unroll
      for (int e = 0; e < NB; ++e) {
        const double l = lam[n * NB + e];
#pragma unroll
        for (int v = 0; v < NB; ++v) acc[v] = fma(blk[e * NB + v], l, acc[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < NB; ++v) g_unew[v * N + c] = acc[v];
  }

  const double pn = u_new[c], swn = u_new[N + c], xn = (NB == 3) ? u_new[2 * N + c] : 0.0;
  const double po = u_old[c], swo = u_old[N + c], xo = (NB == 3) ? u_old[2 * N + c] : 0.0;
  const int fn = (NB == 3) ? (f_new[c] & 1) : 0, fo = (NB == 3) ? (f_old[c] & 1) : 0;
  const double ph = phi[c];

  if (g_uold || g_phi) {
    // the accumulation is linear in the reference porosity: the amounts of
    // the old state per unit phi_ref serve both outputs
    double mo[3], m_p[3], m_sw[3], m_x[3];
    cell_masses<NB, true>(P, T, po, swo, xo, fo, 1.0, mo, m_p, m_sw, m_x);
    if (g_uold) {
      double lph[NB];
#pragma unroll
      for (int e = 0; e < NB; ++e) lph[e] = lc[e] * ph;
      double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int e = 0; e < NB; ++e) {
        g[0] = fma(lph[e], m_p[e], g[0]);
        g[1] = fma(lph[e], m_sw[e], g[1]);
        g[2] = fma(lph[e], m_x[e], g[2]);
      }
#pragma unroll
      for (int v = 0; v < NB; ++v) g_uold[v * N + c] = -scale * g[v];
    }
    if (g_phi) {
      double mn[3];
      cell_masses<NB, false>(P, T, pn, swn, xn, fn, 1.0, mn);
      double g = 0.0;
#pragma unroll
      for (int e = 0; e < NB; ++e) g = fma(lc[e], mn[e] - mo[e], g);
      g_phi[c] = scale * g;
    }
  }

  if (g_lnk) {
    bool has[7];
    neighbours(P, c, has);
    const long long stride[3] = {1, P.nx, P.nxy};
    double g = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (has[4 + d]) {              // + face: this cell is the upstream index i
        const long long n = c + stride[d];
        const double w = wlnk[d * N + c];
        double t = 0.0;
#pragma unroll
        for (int e = 0; e < NB; ++e) t = fma(lc[e] - lam[n * NB + e], face_flux[(d * NB + e) * N + c], t);
        g = fma(w, t, g);
      }
      if (has[2 - d]) {              // - face: this cell is j of the face (n, c)
        const long long n = c - stride[d];
        const double w = wlnk[(3 + d) * N + n];
        double t = 0.0;
#pragma unroll
        for (int e = 0; e < NB; ++e) t = fma(lam[n * NB + e] - lc[e], face_flux[(d * NB + e) * N + n], t);
        g = fma(w, t, g);
      }
    }
    const int ip = perf_of_cell[c];
    if (ip >= 0) {                   // the well index is proportional to k of the cell
      CellQ q{};
      CellAux a{};
      cell_quantities<NB, true>(P, T, pn, swn, xn, fn, ph, q, a);
      double src[3], ds[3][3];
      well_source<NB>(perf[ip], q, a, src, ds);
#pragma unroll
      for (int e = 0; e < NB; ++e) g = fma(-lc[e], src[e], g);
    }
    g_lnk[c] = g;
  }
}

// ------------------------------------------------------------------ wells
template <int NB>
__global__ void well_rate_kernel(Params P, const Table* __restrict__ gT, const double* __restrict__ u,
                                 const int8_t* __restrict__ flag, const double* __restrict__ phi,
                                 const Perf* __restrict__ perf, const int32_t* __restrict__ first,
                                 int nwell, double* __restrict__ q) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwell) return;
  const long long N = P.N;
  double sum[3] = {0.0, 0.0, 0.0};
  for (int k = first[w]; k < first[w + 1]; ++k) {
    const long long c = perf[k].cell;
    CellQ cq{};
    CellAux a{};
    cell_quantities<NB, true>(P, *gT, u[c], u[N + c], (NB == 3) ? u[2 * N + c] : 0.0,
                              (NB == 3) ? (flag[c] & 1) : 0, phi[c], cq, a);
    double src[3], ds[3][3];
    well_source<NB>(perf[k], cq, a, src, ds);
    for (int e = 0; e < NB; ++e) sum[e] += src[e];
  }
  for (int e = 0; e < NB; ++e) q[w * NB + e] = sum[e];
}

}  // namespace

cudaError_t launch_setup(ocp_grid* g, const double* d_lnk, double dx, double dy, double dz,
                         double kz_over_kx, cudaStream_t s) {
  const Params& P = g->prm;
  const unsigned blocks = (unsigned)((P.N + 255) / 256);
  setup_kernel<<<blocks, 256, 0, s>>>(P, d_lnk, dx, dy, dz, kz_over_kx, g->d_trans, g->d_wlnk,
                                      g->d_row_ptr, g->d_col_idx);
  return cudaGetLastError();
}

cudaError_t launch_spmv(const ocp_grid* g, const double* val, double alpha, const double* x, double beta,
                        double* y, int transpose, cudaStream_t s, int nbs, const double* skip) {
  const long long N = g->prm.N;
  const int mode = (beta != 0.0) ? 2 : (alpha != 1.0 ? 1 : 0);
  const unsigned gblocks = (unsigned)((N + kSpmvThreads - 1) / kSpmvThreads);
  const int nb = nbs > 0 ? nbs : g->prm.nb;
  // 2x2 and 1x1 products stage their matrix slices by bulk copy when the
  // matrix is 16-byte aligned (the copy's rule); otherwise, and for 3x3, the
  // register kernel runs.  Both give identical bits.  Every product is a
  // programmatic launch (launch_pdl): it is scheduled while the kernel before
  // it finishes and waits for it before touching memory.
  const bool bulk = ((uintptr_t)val & 15) == 0;
  const unsigned bblocks = (unsigned)((N + kBulkRows - 1) / kBulkRows);
  if (nb == 3) {
    if (transpose) return launch_pdl(spmv_grid_t_kernel<3>, gblocks, kSpmvThreads, 0, s, g->prm, val, alpha, x, beta, y, mode, skip);
    return launch_pdl(spmv_grid_kernel<3>, gblocks, kSpmvThreads, 0, s, g->prm, (const int32_t*)g->d_row_ptr, val, alpha, x, beta, y, mode, skip);
  } else if (nb == 2) {
    if (transpose) return launch_pdl(spmv_grid_t_kernel<2>, gblocks, kSpmvThreads, 0, s, g->prm, val, alpha, x, beta, y, mode, skip);
    if (bulk) return launch_pdl(spmv_bulk_kernel<2>, bblocks, kBulkRows, bulk_smem_bytes<2>(), s, g->prm, (const int32_t*)g->d_row_ptr, (long long)g->nnzb, val, alpha, x, beta, y, mode, g->d_status, skip);
    return launch_pdl(spmv_grid_kernel<2>, gblocks, kSpmvThreads, 0, s, g->prm, (const int32_t*)g->d_row_ptr, val, alpha, x, beta, y, mode, skip);
  } else {
    if (transpose) return launch_pdl(spmv_grid_t_kernel<1>, gblocks, kSpmvThreads, 0, s, g->prm, val, alpha, x, beta, y, mode, skip);
    if (bulk) return launch_pdl(spmv_bulk_kernel<1>, bblocks, kBulkRows, bulk_smem_bytes<1>(), s, g->prm, (const int32_t*)g->d_row_ptr, (long long)g->nnzb, val, alpha, x, beta, y, mode, g->d_status, skip);
    return launch_pdl(spmv_grid_kernel<1>, gblocks, kSpmvThreads, 0, s, g->prm, (const int32_t*)g->d_row_ptr, val, alpha, x, beta, y, mode, skip);
  }
  return cudaGetLastError();
}

cudaError_t launch_vjp(const ocp_grid* g, const double* u_new, const int8_t* f_new, const double* u_old,
                       const int8_t* f_old, double dt, const double* val, const double* face_flux,
                       const double* lam, double* g_unew, double* g_uold, double* g_lnk, double* g_phi,
                       cudaStream_t s) {
  const Params& P = g->prm;
  const unsigned blocks = (unsigned)((P.N + kVjpThreads - 1) / kVjpThreads);
  const double scale = P.vol_rb / dt;
  if (P.nb == 3)
    return launch_pdl(vjp_kernel<3>, blocks, kVjpThreads, 0, s, P, (const Table*)g->d_table, u_new, f_new, u_old,
                      f_old, (const double*)g->d_phi, val, face_flux, (const double*)g->d_wlnk,
                      (const int32_t*)g->d_perf_of_cell, (const Perf*)g->d_perf, scale, lam, g_unew, g_uold, g_lnk,
                      g_phi, g->d_status);
  return launch_pdl(vjp_kernel<2>, blocks, kVjpThreads, 0, s, P, (const Table*)g->d_table, u_new, f_new, u_old,
                    f_old, (const double*)g->d_phi, val, face_flux, (const double*)g->d_wlnk,
                    (const int32_t*)g->d_perf_of_cell, (const Perf*)g->d_perf, scale, lam, g_unew, g_uold, g_lnk,
                    g_phi, g->d_status);
}

cudaError_t launch_well_rates(const ocp_grid* g, const double* u, const int8_t* flag, double* q,
                              cudaStream_t s) {
  if (g->nwell == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((g->nwell + 63) / 64);
  if (g->prm.nb == 3)
    well_rate_kernel<3><<<blocks, 64, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, g->d_perf, g->d_well_first, g->nwell, q);
  else
    well_rate_kernel<2><<<blocks, 64, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, g->d_perf, g->d_well_first, g->nwell, q);
  return cudaGetLastError();
}

}  // namespace ocp
