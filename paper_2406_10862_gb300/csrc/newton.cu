// Newton-step support: the parts of the FIM nonlinear iteration (Sec. 3.2.5,
// steps 2 and 4) around the linearisation -- a block-Jacobi preconditioned
// BiCGSTAB solve on the block-CSR Jacobian (the paper hands this to CPR
// solvers in PETSc/Hypre, Sec. 5.1; here it is a plain GPU Krylov method),
// the update of the primary variables with a saturation chop and the
// saturated/undersaturated phase switch, the adjoint of the well rates, and
// the update of transmissibilities and well indices from a new ln k.
//
// The BiCGSTAB scalars never leave the device: every reduction ends in a
// device scalar that the next kernels read, and the host only reads the
// residual norm to decide when to stop.  Dot products are two-pass with a
// fixed grid, so results are deterministic.
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace ocp {
namespace {

constexpr int kRedBlocks = 304;       // fixed partial-sum grid (2 per SM)
constexpr int kRedThreads = 256;

// scalar slots of the solver
// S_DONE, S_ITER, S_TARGET, S_MAXIT drive the device-side iteration control
enum {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_BETA, S_R0V, S_TS, S_TT, S_RR, S_BB, S_FLAG, S_TMP,
  S_DONE, S_ITER, S_TARGET, S_MAXIT, S_TICKET, S_COUNT
};
// S_TICKET holds a 64-bit counter (not a double): the CTAs of a fused step
// count themselves in, and the last one finishes the step's reductions.
constexpr int kItersPerGraph = 8;     // BiCGSTAB iterations per graph replay

__global__ void __launch_bounds__(kRedThreads) dot_partial(long long n, const double* __restrict__ a,
                                                            const double* __restrict__ b,
                                                            double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads)
    s = fma(a[i], b[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads) dot_final(const double* __restrict__ part, double* out) {
  __shared__ double sh[kRedThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------ fused steps
// The kernels below fuse a vector step with the dot products that follow it.
// They use the same fixed grid and the same element-to-thread assignment,
// per-thread order and tree as dot_partial / dot_final, so every sum is the
// bit-identical value the separate kernels gave.
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* __restrict__ part) {
  __shared__ double sh[NV][kRedThreads];
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) part[q * kRedBlocks + blockIdx.x] = sh[q][0];
}

// element i of the block-Jacobi product D^-1 z (the order of bj_apply_kernel)
template <int NB>
__device__ __forceinline__ double bj_elem(const double* __restrict__ dinv, const double* __restrict__ z, long long i) {
  const long long c = i / NB;
  const int e = (int)(i - c * NB);
  double s = 0.0;
#pragma unroll
  for (int v = 0; v < NB; ++v) s = fma(dinv[c * NB * NB + e * NB + v], z[c * NB + v], s);
  return s;
}

// Totals and the scalar step after them:
//   kFinAlpha: r0.v -> alpha;  kFinOmega: t.s, t.t -> omega;
//   kFinRrRho: r.r -> the loop's test for the next iteration (S_DONE or
//   S_ITER + 1), then r0.r -> rho and beta.
enum { kFinAlpha = 0, kFinOmega = 1, kFinRrRho = 2 };

// The totals of the partials (the order and tree of dot_final), read from
// L2: in the fused kernels other CTAs wrote them moments before.
__device__ __forceinline__ double block_total_cg(const double* part) {
  __shared__ double sh[kRedThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) s += __ldcg(part + i);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

template <int MODE>
__device__ __forceinline__ void finish(const double* part, double* sc) {
  const double a = block_total_cg(part);
  const double b = (MODE == kFinAlpha) ? 0.0 : block_total_cg(part + kRedBlocks);
  if (threadIdx.x != 0) return;
  if constexpr (MODE == kFinAlpha) {
    sc[S_R0V] = a;
    if (a == 0.0) { sc[S_FLAG] = 1.0; sc[S_ALPHA] = 0.0; return; }
    sc[S_ALPHA] = sc[S_RHO] / a;
  } else if constexpr (MODE == kFinOmega) {
    sc[S_TS] = a;
    sc[S_TT] = b;
    if (b == 0.0) { sc[S_OMEGA] = 0.0; return; }   // s == 0: x is already exact
    sc[S_OMEGA] = a / b;
    sc[S_RHO_OLD] = sc[S_RHO];
  } else {
    sc[S_RR] = a;
    const double res = sqrt(a);
    if (sc[S_FLAG] != 0.0 || !(res > sc[S_TARGET]) || !(sc[S_ITER] < sc[S_MAXIT])) {
      sc[S_DONE] = 1.0;
      return;
    }
    sc[S_ITER] += 1.0;
    sc[S_RHO] = b;
    if (sc[S_RHO_OLD] == 0.0 || sc[S_OMEGA] == 0.0) { sc[S_FLAG] = 1.0; sc[S_BETA] = 0.0; return; }
    sc[S_BETA] = (b / sc[S_RHO_OLD]) * (sc[S_ALPHA] / sc[S_OMEGA]);
  }
}

// Every CTA of a fused step takes a ticket after writing its partials; the
// one that takes the last ticket has seen all of them written (each CTA
// fences before its ticket) and finishes the step, then resets the counter.
// The CTAs read every scalar they need before taking their tickets.
template <int MODE>
__device__ __forceinline__ void last_cta_finishes(const double* part, double* sc) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long prev = atomicAdd(reinterpret_cast<unsigned long long*>(sc + S_TICKET), 1ull);
    last = prev == (unsigned long long)(kRedBlocks - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish<MODE>(part, sc);
  if (threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(sc + S_TICKET) = 0ull;
}

// v = D^-1 z, the partials of r0 . v, then alpha
template <int NB>
__global__ void __launch_bounds__(kRedThreads) apply_dot(long long n, const double* __restrict__ dinv,
                                                          const double* __restrict__ z, double* __restrict__ v,
                                                          const double* __restrict__ r0, double* sc,
                                                          double* __restrict__ part) {
  if (sc[S_DONE] != 0.0) return;
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    const double x = bj_elem<NB>(dinv, z, i);
    v[i] = x;
    acc[0] = fma(r0[i], x, acc[0]);
  }
  block_partials<1>(acc, part);
  last_cta_finishes<kFinAlpha>(part, sc);
}

// t = D^-1 z, the partials of t . s and t . t, then omega
template <int NB>
__global__ void __launch_bounds__(kRedThreads) apply_dot2(long long n, const double* __restrict__ dinv,
                                                           const double* __restrict__ z, double* __restrict__ t,
                                                           const double* __restrict__ sv, double* sc,
                                                           double* __restrict__ part) {
  if (sc[S_DONE] != 0.0) return;
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    const double x = bj_elem<NB>(dinv, z, i);
    t[i] = x;
    acc[0] = fma(x, sv[i], acc[0]);
    acc[1] = fma(x, x, acc[1]);
  }
  block_partials<2>(acc, part);
  last_cta_finishes<kFinOmega>(part, sc);
}

// x += alpha p + omega s, r = s - omega t, the partials of r . r and r0 . r,
// then the loop's test, rho and beta
__global__ void __launch_bounds__(kRedThreads) upd_xr_dot(long long n, double* __restrict__ x,
                                                           const double* __restrict__ p, const double* __restrict__ sv,
                                                           double* __restrict__ r, const double* __restrict__ t,
                                                           const double* __restrict__ r0, double* sc,
                                                           double* __restrict__ part) {
  if (sc[S_DONE] != 0.0) return;
  const double al = sc[S_ALPHA], om = sc[S_OMEGA];
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    x[i] = fma(om, sv[i], fma(al, p[i], x[i]));
    const double ri = fma(-om, t[i], sv[i]);
    r[i] = ri;
    acc[0] = fma(ri, ri, acc[0]);
    acc[1] = fma(r0[i], ri, acc[1]);
  }
  block_partials<2>(acc, part);
  last_cta_finishes<kFinRrRho>(part, sc);
}

// the partials of a1 . b1 and a2 . b2 (start of the iteration)
__global__ void __launch_bounds__(kRedThreads) dot2_partial(long long n, const double* __restrict__ a1,
                                                             const double* __restrict__ b1,
                                                             const double* __restrict__ a2,
                                                             const double* __restrict__ b2, double* __restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n; i += (long long)kRedBlocks * kRedThreads) {
    acc[0] = fma(a1[i], b1[i], acc[0]);
    acc[1] = fma(a2[i], b2[i], acc[1]);
  }
  block_partials<2>(acc, part);
}

// The same finish as a one-CTA kernel, after dot2_partial at the start of a solve.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) fin_kernel(const double* __restrict__ part, double* __restrict__ sc) {
  if (sc[S_DONE] != 0.0) return;
  finish<MODE>(part, sc);
}

__global__ void scal_init(double* sc) {
  sc[S_RHO_OLD] = 1.0; sc[S_ALPHA] = 1.0; sc[S_OMEGA] = 1.0; sc[S_FLAG] = 0.0; sc[S_BETA] = 0.0;
  sc[S_DONE] = 0.0; sc[S_ITER] = 0.0;
  *reinterpret_cast<unsigned long long*>(sc + S_TICKET) = 0ull;
}
__global__ void iter_setup(double* sc, double target, double maxit) {
  sc[S_TARGET] = target;
  sc[S_MAXIT] = maxit;
}

// p = r + beta (p - omega v)
__global__ void upd_p(long long n, const double* __restrict__ r, double* __restrict__ p,
                      const double* __restrict__ v, const double* __restrict__ sc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n || sc[S_DONE] != 0.0) return;
  p[i] = fma(sc[S_BETA], fma(-sc[S_OMEGA], v[i], p[i]), r[i]);
}
// s = r - alpha v
__global__ void upd_s(long long n, const double* __restrict__ r, const double* __restrict__ v,
                      double* __restrict__ s, const double* __restrict__ sc) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n || sc[S_DONE] != 0.0) return;
  s[i] = fma(-sc[S_ALPHA], v[i], r[i]);
}
// Inverse of every diagonal block (of its transpose when TRANS).
// With well terms, a perforated cell's block is that of the Schur complement,
// A_cc - bs_c cs_c^T / d_w.
template <int NB>
__global__ void block_jacobi_kernel(Params P, const int32_t* __restrict__ row_ptr, const double* __restrict__ val,
                                    double* __restrict__ dinv, int trans, int* status,
                                    const int32_t* __restrict__ perf_of_cell, const Perf* __restrict__ perf,
                                    WellSchur ws) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= P.N) return;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const int diag = (k > 0) + (j > 0) + (i > 0);
  const double* D = val + ((long long)row_ptr[c] + diag) * NB * NB;
  double a[NB][NB], inv[NB][NB];
  for (int e = 0; e < NB; ++e)
    for (int v = 0; v < NB; ++v) a[e][v] = trans ? D[v * NB + e] : D[e * NB + v];
  if (ws.d) {
    const int ip = perf_of_cell[c];
    if (ip >= 0) {
      const double id = 1.0 / ws.d[perf[ip].well];
      for (int e = 0; e < NB; ++e)
        for (int v = 0; v < NB; ++v) a[e][v] = fma(-ws.bs[ip * NB + e] * id, ws.cs[ip * NB + v], a[e][v]);
    }
  }
  double det;
  if constexpr (NB == 1) {
    det = a[0][0];
    inv[0][0] = 1.0 / det;
  } else if constexpr (NB == 3) {
    const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
    const double id = 1.0 / det;
    inv[0][0] = c00 * id;
    inv[1][0] = c01 * id;
    inv[2][0] = c02 * id;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  } else {
    det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
    const double id = 1.0 / det;
    inv[0][0] = a[1][1] * id;
    inv[0][1] = -a[0][1] * id;
    inv[1][0] = -a[1][0] * id;
    inv[1][1] = a[0][0] * id;
  }
  if (!(det != 0.0) || !finite(det)) atomicOr(status, kStatNonFinite);
  for (int e = 0; e < NB; ++e)
    for (int v = 0; v < NB; ++v) dinv[c * NB * NB + e * NB + v] = inv[e][v];
}

template <int NB>
__global__ void bj_apply_kernel(long long N, const double* __restrict__ dinv, const double* __restrict__ x,
                                double* __restrict__ y) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  double xv[NB];
  for (int v = 0; v < NB; ++v) xv[v] = x[c * NB + v];
  for (int e = 0; e < NB; ++e) {
    double s = 0.0;
    for (int v = 0; v < NB; ++v) s = fma(dinv[c * NB * NB + e * NB + v], xv[v], s);
    y[c * NB + e] = s;
  }
}

// Newton update with a per-cell saturation chop and the phase switch; also
// the largest change of each variable (atomicMax on the bits of |du| >= 0,
// which is exact and order-independent).
template <int NB>
__global__ void newton_update_kernel(Params P, const Table* __restrict__ gT, double* __restrict__ u,
                                     int8_t* __restrict__ flag, const double* __restrict__ du, double scale,
                                     double ds_max, unsigned long long* __restrict__ dmax,
                                     int* __restrict__ nswitch) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const Table& T = *gT;
  double d[3] = {scale * du[c * NB], scale * du[c * NB + 1], NB == 3 ? scale * du[c * NB + 2] : 0.0};
  const int f = (NB == 3) ? flag[c] : 0;
  // saturation chop: scale the cell's saturation changes to at most ds_max
  double big = fabs(d[1]);
  if (NB == 3 && f == 0) big = fmax(big, fabs(d[2]));
  if (big > ds_max) {
    const double sc = ds_max / big;
    d[1] *= sc;
    if (NB == 3 && f == 0) d[2] *= sc;
  }
  atomicMax(&dmax[0], (unsigned long long)__double_as_longlong(fabs(d[0])));
  atomicMax(&dmax[1], (unsigned long long)__double_as_longlong(fabs(d[1])));
  if (NB == 3) atomicMax(&dmax[2 + f], (unsigned long long)__double_as_longlong(fabs(d[2])));
  const double p = u[c] + d[0];
  u[c] = p;
  u[N + c] += d[1];
  if (NB == 3) {
    double x = u[2 * N + c] + d[2];
    // saturated R_s at the new pressure, from the table piece containing p
    const int kp = segment(T.pkey, T.nrow, dkey(p));
    const double rs_sat = fma(p - T.p[kp], T.s[4][kp], T.y[4][kp]);
    int nf = f;
    if (f == 0 && x < 0.0) {            // free gas disappeared: undersaturated at the bubble point
      nf = 1;
      x = rs_sat;
    } else if (f == 1 && x > rs_sat) {  // more gas than the oil can hold: free gas appears
      nf = 0;
      x = 0.0;
    }
    u[2 * N + c] = x;
    if (nf != f) {
      flag[c] = (int8_t)nf;
      atomicAdd(nswitch, 1);
    }
  }
}

// Adjoint of the well rates: for the rate cotangents q_bar[w*nb + e],
// g_u[v*N + c] += sum_e q_bar * dq/du and g_lnk[c] += sum_e q_bar * q
// (the well index is proportional to k of the cell).
template <int NB>
__global__ void well_vjp_kernel(Params P, const Table* __restrict__ gT, const double* __restrict__ u,
                                const int8_t* __restrict__ flag, const double* __restrict__ phi,
                                const Perf* __restrict__ perf, int nperf, const double* __restrict__ qbar,
                                double* __restrict__ g_u, double* __restrict__ g_lnk) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nperf) return;
  const long long N = P.N;
  const Perf w = perf[k];
  const long long c = w.cell;
  CellQ q{};
  CellAux a{};
  cell_quantities<NB, true>(P, *gT, u[c], u[N + c], (NB == 3) ? u[2 * N + c] : 0.0,
                            (NB == 3) ? (flag[c] & 1) : 0, phi[c], q, a, w.kind == 1);
  double src[3], ds[3][3];
  well_source<NB>(w, q, a, src, ds);
  double gl = 0.0;
  for (int v = 0; v < NB; ++v) {
    double s = 0.0;
    for (int e = 0; e < NB; ++e) s = fma(qbar[w.well * NB + e], ds[e][v], s);
    if (g_u) g_u[v * N + c] += s;
  }
  for (int e = 0; e < NB; ++e) gl = fma(qbar[w.well * NB + e], src[e], gl);
  if (g_lnk) g_lnk[c] += gl;
}

__global__ void perf_wi_kernel(Perf* perf, int nperf, const double* __restrict__ lnk) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nperf) return;
  perf[k].wi = exp(lnk[perf[k].cell]) * perf[k].geom;
}

unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_perf_wi(ocp_grid* g, const double* lnk, cudaStream_t s) {
  if (g->nperf == 0) return cudaSuccess;
  perf_wi_kernel<<<nblk(g->nperf, 64), 64, 0, s>>>(g->d_perf, g->nperf, lnk);
  return cudaGetLastError();
}

int64_t solver_work_doubles(const ocp_grid* g) {
  const int64_t n = (int64_t)g->prm.nb * g->prm.N;
  // r, r0, p, v, s, t, y, z; block inverses; two sets of partial sums;
  // scalars; and the reduced right-hand side of the well elimination
  return 9 * n + (int64_t)g->prm.nb * g->prm.nb * g->prm.N + 2 * kRedBlocks + S_COUNT + 8;
}

ocp_status bicgstab_run(ocp_grid* g, const double* val, const WellSchur* ws, const double* b, double* x,
                        double rtol, int maxit, int transpose, double* work, int* iters, double* relres,
                        cudaStream_t s, int nbs) {
  if (!(rtol > 0.0) || maxit < 1) return report(OCP_ERR_INVALID_ARG, "rtol must be > 0 and maxit >= 1");
  const int nb = nbs > 0 ? nbs : g->prm.nb;
  const long long N = g->prm.N, n = nb * N;
  double* r = work;
  double* r0 = r + n;
  double* p = r0 + n;
  double* v = p + n;
  double* sv = v + n;
  double* t = sv + n;
  double* y = t + n;
  double* z = y + n;
  double* dinv = z + n;
  double* part = dinv + (long long)nb * nb * N;     // 2 * kRedBlocks partial sums
  double* sc = part + 2 * kRedBlocks;
  const unsigned bn = nblk(n), bc = nblk(N);
  auto dot = [&](const double* a, const double* c, int slot) {
    dot_partial<<<kRedBlocks, kRedThreads, 0, s>>>(n, a, c, part);
    dot_final<<<1, kRedThreads, 0, s>>>(part, sc + slot);
  };
  auto apply = [&](const double* in, double* out) {
    if (nb == 3) bj_apply_kernel<3><<<bc, 256, 0, s>>>(N, dinv, in, out);
    else if (nb == 2) bj_apply_kernel<2><<<bc, 256, 0, s>>>(N, dinv, in, out);
    else bj_apply_kernel<1><<<bc, 256, 0, s>>>(N, dinv, in, out);
  };
  cudaError_t e = cudaSuccess;
  const WellSchur wsv = ws ? *ws : WellSchur{nullptr, nullptr, nullptr};
  if (nb == 3)
    block_jacobi_kernel<3><<<bc, 256, 0, s>>>(g->prm, g->d_row_ptr, val, dinv, transpose, g->d_status,
                                              g->d_perf_of_cell, g->d_perf, wsv);
  else if (nb == 2)
    block_jacobi_kernel<2><<<bc, 256, 0, s>>>(g->prm, g->d_row_ptr, val, dinv, transpose, g->d_status,
                                              g->d_perf_of_cell, g->d_perf, wsv);
  else
    block_jacobi_kernel<1><<<bc, 256, 0, s>>>(g->prm, g->d_row_ptr, val, dinv, transpose, g->d_status,
                                              g->d_perf_of_cell, g->d_perf, wsv);
  // Left block-Jacobi preconditioning: BiCGSTAB on D^-1 A x = D^-1 b, so the
  // residual that is tested is scaled cell by cell into the units of the
  // unknowns (psi, saturation, scf/stb) and no equation dominates its norm.
  // y = D^-1 b and r = D^-1 (b - A x)
  apply(b, y);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_spmv(g, val, -1.0, x, 1.0, t, transpose, s, nb);
  if (e == cudaSuccess && ws) e = launch_well_schur(g, *ws, 0, 1.0, x, t, nullptr, nullptr, s);
  apply(t, r);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r0, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(double) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(double) * n, s);
  scal_init<<<1, 1, 0, s>>>(sc);
  dot(y, y, S_BB);
  dot(r, r, S_RR);
  double h[S_COUNT];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_bicgstab: %s", cudaGetErrorString(e));
  const double bnorm = std::sqrt(h[S_BB]);
  const double target = rtol * (bnorm > 0.0 ? bnorm : 1.0);
  // One iteration's kernels; the loop's test runs on the device (at the end
  // of the previous iteration, in the last CTA of upd_xr_dot), so kItersPerGraph
  // iterations are captured once into a CUDA graph, kept on the grid for the
  // same buffers, and replayed until S_DONE.
  auto iteration = [&](cudaStream_t cs) {
    auto op_s = [&](const double* in, double* out) {
      cudaError_t err = launch_spmv(g, val, 1.0, in, 0.0, out, transpose, cs, nb, sc + S_DONE);
      if (err == cudaSuccess && ws) err = launch_well_schur(g, *ws, 0, -1.0, in, out, nullptr, nullptr, cs, sc + S_DONE);
      return err;
    };
    cudaError_t err = cudaSuccess;
    // p = r + beta (p - omega v)   (beta from the end of the previous iteration)
    upd_p<<<bn, 256, 0, cs>>>(n, r, p, v, sc);
    // v = D^-1 A p, then alpha = rho / (r0 . v)
    if (err == cudaSuccess) err = op_s(p, z);
    if (nb == 3) apply_dot<3><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, v, r0, sc, part);
    else if (nb == 2) apply_dot<2><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, v, r0, sc, part);
    else apply_dot<1><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, v, r0, sc, part);
    upd_s<<<bn, 256, 0, cs>>>(n, r, v, sv, sc);
    // t = D^-1 A s, then omega = (t . s) / (t . t)
    if (err == cudaSuccess) err = op_s(sv, z);
    if (nb == 3) apply_dot2<3><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, t, sv, sc, part);
    else if (nb == 2) apply_dot2<2><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, t, sv, sc, part);
    else apply_dot2<1><<<kRedBlocks, kRedThreads, 0, cs>>>(n, dinv, z, t, sv, sc, part);
    // x += alpha p + omega s;  r = s - omega t;  then the loop's test, rho and beta
    upd_xr_dot<<<kRedBlocks, kRedThreads, 0, cs>>>(n, x, p, sv, r, t, r0, sc, part);
    return err;
  };
  const void* key[8] = {val, work, x, ws ? ws->bs : nullptr, ws ? ws->cs : nullptr, ws ? ws->d : nullptr,
                        (const void*)(intptr_t)(transpose ? 1 : 0), (const void*)(intptr_t)nb};
  bool same = g->solve_exec != nullptr;
  for (int k = 0; k < 8 && same; ++k) same = g->solve_key[k] == key[k];
  if (!same) {
    if (g->solve_exec) {
      cudaGraphExecDestroy(g->solve_exec);
      g->solve_exec = nullptr;
    }
    if (!g->solve_cap) e = cudaStreamCreateWithFlags(&g->solve_cap, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(g->solve_cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t er = cudaSuccess;
      for (int k = 0; k < kItersPerGraph && er == cudaSuccess; ++k) er = iteration(g->solve_cap);
      e = cudaStreamEndCapture(g->solve_cap, &graph);
      if (e == cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->solve_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_bicgstab capture: %s", cudaGetErrorString(e));
    for (int k = 0; k < 8; ++k) g->solve_key[k] = key[k];
  }
  iter_setup<<<1, 1, 0, s>>>(sc, target, (double)maxit);
  // the loop's first test and the first rho and beta
  dot2_partial<<<kRedBlocks, kRedThreads, 0, s>>>(n, r, r, r0, r, part);
  fin_kernel<kFinRrRho><<<1, kRedThreads, 0, s>>>(part, sc);
  const int max_replays = maxit / kItersPerGraph + 2;
  for (int rep = 0; rep < max_replays; ++rep) {
    e = cudaGraphLaunch(g->solve_exec, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_bicgstab: %s", cudaGetErrorString(e));
    if (h[S_DONE] != 0.0) break;
  }
  const int it = (int)h[S_ITER];
  const double res = std::sqrt(h[S_RR]);
  if (iters) *iters = it;
  if (relres) *relres = bnorm > 0.0 ? res / bnorm : res;
  if (!std::isfinite(res)) return report(OCP_ERR_NONFINITE, "ocp_bicgstab: non-finite residual");
  if (res > target) return report(OCP_ERR_TIMEOUT, "ocp_bicgstab: no convergence in %d iterations (relres %.3e)",
                                  it, bnorm > 0.0 ? res / bnorm : res);
  return OCP_OK;
}

}  // namespace ocp

namespace {

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

extern "C" {

int64_t ocp_solver_work_doubles(const ocp_grid* g) { return g ? ocp::solver_work_doubles(g) : 0; }

ocp_status ocp_bicgstab(ocp_grid* g, const double* val, const double* b, double* x, double rtol, int maxit,
                        int transpose, double* work, int* iters, double* relres, void* stream) {
  using namespace ocp;
  if (!g || !val || !b || !x || !work) return report(OCP_ERR_INVALID_ARG, "grid, val, b, x and work are required");
  if (b == x) return report(OCP_ERR_INVALID_ARG, "b and x must not overlap");
  Guard guard(g->device);
  if (guard.err != cudaSuccess) return report(OCP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(guard.err));
  return bicgstab_run(g, val, nullptr, b, x, rtol, maxit, transpose, work, iters, relres, (cudaStream_t)stream);
}

ocp_status ocp_newton_update(ocp_grid* g, double* u, int8_t* flag, const double* du, double scale,
                             double ds_max, double* du_max, int* nswitch, void* stream) {
  using namespace ocp;
  if (!g || !u || !du || !du_max || !nswitch || (g->prm.nb == 3 && !flag))
    return report(OCP_ERR_INVALID_ARG, "grid, u, flag, du, du_max and nswitch are required");
  if (!(ds_max > 0.0)) return report(OCP_ERR_INVALID_ARG, "ds_max must be > 0");
  Guard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = cudaMemsetAsync(du_max, 0, sizeof(double) * (g->prm.nb + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(nswitch, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(du_max);
    if (g->prm.nb == 3)
      newton_update_kernel<3><<<nblk(g->prm.N), 256, 0, s>>>(g->prm, g->d_table, u, flag, du, scale, ds_max, dm, nswitch);
    else
      newton_update_kernel<2><<<nblk(g->prm.N), 256, 0, s>>>(g->prm, g->d_table, u, flag, du, scale, ds_max, dm, nswitch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_newton_update: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_well_rates_vjp(ocp_grid* g, const double* u, const int8_t* flag, const double* q_bar,
                              double* g_u, double* g_lnk, void* stream) {
  using namespace ocp;
  if (!g || !u || !q_bar || (g->prm.nb == 3 && !flag))
    return report(OCP_ERR_INVALID_ARG, "grid, u, flag and q_bar are required");
  if (g->nperf == 0) return OCP_OK;
  Guard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (g->prm.nb == 3)
    well_vjp_kernel<3><<<nblk(g->nperf, 64), 64, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, g->d_perf, g->nperf,
                                                         q_bar, g_u, g_lnk);
  else
    well_vjp_kernel<2><<<nblk(g->nperf, 64), 64, 0, s>>>(g->prm, g->d_table, u, flag, g->d_phi, g->d_perf, g->nperf,
                                                         q_bar, g_u, g_lnk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_well_rates_vjp: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_grid_update_perm(ocp_grid* g, const double* lnk, void* stream) {
  using namespace ocp;
  if (!g || !lnk) return report(OCP_ERR_INVALID_ARG, "grid and lnk are required");
  Guard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = launch_setup(g, lnk, g->dx, g->dy, g->prm.dz, g->kz_over_kx, s);
  if (e == cudaSuccess) e = launch_perf_wi(g, lnk, s);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_grid_update_perm: %s", cudaGetErrorString(e));
  return OCP_OK;
}

}  // extern "C"
