// FIM linearisation kernels: cell terms, connection terms, assembly.
//
// The Newton linearisation of Sec. 3.2.5 (steps 1 and 3) split the way the
// paper splits the reservoir (Sec. 3.2.3-3.2.4):
//   cell_kernel      PVT/SAT/ROCK properties with derivatives, accumulation
//                    (ACCU) and well (AllWells) terms of every cell;
//   face_kernel      the upwinded two-point flux of every face, computed
//                    exactly once (BulkConn).  The thread of cell c handles
//                    its +x, +y, +z faces: it writes the two off-diagonal
//                    blocks of each face straight into the Jacobian, adds the
//                    face to its own residual and diagonal block, and hands
//                    the + neighbour its share (flux and diagonal block);
//   assemble_kernel  every cell subtracts the shares handed to it and writes
//                    its residual and diagonal block.
// No atomics: every output entry has one writer and a fixed summation order
// (own terms, +x, +y, +z, then -z, -y, -x), independent of the launch shape.
// On GB300 the FP64 pipe, not HBM, bounds these kernels, so each face is
// computed once and results travel through (coalesced, variable-major)
// scratch rather than being recomputed.
#include "ocp_internal.cuh"
#include "kernels.cuh"

namespace ocp {

namespace {

// scratch layout, doubles per cell, variable-major: [field * N + cell]
constexpr int kQ = 25;      // CellQ fields            0 .. 24
constexpr int kSelf = 25;   // own residual (3) + diagonal (9)   25 .. 36
constexpr int kPart = 37;   // after the +faces                  37 .. 48
constexpr int kInc = 49;    // shares handed over, 3 x (F 3 + dj 9)   49 .. 84

// CellQ fields each block size reads (the two-phase path skips the gas and
// dissolved-gas fields).
template <int NB>
__device__ __forceinline__ bool q_used(int f) {
  if (NB == 3) return true;
  return !(f == 2 || f == 4 || f == 9 || f == 10 || f == 11 || f == 18 || f >= 19);
}

template <int NB>
__device__ __forceinline__ void store_q(double* s, long long N, long long c, const CellQ& q) {
  const double* f = reinterpret_cast<const double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    if (q_used<NB>(i)) s[i * N + c] = f[i];
}
template <int NB>
__device__ __forceinline__ void load_q(const double* __restrict__ s, long long N, long long c, CellQ& q) {
  double* f = reinterpret_cast<double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i] = q_used<NB>(i) ? s[i * N + c] : 0.0;
}

template <int NB>
__global__ void __launch_bounds__(256) cell_kernel(Params P, const Table* __restrict__ gT,
                                                   const double* __restrict__ u_new,
                                                   const int8_t* __restrict__ f_new,
                                                   const double* __restrict__ u_old,
                                                   const int8_t* __restrict__ f_old,
                                                   const double* __restrict__ phi,
                                                   const int32_t* __restrict__ perf_of_cell,
                                                   const Perf* __restrict__ perf, double scale,
                                                   double* __restrict__ scr, int* status) {
  __shared__ Table T;
  for (int i = threadIdx.x; i < (int)(sizeof(Table) / 8); i += blockDim.x)
    reinterpret_cast<double*>(&T)[i] = reinterpret_cast<const double*>(gT)[i];
  __syncthreads();
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const double pn = u_new[c], swn = u_new[N + c], xn = (NB == 3) ? u_new[2 * N + c] : 0.0;
  const double po = u_old[c], swo = u_old[N + c], xo = (NB == 3) ? u_old[2 * N + c] : 0.0;
  const int fn = (NB == 3) ? f_new[c] : 0, fo = (NB == 3) ? f_old[c] : 0;
  int bad = 0;
  if (!(finite(pn) && finite(swn) && finite(xn) && finite(po) && finite(swo) && finite(xo))) bad |= kStatNonFinite;
  if ((unsigned)fn > 1u || (unsigned)fo > 1u) bad |= kStatBadFlag;
  if (bad) atomicOr(status, bad);
  // pore volume over dt folded into the porosity: the amounts come out as
  // accumulation terms directly
  const double phs = phi[c] * scale;
  const int ip = perf_of_cell[c];
  const bool inj = ip >= 0 && perf[ip].kind == 1;
  CellQ q{};
  CellAux a{};
  cell_quantities<NB, true>(P, T, pn, swn, xn, fn & 1, phs, q, a, inj);
  double mo[3];
  cell_masses<NB, false>(P, T, po, swo, xo, fo & 1, phs, mo);
  double r[3], dg[3][3];
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    r[e] = a.m[e] - mo[e];
    dg[e][0] = a.m_p[e];
    dg[e][1] = a.m_sw[e];
    dg[e][2] = a.m_x[e];
  }
  if (ip >= 0) {
    // the well terms need the true (unscaled) injector mobility only
    double src[3], ds[3][3];
    well_source<NB>(perf[ip], q, a, src, ds);
    for (int e = 0; e < NB; ++e) {
      r[e] -= src[e];
      for (int v = 0; v < NB; ++v) dg[e][v] -= ds[e][v];
    }
  }
  store_q<NB>(scr, N, c, q);
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    scr[(kSelf + e) * N + c] = r[e];
#pragma unroll
    for (int v = 0; v < NB; ++v) scr[(kSelf + 3 + 3 * e + v) * N + c] = dg[e][v];
  }
}

template <int NB>
__global__ void __launch_bounds__(256) face_kernel(Params P, const double* __restrict__ trans,
                                                   const int32_t* __restrict__ row_ptr,
                                                   double* __restrict__ scr, double* __restrict__ val,
                                                   double* __restrict__ face_flux) {
  constexpr int B2 = NB * NB;
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int i = (int)(c % P.nx);
  const int j = (int)((c / P.nx) % P.ny);
  const int k = (int)(c / P.nxy);
  const bool hm[3] = {i > 0, j > 0, k > 0};
  const bool hp[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  const long long stride[3] = {1, P.nx, P.nxy};
  CellQ a;
  load_q<NB>(scr, N, c, a);
  double r[NB], dg[NB][NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    r[e] = scr[(kSelf + e) * N + c];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[e][v] = scr[(kSelf + 3 + 3 * e + v) * N + c];
  }
  const long long row0 = row_ptr[c];
  int slot = (int)hm[0] + (int)hm[1] + (int)hm[2] + 1;   // first + block of this row
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!hp[d]) {
      if (face_flux)
        for (int e = 0; e < NB; ++e) face_flux[(d * NB + e) * N + c] = 0.0;
      continue;
    }
    const long long n = c + stride[d];
    CellQ b;
    load_q<NB>(scr, N, n, b);
    FaceOut<NB> o;
    const double T = trans[d * N + c];
    if (d == 2) face_terms<NB, true>(T, -P.grav_dz, a, b, o);
    else face_terms<NB, false>(T, 0.0, a, b, o);
    // this row: flux out, diagonal, and the block of the + neighbour
    double* blk = val + (row0 + slot) * B2;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      r[e] += o.F[e];
#pragma unroll
      for (int v = 0; v < NB; ++v) {
        dg[e][v] += o.di[e][v];
        blk[e * NB + v] = o.dj[e][v];
      }
    }
    ++slot;
    // the + neighbour's row: its block of this cell, and its share
    const int slot_n = (d == 0) ? ((int)hm[2] + (int)hm[1]) : (d == 1 ? (int)hm[2] : 0);
    double* nblk = val + ((long long)row_ptr[n] + slot_n) * B2;
    const int base = kInc + 12 * d;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      scr[(base + e) * N + n] = o.F[e];
#pragma unroll
      for (int v = 0; v < NB; ++v) {
        nblk[e * NB + v] = neg(o.di[e][v]);
        scr[(base + 3 + 3 * e + v) * N + n] = o.dj[e][v];
      }
      if (face_flux) face_flux[(d * NB + e) * N + c] = o.F[e];
    }
  }
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    scr[(kPart + e) * N + c] = r[e];
#pragma unroll
    for (int v = 0; v < NB; ++v) scr[(kPart + 3 + 3 * e + v) * N + c] = dg[e][v];
  }
}

template <int NB>
__global__ void __launch_bounds__(256) assemble_kernel(Params P, const int32_t* __restrict__ row_ptr,
                                                       const double* __restrict__ scr,
                                                       double* __restrict__ res, double* __restrict__ val,
                                                       int* status) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int i = (int)(c % P.nx);
  const int j = (int)((c / P.nx) % P.ny);
  const int k = (int)(c / P.nxy);
  const bool hm[3] = {i > 0, j > 0, k > 0};
  double r[NB], dg[NB][NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    r[e] = scr[(kPart + e) * N + c];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[e][v] = scr[(kPart + 3 + 3 * e + v) * N + c];
  }
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (!hm[d]) continue;
    const int base = kInc + 12 * d;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      r[e] -= scr[(base + e) * N + c];
#pragma unroll
      for (int v = 0; v < NB; ++v) dg[e][v] -= scr[(base + 3 + 3 * e + v) * N + c];
    }
  }
  double* out = val + ((long long)row_ptr[c] + (int)hm[0] + (int)hm[1] + (int)hm[2]) * NB * NB;
  bool ok = true;
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    res[c * NB + e] = r[e];
    ok = ok && finite(r[e]);
#pragma unroll
    for (int v = 0; v < NB; ++v) out[e * NB + v] = dg[e][v];
  }
  if (!ok) atomicOr(status, kStatNonFinite);
}

template <int NB>
void launch_all(const ocp_grid* g, double* scratch, const double* u_new, const int8_t* f_new,
                const double* u_old, const int8_t* f_old, double dt, double* res, double* val,
                double* face_flux, cudaStream_t s) {
  const Params& P = g->prm;
  const int threads = 256;
  const unsigned blocks = (unsigned)((P.N + threads - 1) / threads);
  const double scale = P.vol_rb / dt;
  cell_kernel<NB><<<blocks, threads, 0, s>>>(P, g->d_table, u_new, f_new, u_old, f_old, g->d_phi,
                                             g->d_perf_of_cell, g->d_perf, scale, scratch, g->d_status);
  face_kernel<NB><<<blocks, threads, 0, s>>>(P, g->d_trans, g->d_row_ptr, scratch, val, face_flux);
  assemble_kernel<NB><<<blocks, threads, 0, s>>>(P, g->d_row_ptr, scratch, res, val, g->d_status);
}

}  // namespace

// 85 doubles per cell are used; 100 are reserved.
int64_t linearize_scratch_doubles(int64_t N) { return (int64_t)100 * N; }

cudaError_t launch_linearize(const ocp_grid* g, const double* u_new, const int8_t* f_new,
                             const double* u_old, const int8_t* f_old, double dt, double* res,
                             double* val, double* face_flux, cudaStream_t s) {
  if (g->prm.nb == 3) launch_all<3>(g, g->d_scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s);
  else launch_all<2>(g, g->d_scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s);
  return cudaGetLastError();
}

cudaError_t launch_linearize_scratch(const ocp_grid* g, double* scratch, const double* u_new,
                                     const int8_t* f_new, const double* u_old, const int8_t* f_old, double dt,
                                     double* res, double* val, double* face_flux, cudaStream_t s) {
  if (g->prm.nb == 3) launch_all<3>(g, scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s);
  else launch_all<2>(g, scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s);
  return cudaGetLastError();
}

}  // namespace ocp
