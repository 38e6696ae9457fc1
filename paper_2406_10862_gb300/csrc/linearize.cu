// FIM linearisation kernels: cell terms, connection terms, assembly.
//
// The Newton linearisation of Sec. 3.2.5 (steps 1 and 3) split the way the
// paper splits the reservoir (Sec. 3.2.3-3.2.4):
//   cell_kernel      PVT/SAT/ROCK properties with derivatives, accumulation
//                    (ACCU) and well (AllWells) terms of every cell;
//   face_kernel      the upwinded two-point flux of every face, computed
//                    exactly once, with derivatives for both cells (BulkConn);
//   assemble_kernel  every cell writes its own block row and residual (no
//                    atomics), summing in a fixed order: own terms, then faces
//                    -z, -y, -x, +x, +y, +z.
// Intermediate per-cell and per-face results live in the grid's scratch
// buffer, variable-major so that every access is coalesced.
#include "ocp_internal.cuh"
#include "kernels.cuh"

namespace ocp {

namespace {

constexpr int kQ = 25;        // stored CellQ fields
constexpr int kSelf = 25;     // residual (3) + diagonal block (9)
constexpr int kFace = 37;     // 3 directions x (F 3 + di 9 + dj 9)

__device__ __forceinline__ void store_q(double* s, long long N, long long c, const CellQ& q) {
  const double* f = reinterpret_cast<const double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i) s[i * N + c] = f[i];
}
__device__ __forceinline__ void load_q(const double* __restrict__ s, long long N, long long c, CellQ& q) {
  double* f = reinterpret_cast<double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i] = s[i * N + c];
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
  const double ph = phi[c];
  CellQ q{};
  CellAux a{};
  cell_quantities<NB, true>(P, T, pn, swn, xn, fn & 1, ph, q, a);
  double mo[3];
  cell_masses<NB>(P, T, po, swo, xo, fo & 1, ph, mo);
  double r[3], dg[3][3];
  for (int e = 0; e < NB; ++e) {
    r[e] = (a.m[e] - mo[e]) * scale;
    dg[e][0] = a.m_p[e] * scale;
    dg[e][1] = a.m_sw[e] * scale;
    dg[e][2] = a.m_x[e] * scale;
  }
  const int ip = perf_of_cell[c];
  if (ip >= 0) {
    double src[3], ds[3][3];
    well_source<NB>(perf[ip], q, a, src, ds);
    for (int e = 0; e < NB; ++e) {
      r[e] -= src[e];
      for (int v = 0; v < NB; ++v) dg[e][v] -= ds[e][v];
    }
  }
  store_q(scr, N, c, q);
  for (int e = 0; e < NB; ++e) {
    scr[(kSelf + e) * N + c] = r[e];
    for (int v = 0; v < NB; ++v) scr[(kSelf + 3 + 3 * e + v) * N + c] = dg[e][v];
  }
}

template <int NB>
__global__ void __launch_bounds__(256) face_kernel(Params P, const double* __restrict__ trans,
                                                   double* __restrict__ scr,
                                                   double* __restrict__ face_flux) {
  const long long N = P.N;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= N) return;
  const int i = (int)(c % P.nx);
  const int j = (int)((c / P.nx) % P.ny);
  const int k = (int)(c / P.nxy);
  const bool has[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  const long long stride[3] = {1, P.nx, P.nxy};
  CellQ a;
  load_q(scr, N, c, a);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int base = kFace + 21 * d;
    FaceOut<NB> o;
    if (has[d]) {
      CellQ b;
      load_q(scr, N, c + stride[d], b);
      const double T = trans[d * N + c];
      if (d == 2) face_terms<NB, true>(T, -P.grav_dz, a, b, o);
      else face_terms<NB, false>(T, 0.0, a, b, o);
    } else {
      for (int e = 0; e < NB; ++e) {
        o.F[e] = 0.0;
        for (int v = 0; v < NB; ++v) o.di[e][v] = o.dj[e][v] = 0.0;
      }
    }
    for (int e = 0; e < NB; ++e) {
      scr[(base + e) * N + c] = o.F[e];
      for (int v = 0; v < NB; ++v) {
        scr[(base + 3 + 3 * e + v) * N + c] = o.di[e][v];
        scr[(base + 12 + 3 * e + v) * N + c] = o.dj[e][v];
      }
      if (face_flux) face_flux[(d * NB + e) * N + c] = o.F[e];
    }
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
  const bool hp[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  const long long stride[3] = {1, P.nx, P.nxy};
  double r[3], dg[3][3];
  for (int e = 0; e < NB; ++e) {
    r[e] = scr[(kSelf + e) * N + c];
    for (int v = 0; v < NB; ++v) dg[e][v] = scr[(kSelf + 3 + 3 * e + v) * N + c];
  }
  double* out = val + (long long)row_ptr[c] * NB * NB;
  int slot = 0;
  // faces where this cell is the + side: -z, -y, -x
  for (int d = 2; d >= 0; --d) {
    if (!hm[d]) continue;
    const long long n = c - stride[d];
    const int base = kFace + 21 * d;
    for (int e = 0; e < NB; ++e) {
      r[e] -= scr[(base + e) * N + n];
      for (int v = 0; v < NB; ++v) {
        dg[e][v] -= scr[(base + 12 + 3 * e + v) * N + n];
        out[slot * NB * NB + e * NB + v] = -scr[(base + 3 + 3 * e + v) * N + n];
      }
    }
    ++slot;
  }
  const int diag = slot++;
  // faces where this cell is the - side: +x, +y, +z
  for (int d = 0; d < 3; ++d) {
    if (!hp[d]) continue;
    const int base = kFace + 21 * d;
    for (int e = 0; e < NB; ++e) {
      r[e] += scr[(base + e) * N + c];
      for (int v = 0; v < NB; ++v) {
        dg[e][v] += scr[(base + 3 + 3 * e + v) * N + c];
        out[slot * NB * NB + e * NB + v] = scr[(base + 12 + 3 * e + v) * N + c];
      }
    }
    ++slot;
  }
  bool ok = true;
  for (int e = 0; e < NB; ++e) {
    res[c * NB + e] = r[e];
    ok = ok && finite(r[e]);
    for (int v = 0; v < NB; ++v) out[diag * NB * NB + e * NB + v] = dg[e][v];
  }
  if (!ok) atomicOr(status, kStatNonFinite);
}

}  // namespace

int64_t linearize_scratch_doubles(int64_t N) { return (int64_t)(kFace + 63) * N; }

cudaError_t launch_linearize(const ocp_grid* g, const double* u_new, const int8_t* f_new,
                             const double* u_old, const int8_t* f_old, double dt, double* res,
                             double* val, double* face_flux, cudaStream_t s) {
  const Params& P = g->prm;
  const int threads = 256;
  const unsigned blocks = (unsigned)((P.N + threads - 1) / threads);
  const double scale = P.vol_rb / dt;
  if (P.nb == 3) {
    cell_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_table, u_new, f_new, u_old, f_old, g->d_phi,
                                              g->d_perf_of_cell, g->d_perf, scale, g->d_scratch, g->d_status);
    face_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_trans, g->d_scratch, face_flux);
    assemble_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_row_ptr, g->d_scratch, res, val, g->d_status);
  } else {
    cell_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_table, u_new, f_new, u_old, f_old, g->d_phi,
                                              g->d_perf_of_cell, g->d_perf, scale, g->d_scratch, g->d_status);
    face_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_trans, g->d_scratch, face_flux);
    assemble_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_row_ptr, g->d_scratch, res, val, g->d_status);
  }
  return cudaGetLastError();
}

cudaError_t launch_linearize_scratch(const ocp_grid* g, double* scratch, const double* u_new,
                                     const int8_t* f_new, const double* u_old, const int8_t* f_old, double dt,
                                     double* res, double* val, double* face_flux, cudaStream_t s) {
  const Params& P = g->prm;
  const int threads = 256;
  const unsigned blocks = (unsigned)((P.N + threads - 1) / threads);
  const double scale = P.vol_rb / dt;
  if (P.nb == 3) {
    cell_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_table, u_new, f_new, u_old, f_old, g->d_phi,
                                              g->d_perf_of_cell, g->d_perf, scale, scratch, g->d_status);
    face_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_trans, scratch, face_flux);
    assemble_kernel<3><<<blocks, threads, 0, s>>>(P, g->d_row_ptr, scratch, res, val, g->d_status);
  } else {
    cell_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_table, u_new, f_new, u_old, f_old, g->d_phi,
                                              g->d_perf_of_cell, g->d_perf, scale, scratch, g->d_status);
    face_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_trans, scratch, face_flux);
    assemble_kernel<2><<<blocks, threads, 0, s>>>(P, g->d_row_ptr, scratch, res, val, g->d_status);
  }
  return cudaGetLastError();
}

}  // namespace ocp
