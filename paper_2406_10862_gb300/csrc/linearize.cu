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
//
// Every kernel walks a list of tiles -- TPB consecutive cells of one model --
// with its CTAs striding over the list.  A single grid is the one-model case
// (its arguments passed by value, tiles implied); a batch of grids passes a
// device table of per-model arguments and an explicit tile list.  Both run
// the same kernels, so a batched linearisation is bit-identical to the
// per-grid one, whatever the tile size or the number of CTAs.
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
__device__ __forceinline__ void cell_body(const ModelArgs& M, const Table& T, long long c) {
  const Params& P = M.P;
  const long long N = P.N;
  const double* __restrict__ u_new = M.u_new;
  const double* __restrict__ u_old = M.u_old;
  double* __restrict__ scr = M.scr;
  const double pn = u_new[c], swn = u_new[N + c], xn = (NB == 3) ? u_new[2 * N + c] : 0.0;
  const double po = u_old[c], swo = u_old[N + c], xo = (NB == 3) ? u_old[2 * N + c] : 0.0;
  const int fn = (NB == 3) ? M.f_new[c] : 0, fo = (NB == 3) ? M.f_old[c] : 0;
  int bad = 0;
  if (!(finite(pn) && finite(swn) && finite(xn) && finite(po) && finite(swo) && finite(xo))) bad |= kStatNonFinite;
  if ((unsigned)fn > 1u || (unsigned)fo > 1u) bad |= kStatBadFlag;
  if (bad) atomicOr(M.status, bad);
  // pore volume over dt folded into the porosity: the amounts come out as
  // accumulation terms directly
  const double phs = M.phi[c] * M.scale;
  const int ip = M.perf_of_cell[c];
  const bool inj = ip >= 0 && M.perf[ip].kind == 1;
  CellQ q{};
  CellAux a{};
  cell_quantities<NB, true>(P, T, pn, swn, xn, fn & 1, phs, q, a, inj);
  double r[3], dg[3][3];
  if (!M.no_acc) {
    double mo[3];
    cell_masses<NB, false>(P, T, po, swo, xo, fo & 1, phs, mo);
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      r[e] = a.m[e] - mo[e];
      dg[e][0] = a.m_p[e];
      dg[e][1] = a.m_sw[e];
      dg[e][2] = a.m_x[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < NB; ++e) r[e] = dg[e][0] = dg[e][1] = dg[e][2] = 0.0;
  }
  if (ip >= 0) {
    double src[3], ds[3][3];
    Perf w = M.perf[ip];
    if (M.p_bh) w.p_bh = M.p_bh[w.well];
    well_source<NB>(w, q, a, src, ds);
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
__device__ __forceinline__ void face_body(const ModelArgs& M, long long c) {
  constexpr int B2 = NB * NB;
  const Params& P = M.P;
  const long long N = P.N;
  double* __restrict__ scr = M.scr;
  double* __restrict__ val = M.val;
  double* __restrict__ face_flux = M.face_flux;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
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
  const long long row0 = row_start_ijk(P, c, i, j, k);   // the row pointers in closed form: no loads
  int slot = (int)hm[0] + (int)hm[1] + (int)hm[2] + 1;   // first + block of this row
#pragma unroll 1
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
    const double T = M.trans[d * N + c];
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
    double* nblk = val + (row_start_ijk(P, n, i + (d == 0), j + (d == 1), k + (d == 2)) + slot_n) * B2;
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
__device__ __forceinline__ void assemble_body(const ModelArgs& M, long long c) {
  const Params& P = M.P;
  const long long N = P.N;
  const double* __restrict__ scr = M.scr;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
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
  double* out = M.val + (row_start_ijk(P, c, i, j, k) + (int)hm[0] + (int)hm[1] + (int)hm[2]) * NB * NB;
  bool ok = true;
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    M.res[c * NB + e] = r[e];
    ok = ok && finite(r[e]);
#pragma unroll
    for (int v = 0; v < NB; ++v) out[e * NB + v] = dg[e][v];
  }
  if (!ok) atomicOr(M.status, kStatNonFinite);
}

// The model and first cell of tile t.
template <int TPB>
__device__ __forceinline__ const ModelArgs& tile_of(const TileList& L, const ModelArgs& single, int t,
                                                     int& m, long long& c0) {
  if (L.models) {
    const int2 tt = L.tiles[t];
    m = tt.x;
    c0 = tt.y;
    return L.models[m];
  }
  m = 0;
  c0 = (long long)t * TPB;
  return single;
}

template <int NB, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) cell_kernel(TileList L, ModelArgs single) {
  __shared__ Table T;
  int cur = -1;
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<TPB>(L, single, t, m, c0);
    if (m != cur) {                      // the PVT table of this tile's model
      __syncthreads();
      for (int i = threadIdx.x; i < (int)(sizeof(Table) / 8); i += TPB)
        reinterpret_cast<double*>(&T)[i] = reinterpret_cast<const double*>(M.table)[i];
      __syncthreads();
      cur = m;
    }
    const long long c = c0 + threadIdx.x;
    if (c < M.P.N) cell_body<NB>(M, T, c);
  }
}

template <int NB, int TPB>
__global__ void __launch_bounds__(TPB, (NB == 3 ? 384 : 512) / TPB) face_kernel(TileList L, ModelArgs single) {
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<TPB>(L, single, t, m, c0);
    const long long c = c0 + threadIdx.x;
    if (c < M.P.N) face_body<NB>(M, c);
  }
}

template <int NB, int TPB>
__global__ void __launch_bounds__(TPB) assemble_kernel(TileList L, ModelArgs single) {
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<TPB>(L, single, t, m, c0);
    const long long c = c0 + threadIdx.x;
    if (c < M.P.N) assemble_body<NB>(M, c);
  }
}

template <int NB, int TPB>
void launch_stage(int stage, const TileList& L, const ModelArgs& single, int grid, cudaStream_t s) {
  if (stage == 0) cell_kernel<NB, TPB><<<grid, TPB, 0, s>>>(L, single);
  else if (stage == 1) face_kernel<NB, TPB><<<grid, TPB, 0, s>>>(L, single);
  else assemble_kernel<NB, TPB><<<grid, TPB, 0, s>>>(L, single);
}

}  // namespace

// Launches the three stages.  `lists[0]` / `lists[1]` are the tile lists for
// 128 / 256 cells per tile; cfg picks, per stage, the tile size and the grid
// (CTAs per SM times the SM count, or 0 for one CTA per tile; a negative
// count skips the stage, which only the autotuner uses).
cudaError_t launch_tiles(int nb, const TileList* lists, const ModelArgs& single, const LaunchCfg& cfg,
                         int sms, cudaStream_t s) {
  for (int stage = 0; stage < 3; ++stage) {
    if (cfg.ctas_per_sm[stage] < 0) continue;
    const int tpb = cfg.tpb[stage] == 128 ? 128 : 256;
    const TileList& L = lists[tpb == 128 ? 0 : 1];
    if (L.ntiles == 0) continue;
    int grid = cfg.ctas_per_sm[stage] > 0 ? cfg.ctas_per_sm[stage] * sms : L.ntiles;
    if (grid > L.ntiles) grid = L.ntiles;
    if (nb == 3) {
      if (tpb == 128) launch_stage<3, 128>(stage, L, single, grid, s);
      else launch_stage<3, 256>(stage, L, single, grid, s);
    } else {
      if (tpb == 128) launch_stage<2, 128>(stage, L, single, grid, s);
      else launch_stage<2, 256>(stage, L, single, grid, s);
    }
  }
  return cudaGetLastError();
}

ModelArgs model_args(const ocp_grid* g, double* scratch, const double* u_new, const int8_t* f_new,
                     const double* u_old, const int8_t* f_old, double dt, double* res, double* val,
                     double* face_flux) {
  ModelArgs M;
  M.P = g->prm;
  M.table = g->d_table;
  M.trans = g->d_trans;
  M.row_ptr = g->d_row_ptr;
  M.phi = g->d_phi;
  M.perf_of_cell = g->d_perf_of_cell;
  M.perf = g->d_perf;
  M.status = g->d_status;
  M.scr = scratch;
  M.u_new = u_new;
  M.f_new = f_new;
  M.u_old = u_old;
  M.f_old = f_old;
  M.res = res;
  M.val = val;
  M.face_flux = face_flux;
  M.scale = g->prm.vol_rb / dt;
  M.p_bh = nullptr;
  M.no_acc = 0;
  return M;
}

namespace {

cudaError_t launch_single(const ocp_grid* g, double* scratch, const double* u_new, const int8_t* f_new,
                          const double* u_old, const int8_t* f_old, double dt, double* res, double* val,
                          double* face_flux, cudaStream_t s, const double* p_bh = nullptr, int no_acc = 0) {
  ModelArgs M = model_args(g, scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux);
  M.p_bh = p_bh;
  M.no_acc = no_acc;
  TileList lists[2];
  lists[0].models = nullptr;
  lists[0].tiles = nullptr;
  lists[0].ntiles = (int)((g->prm.N + 127) / 128);
  lists[1] = lists[0];
  lists[1].ntiles = (int)((g->prm.N + 255) / 256);
  return launch_tiles(g->prm.nb, lists, M, g->cfg, g->sms, s);
}

}  // namespace

// 85 doubles per cell are used; 100 are reserved.
int64_t linearize_scratch_doubles(int64_t N) { return (int64_t)100 * N; }

cudaError_t launch_linearize(const ocp_grid* g, const double* u_new, const int8_t* f_new,
                             const double* u_old, const int8_t* f_old, double dt, double* res,
                             double* val, double* face_flux, cudaStream_t s, const double* p_bh, int no_acc) {
  return launch_single(g, g->d_scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s, p_bh, no_acc);
}

cudaError_t launch_linearize_scratch(const ocp_grid* g, double* scratch, const double* u_new,
                                     const int8_t* f_new, const double* u_old, const int8_t* f_old, double dt,
                                     double* res, double* val, double* face_flux, cudaStream_t s) {
  return launch_single(g, scratch, u_new, f_new, u_old, f_old, dt, res, val, face_flux, s);
}

}  // namespace ocp
