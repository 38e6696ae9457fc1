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
// The outputs (Jacobian blocks, residual, face fluxes) are written with
// streaming stores (evict-first), so that they do not push out of L2 the
// scratch the next stage still reads (measured 0.2226 -> 0.2184 ms with three
// launches on the 200 000-cell box).
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
// Scratch loads.  COH: the data was written earlier in the same launch by
// another CTA (the ordered launch), so the load goes through L2, which is
// coherent, instead of a possibly stale L1 line; otherwise a plain load.
template <bool COH>
__device__ __forceinline__ double lds(const double* p) {
  if (COH) return __ldcg(p);
  return *p;
}
template <int NB, bool COH = false>
__device__ __forceinline__ void load_q(const double* s, long long N, long long c, CellQ& q) {
  double* f = reinterpret_cast<double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i] = q_used<NB>(i) ? lds<COH>(s + i * N + c) : 0.0;
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

// The +x, +y, +z faces of cell c (BulkConn): the two off-diagonal blocks of
// each face go straight into the Jacobian, the + neighbour's share (flux and
// diagonal block) into its scratch slots, and this row's residual and
// diagonal block -- its own terms plus its + faces -- come back in r, dg.
template <int NB, bool COH>
__device__ __forceinline__ void face_part(const ModelArgs& M, long long c, double (&r)[NB],
                                          double (&dg)[NB][NB]) {
  constexpr int B2 = NB * NB;
  const Params& P = M.P;
  const long long N = P.N;
  double* scr = M.scr;
  double* __restrict__ val = M.val;
  double* __restrict__ face_flux = M.face_flux;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
  const bool hp[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  const long long stride[3] = {1, P.nx, P.nxy};
  CellQ a;
  load_q<NB, COH>(scr, N, c, a);
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    r[e] = lds<COH>(scr + (kSelf + e) * N + c);
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[e][v] = lds<COH>(scr + (kSelf + 3 + 3 * e + v) * N + c);
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
    load_q<NB, COH>(scr, N, n, b);
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
        __stcs(blk + e * NB + v, o.dj[e][v]);
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
        __stcs(nblk + e * NB + v, neg(o.di[e][v]));
        scr[(base + 3 + 3 * e + v) * N + n] = o.dj[e][v];
      }
      if (face_flux) __stcs(face_flux + (d * NB + e) * N + c, o.F[e]);
    }
  }
}

template <int NB>
__device__ __forceinline__ void face_body(const ModelArgs& M, long long c) {
  const long long N = M.P.N;
  double* scr = M.scr;
  double r[NB], dg[NB][NB];
  face_part<NB, false>(M, c, r, dg);
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    scr[(kPart + e) * N + c] = r[e];
#pragma unroll
    for (int v = 0; v < NB; ++v) scr[(kPart + 3 + 3 * e + v) * N + c] = dg[e][v];
  }
}

// Row c of the residual and its diagonal block: r, dg (own terms and + faces)
// minus the shares its - neighbours handed over, in the fixed order -z, -y,
// -x (LinearSystem assembly, one writer per entry).
template <int NB, bool COH>
__device__ __forceinline__ void assemble_rows(const ModelArgs& M, long long c, double (&r)[NB],
                                              double (&dg)[NB][NB]) {
  const Params& P = M.P;
  const long long N = P.N;
  const double* scr = M.scr;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (!hm[d]) continue;
    const int base = kInc + 12 * d;
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      r[e] -= lds<COH>(scr + (base + e) * N + c);
#pragma unroll
      for (int v = 0; v < NB; ++v) dg[e][v] -= lds<COH>(scr + (base + 3 + 3 * e + v) * N + c);
    }
  }
  double* out = M.val + (row_start_ijk(P, c, i, j, k) + (int)hm[0] + (int)hm[1] + (int)hm[2]) * NB * NB;
  bool ok = true;
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    __stcs(M.res + c * NB + e, r[e]);
    ok = ok && finite(r[e]);
#pragma unroll
    for (int v = 0; v < NB; ++v) __stcs(out + e * NB + v, dg[e][v]);
  }
  if (!ok) atomicOr(M.status, kStatNonFinite);
}

template <int NB>
__device__ __forceinline__ void assemble_body(const ModelArgs& M, long long c) {
  const long long N = M.P.N;
  const double* __restrict__ scr = M.scr;
  double r[NB], dg[NB][NB];
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    r[e] = scr[(kPart + e) * N + c];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[e][v] = scr[(kPart + 3 + 3 * e + v) * N + c];
  }
  assemble_rows<NB, false>(M, c, r, dg);
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
  pdl_wait();
  __shared__ Table T;
  __shared__ unsigned long long bar;
  unsigned uses = 0;
  int cur = -1;
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<TPB>(L, single, t, m, c0);
    if (m != cur) {                      // the PVT table of this tile's model
      __syncthreads();
      load_table(T, M.table, bar, uses, M.status);
      cur = m;
    }
    const long long c = c0 + threadIdx.x;
    if (c < M.P.N) cell_body<NB>(M, T, c);
  }
}

template <int NB, int TPB>
__global__ void __launch_bounds__(TPB, (NB == 3 ? 384 : 512) / TPB) face_kernel(TileList L, ModelArgs single) {
  pdl_wait();
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
  pdl_wait();
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<TPB>(L, single, t, m, c0);
    const long long c = c0 + threadIdx.x;
    if (c < M.P.N) assemble_body<NB>(M, c);
  }
}

// -------------------------------------------------- split face and assembly
// For small grids, whose time is the FP64 instruction count of their warps
// (each FP64 warp instruction holds a sub-partition's FP64 unit 64 cycles):
// the face stage with one warp per direction and the assembly with one warp
// per equation, over 32-cell tiles, so that a warp does a third of a cell's
// work.  Same arithmetic in the same order as face_kernel and
// assemble_kernel: bit-identical results.

// Face d of cell c: the blocks and the + neighbour's share as in face_part;
// this row's own terms (F, dF/du_c) go to own[0..12)[lane] for the combine.
template <int NB>
__device__ __forceinline__ void face_dir(const ModelArgs& M, long long c, int d, double (*own)[32], int lane) {
  constexpr int B2 = NB * NB;
  const Params& P = M.P;
  const long long N = P.N;
  double* scr = M.scr;
  double* __restrict__ face_flux = M.face_flux;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
  const bool hp[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  if (!hp[d]) {
    if (face_flux)
      for (int e = 0; e < NB; ++e) __stcs(face_flux + (d * NB + e) * N + c, 0.0);
    return;
  }
  const long long stride = d == 0 ? 1 : (d == 1 ? (long long)P.nx : P.nxy);
  const long long n = c + stride;
  CellQ a, b;
  load_q<NB>(scr, N, c, a);
  load_q<NB>(scr, N, n, b);
  FaceOut<NB> o;
  const double T = M.trans[d * N + c];
  if (d == 2) face_terms<NB, true>(T, -P.grav_dz, a, b, o);
  else face_terms<NB, false>(T, 0.0, a, b, o);
  const int slot = (int)hm[0] + (int)hm[1] + (int)hm[2] + 1 + (d > 0 && hp[0]) + (d > 1 && hp[1]);
  double* blk = M.val + (row_start_ijk(P, c, i, j, k) + slot) * B2;
  const int slot_n = (d == 0) ? ((int)hm[2] + (int)hm[1]) : (d == 1 ? (int)hm[2] : 0);
  double* nblk = M.val + (row_start_ijk(P, n, i + (d == 0), j + (d == 1), k + (d == 2)) + slot_n) * B2;
  const int base = kInc + 12 * d;
#pragma unroll
  for (int e = 0; e < NB; ++e) {
    own[e][lane] = o.F[e];
    scr[(base + e) * N + n] = o.F[e];
#pragma unroll
    for (int v = 0; v < NB; ++v) {
      own[3 + 3 * e + v][lane] = o.di[e][v];
      __stcs(blk + e * NB + v, o.dj[e][v]);
      __stcs(nblk + e * NB + v, neg(o.di[e][v]));
      scr[(base + 3 + 3 * e + v) * N + n] = o.dj[e][v];
    }
    if (face_flux) __stcs(face_flux + (d * NB + e) * N + c, o.F[e]);
  }
}

template <int NB>
__global__ void __launch_bounds__(96) face_split_kernel(TileList L, ModelArgs single) {
  pdl_wait();
  __shared__ double own[3][12][32];      // [direction][F, dF/du_c][lane]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<32>(L, single, t, m, c0);
    const long long N = M.P.N;
    const long long c = c0 + lane;
    if (c < N) face_dir<NB>(M, c, w, own[w], lane);
    __syncthreads();
    if (c < N && w < NB) {               // warp e: equation e of this row, own terms + faces x, y, z
      int i, j, k;
      cell_ijk(M.P, c, i, j, k);
      const bool hp[3] = {i + 1 < M.P.nx, j + 1 < M.P.ny, k + 1 < M.P.nz};
      double* scr = M.scr;
      const int e = w;
      double r = scr[(kSelf + e) * N + c];
      double dg[NB];
#pragma unroll
      for (int v = 0; v < NB; ++v) dg[v] = scr[(kSelf + 3 + 3 * e + v) * N + c];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!hp[d]) continue;
        r += own[d][e][lane];
#pragma unroll
        for (int v = 0; v < NB; ++v) dg[v] += own[d][3 + 3 * e + v][lane];
      }
      scr[(kPart + e) * N + c] = r;
#pragma unroll
      for (int v = 0; v < NB; ++v) scr[(kPart + 3 + 3 * e + v) * N + c] = dg[v];
    }
    __syncthreads();                     // own[] is reused by the next tile
  }
}

template <int NB>
__global__ void __launch_bounds__(96) assemble_split_kernel(TileList L, ModelArgs single) {
  pdl_wait();
  const int e = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (e >= NB) return;
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<32>(L, single, t, m, c0);
    const long long N = M.P.N;
    const long long c = c0 + lane;
    if (c >= N) continue;
    const double* scr = M.scr;
    int i, j, k;
    cell_ijk(M.P, c, i, j, k);
    const bool hm[3] = {i > 0, j > 0, k > 0};
    double r = scr[(kPart + e) * N + c];
    double dg[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[v] = scr[(kPart + 3 + 3 * e + v) * N + c];
#pragma unroll
    for (int d = 2; d >= 0; --d) {
      if (!hm[d]) continue;
      const int base = kInc + 12 * d;
      r -= scr[(base + e) * N + c];
#pragma unroll
      for (int v = 0; v < NB; ++v) dg[v] -= scr[(base + 3 + 3 * e + v) * N + c];
    }
    double* out = M.val + (row_start_ijk(M.P, c, i, j, k) + (int)hm[0] + (int)hm[1] + (int)hm[2]) * NB * NB;
    __stcs(M.res + c * NB + e, r);
#pragma unroll
    for (int v = 0; v < NB; ++v) __stcs(out + e * NB + v, dg[v]);
    if (!finite(r)) atomicOr(M.status, kStatNonFinite);
  }
}

// ------------------------------------------------------------ ordered launch
// One persistent launch whose CTAs claim work items in a fixed global order
// from a device counter.  An item is the cell stage or the face-and-assembly
// stage of one tile.  Every item an item depends on comes earlier in the
// order, and items are only claimed by running CTAs, so every wait ends: the
// earliest unfinished item never waits.  The waits are nonetheless bounded;
// one that expires sets the status word's timeout bit and the item proceeds.
//
// Order of one model's items (n tiles of T cells, D = ceil(nxy / T) + 1):
// MODE 1 (cell stage run before, by cell_kernel): face(0), face(1), ...;
// MODE 2: cell(0) .. cell(D'-1), then cell(D'+p), face(p) for p = 0, 1, ...,
// then the last D' faces, D' = min(D, n): a face item needs the cells of its
// tile and of the tiles holding its + neighbours, at most ceil(nxy / T) tiles
// ahead.  Models follow one another in the batch's order.
//
// A face item computes its cells' + faces (writing their shares), marks its
// tile's face stage done, waits for the face stages of the tiles holding its
// cells' - neighbours, and assembles its rows: the same arithmetic in the
// same order as face_kernel + assemble_kernel, so results are bit-identical.
constexpr int kWaitLimit = 1 << 22;     // polls of a flag, about 0.4 s at 100 ns each

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Polls *f until it is set, at most kWaitLimit times; false if it never was.
__device__ __forceinline__ bool wait_flag(const int* f) {
  for (int it = 0; it < kWaitLimit; ++it) {
    if (ld_acquire(f)) return true;
    __nanosleep(100);
  }
  return false;
}

// Item k of one model with n tiles in MODE 2: kind 0 cell, 1 face; its tile.
__device__ __forceinline__ void decode_mode2(long long k, long long n, long long D, int& kind, long long& t) {
  const long long Dp = D < n ? D : n;
  if (k < Dp) { kind = 0; t = k; return; }
  const long long j = k - Dp;
  if (j < 2 * (n - Dp)) {
    kind = (int)(j & 1);
    t = kind ? (j >> 1) : Dp + (j >> 1);
    return;
  }
  kind = 1;
  t = n - Dp + (j - 2 * (n - Dp));
}

// Waits (threads 0..5, one flag each) for the tiles holding the cells of up
// to three inclusive cell ranges [lo[q], hi[q]], clamped to [0, N), other
// than tile `self`; returns after a barrier.  Sets the timeout bit on expiry.
template <int TPB>
__device__ __forceinline__ void wait_tiles(const int* flags, const long long (&lo)[3], const long long (&hi)[3],
                                           long long N, long long self, int* status) {
  const int q = threadIdx.x >> 1, side = threadIdx.x & 1;
  if (threadIdx.x < 6) {
    long long a = lo[q] < 0 ? 0 : lo[q];
    long long b = hi[q] >= N ? N - 1 : hi[q];
    if (a <= b) {
      const long long t = side ? b / TPB : a / TPB;    // a range spans at most two tiles
      if (t != self && !wait_flag(flags + t)) atomicOr(status, kStatTimeout);
    }
  }
  __syncthreads();
}

template <int NB, int TPB, int MODE>
__global__ void __launch_bounds__(TPB, (NB == 3 ? 384 : 512) / TPB) ordered_kernel(OrderedList O,
                                                                                    ModelArgs single) {
  pdl_wait();
  __shared__ Table T;
  __shared__ unsigned long long bar;
  __shared__ long long s_tile;
  __shared__ int s_model, s_kind, s_stop;
  unsigned uses = 0;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long item = (long long)atomicAdd(O.counter, 1u);
      s_stop = item >= O.nitems;
      if (!s_stop) {
        int m = 0;
        long long k = item;
        if (O.models) {                       // the model holding the item (binary search)
          int lo = 0, hi = O.nmodels - 1;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((long long)MODE * O.tile_start[mid] <= item) lo = mid; else hi = mid - 1;
          }
          m = lo;
          k = item - (long long)MODE * O.tile_start[m];
        }
        const ModelArgs& M = O.models ? O.models[O.order[m]] : single;
        const long long n = (M.P.N + TPB - 1) / TPB;
        int kind = 1;
        long long t = k;
        if (MODE == 2) decode_mode2(k, n, (M.P.nxy + TPB - 1) / TPB + 1, kind, t);
        s_model = m;
        s_kind = kind;
        s_tile = t;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int mo = s_model, kind = s_kind;
    const long long t = s_tile;
    __syncthreads();                          // everyone has read the item before it is overwritten
    const ModelArgs& M = O.models ? O.models[O.order[mo]] : single;
    const long long N = M.P.N, nx = M.P.nx, nxy = M.P.nxy;
    const long long fbase = O.models ? O.tile_start[mo] : 0;
    const long long c0 = t * TPB, c1 = (c0 + TPB < N) ? c0 + TPB : N;
    const long long c = c0 + threadIdx.x;
    if (MODE == 2 && kind == 0) {
      if (mo != cur) {                        // the PVT table of this model (no thread reads the
        load_table(T, M.table, bar, uses, M.status);   // previous one: every item ends past a barrier)
        cur = mo;
      }
      if (c < N) cell_body<NB>(M, T, c);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(O.flag_cell + fbase + t, 1);
      }
      continue;
    }
    if (MODE == 2) {                          // cells of this tile and of its + neighbours
      const long long lo[3] = {c0, c0 + nx, c0 + nxy}, hi[3] = {c1, c1 - 1 + nx, c1 - 1 + nxy};
      wait_tiles<TPB>(O.flag_cell + fbase, lo, hi, N, -1, M.status);
    }
    double r[NB], dg[NB][NB];
    if (c < N) face_part<NB, MODE == 2>(M, c, r, dg);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(O.flag_face + fbase + t, 1);
    }
    {                                          // shares from the - neighbours' tiles
      const long long lo[3] = {c0 - 1, c0 - nx, c0 - nxy}, hi[3] = {c1 - 2, c1 - 1 - nx, c1 - 1 - nxy};
      wait_tiles<TPB>(O.flag_face + fbase, lo, hi, N, t, M.status);
    }
    if (c < N) assemble_rows<NB, true>(M, c, r, dg);
  }
}

template <int NB, int TPB>
void launch_stage(int stage, const TileList& L, const ModelArgs& single, int grid, cudaStream_t s) {
  if (stage == 0) launch_pdl(cell_kernel<NB, TPB>, grid, TPB, 0, s, L, single);
  else if (stage == 1) launch_pdl(face_kernel<NB, TPB>, grid, TPB, 0, s, L, single);
  else launch_pdl(assemble_kernel<NB, TPB>, grid, TPB, 0, s, L, single);
}

template <int NB, int TPB, int MODE>
cudaError_t launch_ordered_t(const OrderedList& O, const ModelArgs& single, int ctas_per_sm, int sms,
                             cudaStream_t s) {
  int per_sm = ctas_per_sm;
  if (per_sm <= 0) {                     // as many CTAs as fit at once
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ordered_kernel<NB, TPB, MODE>, TPB, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  long long grid = (long long)per_sm * (sms > 0 ? sms : 1);
  if (grid > O.nitems) grid = O.nitems;
  if (grid < 1) return cudaSuccess;
  return launch_pdl(ordered_kernel<NB, TPB, MODE>, (unsigned)grid, TPB, 0, s, O, single);
}

template <int NB, int TPB>
cudaError_t launch_ordered_nb(int mode, const OrderedList& O, const ModelArgs& single, int ctas_per_sm, int sms,
                              cudaStream_t s) {
  if (mode == 2) return launch_ordered_t<NB, TPB, 2>(O, single, ctas_per_sm, sms, s);
  return launch_ordered_t<NB, TPB, 1>(O, single, ctas_per_sm, sms, s);
}

}  // namespace

// The ordered launch (cfg.ordered 1 or 2) at tile size cfg.tpb[1].  `O`
// holds the model list (or none for `single`), the tile counts, and the
// counter and flags, which the caller has zeroed on the stream.  With mode 1
// the cell stage is launched first, over `lists`.
cudaError_t launch_ordered(int nb, const TileList* lists, OrderedList O, const ModelArgs& single,
                           const LaunchCfg& cfg, int sms, cudaStream_t s) {
  const int tpb = cfg.tpb[1];
  const int ti = tile_index(tpb);
  if (ti < 0 || (cfg.ordered != 1 && cfg.ordered != 2)) return cudaErrorInvalidValue;
  if (cfg.ordered == 1) {
    LaunchCfg cell = cfg;
    cell.ctas_per_sm[1] = cell.ctas_per_sm[2] = -1;    // the cell stage alone
    cell.ordered = 0;
    cudaError_t e = launch_tiles(nb, lists, single, cell, sms, s);
    if (e != cudaSuccess) return e;
  }
  O.nitems *= cfg.ordered;                // nitems holds the tile count
#define OCP_ORD(NB)                                                                              \
  switch (ti) {                                                                                  \
    case 0: return launch_ordered_nb<NB, 32>(cfg.ordered, O, single, cfg.ctas_per_sm[1], sms, s); \
    case 1: return launch_ordered_nb<NB, 64>(cfg.ordered, O, single, cfg.ctas_per_sm[1], sms, s); \
    case 2: return launch_ordered_nb<NB, 128>(cfg.ordered, O, single, cfg.ctas_per_sm[1], sms, s); \
    default: return launch_ordered_nb<NB, 256>(cfg.ordered, O, single, cfg.ctas_per_sm[1], sms, s); \
  }
  if (nb == 3) {
    OCP_ORD(3)
  } else {
    OCP_ORD(2)
  }
#undef OCP_ORD
}

// Launches the three stages.  `lists[t]` is the tile list for
// kTileSizes[t] cells per tile; cfg picks, per stage, the tile size and the
// grid (CTAs per SM times the SM count, or 0 for one CTA per tile; a
// negative count skips the stage, which only the autotuner uses).
cudaError_t launch_tiles(int nb, const TileList* lists, const ModelArgs& single, const LaunchCfg& cfg,
                         int sms, cudaStream_t s) {
  for (int stage = 0; stage < 3; ++stage) {
    if (cfg.ctas_per_sm[stage] < 0) continue;
    if (cfg.ordered == 3 && stage > 0) {   // the split face and assembly stages, 32-cell tiles
      const TileList& L = lists[0];
      if (L.ntiles == 0) continue;
      int grid = cfg.ctas_per_sm[stage] > 0 ? cfg.ctas_per_sm[stage] * sms : L.ntiles;
      if (grid > L.ntiles) grid = L.ntiles;
      cudaError_t e;
      if (nb == 3) e = stage == 1 ? launch_pdl(face_split_kernel<3>, grid, 96, 0, s, L, single)
                                  : launch_pdl(assemble_split_kernel<3>, grid, 96, 0, s, L, single);
      else e = stage == 1 ? launch_pdl(face_split_kernel<2>, grid, 96, 0, s, L, single)
                          : launch_pdl(assemble_split_kernel<2>, grid, 96, 0, s, L, single);
      if (e != cudaSuccess) return e;
      continue;
    }
    const int t = tile_index(cfg.tpb[stage]);
    if (t < 0) return cudaErrorInvalidValue;
    const TileList& L = lists[t];
    if (L.ntiles == 0) continue;
    int grid = cfg.ctas_per_sm[stage] > 0 ? cfg.ctas_per_sm[stage] * sms : L.ntiles;
    if (grid > L.ntiles) grid = L.ntiles;
#define OCP_STAGE(NB)                                                   \
    switch (t) {                                                        \
      case 0: launch_stage<NB, 32>(stage, L, single, grid, s); break;   \
      case 1: launch_stage<NB, 64>(stage, L, single, grid, s); break;   \
      case 2: launch_stage<NB, 128>(stage, L, single, grid, s); break;  \
      default: launch_stage<NB, 256>(stage, L, single, grid, s); break; \
    }
    if (nb == 3) {
      OCP_STAGE(3)
    } else {
      OCP_STAGE(2)
    }
#undef OCP_STAGE
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
  TileList lists[kNumTileSizes];
  for (int t = 0; t < kNumTileSizes; ++t) {
    lists[t].models = nullptr;
    lists[t].tiles = nullptr;
    lists[t].ntiles = (int)((g->prm.N + kTileSizes[t] - 1) / kTileSizes[t]);
  }
  if (g->cfg.ordered == 0 || g->cfg.ordered == 3) return launch_tiles(g->prm.nb, lists, M, g->cfg, g->sms, s);
  const long long nmax = (g->prm.N + 31) / 32;       // flags sized for the smallest tiles
  cudaError_t e = cudaMemsetAsync(g->d_sync, 0, sizeof(unsigned) * (1 + 2 * nmax), s);
  if (e != cudaSuccess) return e;
  OrderedList O{};
  O.counter = g->d_sync;
  O.flag_cell = reinterpret_cast<int*>(g->d_sync + 1);
  O.flag_face = reinterpret_cast<int*>(g->d_sync + 1 + nmax);
  O.nitems = (g->prm.N + g->cfg.tpb[1] - 1) / g->cfg.tpb[1];
  return launch_ordered(g->prm.nb, lists, O, M, g->cfg, g->sms, s);
}

}  // namespace

cudaError_t preload_linearize(int nb) {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess;
#define OCP_LOAD(NB, TPB)                                                              \
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, cell_kernel<NB, TPB>);           \
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, face_kernel<NB, TPB>);           \
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, assemble_kernel<NB, TPB>);       \
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, ordered_kernel<NB, TPB, 1>);     \
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, ordered_kernel<NB, TPB, 2>);
  if (nb == 3) {
    OCP_LOAD(3, 32) OCP_LOAD(3, 64) OCP_LOAD(3, 128) OCP_LOAD(3, 256)
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, face_split_kernel<3>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, assemble_split_kernel<3>);
  } else {
    OCP_LOAD(2, 32) OCP_LOAD(2, 64) OCP_LOAD(2, 128) OCP_LOAD(2, 256)
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, face_split_kernel<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, assemble_split_kernel<2>);
  }
#undef OCP_LOAD
  return e;
}

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
