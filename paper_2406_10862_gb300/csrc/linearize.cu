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

// Drops from L2, without writing them back to DRAM, the 128-byte lines of
// scratch fields [f0, f1) that hold only cells [c0, c0 + TPB) (clamped to
// N): called once every reader of those cells' scratch is done, so that dead
// scratch costs no DRAM write.  Lines shared with other cells are left
// alone.  All threads of the CTA call it, after a barrier.
template <int TPB>
__device__ __forceinline__ void discard_scratch(const double* s, long long N, long long c0, int f0, int f1) {
  constexpr int kPer = TPB / 16 >= 8 ? TPB / 8 : 8;      // power of two above the lines a range can touch
  const long long c1 = c0 + TPB < N ? c0 + TPB : N;
  for (int k = threadIdx.x; k < (f1 - f0) * kPer; k += blockDim.x) {
    const int f = f0 + k / kPer, j = k % kPer;
    const uintptr_t a = (uintptr_t)(s + f * N + c0), b = (uintptr_t)(s + f * N + c1);
    const uintptr_t line = ((a + 127) & ~(uintptr_t)127) + 128 * (uintptr_t)j;
    if (line + 128 <= b) asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
  }
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
    // explicitly rounded differences here and below: the terms may come
    // from other warps (the one-cluster launch), so that no product is ever
    // fused into these subtractions and every launch shape gives the same bits
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      r[e] = __dsub_rn(a.m[e], mo[e]);
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
      r[e] = __dsub_rn(r[e], src[e]);
      for (int v = 0; v < NB; ++v) dg[e][v] = __dsub_rn(dg[e][v], ds[e][v]);
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
template <int NB, bool COH>
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
  load_q<NB, COH>(scr, N, c, a);
  load_q<NB, COH>(scr, N, n, b);
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

// One 32-cell tile of the split face stage (96 threads): warp d computes
// direction d of every cell of the tile, then warp e < NB adds equation e's
// own terms and faces x, y, z.  Ends with the own[] buffer free again.
template <int NB, bool COH>
__device__ __forceinline__ void face_split_tile(const ModelArgs& M, long long c0, double (*own)[12][32]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long N = M.P.N;
  const long long c = c0 + lane;
  if (c < N) face_dir<NB, COH>(M, c, w, own[w], lane);
  __syncthreads();
  if (c < N && w < NB) {               // warp e: equation e of this row, own terms + faces x, y, z
    int i, j, k;
    cell_ijk(M.P, c, i, j, k);
    const bool hp[3] = {i + 1 < M.P.nx, j + 1 < M.P.ny, k + 1 < M.P.nz};
    double* scr = M.scr;
    const int e = w;
    double r = lds<COH>(scr + (kSelf + e) * N + c);
    double dg[NB];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[v] = lds<COH>(scr + (kSelf + 3 + 3 * e + v) * N + c);
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
  __syncthreads();                     // own[] is free for the next tile
}

// Equation e of row c in the split assembly: its own terms and + faces
// minus the shares of the - neighbours, in the order -z, -y, -x.
template <int NB, bool COH>
__device__ __forceinline__ void assemble_finish(const ModelArgs& M, long long c, int e, double r, double (&dg)[NB]) {
  const long long N = M.P.N;
  const double* scr = M.scr;
  int i, j, k;
  cell_ijk(M.P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (!hm[d]) continue;
    const int base = kInc + 12 * d;
    r -= lds<COH>(scr + (base + e) * N + c);
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[v] -= lds<COH>(scr + (base + 3 + 3 * e + v) * N + c);
  }
  double* out = M.val + (row_start_ijk(M.P, c, i, j, k) + (int)hm[0] + (int)hm[1] + (int)hm[2]) * NB * NB;
  __stcs(M.res + c * NB + e, r);
#pragma unroll
  for (int v = 0; v < NB; ++v) __stcs(out + e * NB + v, dg[v]);
  if (!finite(r)) atomicOr(M.status, kStatNonFinite);
}

template <int NB, bool COH>
__device__ __forceinline__ void assemble_split_row(const ModelArgs& M, long long c, int e) {
  const long long N = M.P.N;
  const double* scr = M.scr;
  const double r = lds<COH>(scr + (kPart + e) * N + c);
  double dg[NB];
#pragma unroll
  for (int v = 0; v < NB; ++v) dg[v] = lds<COH>(scr + (kPart + 3 + 3 * e + v) * N + c);
  assemble_finish<NB, COH>(M, c, e, r, dg);
}

template <int NB>
__global__ void __launch_bounds__(96) face_split_kernel(TileList L, ModelArgs single) {
  pdl_wait();
  __shared__ double own[3][12][32];      // [direction][F, dF/du_c][lane]
  for (int t = blockIdx.x; t < L.ntiles; t += gridDim.x) {
    int m;
    long long c0;
    const ModelArgs& M = tile_of<32>(L, single, t, m, c0);
    face_split_tile<NB, false>(M, c0, own);
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
    const long long c = c0 + lane;
    if (c < M.P.N) assemble_split_row<NB, false>(M, c, e);
  }
}

// -------------------------------------------------------- one-cluster launch
// A grid of at most kMaxClusterTiles 32-cell tiles linearised by one
// thread-block cluster, CTA t (cluster rank t) owning tile t, in three
// stages separated by cluster barriers instead of launch boundaries.  The
// stages exchange data through distributed shared memory rather than
// scratch: each CTA keeps its cells' quantities in its own shared memory,
// where the face stage of the CTA holding a - neighbour reads them, and that
// face stage writes the neighbour's share straight into the shared memory of
// the CTA owning the neighbour.  barrier.cluster.arrive.release orders those
// accesses before barrier.cluster.wait.acquire returns in every CTA; a CTA
// arrives as soon as its writes for the others are done and waits only
// before it reads theirs, doing its own CTA's work in between.  Every thread
// reaches every barrier, and no CTA touches another's shared memory after
// the last one.
//
// Such grids are latency bound: each FP64 warp instruction holds an SM
// sub-partition's FP64 unit 64 cycles, so a stage takes about the FP64
// instruction count of its busiest sub-partition.  Both stages are
// therefore spread over more warps than the tile kernels use:
//   cell stage: warp 0 the PVT properties at the new state, warp 1 the
//   relative permeabilities, warp 3 the amounts at the old state; then
//   warp 0 the water and oil amounts and accumulation terms, warp 3 the gas
//   ones, warp 2 the densities, mobilities and well terms, warp 1 the
//   capillary pressures;
//   face stage: one warp per direction and phase, placed so that the four
//   sub-partitions get about equal FP64 work, the gas component's
//   dissolved-gas term added by the gas warp once the oil warp's phase flux
//   is in shared memory; then one warp per equation adds the faces to the
//   cell's own terms and, after the second barrier, subtracts the shares of
//   the - neighbours.
// Every quantity is computed by the same expressions as in the tile kernels
// (the differences that take terms computed by other warps are explicitly
// rounded there too), so the results are bit-identical to theirs.
constexpr int kClusterThreads = 288;   // 9 warps: 3 directions x 3 phases in the face stage

struct ClusterCellBuf {                // cell stage, per lane
  Pvt f[32];                           // warp 0 -> warps 1, 2, 3
  KrSide kg[32];                       // warp 2 -> warp 1
  Kr k[32];                            // warp 1 -> warp 2
  double mo[3][32];                    // warp 3 -> warps 0, 3
  double src[3][32], ds[3][3][32];     // warps 1, 2 -> warps 0, 3 (perforated cells)
  double qg[3][32];                    // warp 1 -> warp 2: producers' free-gas rate
};
struct ClusterFaceBuf {                // face stage, per lane
  double own[3][12][32];               // [direction][F, dF/du_c][lane]
  double oil[3][7][32];                // [direction][F, di, dj of the oil phase][lane]
  int up_o[3][32];
};
struct ClusterShared {                 // read and written by the other CTAs of the cluster
  double q[kQ][32];                    // CellQ fields of the tile's cells
  double share[3][12][32];             // [direction][F, dF/du_-][lane]: the - neighbour's share
};
// The Jacobian rows of the tile's cells are assembled in shared memory (the
// - neighbour blocks written there by the CTAs holding those neighbours) and
// stored with coalesced stores at the end: at most 7 blocks per row.  The
// dynamic shared memory is sized above half an SM's so that the CTAs of the
// cluster run on different SMs (their FP64 units set the time).
constexpr int kClusterStageBlocks = 32 * 7;
constexpr int kClusterDynSmem = 120 * 1024;
static_assert(kClusterStageBlocks * 9 * (int)sizeof(double) <= kClusterDynSmem, "staged rows exceed the buffer");
// Block index of the first block of row c, for 0 <= c <= N (N: the total).
__device__ __forceinline__ long long row_start_any(const Params& P, long long c) {
  if (c >= P.N) return 7 * P.N - 2 * ((long long)P.ny * P.nz + (long long)P.nx * P.nz + P.nxy);
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  return row_start_ijk(P, c, i, j, k);
}

// Face-stage task of warp w: direction kTaskD, phase kTaskPh (0 water, 1
// oil, 2 gas; -1 none).  Warp w runs on sub-partition w % 4; with three
// phases each sub-partition gets about 50 FP64 instructions per cell (a gas
// task, which also adds the dissolved gas, counts for about two others).
// Two bits per warp, warp w at bits 2w: three phases d = 0 0 1 2 1 1 2 2 0,
// ph = 0 2 2 2 0 1 1 0 1; two phases d = 0 0 1 1 2 2, ph = 0 1 0 1 1 0, and
// 3 (none) for warps 6..8.
__device__ __forceinline__ void face_task(int nb, int w, int& d, int& ph) {
  const unsigned dk = nb == 3 ? 42384u : 2640u, pk = nb == 3 ? 70824u : 258372u;
  d = (int)((dk >> (2 * w)) & 3u);
  ph = (int)((pk >> (2 * w)) & 3u);
  if (ph == 3) ph = -1;
}

// The cluster barrier in its two halves.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Distributed shared memory: the address of `p` (a variable of this CTA's
// shared memory) in the window of cluster rank `rank`, and 8-byte accesses
// through such addresses.
__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ double dsmem_ld(unsigned a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void dsmem_st(unsigned a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// CellQ fields [lo, hi) that the block size uses, into the tile's q[][lane].
template <int NB>
__device__ __forceinline__ void put_q(double (*qs)[32], int lane, const CellQ& q, int lo, int hi) {
  const double* f = reinterpret_cast<const double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    if (i >= lo && i < hi && q_used<NB>(i)) qs[i][lane] = f[i];
}
// The CellQ fields of one phase (0 water, 1 oil, 2 gas with the dissolved-gas
// ratio; the others left zero) of lane `lane` of the tile whose q[][] is at
// cluster address `a` (dsmem_addr of q[0][0]).
__host__ __device__ constexpr bool q_of_phase(int i, int ph) {
  // water pw dpw_sw rw rw_p lw lw_p lw_sw; oil p ro ro_p ro_x lo lo_p lo_sw lo_x;
  // gas pg dpg_x rg rg_p lg lg_p lg_x rs rs_p rs_x
  const bool w = i == 1 || i == 3 || i == 5 || i == 6 || i == 12 || i == 13 || i == 14;
  const bool o = i == 0 || i == 7 || i == 8 || i == 9 || i == 15 || i == 16 || i == 17 || i == 18;
  const bool g = i == 2 || i == 4 || i == 10 || i == 11 || i == 19 || i == 20 || i == 21 || i >= 22;
  return ph == 0 ? w : (ph == 1 ? o : g);
}
template <int NB, int PH>
__device__ __forceinline__ void get_q_phase(unsigned a, int lane, CellQ& q) {
  double* f = reinterpret_cast<double*>(&q);
#pragma unroll
  for (int i = 0; i < kQ; ++i) f[i] = (q_of_phase(i, PH) && q_used<NB>(i)) ? dsmem_ld(a + 8u * (32u * i + lane)) : 0.0;
}
// The quantities of phase PH of this cell (a, this CTA) and of its +
// neighbour (b, lane ln of CTA rank), and the phase's flux across the face.
template <int NB, int PH>
__device__ __forceinline__ void phase_face(unsigned qa, int lane, unsigned qb, int ln, bool grav, double T,
                                           double hz, CellQ& a, CellQ& b, double& F, double (&di)[3],
                                           double (&dj)[3], bool& up) {
  get_q_phase<NB, PH>(qa, lane, a);
  get_q_phase<NB, PH>(qb, ln, b);
  if (PH == 0) {
    if (grav) water_flux<NB, true>(T, hz, a, b, F, di, dj, up);
    else water_flux<NB, false>(T, hz, a, b, F, di, dj, up);
  } else if (PH == 1) {
    if (grav) oil_flux<NB, true>(T, hz, a, b, F, di, dj, up);
    else oil_flux<NB, false>(T, hz, a, b, F, di, dj, up);
  } else {
    if (grav) gas_flux<NB, true>(T, hz, a, b, F, di, dj, up);
    else gas_flux<NB, false>(T, hz, a, b, F, di, dj, up);
  }
}

// A cell's inputs, loaded by each cell-stage warp while the PVT table's copy
// is in flight (one round of memory latency; nothing uses them before the
// wait for the table).
struct CellIn {
  double pn, swn, xn, po, swo, xo, phi;
  int fn, fo, ip;
};
template <int NB>
__device__ __forceinline__ void load_cell_in(const ModelArgs& M, long long c, CellIn& in) {
  const long long N = M.P.N;
  in.pn = M.u_new[c];
  in.swn = M.u_new[N + c];
  in.xn = (NB == 3) ? M.u_new[2 * N + c] : 0.0;
  in.po = M.u_old[c];
  in.swo = M.u_old[N + c];
  in.xo = (NB == 3) ? M.u_old[2 * N + c] : 0.0;
  in.fn = (NB == 3) ? M.f_new[c] : 0;
  in.fo = (NB == 3) ? M.f_old[c] : 0;
  in.phi = M.phi[c];
  in.ip = M.perf_of_cell[c];
}

// Barrier of warps 1 and 2 only (named barrier `id`, 64 threads).
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// The cell stage of tile c0 (warps 0..3, one cell per lane): the cells'
// quantities go to qs, their own residual and diagonal block to self.
// Phase A: warp 0 the PVT properties at the new state, warps 1 and 2 the
// water and gas sides of the relative permeabilities (warp 1 then combines
// them), warp 3 the amounts at the old state.  Phase B: warp 0 the water and
// oil amounts and their accumulation terms, warp 3 the gas ones, warp 1 the
// capillary pressures and the water and gas densities and mobilities, warp 2
// the oil ones and (tiles with perforated cells) the well terms.  Phase C
// (such tiles): warps 0 and 3 subtract the well terms.
template <int NB>
__device__ __forceinline__ void cluster_cell_stage(const ModelArgs& M, const Table& T, long long c0,
                                                   const CellIn& in, ClusterCellBuf& B, double (*qs)[32],
                                                   double (*self)[32]) {
  const Params& P = M.P;
  const long long N = P.N;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c = c0 + lane;
  const bool live = c < N;
  const int ip = (live && w < 4) ? in.ip : -1;
  // pore volume over dt folded into the porosity, as in cell_body
  const double pn = in.pn, swn = in.swn, phs = in.phi * M.scale;
  const int flag = in.fn & 1;
  const bool tile_well = __any_sync(0xffffffffu, ip >= 0);   // the same in warps 0..3
  Pvt f;
  Kr k;
  if (w == 0) {                         // PVT at the new state
    if (live) {
      int bad = 0;
      if (!(finite(pn) && finite(swn) && finite(in.xn) && finite(in.po) && finite(in.swo) && finite(in.xo)))
        bad |= kStatNonFinite;
      if ((unsigned)in.fn > 1u || (unsigned)in.fo > 1u) bad |= kStatBadFlag;
      if (bad) atomicOr(M.status, bad);
      pvt<NB, true>(P, T, pn, in.xn, flag, f);
      B.f[lane] = f;
    }
  } else if (w == 1) {                  // relative permeabilities: water side, then both
    KrSide kw;
    if (live) rel_perm_w(P, swn, kw);
    if (NB == 3) pair_sync(1);
    if (live) {
      KrSide kg{};
      if (NB == 3) kg = B.kg[lane];
      rel_perm_combine<NB>(P, kw, kg, flag, k);
      B.k[lane] = k;
    }
  } else if (w == 2) {                  // relative permeabilities: gas side
    if (NB == 3) {
      if (live) {
        KrSide kg;
        rel_perm_g(P, flag == 0 ? in.xn : 0.0, kg);
        B.kg[lane] = kg;
      }
      pair_sync(1);
    }
  } else if (w == 3 && live && !M.no_acc) {   // the amounts at the old state
    double mo[3];
    cell_masses<NB, false>(P, T, in.po, in.swo, in.xo, in.fo & 1, phs, mo);
#pragma unroll
    for (int e = 0; e < NB; ++e) B.mo[e][lane] = mo[e];
  }
  __syncthreads();
  // rows e0 <= e < e1 of the own terms: warp 0 water and oil, warp 3 gas
  const int e0 = w == 0 ? 0 : 2, e1 = w == 0 ? 2 : NB;
  const bool rows = live && (w == 0 || (NB == 3 && w == 3));
  double r[3] = {0.0, 0.0, 0.0}, dg[3][3] = {};
  if (rows) {
    if (w == 3) f = B.f[lane];
    double m[3], m_p[3], m_sw[3], m_x[3];
    if (w == 0) masses<NB, true, 0>(P, f, pn, swn, phs, m, m_p, m_sw, m_x);
    else masses<NB, true, 1>(P, f, pn, swn, phs, m, m_p, m_sw, m_x);
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      if (e < e0 || e >= e1) continue;
      if (!M.no_acc) {
        r[e] = __dsub_rn(m[e], B.mo[e][lane]);
        dg[e][0] = m_p[e];
        dg[e][1] = m_sw[e];
        dg[e][2] = m_x[e];
      } else {
        r[e] = dg[e][0] = dg[e][1] = dg[e][2] = 0.0;
      }
    }
  } else if (w == 1) {                  // capillary pressures, water and gas densities and mobilities
    if (live) {
      f = B.f[lane];
      CellQ q{};
      cap_pressure<NB>(P, pn, k, q);
      dens_mob<NB, true, false>(P, f, k, q);
      put_q<NB>(qs, lane, q, 0, 7);      // p pw pg dpw_sw dpg_x rw rw_p
      put_q<NB>(qs, lane, q, 10, 15);    // rg rg_p lw lw_p lw_sw
      put_q<NB>(qs, lane, q, 19, kQ);    // lg lg_p lg_x rs rs_p rs_x
      if (ip >= 0) {                    // producers: the water row and the free gas
        Perf wl = M.perf[ip];
        if (M.p_bh) wl.p_bh = M.p_bh[wl.well];
        if (wl.kind == 0) {
          double src = 0.0, d[3] = {0.0, 0.0, 0.0}, qg[3] = {0.0, 0.0, 0.0};
          if (positive(q.p - wl.p_bh)) {
            const double g = wl.p_bh - q.p;
            well_prod_water(wl, q, g, src, d);
            if (NB == 3) well_prod_gas_free(wl, q, g, qg);
          }
          B.src[0][lane] = src;
#pragma unroll
          for (int v = 0; v < NB; ++v) B.ds[0][v][lane] = d[v];
#pragma unroll
          for (int v = 0; v < 3; ++v) B.qg[v][lane] = qg[v];
        }
      }
    }
    if (tile_well) pair_sync(2);
  } else if (w == 2) {                  // oil density and mobility, well terms
    CellQ q{};
    if (live) {
      f = B.f[lane];
      k = B.k[lane];
      dens_mob<NB, false, true>(P, f, k, q);
      put_q<NB>(qs, lane, q, 7, 10);     // ro, ro_p, ro_x
      put_q<NB>(qs, lane, q, 15, 19);    // lo, lo_p, lo_sw, lo_x
    }
    if (tile_well) {
      Perf wl{};
      double src[3] = {0.0, 0.0, 0.0}, ds[3][3] = {};
      bool prod = false;
      if (ip >= 0) {
        wl = M.perf[ip];
        if (M.p_bh) wl.p_bh = M.p_bh[wl.well];
        q.p = pn;
        prod = wl.kind == 0 && positive(q.p - wl.p_bh);
        if (prod) well_prod_oil(wl, q, wl.p_bh - q.p, src[1], ds[1]);
      }
      pair_sync(2);
      if (ip >= 0) {
        if (wl.kind == 0) {             // producers: the oil row, then the gas component
          if (NB == 3 && prod) {
            q.rs = qs[22][lane];
            q.rs_p = qs[23][lane];
            q.rs_x = qs[24][lane];
            const double qg[3] = {B.qg[0][lane], B.qg[1][lane], B.qg[2][lane]};
            well_prod_gas(q, src[1], ds[1], qg, src[2], ds[2]);
          }
#pragma unroll
          for (int e = 1; e < NB; ++e) {
            B.src[e][lane] = src[e];
#pragma unroll
            for (int v = 0; v < NB; ++v) B.ds[e][v][lane] = ds[e][v];
          }
        } else {                        // injectors: the injected phase's row
          CellQ qa;
          double* fq = reinterpret_cast<double*>(&qa);
#pragma unroll
          for (int i = 0; i < kQ; ++i) fq[i] = q_used<NB>(i) ? qs[i][lane] : 0.0;
          qa.p = pn;
          CellAux a{};
          total_mob<NB>(P, f, k, true, a);
          well_source<NB>(wl, qa, a, src, ds);
#pragma unroll
          for (int e = 0; e < NB; ++e) {
            B.src[e][lane] = src[e];
#pragma unroll
            for (int v = 0; v < NB; ++v) B.ds[e][v][lane] = ds[e][v];
          }
        }
      }
    }
  }
  __syncthreads();
  if (rows) {                           // minus the well terms; own terms to shared memory
    if (ip >= 0) {
#pragma unroll
      for (int e = 0; e < NB; ++e) {
        if (e < e0 || e >= e1) continue;
        r[e] = __dsub_rn(r[e], B.src[e][lane]);
#pragma unroll
        for (int v = 0; v < NB; ++v) dg[e][v] = __dsub_rn(dg[e][v], B.ds[e][v][lane]);
      }
    }
#pragma unroll
    for (int e = 0; e < NB; ++e) {
      if (e < e0 || e >= e1) continue;
      self[e][lane] = r[e];
#pragma unroll
      for (int v = 0; v < NB; ++v) self[3 + 3 * e + v][lane] = dg[e][v];
    }
  }
}

// Row e of face d's outputs (as face_dir writes them for every row): this
// row's block of the neighbour into the tile's staged rows at blk, the
// neighbour row's block of this cell at cluster address nblk and the
// neighbour's share at cluster address sh (share[d][0][lane of the
// neighbour]), both in the CTA holding the neighbour.
template <int NB>
__device__ __forceinline__ void face_row(const ModelArgs& M, long long c, int d, int e, double* blk, unsigned nblk,
                                         double F, const double (&di)[3], const double (&dj)[3], double (*own)[32],
                                         int lane, unsigned sh) {
  const long long N = M.P.N;
  own[e][lane] = F;
  dsmem_st(sh + 256u * e, F);
#pragma unroll
  for (int v = 0; v < NB; ++v) {
    own[3 + 3 * e + v][lane] = di[v];
    blk[e * NB + v] = dj[v];
    dsmem_st(nblk + 8u * (e * NB + v), neg(di[v]));
    dsmem_st(sh + 256u * (3 + 3 * e + v), dj[v]);
  }
  if (M.face_flux) __stcs(M.face_flux + (d * NB + e) * N + c, F);
}

// The face stage of tile c0, entered after the CTA's arrival at the first
// cluster barrier: warp w computes its task's phase of its direction for
// every cell (Tf its face's transmissibility, loaded at the start of the
// kernel); the CTA then arrives at the second barrier, and warp e < NB adds
// its equation's faces to the own terms in self[] and returns them in r, dg.
template <int NB>
__device__ __forceinline__ void cluster_face_stage(const ModelArgs& M, long long c0, double Tf, ClusterFaceBuf& B,
                                                   ClusterShared& S, double* stage, const double (*self)[32],
                                                   double& r, double (&dg)[NB]) {
  constexpr int B2 = NB * NB;
  const Params& P = M.P;
  const long long N = P.N;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c = c0 + lane;
  int d, ph;
  face_task(NB, w, d, ph);
  const bool active = c < N && ph >= 0;
  int i = 0, j = 0, k = 0;
  if (c < N) cell_ijk(P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
  const bool hp[3] = {i + 1 < P.nx, j + 1 < P.ny, k + 1 < P.nz};
  const bool has = active && hp[d];
  const long long n = has ? c + (d == 0 ? 1 : (d == 1 ? (long long)P.nx : P.nxy)) : 0;
  double* blk = nullptr;
  unsigned nblk = 0;
  CellQ a{}, b{};
  double Fp = 0.0, di[3] = {0.0, 0.0, 0.0}, dj[3] = {0.0, 0.0, 0.0};
  cluster_wait();                        // every CTA's cell quantities are in its shared memory
  unsigned sh = 0;
  if (active) {
    if (!has) {
      if (M.face_flux) __stcs(M.face_flux + (d * NB + ph) * N + c, 0.0);
    } else {
      const unsigned rank = (unsigned)(n >> 5), ln = (unsigned)(n & 31);
      const unsigned qa = dsmem_addr(&S.q[0][0], blockIdx.x), qb = dsmem_addr(&S.q[0][0], rank);
      sh = dsmem_addr(&S.share[d][0][ln], rank);
      const double hz = d == 2 ? -P.grav_dz : 0.0;
      bool up;
      if (ph == 0) phase_face<NB, 0>(qa, lane, qb, (int)ln, d == 2, Tf, hz, a, b, Fp, di, dj, up);
      else if (ph == 1) phase_face<NB, 1>(qa, lane, qb, (int)ln, d == 2, Tf, hz, a, b, Fp, di, dj, up);
      else phase_face<NB, 2>(qa, lane, qb, (int)ln, d == 2, Tf, hz, a, b, Fp, di, dj, up);
      const int slot = (int)hm[0] + (int)hm[1] + (int)hm[2] + 1 + (d > 0 && hp[0]) + (d > 1 && hp[1]);
      blk = stage + (row_start_ijk(P, c, i, j, k) - row_start_any(P, c0) + slot) * B2;
      const int slot_n = (d == 0) ? ((int)hm[2] + (int)hm[1]) : (d == 1 ? (int)hm[2] : 0);
      const long long nb0 = row_start_any(P, (long long)rank * 32);
      nblk = dsmem_addr(stage + (row_start_ijk(P, n, i + (d == 0), j + (d == 1), k + (d == 2)) - nb0 + slot_n) * B2,
                        rank);
      if (ph < 2) face_row<NB>(M, c, d, ph, blk, nblk, Fp, di, dj, B.own[d], lane, sh);
      if (NB == 3 && ph == 1) {
        B.oil[d][0][lane] = Fp;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          B.oil[d][1 + v][lane] = di[v];
          B.oil[d][4 + v][lane] = dj[v];
        }
        B.up_o[d][lane] = up;
      }
    }
  }
  if (NB == 3) {
    __syncthreads();
    if (active && has && ph == 2) {     // the gas component: free gas plus gas dissolved in the oil
      double di_o[3], dj_o[3], F, dig[3], djg[3];
      const double Fo = B.oil[d][0][lane];
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        di_o[v] = B.oil[d][1 + v][lane];
        dj_o[v] = B.oil[d][4 + v][lane];
      }
      gas_component(a, b, B.up_o[d][lane] != 0, Fo, di_o, dj_o, Fp, di, dj, F, dig, djg);
      face_row<NB>(M, c, d, 2, blk, nblk, F, dig, djg, B.own[d], lane, sh);
    }
  }
  __syncthreads();
  cluster_arrive();                      // this CTA's shares are in the other CTAs' shared memory
  if (c < N && w < NB) {                // warp e: equation e, own terms + faces x, y, z
    const int e = w;
    r = self[e][lane];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[v] = self[3 + 3 * e + v][lane];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      if (!hp[dd]) continue;
      r += B.own[dd][e][lane];
#pragma unroll
      for (int v = 0; v < NB; ++v) dg[v] += B.own[dd][3 + 3 * e + v][lane];
    }
  }
}

// Equation e of row c: r, dg (own terms and + faces) minus the shares of the
// - neighbours in share[][][lane], in the order -z, -y, -x (as
// assemble_finish); the diagonal block goes to the staged rows.
template <int NB>
__device__ __forceinline__ void cluster_assemble(const ModelArgs& M, long long c0, long long c, int e, double r,
                                                 double (&dg)[NB], const double (*share)[12][32], double* stage,
                                                 int lane) {
  int i, j, k;
  cell_ijk(M.P, c, i, j, k);
  const bool hm[3] = {i > 0, j > 0, k > 0};
#pragma unroll
  for (int d = 2; d >= 0; --d) {
    if (!hm[d]) continue;
    r -= share[d][e][lane];
#pragma unroll
    for (int v = 0; v < NB; ++v) dg[v] -= share[d][3 + 3 * e + v][lane];
  }
  double* out = stage + (row_start_ijk(M.P, c, i, j, k) - row_start_any(M.P, c0) + (int)hm[0] + (int)hm[1] +
                         (int)hm[2]) * NB * NB;
  __stcs(M.res + c * NB + e, r);
#pragma unroll
  for (int v = 0; v < NB; ++v) out[e * NB + v] = dg[v];
  if (!finite(r)) atomicOr(M.status, kStatNonFinite);
}

template <int NB>
__global__ void __launch_bounds__(kClusterThreads) cluster_kernel(const ModelArgs* models, ModelArgs single) {
  pdl_wait();
  __shared__ Table T;
  __shared__ unsigned long long bar;
  __shared__ double self[12][32];
  __shared__ ClusterShared S;
  __shared__ union {
    ClusterCellBuf cell;
    ClusterFaceBuf face;
  } buf;
  extern __shared__ __align__(16) double stage[];   // kClusterStageBlocks blocks
  unsigned uses = 0;
  // the model's arguments by value: read once, and no store can alias them
  const ModelArgs M = models ? models[0] : single;
  const long long c0 = (long long)blockIdx.x * 32;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c = c0 + lane;
  // the PVT table's copy first, then the cell stage's inputs and the face
  // stage's transmissibility while it is on its way
  table_copy_issue(T, M.table, bar, uses);
  CellIn in{};
  if (w < 4 && c < M.P.N) load_cell_in<NB>(M, c, in);
  double Tf = 0.0;
  {
    int d, ph;
    face_task(NB, w, d, ph);
    if (ph >= 0 && c < M.P.N) Tf = M.trans[d * M.P.N + c];
  }
  table_copy_wait(bar, uses, M.status);
  cluster_cell_stage<NB>(M, T, c0, in, buf.cell, S.q, self);
  __syncthreads();                       // the CTA's own quantities and self[] are complete
  cluster_arrive();
  double r = 0.0, dg[NB];
  cluster_face_stage<NB>(M, c0, Tf, buf.face, S, stage, self, r, dg);   // waits, and arrives again
  cluster_wait();                        // every share and block is in its CTA's shared memory
  if (w < NB && c < M.P.N) cluster_assemble<NB>(M, c0, c, w, r, dg, S.share, stage, lane);
  __syncthreads();
  // the tile's Jacobian rows, contiguous in val, with coalesced stores
  const long long b0 = row_start_any(M.P, c0);
  const long long nv = (row_start_any(M.P, c0 + 32 < M.P.N ? c0 + 32 : M.P.N) - b0) * NB * NB;
  for (long long q = threadIdx.x; q < nv; q += kClusterThreads) __stcs(M.val + b0 * NB * NB + q, stage[q]);
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
  int dead = -1;                            // model and first cell of the tile whose scratch died
  long long dead_c0 = 0;                    // in the previous face item
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
    if (dead >= 0) {                          // every thread is past the previous item
      const ModelArgs& D = O.models ? O.models[O.order[dead]] : single;
      discard_scratch<TPB>(D.scr, D.P.N, dead_c0, 0, kSelf + 12);
      discard_scratch<TPB>(D.scr, D.P.N, dead_c0, kInc, kInc + 36);
      dead = -1;
    }
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
    // The tile's scratch is now dead: its shares were just read, its own
    // terms in its face stage, and its cell quantities by its own face stage
    // and by the face stages of the tiles holding its cells' - neighbours,
    // which the wait above saw finish.  Its L2 lines are dropped after the
    // next item's barrier (every thread is past the assembly then).
    dead = mo;
    dead_c0 = c0;
  }
  if (dead >= 0) {
    const ModelArgs& D = O.models ? O.models[O.order[dead]] : single;
    discard_scratch<TPB>(D.scr, D.P.N, dead_c0, 0, kSelf + 12);
    discard_scratch<TPB>(D.scr, D.P.N, dead_c0, kInc, kInc + 36);
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

// The one-cluster launch (cfg.ordered 4) of the first model of `models`, or
// of `single` when models is null: one CTA per 32-cell tile, all of them one
// cluster.  The model must have at most max_tiles tiles (the largest cluster
// this device runs, cluster_max_tiles).
cudaError_t launch_cluster(int nb, const ModelArgs* models, const ModelArgs& single, long long N, int max_tiles,
                           cudaStream_t s) {
  const long long nt = (N + 31) / 32;
  if (nt < 1 || nt > max_tiles || nt > kMaxClusterTiles) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nt);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = kClusterDynSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)nt;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  if (nb == 3) return cudaLaunchKernelEx(&cfg, cluster_kernel<3>, models, single);
  return cudaLaunchKernelEx(&cfg, cluster_kernel<2>, models, single);
}

// The largest cluster of cluster_kernel the current device can run (at most
// kMaxClusterTiles), or 0 if it runs none.  Clusters above 8 CTAs are
// non-portable and allowed explicitly on the kernel (preload_linearize).
int cluster_max_tiles(int nb) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kMaxClusterTiles);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = kClusterDynSmem;
  int n = 0;
  const cudaError_t e = nb == 3 ? cudaOccupancyMaxPotentialClusterSize(&n, (const void*)cluster_kernel<3>, &cfg)
                                : cudaOccupancyMaxPotentialClusterSize(&n, (const void*)cluster_kernel<2>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n < kMaxClusterTiles ? n : kMaxClusterTiles;
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
  if (g->cfg.ordered == 4) return launch_cluster(g->prm.nb, nullptr, M, g->prm.N, g->max_cluster, s);
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cluster_kernel<3>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cluster_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterDynSmem);
  } else {
    OCP_LOAD(2, 32) OCP_LOAD(2, 64) OCP_LOAD(2, 128) OCP_LOAD(2, 256)
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, face_split_kernel<2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, assemble_split_kernel<2>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cluster_kernel<2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cluster_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterDynSmem);
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
