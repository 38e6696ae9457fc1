// Adaptive coupling of subdomains (Sec. 4, steps 1-3).
//
// Subdomains are the boxes of a px x py x pz split of the grid.
//   mark_kernel        step 1: a cell is marked when one of its phase
//                      saturations moved by more than the threshold over the
//                      step; its subdomain is flagged, and (step 2, rule b)
//                      every subdomain that sees it as a ghost cell is
//                      coupled with the subdomain owning it;
//   components_kernel  step 2, rule a: a flagged subdomain is coupled with
//                      all its neighbouring subdomains; step 3: connected
//                      components by lock-free union-find in one CTA, in
//                      shared memory for up to 6000 subdomains (each root is
//                      its tree's smallest member, so the labels -- the
//                      smallest subdomain index of each component -- do not
//                      depend on thread order).
// Couplings are 6-bit masks per subdomain (+x, -x, +y, -y, +z, -z), set with
// atomicOr, so the result does not depend on thread order.
#include <cmath>

#include "kernels.cuh"
#include "ocp_internal.cuh"

namespace ocp {
namespace {

struct Boxes {
  int px, py, pz;
};

__device__ __forceinline__ int part(int idx, int n, int parts) { return (int)(((long long)idx * parts) / n); }

__device__ __forceinline__ int sub_of(const Params& P, const Boxes& B, int i, int j, int k) {
  return part(i, P.nx, B.px) + B.px * (part(j, P.ny, B.py) + B.py * part(k, P.nz, B.pz));
}

// FP32 value of a double read from its high word alone: the significand is
// truncated to 20 bits (relative error below 2^-20), magnitudes below 2^-126
// read as zero, and 2^127 and above (inf, NaN) read as inf.  Integer
// instructions only: on this GPU FP64 instructions, conversions included,
// are the scarce resource, integer and FP32 ones are not.
__device__ __forceinline__ float approx_f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned m = hi & 0x7fffffffu, sgn = hi & 0x80000000u;
  unsigned fb;
  if (m < (897u << 20)) fb = sgn;
  else if (m >= (1151u << 20)) fb = sgn | 0x7f800000u;
  else fb = sgn | ((m - (896u << 20)) << 3);
  return __uint_as_float(fb);
}

// Step 1's test, max_alpha |S_alpha,new - S_alpha,old| > thr, decided in FP32
// where the FP32 value is farther from thr than its error bound, else in FP64
// exactly as the definition reads (NaN in any phase leaves the cell unmarked,
// as a NaN maximum compares false).  The FP32 error is below 2^-19 (1 + sum
// of the four |S| read), the threshold's below 2^-20 thr; the margin takes
// 2^-16 (1 + sum) + 2^-19 thr, eight times that, and is inf (so FP64 decides)
// for inputs of 2^127 or more.
template <int NB>
__device__ __forceinline__ bool changed_cell(const double* __restrict__ u_new, const int8_t* __restrict__ f_new,
                                             const double* __restrict__ u_old, const int8_t* __restrict__ f_old,
                                             long long N, long long c, float thr_f, double thr) {
  const double wn = u_new[N + c], wo = u_old[N + c];
  // the third variable is loaded whatever the flag (no load waits on another)
  const double xn = NB == 3 ? u_new[2 * N + c] : 0.0, xo = NB == 3 ? u_old[2 * N + c] : 0.0;
  const double gn = (NB == 3 && f_new[c] == 0) ? xn : 0.0;
  const double go = (NB == 3 && f_old[c] == 0) ? xo : 0.0;
  const float a = approx_f(wn), b = approx_f(gn), cc = approx_f(wo), d = approx_f(go);
  const float dw = fabsf(a - cc), dg = fabsf(b - d);
  const float dox = fabsf(((1.0f - a) - b) - ((1.0f - cc) - d));
  const float ch = fmaxf(fmaxf(dw, dox), dg);
  const float margin = 0x1p-16f * (1.0f + fabsf(a) + fabsf(b) + fabsf(cc) + fabsf(d)) + 0x1p-19f * thr_f;
  if (ch > thr_f + margin) return true;
  if (ch < thr_f - margin) return false;
  const double ew = fabs(wn - wo);
  const double eo = fabs(((1.0 - wn) - gn) - ((1.0 - wo) - go));
  const double eg = fabs(gn - go);
  if (isnan(ew) || isnan(eo) || isnan(eg)) return false;
  return fmax(fmax(ew, eo), eg) > thr;
}

template <int NB>
__global__ void mark_kernel(Params P, Boxes B, const double* __restrict__ u_new, const int8_t* __restrict__ f_new,
                            const double* __restrict__ u_old, const int8_t* __restrict__ f_old, double thr,
                            int* __restrict__ sub_flag, unsigned* __restrict__ mask, int* __restrict__ nmarked) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const float thr_f = approx_f(thr);
  const bool mk = c < P.N && changed_cell<NB>(u_new, f_new, u_old, f_old, P.N, c, thr_f, thr);
  // one counter update per warp (blocks are whole warps)
  const unsigned bal = __ballot_sync(0xffffffffu, mk);
  if ((threadIdx.x & 31) == 0 && bal) atomicAdd(nmarked, __popc(bal));
  if (!mk) return;
  int i, j, k;
  cell_ijk(P, c, i, j, k);
  const int s = sub_of(P, B, i, j, k);
  // most marked cells find their box already flagged: read before the atomic
  if (!*(volatile const int*)&sub_flag[s]) atomicOr(&sub_flag[s], 1);
  // rule (b): this cell is a ghost of every other subdomain it touches
  const int di[6] = {1, -1, 0, 0, 0, 0}, dj[6] = {0, 0, 1, -1, 0, 0}, dk[6] = {0, 0, 0, 0, 1, -1};
  for (int d = 0; d < 6; ++d) {
    const int a2 = i + di[d], b2 = j + dj[d], e2 = k + dk[d];
    if (a2 < 0 || a2 >= P.nx || b2 < 0 || b2 >= P.ny || e2 < 0 || e2 >= P.nz) continue;
    const int t = sub_of(P, B, a2, b2, e2);
    if (t == s) continue;
    atomicOr(&mask[s], 1u << d);          // s sees t across direction d
    atomicOr(&mask[t], 1u << (d ^ 1));    // and t sees s the other way
  }
}

__device__ __forceinline__ int box_nbr(const Boxes& B, int s, int d) {
  const int bx = s % B.px, by = (s / B.px) % B.py, bz = s / (B.px * B.py);
  int x = bx, y = by, z = bz;
  if (d == 0) ++x; else if (d == 1) --x; else if (d == 2) ++y; else if (d == 3) --y; else if (d == 4) ++z; else --z;
  if (x < 0 || x >= B.px || y < 0 || y >= B.py || z < 0 || z >= B.pz) return -1;
  return x + B.px * (y + B.py * z);
}

constexpr int kCompThreads = 1024;
constexpr int kSmemSubs = 6000;   // parents + masks (48 000 B) + two counters fit in 48 KB

// Root of x's tree.  Parents only ever point to smaller indices, so the walk
// ends within S steps; path halving (a node's parent replaced by its
// grandparent, still an ancestor) keeps trees shallow.  The step bound makes
// the walk finite whatever happens; exceeding it sets *err.
__device__ __forceinline__ int uf_find(volatile int* parent, int x, int S, int* err) {
  for (int step = 0; step <= S; ++step) {
    const int p = parent[x];
    if (p == x) return x;
    const int gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = gp;
  }
  atomicOr(err, 1);
  return x;
}

// Join the trees of a and b, hooking the larger root under the smaller one
// with a compare-and-swap that only succeeds while it is still a root.  A
// failed swap means another thread linked that root; there are at most S - 1
// links in all, so the retries are bounded (counted in *retries).
__device__ __forceinline__ void uf_union(volatile int* parent, int* parent_atomic, int a, int b, int S, int* err,
                                         int* retries) {
  for (int attempt = 0; attempt <= S; ++attempt) {
    int ra = uf_find(parent, a, S, err), rb = uf_find(parent, b, S, err);
    if (ra == rb) return;
    if (ra > rb) {
      const int t = ra;
      ra = rb;
      rb = t;
    }
    if (atomicCAS(&parent_atomic[rb], rb, ra) == rb) return;
    atomicAdd(retries, 1);
  }
  atomicOr(err, 1);
}

// Step 2 rule (a) and step 3 in one CTA: union-find over the coupling edges.
// Every tree's root is its smallest member, so the labels are the smallest
// subdomain index of each component whatever the order of the unions.  With
// SMEM the parents and masks live in shared memory (S <= kSmemSubs), else in
// the global work arrays.
template <bool SMEM>
__global__ void __launch_bounds__(kCompThreads) components_kernel(Boxes B, const int* __restrict__ sub_flag,
                                                                   unsigned* mask_g, int* labels_g, int* stats) {
  extern __shared__ int smem[];
  __shared__ int err, retries;
  const int S = B.px * B.py * B.pz;
  int* par = SMEM ? smem : labels_g;
  unsigned* msk = SMEM ? reinterpret_cast<unsigned*>(smem + S) : mask_g;
  if (threadIdx.x == 0) err = retries = 0;
  for (int s = threadIdx.x; s < S; s += kCompThreads) {
    par[s] = s;
    if (SMEM) msk[s] = mask_g[s];
  }
  __syncthreads();
  // rule (a): a flagged subdomain is coupled with all its neighbouring subdomains
  for (int s = threadIdx.x; s < S; s += kCompThreads) {
    if (!sub_flag[s]) continue;
    for (int d = 0; d < 6; ++d) {
      const int t = box_nbr(B, s, d);
      if (t < 0) continue;
      atomicOr(&msk[s], 1u << d);
      atomicOr(&msk[t], 1u << (d ^ 1));
    }
  }
  __syncthreads();
  // every edge once, from its endpoint in the + direction's lower side
  for (int s = threadIdx.x; s < S; s += kCompThreads) {
    const unsigned bits = msk[s];
    for (int d = 0; d < 6; d += 2)
      if (bits & (1u << d)) uf_union(par, par, s, box_nbr(B, s, d), S, &err, &retries);
  }
  __syncthreads();
  // roots are final now; in the global path the finds may still halve paths
  // in the parent array, which is the label array, so the roots go through
  // the mask array (no longer needed) before they are written as labels
  for (int s = threadIdx.x; s < S; s += kCompThreads) {
    const int r = uf_find(par, s, S, &err);
    if (SMEM) labels_g[s] = r;
    else mask_g[s] = (unsigned)r;
  }
  __syncthreads();
  if (!SMEM)
    for (int s = threadIdx.x; s < S; s += kCompThreads) labels_g[s] = (int)mask_g[s];
  if (threadIdx.x == 0) {
    stats[0] = retries;
    stats[1] = err;
  }
}

}  // namespace
}  // namespace ocp

extern "C" {

int64_t ocp_coupling_work_ints(int px, int py, int pz) {
  if (px < 1 || py < 1 || pz < 1) return 0;
  return 2 * (int64_t)px * py * pz + 4;
}

ocp_status ocp_coupling_components(ocp_grid* g, const double* u_new, const int8_t* flag_new, const double* u_old,
                                   const int8_t* flag_old, double threshold, int px, int py, int pz,
                                   int32_t* labels, int32_t* work, void* stream) {
  using namespace ocp;
  if (!g || !u_new || !u_old || !labels || !work || (g->prm.nb == 3 && (!flag_new || !flag_old)))
    return report(OCP_ERR_INVALID_ARG, "grid, states, flags, labels and work are required");
  if (px < 1 || py < 1 || pz < 1 || px > g->prm.nx || py > g->prm.ny || pz > g->prm.nz)
    return report(OCP_ERR_INVALID_ARG, "subdomain counts must be in [1, cells per direction]");
  if (!(threshold >= 0.0) || !std::isfinite(threshold)) return report(OCP_ERR_INVALID_ARG, "bad threshold");
  const int S = px * py * pz;
  int prev = -1;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess && prev != g->device) e = cudaSetDevice(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  int* sub_flag = work;
  unsigned* mask = reinterpret_cast<unsigned*>(work + S);
  int* nmarked = work + 2 * S;
  int* stats = work + 2 * S + 1;   // union retries, error flag
  if (e == cudaSuccess) e = cudaMemsetAsync(work, 0, sizeof(int32_t) * (2 * (size_t)S + 4), s);
  Boxes B{px, py, pz};
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)((g->prm.N + 255) / 256);   // 256 = whole warps, as mark_kernel needs
    if (g->prm.nb == 3)
      mark_kernel<3><<<blocks, 256, 0, s>>>(g->prm, B, u_new, flag_new, u_old, flag_old, threshold, sub_flag, mask, nmarked);
    else
      mark_kernel<2><<<blocks, 256, 0, s>>>(g->prm, B, u_new, flag_new, u_old, flag_old, threshold, sub_flag, mask, nmarked);
    if (S <= kSmemSubs)
      components_kernel<true><<<1, kCompThreads, 8 * (size_t)S, s>>>(B, sub_flag, mask, labels, stats);
    else
      components_kernel<false><<<1, kCompThreads, 0, s>>>(B, sub_flag, mask, labels, stats);
    e = cudaGetLastError();
  }
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return report(OCP_ERR_CUDA, "ocp_coupling_components: %s", cudaGetErrorString(e));
  return OCP_OK;
}

}  // extern "C"
