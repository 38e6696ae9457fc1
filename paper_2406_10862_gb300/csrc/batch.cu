// Batched ensemble: many grids linearised by one pass of the tile kernels.
//
// The per-model arguments live in a device table, the tile lists hold
// (model, first cell) pairs with the largest models first, and every CTA of
// a stage strides over the list; the three stages (cell, face, assemble) can
// be captured once into a CUDA graph and replayed.  Because the single-grid
// path runs the same kernels, a batched linearisation is bit-identical to
// linearising each grid on its own, for every launch shape.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "ocp_internal.cuh"

struct ocp_batch {
  int device = 0;
  int nb = 0;
  int sms = 0;
  std::vector<ocp_grid*> grids;
  ocp::ModelArgs* h_models = nullptr;   // pinned staging of the argument table
  ocp::ModelArgs* d_models = nullptr;
  int2* d_tiles[ocp::kNumTileSizes] = {};
  int ntiles[ocp::kNumTileSizes] = {};
  // ordered launch: models largest first, tiles of the models before each
  // (per tile size), and the item counter plus cell and face flags
  int* d_order = nullptr;
  long long* d_tile_start[ocp::kNumTileSizes] = {};
  unsigned* d_sync = nullptr;
  long long nsync_tiles = 0;             // flags per stage (tiles of 32 cells)
  ocp::LaunchCfg cfg;
  bool io_set = false;
  bool dirty = true;                     // host table newer than the device one
  double dt = -1.0;
  cudaStream_t cap = nullptr;            // private stream for graph capture
  cudaGraphExec_t exec = nullptr;
  long long ncell = 0;
};

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

void free_batch(ocp_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFreeHost(b->h_models);
  cudaFree(b->d_models);
  for (int t = 0; t < ocp::kNumTileSizes; ++t) {
    cudaFree(b->d_tiles[t]);
    cudaFree(b->d_tile_start[t]);
  }
  cudaFree(b->d_order);
  cudaFree(b->d_sync);
  delete b;
}

void lists_of(const ocp_batch* b, ocp::TileList* L) {
  for (int k = 0; k < ocp::kNumTileSizes; ++k) {
    L[k].models = b->d_models;
    L[k].tiles = b->d_tiles[k];
    L[k].ntiles = b->ntiles[k];
  }
}

// Upload the argument table if it changed (stream-ordered after earlier work
// on `s`; the host copy is not touched again until the upload has finished).
cudaError_t upload(ocp_batch* b, double dt, cudaStream_t s) {
  if (dt != b->dt) {
    for (size_t m = 0; m < b->grids.size(); ++m) b->h_models[m].scale = b->grids[m]->prm.vol_rb / dt;
    b->dt = dt;
    b->dirty = true;
  }
  if (!b->dirty) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(b->d_models, b->h_models, sizeof(ocp::ModelArgs) * b->grids.size(),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) b->dirty = false;
  return e;
}

// The largest one-cluster launch a batch may take: only a batch of one
// grid, and only as large as its device runs.
int cluster_tiles(const ocp_batch* b) { return b->grids.size() == 1 ? b->grids[0]->max_cluster : 0; }

cudaError_t run_cfg(ocp_batch* b, const ocp::LaunchCfg& cfg, cudaStream_t s) {
  ocp::TileList L[ocp::kNumTileSizes];
  lists_of(b, L);
  ocp::ModelArgs unused{};
  if (cfg.ordered == 0 || cfg.ordered == 3) return ocp::launch_tiles(b->nb, L, unused, cfg, b->sms, s);
  if (cfg.ordered == 4) return ocp::launch_cluster(b->nb, b->d_models, unused, b->grids[0]->prm.N, cluster_tiles(b), s);
  const int ti = ocp::tile_index(cfg.tpb[1]);
  if (ti < 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(unsigned) * (1 + 2 * b->nsync_tiles), s);
  if (e != cudaSuccess) return e;
  ocp::OrderedList O{};
  O.models = b->d_models;
  O.order = b->d_order;
  O.tile_start = b->d_tile_start[ti];
  O.nmodels = (int)b->grids.size();
  O.nitems = b->ntiles[ti];
  O.counter = b->d_sync;
  O.flag_cell = reinterpret_cast<int*>(b->d_sync + 1);
  O.flag_face = reinterpret_cast<int*>(b->d_sync + 1 + b->nsync_tiles);
  return ocp::launch_ordered(b->nb, L, O, unused, cfg, b->sms, s);
}

cudaError_t run(ocp_batch* b, cudaStream_t s) { return run_cfg(b, b->cfg, s); }

ocp_status check_shape(const ocp_launch_shape* sh) {
  if (!sh) return ocp::report(OCP_ERR_INVALID_ARG, "launch shape is NULL");
  for (int s = 0; s < 3; ++s) {
    if (ocp::tile_index(sh->cells_per_tile[s]) < 0)
      return ocp::report(OCP_ERR_INVALID_ARG, "cells_per_tile must be 32, 64, 128 or 256");
    if (sh->ctas_per_sm[s] < 0 || sh->ctas_per_sm[s] > 64)
      return ocp::report(OCP_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 64]");
  }
  if (sh->ordered < 0 || sh->ordered > 4) return ocp::report(OCP_ERR_INVALID_ARG, "ordered must be 0, 1, 2, 3 or 4");
  return OCP_OK;
}

// ordered = 4 needs a model of at most `max_tiles` 32-cell tiles.
ocp_status check_cluster(const ocp_launch_shape* sh, long long N, int max_tiles) {
  if (sh->ordered == 4 && (N + 31) / 32 > max_tiles)
    return ocp::report(OCP_ERR_INVALID_ARG,
                       "ordered = 4 needs one grid of at most %d 32-cell tiles on this device (has %lld)", max_tiles,
                       (N + 31) / 32);
  return OCP_OK;
}

}  // namespace

extern "C" {

ocp_status ocp_batch_create(ocp_grid* const* grids, int n, ocp_batch** out) {
  if (!out) return ocp::report(OCP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grids || n < 1) return ocp::report(OCP_ERR_INVALID_ARG, "need at least one grid");
  for (int m = 0; m < n; ++m) {
    if (!grids[m]) return ocp::report(OCP_ERR_INVALID_ARG, "grid %d is NULL", m);
    if (grids[m]->device != grids[0]->device) return ocp::report(OCP_ERR_INVALID_ARG, "grids are on different devices");
    if (grids[m]->prm.nb != grids[0]->prm.nb) return ocp::report(OCP_ERR_INVALID_ARG, "grids mix block sizes");
  }
  ocp_batch* b = new (std::nothrow) ocp_batch();
  if (!b) return ocp::report(OCP_ERR_OOM, "host allocation failed");
  b->device = grids[0]->device;
  b->nb = grids[0]->prm.nb;
  b->sms = grids[0]->sms;
  b->grids.assign(grids, grids + n);
  for (int m = 0; m < n; ++m) b->ncell += grids[m]->prm.N;
  b->cfg = ocp::default_cfg(b->ncell, b->sms, n == 1 ? grids[0]->max_cluster : 0);    // until tuned or set
  // largest models first
  std::vector<int> order(n);
  for (int m = 0; m < n; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return grids[a]->prm.N > grids[c]->prm.N; });
  std::vector<int2> tiles[ocp::kNumTileSizes];
  for (int k = 0; k < ocp::kNumTileSizes; ++k)
    for (int m : order)
      for (long long c0 = 0; c0 < grids[m]->prm.N; c0 += ocp::kTileSizes[k])
        tiles[k].push_back(make_int2(m, (int)c0));
  Guard guard(b->device);
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_models, sizeof(ocp::ModelArgs) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_models, sizeof(ocp::ModelArgs) * n);
  // the ordered launch's model order and per-model tile offsets
  std::vector<long long> tstart[ocp::kNumTileSizes];
  for (int k = 0; k < ocp::kNumTileSizes; ++k) {
    tstart[k].push_back(0);
    for (int m : order) tstart[k].push_back(tstart[k].back() + (grids[m]->prm.N + ocp::kTileSizes[k] - 1) / ocp::kTileSizes[k]);
  }
  b->nsync_tiles = tstart[0].back();
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_order, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_sync, sizeof(unsigned) * (1 + 2 * b->nsync_tiles));
  for (int k = 0; k < ocp::kNumTileSizes && e == cudaSuccess; ++k) {
    e = cudaMalloc((void**)&b->d_tile_start[k], sizeof(long long) * tstart[k].size());
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_tile_start[k], tstart[k].data(), sizeof(long long) * tstart[k].size(),
                     cudaMemcpyHostToDevice);
  }
  for (int k = 0; k < ocp::kNumTileSizes && e == cudaSuccess; ++k) {
    b->ntiles[k] = (int)tiles[k].size();
    e = cudaMalloc((void**)&b->d_tiles[k], sizeof(int2) * tiles[k].size());
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_tiles[k], tiles[k].data(), sizeof(int2) * tiles[k].size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    free_batch(b);
    return ocp::report(e == cudaErrorMemoryAllocation ? OCP_ERR_OOM : OCP_ERR_CUDA, "ocp_batch_create: %s",
                       cudaGetErrorString(e));
  }
  *out = b;
  return OCP_OK;
}

ocp_status ocp_batch_destroy(ocp_batch* b) {
  if (!b) return OCP_OK;
  Guard guard(b->device);
  free_batch(b);
  return OCP_OK;
}

ocp_status ocp_batch_set_io(ocp_batch* b, const ocp_batch_io* io) {
  if (!b || !io) return ocp::report(OCP_ERR_INVALID_ARG, "batch and io are required");
  for (size_t m = 0; m < b->grids.size(); ++m) {
    const ocp_batch_io& x = io[m];
    if (!x.u_new || !x.u_old || !x.residual || !x.bsr_val || (b->nb == 3 && (!x.flag_new || !x.flag_old)))
      return ocp::report(OCP_ERR_INVALID_ARG, "model %d: missing input or output pointer", (int)m);
  }
  Guard guard(b->device);
  // the previous table may still be in flight: wait for the device first
  cudaError_t e = guard.err == cudaSuccess ? cudaDeviceSynchronize() : guard.err;
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_batch_set_io: %s", cudaGetErrorString(e));
  for (size_t m = 0; m < b->grids.size(); ++m) {
    const ocp_batch_io& x = io[m];
    b->h_models[m] = ocp::model_args(b->grids[m], b->grids[m]->d_scratch, x.u_new, x.flag_new, x.u_old,
                                     x.flag_old, 1.0, x.residual, x.bsr_val, x.face_flux);
  }
  b->io_set = true;
  b->dirty = true;
  b->dt = -1.0;
  return OCP_OK;
}

ocp_status ocp_batch_linearize(ocp_batch* b, double dt, void* stream) {
  if (!b) return ocp::report(OCP_ERR_INVALID_ARG, "batch is NULL");
  if (!b->io_set) return ocp::report(OCP_ERR_INVALID_ARG, "ocp_batch_set_io has not been called");
  if (!(std::isfinite(dt) && dt > 0.0)) return ocp::report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(b->device);
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = upload(b, dt, (cudaStream_t)stream);
  if (e == cudaSuccess) e = run(b, (cudaStream_t)stream);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_batch_linearize: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_batch_graph_launch(ocp_batch* b, double dt, void* stream) {
  if (!b) return ocp::report(OCP_ERR_INVALID_ARG, "batch is NULL");
  if (!b->io_set) return ocp::report(OCP_ERR_INVALID_ARG, "ocp_batch_set_io has not been called");
  if (!(std::isfinite(dt) && dt > 0.0)) return ocp::report(OCP_ERR_INVALID_ARG, "dt must be finite and > 0");
  Guard guard(b->device);
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = upload(b, dt, (cudaStream_t)stream);
  if (e == cudaSuccess && !b->exec) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t er = run(b, b->cap);
      e = cudaStreamEndCapture(b->cap, &graph);
      if (e == cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_batch_graph_launch: %s", cudaGetErrorString(e));
  return OCP_OK;
}

ocp_status ocp_batch_set_shape(ocp_batch* b, const ocp_launch_shape* sh) {
  if (!b) return ocp::report(OCP_ERR_INVALID_ARG, "batch is NULL");
  ocp_status st = check_shape(sh);
  if (st == OCP_OK) st = check_cluster(sh, b->grids.size() == 1 ? b->grids[0]->prm.N : b->ncell, cluster_tiles(b));
  if (st != OCP_OK) return st;
  for (int s = 0; s < 3; ++s) {
    b->cfg.tpb[s] = sh->cells_per_tile[s];
    b->cfg.ctas_per_sm[s] = sh->ctas_per_sm[s];
  }
  b->cfg.ordered = sh->ordered;
  if (b->exec) {                       // the captured graph has the old shape
    Guard guard(b->device);
    cudaDeviceSynchronize();
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return OCP_OK;
}

ocp_status ocp_batch_get_shape(const ocp_batch* b, ocp_launch_shape* sh) {
  if (!b || !sh) return ocp::report(OCP_ERR_INVALID_ARG, "batch and shape are required");
  for (int s = 0; s < 3; ++s) {
    sh->cells_per_tile[s] = b->cfg.tpb[s];
    sh->ctas_per_sm[s] = b->cfg.ctas_per_sm[s];
  }
  sh->ordered = b->cfg.ordered;
  return OCP_OK;
}

ocp_status ocp_batch_tune(ocp_batch* b, double dt, int reps, ocp_launch_shape* best, void* stream) {
  if (!b) return ocp::report(OCP_ERR_INVALID_ARG, "batch is NULL");
  if (!b->io_set) return ocp::report(OCP_ERR_INVALID_ARG, "ocp_batch_set_io has not been called");
  if (!(std::isfinite(dt) && dt > 0.0) || reps < 1) return ocp::report(OCP_ERR_INVALID_ARG, "bad dt or reps");
  Guard guard(b->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = upload(b, dt, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int ctas[6] = {0, 1, 2, 4, 8, 16};
  ocp::TileList L[ocp::kNumTileSizes];
  lists_of(b, L);
  ocp::ModelArgs unused{};
  ocp::LaunchCfg cur = b->cfg;
  cur.ordered = 0;                      // the stages are tuned as three plain launches
  for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
    float best_ms = 1e30f;
    ocp::LaunchCfg pick = cur;
    for (int ti = 0; ti < ocp::kNumTileSizes && e == cudaSuccess; ++ti)
      for (int ci = 0; ci < 6 && e == cudaSuccess; ++ci) {
        ocp::LaunchCfg c = cur;
        c.tpb[stage] = ocp::kTileSizes[ti];
        c.ctas_per_sm[stage] = ctas[ci];
        std::vector<float> t;
        for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
          // earlier stages with the current choice, then the timed stage alone
          ocp::LaunchCfg pre = cur, one = c;
          e = ocp::launch_tiles(b->nb, L, unused, pre, b->sms, s);   // a full pass makes every input valid
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          // run only `stage`: the other stages get an empty grid via a copy with zero tiles
          if (e == cudaSuccess) {
            ocp::LaunchCfg only = one;
            for (int q = 0; q < 3; ++q)
              if (q != stage) only.ctas_per_sm[q] = -1;
            e = ocp::launch_tiles(b->nb, L, unused, only, b->sms, s);
          }
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (r > 0) t.push_back(ms);
        }
        if (e != cudaSuccess) break;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (med < best_ms) {
          best_ms = med;
          pick = c;
        }
      }
    cur = pick;
  }
  // then the whole pass: the three launches as tuned against the ordered
  // launches (modes 1 and 2, every tile size, occupancy-sized or 1, 2, 4
  // CTAs per SM); the fastest is kept
  auto time_pass = [&](const ocp::LaunchCfg& c, float& med) {
    std::vector<float> t;
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = run_cfg(b, c, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) t.push_back(ms);
    }
    if (e == cudaSuccess) {
      std::sort(t.begin(), t.end());
      med = t[t.size() / 2];
    }
  };
  if (e == cudaSuccess) {
    float best_ms = 1e30f;
    time_pass(cur, best_ms);
    const int octas[4] = {0, 1, 2, 4};
    ocp::LaunchCfg base = cur;
    for (int mode = 3; mode <= 4 && e == cudaSuccess; ++mode) {   // the split face and assembly stages,
      if (mode == 4 && (b->ncell + 31) / 32 > cluster_tiles(b)) break;   // as three launches or one cluster
      ocp::LaunchCfg c = base;
      c.ordered = mode;
      c.ctas_per_sm[1] = c.ctas_per_sm[2] = 0;
      float ms = 1e30f;
      time_pass(c, ms);
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        cur = c;
      }
    }
    for (int mode = 1; mode <= 2 && e == cudaSuccess; ++mode)
      for (int ti = 0; ti < ocp::kNumTileSizes && e == cudaSuccess; ++ti)
        for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
          ocp::LaunchCfg c = base;
          c.ordered = mode;
          c.tpb[1] = ocp::kTileSizes[ti];
          c.ctas_per_sm[1] = octas[ci];
          float ms = 1e30f;
          time_pass(c, ms);
          if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            cur = c;
          }
        }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_batch_tune: %s", cudaGetErrorString(e));
  ocp_launch_shape sh;
  for (int q = 0; q < 3; ++q) {
    sh.cells_per_tile[q] = cur.tpb[q];
    sh.ctas_per_sm[q] = cur.ctas_per_sm[q];
  }
  sh.ordered = cur.ordered;
  if (best) *best = sh;
  return ocp_batch_set_shape(b, &sh);
}

ocp_status ocp_batch_get_status(ocp_batch* b, void* stream) {
  if (!b) return ocp::report(OCP_ERR_INVALID_ARG, "batch is NULL");
  ocp_status worst = OCP_OK;
  for (ocp_grid* g : b->grids) {
    ocp_status st = ocp_get_status(g, stream);
    if (st != OCP_OK && worst == OCP_OK) worst = st;
  }
  return worst;
}

ocp_status ocp_grid_set_shape(ocp_grid* g, const ocp_launch_shape* sh) {
  if (!g) return ocp::report(OCP_ERR_INVALID_ARG, "grid is NULL");
  ocp_status st = check_shape(sh);
  if (st == OCP_OK) st = check_cluster(sh, g->prm.N, g->max_cluster);
  if (st != OCP_OK) return st;
  for (int s = 0; s < 3; ++s) {
    g->cfg.tpb[s] = sh->cells_per_tile[s];
    g->cfg.ctas_per_sm[s] = sh->ctas_per_sm[s];
  }
  g->cfg.ordered = sh->ordered;
  return OCP_OK;
}

ocp_status ocp_grid_get_shape(const ocp_grid* g, ocp_launch_shape* sh) {
  if (!g || !sh) return ocp::report(OCP_ERR_INVALID_ARG, "grid and shape are required");
  for (int s = 0; s < 3; ++s) {
    sh->cells_per_tile[s] = g->cfg.tpb[s];
    sh->ctas_per_sm[s] = g->cfg.ctas_per_sm[s];
  }
  sh->ordered = g->cfg.ordered;
  return OCP_OK;
}

ocp_status ocp_grid_cluster_tiles(const ocp_grid* g, int* tiles) {
  if (!g || !tiles) return ocp::report(OCP_ERR_INVALID_ARG, "grid and tiles are required");
  *tiles = g->max_cluster;
  return OCP_OK;
}

}  // extern "C"
