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
  int2* d_tiles[2] = {nullptr, nullptr};
  int ntiles[2] = {0, 0};
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
  cudaFree(b->d_tiles[0]);
  cudaFree(b->d_tiles[1]);
  delete b;
}

void lists_of(const ocp_batch* b, ocp::TileList* L) {
  for (int k = 0; k < 2; ++k) {
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

cudaError_t run(ocp_batch* b, cudaStream_t s) {
  ocp::TileList L[2];
  lists_of(b, L);
  ocp::ModelArgs unused{};
  return ocp::launch_tiles(b->nb, L, unused, b->cfg, b->sms, s);
}

ocp_status check_shape(const ocp_launch_shape* sh) {
  if (!sh) return ocp::report(OCP_ERR_INVALID_ARG, "launch shape is NULL");
  for (int s = 0; s < 3; ++s) {
    if (sh->cells_per_tile[s] != 128 && sh->cells_per_tile[s] != 256)
      return ocp::report(OCP_ERR_INVALID_ARG, "cells_per_tile must be 128 or 256");
    if (sh->ctas_per_sm[s] < 0 || sh->ctas_per_sm[s] > 64)
      return ocp::report(OCP_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 64]");
  }
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
  b->cfg = grids[0]->cfg;
  // largest models first
  std::vector<int> order(n);
  for (int m = 0; m < n; ++m) order[m] = m;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return grids[a]->prm.N > grids[c]->prm.N; });
  std::vector<int2> tiles[2];
  const int tpb[2] = {128, 256};
  for (int k = 0; k < 2; ++k)
    for (int m : order)
      for (long long c0 = 0; c0 < grids[m]->prm.N; c0 += tpb[k]) tiles[k].push_back(make_int2(m, (int)c0));
  for (int m = 0; m < n; ++m) b->ncell += grids[m]->prm.N;
  Guard guard(b->device);
  cudaError_t e = guard.err;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_models, sizeof(ocp::ModelArgs) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_models, sizeof(ocp::ModelArgs) * n);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
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
  if (st != OCP_OK) return st;
  for (int s = 0; s < 3; ++s) {
    b->cfg.tpb[s] = sh->cells_per_tile[s];
    b->cfg.ctas_per_sm[s] = sh->ctas_per_sm[s];
  }
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
  const int tpbs[2] = {128, 256};
  const int ctas[6] = {0, 1, 2, 4, 8, 16};
  ocp::TileList L[2];
  lists_of(b, L);
  ocp::ModelArgs unused{};
  ocp::LaunchCfg cur = b->cfg;
  for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
    float best_ms = 1e30f;
    ocp::LaunchCfg pick = cur;
    for (int ti = 0; ti < 2 && e == cudaSuccess; ++ti)
      for (int ci = 0; ci < 6 && e == cudaSuccess; ++ci) {
        ocp::LaunchCfg c = cur;
        c.tpb[stage] = tpbs[ti];
        c.ctas_per_sm[stage] = ctas[ci];
        std::vector<float> t;
        for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
          // earlier stages with the current choice, then the timed stage alone
          ocp::LaunchCfg pre = cur, one = c;
          e = ocp::launch_tiles(b->nb, L, unused, pre, b->sms, s);   // a full pass makes every input valid
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          // run only `stage`: the other stages get an empty grid via a copy with zero tiles
          if (e == cudaSuccess) {
            ocp::TileList Ls[2] = {L[0], L[1]};
            ocp::LaunchCfg only = one;
            for (int q = 0; q < 3; ++q)
              if (q != stage) only.ctas_per_sm[q] = -1;
            e = ocp::launch_tiles(b->nb, Ls, unused, only, b->sms, s);
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
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return ocp::report(OCP_ERR_CUDA, "ocp_batch_tune: %s", cudaGetErrorString(e));
  ocp_launch_shape sh;
  for (int q = 0; q < 3; ++q) {
    sh.cells_per_tile[q] = cur.tpb[q];
    sh.ctas_per_sm[q] = cur.ctas_per_sm[q];
  }
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
  if (st != OCP_OK) return st;
  for (int s = 0; s < 3; ++s) {
    g->cfg.tpb[s] = sh->cells_per_tile[s];
    g->cfg.ctas_per_sm[s] = sh->ctas_per_sm[s];
  }
  return OCP_OK;
}

}  // extern "C"
