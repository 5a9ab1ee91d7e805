// Launch-configuration autotuner.
//
// The fastest tiling depends on the grid: shallow grids (nz <= 16) favour
// whole-column tiles, small ones a persistent launch (one CTA per tile for the whole
// run), large ones streaming tiles whose row count trades halo traffic against
// shared memory and occupancy, and temporally blocked passes for their unprotected
// sweeps; batches of uneven grids favour the batched launches.
// abft_tune times short runs of every distinct candidate on the GPU, through the
// public calls only, and returns the fastest as an abft_options.  Results are kept
// per (shapes, mode, accumulation, Delta) for the life of the process, so tuning a
// shape again costs nothing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "abft.h"
#include "abft_internal.h"

namespace {

struct Cand {
  int tile_y, shallow, persistent, batch, depth;
};

struct Result {
  abft_options best;
  double us;
};

std::mutex g_lock;
std::map<std::string, Result> g_cache;

std::string key_of(const abft_grid* g, int n, const abft_options* o, int mode, int sweeps) {
  std::string k;
  char b[96];
  snprintf(b, sizeof b, "m%d a%d d%d s%d t%d b%d v%d|", mode, o->acc, o->delta, sweeps, o->track_residual,
           o->boundary, o->vectors);
  k += b;
  for (int i = 0; i < n; ++i) {
    snprintf(b, sizeof b, "%d,%d,%d;", g[i].nx, g[i].ny, g[i].nz);
    k += b;
  }
  return k;
}

// the settings a candidate actually changes for these grids (so equivalent candidates
// are timed once): per grid the tile class, then persistence, batching and depth
std::string effect_of(const abft_grid* g, int n, const Cand& c, int mode, int bc, int acc) {
  std::string e;
  char b[32];
  for (int i = 0; i < n; ++i) {
    const bool sh = c.shallow && g[i].nz <= abft::kShallowMaxZ;
    const int auto_rows = c.tile_y == 0 && n == 1 ? abft::balanced_shallow_rows(g[i]) : 8;
    const int ty = sh ? (c.tile_y == 16 && g[i].nz <= 8 ? 16 : auto_rows) : (c.tile_y == 0 ? 16 : c.tile_y);
    snprintf(b, sizeof b, "%d%d;", sh ? 1 : 0, ty);
    e += b;
  }
  snprintf(b, sizeof b, "p%db%dd%d", n > 1 && c.batch ? 0 : c.persistent, n > 1 ? c.batch : 0,
           bc != ABFT_BC_CLAMP || (mode == ABFT_MODE_ONLINE && (n > 1 || acc != ABFT_ACC_FP32)) ? 1 : c.depth);
  return e + b;
}

// temporal depth matters for clamped grids: unprotected sweeps (mode NONE, offline
// windows) and online checks of a single grid with FP32 checksums
std::vector<Cand> candidates(const abft_grid* g, int n, int mode, int bc, int acc) {
  std::vector<Cand> out;
  std::vector<std::string> seen;
  for (int depth : {1, 2, 3, 4})
    for (int batch : {1, 0})
      for (int persistent : {1, 0})
        for (int shallow : {1, 0})
          for (int ty : {0, 8, 16, 32}) {  // 0: the library's default height
            const Cand c{ty, shallow, persistent, batch, depth};
            const std::string e = effect_of(g, n, c, mode, bc, acc);
            if (std::find(seen.begin(), seen.end(), e) != seen.end()) continue;
            seen.push_back(e);
            out.push_back(c);
          }
  return out;
}

abft_options with(const abft_options& base, const Cand& c) {
  abft_options o = base;
  o.tile_y = c.tile_y;
  o.shallow = c.shallow;
  o.persistent = c.persistent;
  o.batch = c.batch;
  o.depth = c.depth;
  return o;
}

}  // namespace

extern "C" ABFT_API size_t abft_tune_workspace_bytes(const abft_grid* grids, int32_t n_grids,
                                                     const abft_options* base) {
  if (!grids || n_grids < 1 || !base) return 0;
  size_t m = 0;
  for (const Cand& c : candidates(grids, n_grids, ABFT_MODE_NONE, base->boundary, base->acc)) {
    const abft_options o = with(*base, c);
    const size_t b = abft_workspace_bytes(grids, n_grids, &o);
    if (b == 0) return 0;
    m = std::max(m, b);
  }
  return m;
}

extern "C" ABFT_API abft_status abft_tune(const abft_grid* grids, int32_t n_grids, const float* const* temp,
                                          const float* const* power, const abft_coeffs* coeffs,
                                          const abft_options* base, int32_t mode, int32_t sweeps,
                                          void* workspace, size_t workspace_bytes, abft_options* best,
                                          double* best_us_per_sweep) {
  if (!grids || n_grids < 1 || !temp || !power || !coeffs || !base || !workspace || !best || !best_us_per_sweep)
    return ABFT_E_INVAL;
  if (mode < 0 || mode > 2 || sweeps < 1 || sweeps > 100000) return ABFT_E_INVAL;
  const std::string key = key_of(grids, n_grids, base, mode, sweeps);
  {
    std::lock_guard<std::mutex> hold(g_lock);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      abft_options o = it->second.best;
      o.stream = base->stream;
      *best = o;
      *best_us_per_sweep = it->second.us;
      return ABFT_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(base->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ABFT_E_CUDA;
  double best_us = -1.0;
  abft_options win = *base;
  abft_status st = ABFT_OK;
  for (const Cand& c : candidates(grids, n_grids, mode, base->boundary, base->acc)) {
    const abft_options o = with(*base, c);
    const size_t need = abft_workspace_bytes(grids, n_grids, &o);
    if (need == 0 || need > workspace_bytes) continue;
    abft_ctx* ctx = nullptr;
    st = abft_init(&ctx, grids, n_grids, temp, power, coeffs, &o, workspace, workspace_bytes);
    if (st != ABFT_OK) break;
    float ms = 0.f;
    st = abft_step(ctx, 2, mode);  // warm-up: first launches, graph capture
    if (st == ABFT_OK && cudaEventRecord(e0, s) != cudaSuccess) st = ABFT_E_CUDA;
    if (st == ABFT_OK) st = abft_step(ctx, sweeps, mode);
    if (st == ABFT_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = ABFT_E_CUDA;
    abft_destroy(ctx);
    if (st != ABFT_OK) break;
    const double us = ms * 1e3 / sweeps;
    if (best_us < 0 || us < best_us) {
      best_us = us;
      win = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ABFT_OK) return st;
  if (best_us < 0) return ABFT_E_NOMEM;  // no candidate fitted the workspace
  *best = win;
  *best_us_per_sweep = best_us;
  std::lock_guard<std::mutex> hold(g_lock);
  g_cache[key] = Result{win, best_us};
  return ABFT_OK;
}
