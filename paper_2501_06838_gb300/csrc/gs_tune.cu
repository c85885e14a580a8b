// Autotuner of the render's launch parameters (tile edge, shared-memory batch,
// binning, raster layout, adjoint), behind gs_tune in include/gs.h. Host code: it times the public
// entry points with CUDA events on the caller's workload and keeps the
// fastest choice per workload signature in an optional JSON-lines cache.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gs.h"
#include "gs_internal.cuh"

namespace gs {
void set_last_error(const char* msg);
}

namespace {

struct Cand {
  int tile, batch, binning, raster, adjoint;
};

std::string signature(int32_t n_images, const gs_gaussians* g, const gs_view* v, bool adj,
                      int64_t pairs16) {
  cudaDeviceProp prop;
  int dev = 0;
  std::string name = "gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  double px = 0.0;
  for (int i = 0; i < n_images; ++i) px += (double)v[i].out_h * v[i].out_w;
  const int lpx = (int)std::lround(std::log2(std::max(px, 1.0)));
  const int limg = (int)std::lround(std::log2((double)n_images));
  const int lppp = (int)std::lround(std::log2(std::max((double)pairs16, 1.0) / std::max(px, 1.0) * 256.0));
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s|dt%d|%s|px%d|img%d|ppp%d|head%d", name.c_str(), g[0].dtype,
                adj ? "fwdbwd" : "fwd", lpx, limg, lppp, g[0].head ? 1 : 0);
  return buf;
}

// The cache is JSON lines, one object per tuned workload:
//   {"signature": "...", "tile": 16, "batch": 32, "binning": 2, "adjoint": 1, "raster": 1,
//    "ms": 0.125}
// (written by cache_append; other lines are skipped).
bool cache_lookup(const char* path, const std::string& sig, gs_tuning* out) {
  if (!path) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512], key[256];
  gs_tuning t{};
  bool found = false;
  while (std::fgets(line, sizeof(line), f)) {
    if (std::sscanf(line,
                    " {\"signature\": \"%255[^\"]\", \"tile\": %d, \"batch\": %d, "
                    "\"binning\": %d, \"adjoint\": %d, \"raster\": %d, \"ms\": %f}",
                    key, &t.tile, &t.batch, &t.binning, &t.adjoint, &t.raster, &t.ms) == 7 &&
        sig == key) {
      *out = t;   // the last matching line wins
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_append(const char* path, const std::string& sig, const gs_tuning& t) {
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f,
               "{\"signature\": \"%s\", \"tile\": %d, \"batch\": %d, \"binning\": %d, "
               "\"adjoint\": %d, \"raster\": %d, \"ms\": %.6f}\n",
               sig.c_str(), t.tile, t.batch, t.binning, t.adjoint, t.raster, t.ms);
  std::fclose(f);
}

}  // namespace

extern "C" gs_status gs_tune(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                             float* const* outs, const float* const* grad_outs,
                             float* const* grads, void* ws, size_t ws_bytes, void* stream,
                             int32_t reps, const char* cache_path, gs_tuning* best) {
  if (!best || !g || !v || n_images < 1 || !outs) {
    gs::set_last_error("gs_tune: null argument or n_images < 1");
    return GS_ERR_INVALID;
  }
  if (reps < 1 || reps > 100) {
    gs::set_last_error("gs_tune: reps must be in 1..100");
    return GS_ERR_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool adj = grad_outs && grads;
  std::vector<gs_view> vv(v, v + n_images);
  auto with = [&](const Cand& c) {
    for (auto& x : vv) {
      x.tile = c.tile;
      x.batch = c.batch;
      x.binning = c.binning;
      x.raster = c.raster;
      x.adjoint = c.adjoint;
    }
  };
  bool grid_ok = true;
  for (int i = 0; i < n_images; ++i)
    if (g[i].ref_grid_m == 0 || v[i].out_w > 32767 || v[i].out_h > 32767) grid_ok = false;

  with(Cand{16, 32, GS_BINNING_SORT, GS_RASTER_TILE, GS_ADJOINT_TILE});
  int64_t pairs16 = 0;
  gs_status st = gs_count_pairs(n_images, g, vv.data(), ws, ws_bytes, stream, &pairs16);
  if (st != GS_OK) return st;
  const std::string sig = signature(n_images, g, v, adj, pairs16);
  if (cache_lookup(cache_path, sig, best)) {
    best->from_cache = 1;
    best->n_timed = 0;
    return GS_OK;
  }

  // launch layouts, each with the tile adjoint and, at tile 16, also with the
  // quadrant adjoint (which helps where windows are small, so it competes with
  // the smaller tiles rather than only with the winner)
  std::vector<Cand> cands;
  auto layout = [&](int tile, int batch, int binning, int raster) {
    cands.push_back(Cand{tile, batch, binning, raster, GS_ADJOINT_TILE});
    if (adj && tile == 16) cands.push_back(Cand{tile, batch, binning, raster, GS_ADJOINT_QUADRANT});
  };
  for (int tile : {16, 8, 32})
    for (int b : {1, 2}) {
      const int batch = (tile == 32 ? 64 : 32) * b;
      layout(tile, batch, GS_BINNING_SORT, GS_RASTER_TILE);
      if (grid_ok) {
        layout(tile, batch, GS_BINNING_GRID, GS_RASTER_TILE);
        if (tile == 16) layout(tile, batch, GS_BINNING_GRID, GS_RASTER_PAIR);
      }
    }
  // then the fastest of those with the Gaussian-warp adjoint
  const size_t n_layouts = cands.size();
  if (adj) cands.push_back(Cand{16, 32, GS_BINNING_SORT, GS_RASTER_TILE, GS_ADJOINT_GAUSSIAN});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    gs::set_last_error("gs_tune: cudaEventCreate failed");
    return GS_ERR_CUDA;
  }
  gs_tuning win{};
  win.ms = INFINITY;
  int timed = 0;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    if (ci >= n_layouts) {   // the fastest layout so far, with the Gaussian-warp adjoint
      if (timed == 0) break;   // no layout ran
      cands[ci] = Cand{win.tile, win.batch, win.binning, win.raster, cands[ci].adjoint};
    }
    const Cand c = cands[ci];
    with(c);
    // does the pair list fit? (tile size changes the pair count)
    int64_t need = 0;
    if (gs_count_pairs(n_images, g, vv.data(), ws, ws_bytes, stream, &need) != GS_OK) continue;
    if (gs_workspace_size(n_images, g, vv.data(), need) > ws_bytes) continue;
    auto call = [&]() -> gs_status {
      gs_status r = gs_render_batched(n_images, g, vv.data(), outs, ws, ws_bytes, stream);
      if (r == GS_OK && adj) r = gs_render_batched_bwd(n_images, g, vv.data(), grad_outs, grads, ws,
                                                       ws_bytes, stream);
      return r;
    };
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) ok = call() == GS_OK;
    std::vector<float> ts;
    for (int k = 0; k < reps && ok; ++k) {
      cudaEventRecord(e0, s);
      ok = call() == GS_OK;
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        ts.push_back(ms);
      else
        ok = false;
    }
    if (ok) ok = gs_sync_status(ws, stream) == GS_OK;
    if (!ok || ts.empty()) continue;
    std::sort(ts.begin(), ts.end());
    const float med = ts[ts.size() / 2];
    ++timed;
    if (med < win.ms) {
      win.tile = c.tile;
      win.batch = c.batch;
      win.binning = c.binning;
      win.raster = c.raster;
      win.adjoint = c.adjoint;
      win.ms = med;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (timed == 0) {
    gs::set_last_error("gs_tune: no candidate ran (workspace too small or invalid input)");
    return GS_ERR_CAPACITY;
  }
  win.from_cache = 0;
  win.n_timed = timed;
  *best = win;
  cache_append(cache_path, sig, win);
  return GS_OK;
}
