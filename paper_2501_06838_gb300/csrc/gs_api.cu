// C-ABI entry points (include/gs.h): argument validation, workspace layout,
// and the launch sequence of the render and its adjoint. All device work is
// in the kernels of gs_preprocess.cu, gs_binning.cu and gs_raster.cu.
#include <atomic>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gs.h"
#include "gs_internal.cuh"

namespace gs {
int scan_parts_needed(int64_t n);
int sort_blocks_needed(int64_t capacity);
}  // namespace gs

namespace {

using namespace gs;

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

// ---------------------------------------------------------------------------
// Launch accounting and optional per-kernel event timing.
// ---------------------------------------------------------------------------
struct TimedLaunch {
  int id;
  cudaEvent_t a, b;
  bool graph;   // recorded under stream capture: event-record nodes, re-recorded by every replay
};
std::mutex g_tmu;
std::atomic<uint32_t> g_timing_mask{0u};
std::vector<TimedLaunch> g_timed;
std::vector<cudaEvent_t> g_event_pool;
thread_local cudaEvent_t g_pending_start = nullptr;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

const char* kKernelNames[kKNumKernels] = {
    "setup",      "preprocess",    "reserved",      "scan_top",   "radix_rowscan",
    "emit",       "radix_hist",    "radix_scatter", "ranges",     "raster_fwd",
    "raster_bwd", "preprocess_bwd", "reserved12",    "raster_bwd_gw"};

gs_status fail(gs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

gs_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return GS_ERR_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t hdr, images, records, trect, counts, parts, keys0, vals0, keys1, vals1, hist, hscan,
      ranges, grec, win, ext, tcount, total;
  int64_t n, capacity;
  int tiles, sort_blocks, scan_parts;
};

// grid: grid-implicit binning keeps one pair array (the per-tile lists the
// forward leaves for the adjoint) and no sort buffers.
Layout make_layout(int n_images, int64_t n, int64_t tiles, int64_t capacity, bool grid) {
  Layout L;
  L.n = n;
  L.capacity = capacity;
  L.tiles = (int)tiles;
  L.sort_blocks = grid ? 0 : sort_blocks_needed(capacity);
  const int64_t hist_n = 512LL * L.sort_blocks;   // up to 9-bit digits
  L.scan_parts = scan_parts_needed(n) + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.hdr = take(sizeof(Header));
  L.images = take(sizeof(ImageDesc) * (size_t)n_images);
  L.records = take(64 * (size_t)n);
  L.trect = take(16 * (size_t)n);
  L.counts = take(4 * (size_t)n);
  L.parts = take(8 * (size_t)L.scan_parts);
  const size_t sortcap = grid ? 0 : (size_t)capacity;
  L.keys0 = take(4 * sortcap);
  L.vals0 = take(4 * (size_t)capacity);
  L.keys1 = take(4 * sortcap);
  L.vals1 = take(4 * sortcap);
  L.hist = take(4 * (size_t)hist_n);
  L.hscan = take(4 * 512);
  L.ranges = take(8 * (size_t)tiles);
  L.grec = take(48 * (size_t)n);
  L.win = take(8 * (size_t)n);
  L.ext = take(16 * (size_t)n_images);
  L.tcount = take(4 * (size_t)tiles);
  L.total = o;
  return L;
}

int tile_of(const gs_view& v) { return v.tile == 0 ? 16 : v.tile; }
int batch_of(const gs_view& v) { return v.batch; }   // 0: the tile's smaller batch
int shift_of(int tile) { return tile == 8 ? 3 : tile == 32 ? 5 : 4; }

struct Problem {
  int n_images;
  int64_t n;
  int64_t tiles;
  int tile, batch;
  int adjoint;   // gs_adjoint resolved: 1 tile, 2 Gaussian-warp, 3 tile quadrants
  int grid;      // gs_binning resolved: 1 grid-implicit, 0 sorted pair list
  int pair;      // gs_raster resolved: 1 one warp per pair of tiles, 0 per tile
};

gs_status validate(int32_t n_images, const gs_gaussians* g, const gs_view* v, Problem* P) {
  if (n_images < 1) return fail(GS_ERR_INVALID, "n_images must be >= 1 (got %lld)", (long long)n_images);
  if (!g || !v) return fail(GS_ERR_INVALID, "null gaussians or view array");
  P->n_images = n_images;
  P->n = 0;
  P->tiles = 0;
  P->tile = tile_of(v[0]);
  P->batch = batch_of(v[0]);
  bool grid_ok = true;   // every image on a reference grid, coordinates fit int16
  bool sigma_windows = true, large_scale = false;   // for the AUTO raster layout and adjoint
  bool truncated = true;                             // every window a k-sigma box (trunc_k > 0)
  for (int i = 0; i < n_images; ++i) {
    const gs_gaussians& G = g[i];
    const gs_view& V = v[i];
    if (G.n < 0) return fail(GS_ERR_INVALID, "image %lld: n < 0", (long long)i);
    if (G.dtype < 0 || G.dtype > 2) return fail(GS_ERR_INVALID, "image %lld: unknown dtype", (long long)i);
    const int m = G.ref_grid_m;
    if (!(m == 0 || m == 1 || m == 4 || m == 9 || m == 16))
      return fail(GS_ERR_INVALID, "image %lld: ref_grid_m must be 0, 1, 4, 9 or 16", (long long)i);
    if (V.lr_h < 1 || V.lr_w < 1 || V.out_h < 1 || V.out_w < 1)
      return fail(GS_ERR_INVALID, "image %lld: sizes must be >= 1", (long long)i);
    if (!(V.scale > 0.0f) || !std::isfinite(V.scale))
      return fail(GS_ERR_INVALID, "image %lld: scale must be finite and > 0", (long long)i);
    if (!std::isfinite(V.trunc_k)) return fail(GS_ERR_INVALID, "image %lld: trunc_k not finite", (long long)i);
    if (V.norm != 0 && V.norm != 1) return fail(GS_ERR_INVALID, "image %lld: unknown norm", (long long)i);
    if (V.window != 0 && V.window != 1)
      return fail(GS_ERR_INVALID, "image %lld: unknown window", (long long)i);
    if (V.align != 0 && V.align != 1) return fail(GS_ERR_INVALID, "image %lld: unknown align", (long long)i);
    if (V.align == 1 && !(V.scale < 8388608.0f))
      return fail(GS_ERR_INVALID, "image %lld: half-pixel alignment needs scale < 2^23", (long long)i);
    if (V.adjoint < 0 || V.adjoint > 3) return fail(GS_ERR_INVALID, "image %lld: unknown adjoint", (long long)i);
    if (V.adjoint != v[0].adjoint)
      return fail(GS_ERR_INVALID, "image %lld: adjoint differs from image 0", (long long)i);
    if (V.binning < 0 || V.binning > 2) return fail(GS_ERR_INVALID, "image %lld: unknown binning", (long long)i);
    if (V.row0 < 0) return fail(GS_ERR_INVALID, "image %lld: row0 < 0", (long long)i);
    if (V.binning != v[0].binning)
      return fail(GS_ERR_INVALID, "image %lld: binning differs from image 0", (long long)i);
    if (V.raster < 0 || V.raster > 2) return fail(GS_ERR_INVALID, "image %lld: unknown raster", (long long)i);
    if (V.raster != v[0].raster)
      return fail(GS_ERR_INVALID, "image %lld: raster differs from image 0", (long long)i);
    if (V.window != GS_WINDOW_SIGMA) sigma_windows = false;
    if (V.scale >= 6.0f) large_scale = true;
    if (!(V.trunc_k > 0.0f)) truncated = false;
    if (G.ref_grid_m == 0 || V.out_w > 32767 || V.out_h > 32767) grid_ok = false;
    const double sh = std::floor((double)V.scale * V.lr_h) + 1.0;
    const double sw = std::floor((double)V.scale * V.lr_w) + 1.0;
    if ((double)V.out_h + (double)V.row0 > sh || (double)V.out_w > sw)
      return fail(GS_ERR_INVALID, "image %lld: output larger than floor(s * lr) + 1", (long long)i);
    if (tile_of(V) != P->tile || batch_of(V) != P->batch)
      return fail(GS_ERR_INVALID, "image %lld: tile/batch differ from image 0", (long long)i);
    if (m > 0 && G.n != (int64_t)m * V.lr_h * V.lr_w)
      return fail(GS_ERR_INVALID, "image %lld: n != m * lr_h * lr_w", (long long)i);
    if (G.n > 0 && (!G.offset || !G.sigma || !G.rho || !G.rgb || !G.alpha))
      return fail(GS_ERR_INVALID, "image %lld: null parameter pointer", (long long)i);
    if (G.head) {
      const gs_head& Hd = *G.head;
      if (!(Hd.sigma_span > 0.0f) || !(Hd.sigma_lo >= 0.0f) || !std::isfinite(Hd.sigma_span) ||
          !std::isfinite(Hd.sigma_lo) || !(std::fabs(Hd.rho_scale) <= 1.0f) ||
          !std::isfinite(Hd.offset_scale) || (Hd.offset_tanh != 0 && Hd.offset_tanh != 1) ||
          Hd.reserved[0] || Hd.reserved[1] || Hd.reserved[2])
        return fail(GS_ERR_INVALID, "image %lld: invalid head (sigma_lo >= 0, sigma_span > 0, "
                    "|rho_scale| <= 1, offset_tanh 0 or 1, reserved 0)", (long long)i);
    }
    const int t = P->tile;
    const int64_t tx = (V.out_w + t - 1) / t, ty = (V.out_h + t - 1) / t;
    P->n += G.n;
    P->tiles += tx * ty;
  }
  if (!(P->tile == 8 || P->tile == 16 || P->tile == 32))
    return fail(GS_ERR_INVALID, "tile must be 8, 16 or 32 (got %lld)", (long long)P->tile);
  // the raster stages one or two Gaussians per thread of its block per round
  // (32 threads at tile 8 and 16, 64 at tile 32): only those batches run
  const bool batch_ok = P->batch == 0 || (P->tile == 32 ? (P->batch == 64 || P->batch == 128)
                                                         : (P->batch == 32 || P->batch == 64));
  if (!batch_ok)
    return fail(GS_ERR_INVALID,
                "batch must be 0 (default) or a batch the raster runs: 32 or 64 Gaussians per "
                "shared-memory round at tile 8 and 16, 64 or 128 at tile 32 (got %lld at tile %lld)",
                (long long)P->batch, (long long)P->tile);
  if (v[0].binning == GS_BINNING_GRID && !grid_ok)
    return fail(GS_ERR_UNSUPPORTED,
                "grid binning needs every image on a reference grid (ref_grid_m > 0) and outputs "
                "of at most 32767 px a side");
  P->grid = (v[0].binning == GS_BINNING_GRID || (v[0].binning == GS_BINNING_AUTO && grid_ok)) ? 1 : 0;
  const bool pair_ok = P->grid && P->tile == 16;
  if (v[0].raster == GS_RASTER_PAIR && !pair_ok)
    return fail(GS_ERR_UNSUPPORTED, "raster PAIR needs grid binning and tile 16");
  P->pair = (v[0].raster == GS_RASTER_PAIR ||
             (v[0].raster == GS_RASTER_AUTO && pair_ok && sigma_windows && large_scale)) ? 1 : 0;
  if (v[0].adjoint == GS_ADJOINT_QUADRANT && P->tile != 16)
    return fail(GS_ERR_UNSUPPORTED, "adjoint QUADRANT needs tile 16");
  // AUTO: quadrants at tile 16 where every view has truncated SIGMA windows at
  // scale < 6 (small windows, where they measured faster), else whole tiles
  const bool quad_auto = P->tile == 16 && sigma_windows && truncated && !large_scale;
  P->adjoint = v[0].adjoint == GS_ADJOINT_GAUSSIAN ? GS_ADJOINT_GAUSSIAN
               : (v[0].adjoint == GS_ADJOINT_QUADRANT ||
                  (v[0].adjoint == GS_ADJOINT_AUTO && quad_auto)) ? GS_ADJOINT_QUADRANT
                                                                  : GS_ADJOINT_TILE;
  if (P->n >= (1LL << 31)) return fail(GS_ERR_UNSUPPORTED, "more than 2^31 - 1 Gaussians");
  if (P->tiles >= (1LL << 24)) return fail(GS_ERR_UNSUPPORTED, "more than 2^24 tiles");
  return GS_OK;
}

int64_t capacity_for(const Problem& P, size_t bytes) {
  int64_t lo = 0, hi = (1LL << 31) - 1;
  if (make_layout(P.n_images, P.n, P.tiles, 0, P.grid).total > bytes) return -1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo + 1) / 2;
    if (make_layout(P.n_images, P.n, P.tiles, mid, P.grid).total <= bytes) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Significant bits of the largest tile key, and the radix passes that sort them
// (at most 9 bits per pass, as launch_sort does).
int key_bits(int64_t tiles) {
  int bits = 0;
  while (bits < 32 && ((tiles - 1) >> bits) > 0) ++bits;
  return bits;
}
int radix_passes(int64_t tiles) { return (key_bits(tiles) + 8) / 9; }

struct Call {
  Problem P;
  Layout L;
  Ws w;
  int passes;
};

gs_status prepare(int32_t n_images, const gs_gaussians* g, const gs_view* v, void* ws,
                  size_t ws_bytes, Call* c) {
  gs_status st = validate(n_images, g, v, &c->P);
  if (st != GS_OK) return st;
  if (!ws) return fail(GS_ERR_INVALID, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0)
    return fail(GS_ERR_INVALID, "workspace must be 256-byte aligned");
  const int64_t cap = capacity_for(c->P, ws_bytes);
  if (cap < 0) return fail(GS_ERR_INVALID, "workspace too small (%lld bytes)", (long long)ws_bytes);
  c->L = make_layout(n_images, c->P.n, c->P.tiles, cap, c->P.grid);
  char* b = static_cast<char*>(ws);
  const Layout& L = c->L;
  Ws& w = c->w;
  w.hdr = reinterpret_cast<Header*>(b + L.hdr);
  w.images = reinterpret_cast<ImageDesc*>(b + L.images);
  w.records = reinterpret_cast<float4*>(b + L.records);
  w.trect = reinterpret_cast<uint4*>(b + L.trect);
  w.counts = reinterpret_cast<uint32_t*>(b + L.counts);
  w.parts = reinterpret_cast<unsigned long long*>(b + L.parts);
  w.keys[0] = reinterpret_cast<uint32_t*>(b + L.keys0);
  w.vals[0] = reinterpret_cast<uint32_t*>(b + L.vals0);
  w.keys[1] = reinterpret_cast<uint32_t*>(b + L.keys1);
  w.vals[1] = reinterpret_cast<uint32_t*>(b + L.vals1);
  w.hist = reinterpret_cast<uint32_t*>(b + L.hist);
  w.hscan = reinterpret_cast<uint32_t*>(b + L.hscan);
  w.ranges = reinterpret_cast<uint2*>(b + L.ranges);
  w.grec = reinterpret_cast<float*>(b + L.grec);
  w.win = reinterpret_cast<short4*>(b + L.win);
  w.ext = reinterpret_cast<int4*>(b + L.ext);
  w.tcount = reinterpret_cast<uint32_t*>(b + L.tcount);
  w.grid = c->P.grid;
  w.direct = 0;
  w.grad_out0 = nullptr;
  w.grads0 = nullptr;
  w.n = c->P.n;
  w.capacity = cap;
  w.n_images = n_images;
  w.tiles = (int)c->P.tiles;
  w.tile = c->P.tile;
  w.tile_shift = shift_of(c->P.tile);
  w.sort_blocks = L.sort_blocks;
  w.scan_parts = L.scan_parts;
  c->passes = radix_passes(c->P.tiles);
  // horizontal pairs of tiles (the forward's launch unit for grid binning at tile 16)
  int64_t pairs = 0;
  for (int i = 0; i < n_images; ++i) {
    const int64_t tx = (v[i].out_w + c->P.tile - 1) / c->P.tile;
    const int64_t ty = (v[i].out_h + c->P.tile - 1) / c->P.tile;
    pairs += ty * ((tx + 1) / 2);
  }
  w.n_pairs = (int32_t)pairs;
  w.pair = c->P.pair;
  w.adjoint = c->P.adjoint;
  // blocks of LR cells (the Gaussian-warp adjoint's block form), when
  // every image's Gaussians sit on a reference grid
  int64_t gblocks = 0;
  for (int i = 0; i < n_images; ++i) {
    if (g[i].ref_grid_m == 0) { gblocks = 0; break; }
    gblocks += (int64_t)((v[i].lr_h + kGbCellsY - 1) / kGbCellsY) *
               ((v[i].lr_w + kGbCellsX - 1) / kGbCellsX);
  }
  w.n_gblocks = gblocks < (1LL << 31) ? (int32_t)gblocks : 0;
  return GS_OK;
}

gs_status upload_images(const Call& c, const gs_gaussians* g, const gs_view* v, float* const* outs,
                        const float* const* grad_outs, float* const* grads, int reset,
                        cudaStream_t s) {
  int64_t gbase = 0;
  int tbase = 0, pbase = 0, bbase = 0;
  const int tile = c.P.tile;
  for (int first = 0; first < c.P.n_images; first += kSetupChunk) {
    SetupChunk ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.first = first;
    ch.count = c.P.n_images - first < kSetupChunk ? c.P.n_images - first : kSetupChunk;
    ch.reset = (reset && first == 0) ? 1 : 0;
    ch.reset_ext = reset ? 1 : 0;
    for (int k = 0; k < ch.count; ++k) {
      const int i = first + k;
      ImageDesc& d = ch.d[k];
      d.off = g[i].offset;
      d.sig = g[i].sigma;
      d.rho = g[i].rho;
      d.rgb = g[i].rgb;
      d.alpha = g[i].alpha;
      d.out = outs ? outs[i] : nullptr;
      d.grad_out = grad_outs ? grad_outs[i] : nullptr;
      d.grads = grads ? grads[i] : nullptr;
      d.n = g[i].n;
      d.g_base = gbase;
      d.dtype = g[i].dtype;
      d.m = g[i].ref_grid_m;
      d.lr_h = v[i].lr_h;
      d.lr_w = v[i].lr_w;
      d.out_h = v[i].out_h;
      d.out_w = v[i].out_w;
      d.row0 = v[i].row0;
      d.scale = v[i].scale;
      d.trunc_k = v[i].trunc_k;
      d.flags = (v[i].norm == GS_NORM_PEAK ? kFlagPeak : 0) |
                (v[i].window == GS_WINDOW_RATIO ? kFlagRatio : 0) |
                (v[i].align == GS_ALIGN_HALF ? kFlagHalf : 0) |
                (g[i].head ? kFlagHead : 0) |
                (g[i].head && g[i].head->offset_tanh ? kFlagOffsetTanh : 0);
      if (g[i].head) {
        d.h_sigma_lo = g[i].head->sigma_lo;
        d.h_sigma_span = g[i].head->sigma_span;
        d.h_rho_scale = g[i].head->rho_scale;
        d.h_offset_scale = g[i].head->offset_scale;
      }
      d.tiles_x = (v[i].out_w + tile - 1) / tile;
      d.tiles_y = (v[i].out_h + tile - 1) / tile;
      d.t_base = tbase;
      d.p_base = pbase;
      d.b_base = bbase;
      gbase += g[i].n;
      bbase += ((v[i].lr_h + kGbCellsY - 1) / kGbCellsY) * ((v[i].lr_w + kGbCellsX - 1) / kGbCellsX);
      tbase += d.tiles_x * d.tiles_y;
      pbase += d.tiles_y * ((d.tiles_x + 1) / 2);
    }
    cudaError_t e = launch_setup(ch, c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "setup");
  }
  return GS_OK;
}

gs_status run_forward(int32_t n_images, const gs_gaussians* g, const gs_view* v, float* const* outs,
                      void* ws, size_t ws_bytes, cudaStream_t s) {
  Call c;
  gs_status st = prepare(n_images, g, v, ws, ws_bytes, &c);
  if (st != GS_OK) return st;
  if (!outs) return fail(GS_ERR_INVALID, "null output array");
  for (int i = 0; i < n_images; ++i)
    if (!outs[i]) return fail(GS_ERR_INVALID, "null output pointer for image %lld", (long long)i);
  st = upload_images(c, g, v, outs, nullptr, nullptr, 1, s);
  if (st != GS_OK) return st;
  cudaError_t e;
  if (c.w.grid) {
    // grid-implicit binning: the footprint pass records per-row differences of
    // the pairs per tile (into the array the setup kernel cleared) and the
    // reach; the raster sums its tile's count, enumerates the tile's
    // candidates and leaves the tile's list for the adjoint (no sort)
    e = launch_preprocess(c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "preprocess");
    e = launch_raster_fwd(c.w, nullptr, c.P.batch, s);
    if (e != cudaSuccess) return cuda_fail(e, "raster_fwd");
    return GS_OK;
  }
  e = launch_preprocess(c.w, s);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess");
  if (c.w.n > 0) {
    e = launch_scan_counts(c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan");
    e = launch_emit(c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "emit");
  }
  int fb = 0;
  e = launch_sort(c.w, key_bits(c.P.tiles), s, &fb);
  if (e != cudaSuccess) return cuda_fail(e, "sort");
  e = launch_ranges(c.w, c.w.keys[fb], s);
  if (e != cudaSuccess) return cuda_fail(e, "ranges");
  e = launch_raster_fwd(c.w, c.w.vals[fb], c.P.batch, s);
  if (e != cudaSuccess) return cuda_fail(e, "raster_fwd");
  return GS_OK;
}

gs_status run_backward(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                       const float* const* grad_outs, float* const* grads, void* ws,
                       size_t ws_bytes, cudaStream_t s) {
  Call c;
  gs_status st = prepare(n_images, g, v, ws, ws_bytes, &c);
  if (st != GS_OK) return st;
  if (!grad_outs || !grads) return fail(GS_ERR_INVALID, "null gradient arrays");
  for (int i = 0; i < n_images; ++i) {
    if (!grad_outs[i]) return fail(GS_ERR_INVALID, "null grad_out pointer for image %lld", (long long)i);
    if (g[i].n > 0 && !grads[i]) return fail(GS_ERR_INVALID, "null grads pointer for image %lld", (long long)i);
  }
  if (n_images == 1) {
    // the image table is the forward's; the gradient pointers go by value
    c.w.direct = 1;
    c.w.grad_out0 = grad_outs[0];
    c.w.grads0 = grads[0];
  } else {
    st = upload_images(c, g, v, nullptr, grad_outs, grads, 0, s);
    if (st != GS_OK) return st;
  }
  if (c.w.n == 0) return GS_OK;
  cudaError_t e;
  if (c.P.adjoint != GS_ADJOINT_GAUSSIAN) {
    // the tile adjoint adds into the record-space accumulators, which the
    // forward's footprint pass zeroed and each chain rule clears after use
    const int fb = c.passes & 1;
    e = launch_raster_bwd_tile(c.w, c.w.grid ? c.w.vals[0] : c.w.vals[fb],
                               c.P.adjoint == GS_ADJOINT_QUADRANT, s);
    if (e != cudaSuccess) return cuda_fail(e, "raster_bwd");
  } else {
    // one warp per Gaussian writes all its moments: no clearing, no atomics
    // (blocks of LR cells staging the gradient in shared memory when the
    // Gaussians sit on a reference grid)
    e = c.w.n_gblocks > 0 ? launch_raster_bwd_gblock(c.w, s) : launch_raster_bwd_gw(c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "raster_bwd_gw");
  }
  e = launch_preprocess_bwd(c.w, s);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess_bwd");
  return GS_OK;
}

gs_status map_status(uint32_t bits) {
  if (bits & kStInvalid) return GS_ERR_INVALID;
  if (bits & kStCapacity) return GS_ERR_CAPACITY;
  if (bits & kStTimeout) return GS_ERR_TIMEOUT;
  if (bits & kStInternal) return GS_ERR_INTERNAL;
  return GS_OK;
}

const char* status_text(uint32_t bits) {
  if (bits & kStInvalid) return "a Gaussian parameter is non-finite or out of range";
  if (bits & kStCapacity) return "more (tile, Gaussian) pairs than the workspace capacity";
  if (bits & kStTimeout) return "a bounded device wait gave up";
  if (bits & kStInternal) return "internal consistency check failed";
  return "";
}

}  // namespace

namespace gs {

void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

int resident_grid(const void* kernel, int threads, int64_t work) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> cache;   // (kernel, device) -> CTAs
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return (int)work; }
  int ctas = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& e : cache)
      if (e.first.first == kernel && e.first.second == dev) ctas = e.second;
  }
  if (ctas == 0) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        per_sm < 1 || sms < 1) {
      cudaGetLastError();
      return (int)work;
    }
    ctas = per_sm * sms;
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back({{kernel, dev}, ctas});
  }
  return (int)(work < ctas ? work : ctas);
}

bool chain_overlap() {
  static const bool on = std::getenv("GS_NO_PDL") == nullptr;
  return on;
}

namespace {
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}
}  // namespace

void launch_begin(int id, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!((g_timing_mask.load(std::memory_order_relaxed) >> id) & 1u)) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t a = take_event();
  if (a) cudaEventRecordWithFlags(a, s, capturing(s) ? cudaEventRecordExternal : cudaEventRecordDefault);
  g_pending_start = a;
}

void launch_end(int id, cudaStream_t s) {
  if (!((g_timing_mask.load(std::memory_order_relaxed) >> id) & 1u)) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  cudaEvent_t a = g_pending_start;
  g_pending_start = nullptr;
  if (!a) return;
  cudaEvent_t b = take_event();
  if (!b) { g_event_pool.push_back(a); return; }
  const bool cap = capturing(s);
  cudaEventRecordWithFlags(b, s, cap ? cudaEventRecordExternal : cudaEventRecordDefault);
  g_timed.push_back(TimedLaunch{id, a, b, cap});
}

}  // namespace gs

extern "C" {

size_t gs_workspace_size(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                         int64_t pair_capacity) {
  Problem P;
  if (validate(n_images, g, v, &P) != GS_OK) return 0;
  if (pair_capacity < 0 || pair_capacity >= (1LL << 31)) {
    fail(GS_ERR_INVALID, "pair_capacity out of range (%lld)", (long long)pair_capacity);
    return 0;
  }
  return make_layout(n_images, P.n, P.tiles, pair_capacity, P.grid).total;
}

gs_status gs_count_pairs(int32_t n_images, const gs_gaussians* g, const gs_view* v, void* ws,
                         size_t ws_bytes, void* stream, int64_t* pairs_out) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!pairs_out) return fail(GS_ERR_INVALID, "null pairs_out");
  Call c;
  gs_status st = prepare(n_images, g, v, ws, ws_bytes, &c);
  if (st != GS_OK) return st;
  st = upload_images(c, g, v, nullptr, nullptr, nullptr, 1, s);
  if (st != GS_OK) return st;
  c.w.grid = 0;   // the count is the same either way; take it from the scan
  cudaError_t e = launch_preprocess(c.w, s);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess");
  if (c.w.n > 0) {
    e = launch_scan_counts(c.w, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan");
  }
  Header h;
  e = cudaMemcpyAsync(&h, c.w.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "count_pairs readback");
  *pairs_out = (int64_t)h.pairs;
  if (h.status & kStInvalid) return fail(GS_ERR_INVALID, "%s", status_text(kStInvalid));
  return GS_OK;
}

gs_status gs_render_fwd(const gs_gaussians* g, const gs_view* v, float* out, void* ws,
                        size_t ws_bytes, void* stream) {
  float* outs[1] = {out};
  return run_forward(1, g, v, outs, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

gs_status gs_render_bwd(const gs_gaussians* g, const gs_view* v, const float* grad_out,
                        float* grads, void* ws, size_t ws_bytes, void* stream) {
  const float* go[1] = {grad_out};
  float* gr[1] = {grads};
  return run_backward(1, g, v, go, gr, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

gs_status gs_render_batched(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                            float* const* outs, void* ws, size_t ws_bytes, void* stream) {
  return run_forward(n_images, g, v, outs, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

gs_status gs_render_batched_bwd(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                                const float* const* grad_outs, float* const* grads, void* ws,
                                size_t ws_bytes, void* stream) {
  return run_backward(n_images, g, v, grad_outs, grads, ws, ws_bytes,
                      static_cast<cudaStream_t>(stream));
}

gs_status gs_sync_status(void* ws, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!ws) return fail(GS_ERR_INVALID, "null workspace");
  Header* hdr = static_cast<Header*>(ws);
  uint32_t bits = 0;
  cudaError_t e = cudaMemcpyAsync(&bits, &hdr->status, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&hdr->status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "sync_status");
  gs_status st = map_status(bits);
  if (st != GS_OK) fail(st, "%s", status_text(bits));
  return st;
}

gs_status gs_read_stats(void* ws, void* stream, gs_stats* out) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!ws || !out) return fail(GS_ERR_INVALID, "null argument");
  Header h;
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(Header), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "read_stats");
  out->tile_pairs = (int64_t)h.pairs;
  out->pixel_pairs = (int64_t)h.pixel_pairs;
  out->capacity = (int64_t)h.capacity;
  out->n_gaussians = (int64_t)h.reserved[0];
  out->n_tiles = (int32_t)h.reserved[1];
  out->status = (int32_t)map_status(h.status);
  out->raster = h.reserved[2] ? GS_RASTER_PAIR : GS_RASTER_TILE;
  out->adjoint = (int32_t)h.reserved[3];
  return GS_OK;
}

const char* gs_last_error(void) { return g_last_error.c_str(); }

const char* gs_status_string(int32_t status) {
  switch (status) {
    case GS_OK: return "GS_OK";
    case GS_ERR_INVALID: return "GS_ERR_INVALID";
    case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
    case GS_ERR_CUDA: return "GS_ERR_CUDA";
    case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
    case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
    case GS_ERR_INTERNAL: return "GS_ERR_INTERNAL";
    default: return "GS_UNKNOWN";
  }
}

int64_t gs_launch_count(void) { return g_launches.load(); }

gs_status gs_timing_enable(int32_t kernel_mask) {
  g_timing_mask.store((uint32_t)kernel_mask);
  return GS_OK;
}

int32_t gs_timing_read(double* ms_out, int64_t* count_out, int32_t n) {
  std::lock_guard<std::mutex> lk(g_tmu);
  std::vector<TimedLaunch> keep;
  for (const TimedLaunch& t : g_timed) {
    cudaEventSynchronize(t.b);
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess && t.id < n) {
      if (ms_out) ms_out[t.id] += ms;
      if (count_out) count_out[t.id] += 1;
    } else {
      cudaGetLastError();   // a captured pair not yet replayed: no time to add
    }
    if (t.graph) {
      keep.push_back(t);
    } else {
      g_event_pool.push_back(t.a);
      g_event_pool.push_back(t.b);
    }
  }
  g_timed.swap(keep);
  return kKNumKernels;
}

gs_status gs_timing_release(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  std::vector<TimedLaunch> keep;
  for (const TimedLaunch& t : g_timed) {
    if (t.graph) {
      g_event_pool.push_back(t.a);
      g_event_pool.push_back(t.b);
    } else {
      keep.push_back(t);
    }
  }
  g_timed.swap(keep);
  return GS_OK;
}

const char* gs_kernel_name(int32_t id) {
  if (id < 0 || id >= kKNumKernels) return "";
  return kKernelNames[id];
}

const char* gs_version(void) { return "gs 0.1 sm_103a"; }

}  // extern "C"
