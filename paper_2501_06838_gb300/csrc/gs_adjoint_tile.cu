// Tile adjoint of the scale-aware 2D Gaussian render (GSASR, arXiv 2501.06838,
// Eq. 4 with the Algorithm-1 window; differentiable render, Sec. 3.1 "Fast
// Rasterization" and Sec. 3.2 "Rendering"), one lane per Gaussian.
//
// The exponent of a record is the completed square (log2 units, HR pixels)
//   e = -d^2 + g Y^2 + l,   d = sA X - sK Y,   X = x - cx, Y = y - cy,
// and the render adds c_k 2^e to channel k (c the record colour alpha * rgb).
// For every (tile, Gaussian) pair of the forward's per-tile lists this kernel
// adds the Gaussian's record-space moments over the tile's pixels,
//   Sd = sum Gw d, SY = sum Gw Y, Sdd = sum Gw d^2, SdY = sum Gw d Y,
//   SYY = sum Gw Y^2, C_k = sum g_k 2^e,   Gw = (sum_k g_k c_k) 2^e,
// (g = dL/dI) to the Gaussian's accumulator with one atomic per value. The
// moments are taken in the exponent's own coordinates (d, Y), not in (X, Y):
// for |rho| -> 1 the X moments enter the chain rule with coefficients of
// order 1/(1 - rho^2)^2 that cancel to order 1/(1 - rho^2), which float32
// moments cannot resolve; in (d, Y) no such cancellation occurs.
//
// Layout: one warp per tile, walking the tile's list in chunks of 32 entries;
// lane l owns the chunk's l-th Gaussian. The warp first stages the tile's
// upstream gradient in shared memory, two columns per entry:
//   sgA[r][j] = (g_r(2j), g_r(2j + 1), g_g(2j), g_g(2j + 1)),  sgB[r][j] = (g_b(2j), g_b(2j + 1)).
// All lanes then walk the tile's pixels in the same order (row by row, two
// columns at a time), so every shared-memory read is a broadcast, and each
// lane evaluates its own Gaussian there in packed FP32x2 arithmetic:
//   d = Xs - sK Y (one fused step), e = R - d^2, w = 2^e   (Xs = sA X per
//   column, R = g Y^2 + l per row),
//   G = g . c, C_k += g_k w, Gw = G w, per row A0 += Gw, A1 += Gw d, A2 += Gw d^2,
// and after each row folds (A0, A1, A2) into the moments with that row's Y:
//   SY += Y A0, SYY += Y^2 A0, Sd += A1, SdY += Y A1, Sdd += A2.
// Per pixel that is 13 FP32 lane-operations (two pixels per packed
// instruction) and one MUFU.EX2; no cross-lane reduction. Window masks are in
// the operands (Xs = 1e18 outside the window's columns, so that d stays finite
// and every product with w = +0 is 0; R = -inf outside its rows); rows that no
// lane's window reaches are skipped.
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr float kInfG = __builtin_huge_valf();
constexpr float kFarG = 1e18f;   // masked column: d^2 = 1e36 (finite), e = -1e36, w = +0

__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }

// Stages the upstream gradient of the E x E pixel block at image column ox,
// image row oy (0 outside the output) into sgA/sgB, E * E / 2 entries each.
template <int E>
__device__ __forceinline__ void stage_grad(const Ws& w, const ImageDesc* D, int ox, int oy,
                                           float4* sgA, float2* sgB) {
  constexpr int CP = E / 2;
  const int H = D->out_h, W = D->out_w;
  const int64_t plane = (int64_t)H * W;
  const float* go = w.direct ? w.grad_out0 : D->grad_out;
  float* fa = reinterpret_cast<float*>(sgA);
  float* fb = reinterpret_cast<float*>(sgB);
  for (int idx = threadIdx.x; idx < E * E; idx += 32) {
    const int r = idx / E, x = idx - r * E;
    const int gx = ox + x, gy = oy - D->row0 + r;
    const bool in = gx < W && gy < H;
    const int64_t o = in ? (int64_t)gy * W + gx : 0;   // always a valid address
    const float vr = __ldg(go + o), vg = __ldg(go + plane + o), vb = __ldg(go + 2 * plane + o);
    const int e = r * CP + (x >> 1), hb = x & 1;
    fa[4 * e + hb] = in ? vr : 0.0f;
    fa[4 * e + 2 + hb] = in ? vg : 0.0f;
    fb[2 * e + hb] = in ? vb : 0.0f;
  }
  __syncwarp();
}

// One chunk of the E x E block at (ox, oy): lane l adds Gaussian gid's
// moments over the block (valid false: an empty lane). A Gaussian whose
// window misses the block adds nothing.
template <int E>
__device__ __forceinline__ void bwd_chunk(const Ws& w, uint32_t gid, bool valid, int ox, int oy,
                                          const float4* sgA, const float2* sgB) {
  constexpr int CP = E / 2;                 // column pairs per block row
  constexpr int SEG = E < 16 ? E : 16;      // columns per register table
  constexpr int SP = SEG / 2;               // column pairs per table
  float4 f[kRecordF4];
  if (valid) {
    const float4* rec = w.records + (int64_t)gid * kRecordF4;
#pragma unroll
    for (int q = 0; q < kRecordF4; ++q) f[q] = rec[q];
  }
  // the Gaussian's record in tile-local coordinates
  float cxl = 0.f, cyl = 0.f, sA = 0.f, sK = 0.f, gy2 = 0.f, l = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
  int lx0 = 1, lx1 = 0, ly0 = E, ly1 = -1;
  if (valid) {
    cxl = __fadd_rn(__fsub_rn(f[0].x, (float)ox), f[0].y);
    cyl = __fadd_rn(__fsub_rn(f[0].z, (float)oy), f[0].w);
    sA = f[1].x; sK = f[1].y; gy2 = f[1].z; l = f[1].w;
    cr = f[2].x; cg = f[2].y; cb = f[2].z;
    lx0 = max(__float_as_int(f[3].x) - ox, 0);
    lx1 = min(__float_as_int(f[3].y) - ox, E - 1);
    ly0 = max(__float_as_int(f[3].z) - oy, 0);
    ly1 = min(__float_as_int(f[3].w) - oy, E - 1);
    if (lx0 > lx1 || ly0 > ly1) { ly0 = E; ly1 = -1; }
  }
  // rows some lane's window reaches
  const int rlo = __reduce_min_sync(0xffffffffu, ly0);
  const int rhi = __reduce_max_sync(0xffffffffu, ly1);

  const float2 cr2 = p2(cr, cr), cg2 = p2(cg, cg), cb2 = p2(cb, cb), nsK2 = p2(-sK, -sK);
  float2 Cr = p2(0.f, 0.f), Cg = Cr, Cb = Cr;
  float Sd = 0.f, SY = 0.f, Sdd = 0.f, SdY = 0.f, SYY = 0.f;
#pragma unroll
  for (int seg = 0; seg < E / SEG; ++seg) {
    // per column pair: Xs = sA X (kFarG outside the window)
    float2 Xs2[SP];
#pragma unroll
    for (int j = 0; j < SP; ++j) {
      const int c0 = seg * SEG + 2 * j, c1 = c0 + 1;
      const float a = __fsub_rn((float)c0, cxl), b = __fsub_rn((float)c1, cxl);
      Xs2[j] = p2((c0 >= lx0 && c0 <= lx1) ? sA * a : kFarG,
                  (c1 >= lx0 && c1 <= lx1) ? sA * b : kFarG);
    }
    for (int r = rlo; r <= rhi; ++r) {
      const float Y = __fsub_rn((float)r, cyl);
      const float R = (r >= ly0 && r <= ly1) ? fmaf(gy2 * Y, Y, l) : -kInfG;
      const float2 Y2 = p2(Y, Y), R2 = p2(R, R);
      const float4* ga = sgA + r * CP + seg * SP;
      const float2* gb = sgB + r * CP + seg * SP;
      float2 A0, A1, A2;
#pragma unroll
      for (int j = 0; j < SP; ++j) {
        const float4 q = ga[j];
        const float2 gbj = gb[j];
        const float2 gr2 = p2(q.x, q.y), gg2 = p2(q.z, q.w);
        const float2 d = __ffma2_rn(nsK2, Y2, Xs2[j]);   // one rounding: d cancels for |rho| -> 1
        const float2 e = __ffma2_rn(p2(-d.x, -d.y), d, R2);
        const float2 wv = p2(ex2_approx(e.x), ex2_approx(e.y));
        const float2 G = __ffma2_rn(gbj, cb2, __ffma2_rn(gg2, cg2, __fmul2_rn(gr2, cr2)));
        Cr = __ffma2_rn(gr2, wv, Cr);
        Cg = __ffma2_rn(gg2, wv, Cg);
        Cb = __ffma2_rn(gbj, wv, Cb);
        const float2 Gw = __fmul2_rn(G, wv);
        const float2 Gwd = __fmul2_rn(Gw, d);
        if (j == 0) {
          A0 = Gw;
          A1 = Gwd;
          A2 = __fmul2_rn(Gwd, d);
        } else {
          A0 = __fadd2_rn(A0, Gw);
          A1 = __fadd2_rn(A1, Gwd);
          A2 = __ffma2_rn(Gwd, d, A2);
        }
      }
      const float a0 = A0.x + A0.y, a1 = A1.x + A1.y, a2 = A2.x + A2.y;
      const float ty = Y * a0;
      SY += ty;
      SYY = fmaf(ty, Y, SYY);
      Sd += a1;
      SdY = fmaf(Y, a1, SdY);
      Sdd += a2;
    }
  }
  if (valid) {
    const float v[8] = {Sd, SY, Sdd, SdY, SYY, Cr.x + Cr.y, Cg.x + Cg.y, Cb.x + Cb.y};
    float* acc = w.grec + (int64_t)gid * 12;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (v[k] != 0.0f) atomicAdd(acc + k, v[k]);
  }
}

// The adjoint of tile t by one warp, over the tile's whole list.
template <int TILE>
__device__ __forceinline__ void bwd_one_tile(const Ws& w, const uint32_t* vals, int t, float4* sgA,
                                             float2* sgB) {
  const uint2 range = w.ranges[t];
  const int n = (int)range.y - (int)range.x;
  if (n <= 0) return;   // no Gaussian meets this tile (uniform)
  const int lane = threadIdx.x;
  // tile origin (image rows: a band's output holds rows row0 ..)
  const int im = image_of_tile(w.images, w.n_images, t);
  const ImageDesc* D = &w.images[im];
  const int lt = t - D->t_base;
  const int tyi = lt / D->tiles_x;
  const int ox = (lt - tyi * D->tiles_x) * TILE;
  const int oy = tyi * TILE + D->row0;
  stage_grad<TILE>(w, D, ox, oy, sgA, sgB);
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint32_t gid = i < n ? __ldg(vals + range.x + i) : 0xffffffffu;
    bwd_chunk<TILE>(w, gid, gid < (uint32_t)w.n, ox, oy, sgA, sgB);   // the list holds Gaussian ids
  }
}

// The adjoint of quadrant q (0..3, row-major) of 16 x 16 tile t by one warp:
// the tile's list is filtered to the Gaussians whose window meets the 8 x 8
// quadrant (a ballot per 32 entries into a shared queue of at most 63 ids),
// and the quadrant is evaluated in chunks of 32 of those. Every pixel pair the
// tile-16 walk would evaluate for a Gaussian that misses the quadrant is
// skipped, at the cost of reading the tile's list and windows four times.
__device__ __forceinline__ void bwd_one_quadrant(const Ws& w, const uint32_t* vals, int t, int q,
                                                 float4* sgA, float2* sgB, uint32_t* qids) {
  const uint2 range = w.ranges[t];
  const int n = (int)range.y - (int)range.x;
  if (n <= 0) return;   // no Gaussian meets this tile (uniform)
  const int lane = threadIdx.x;
  const int im = image_of_tile(w.images, w.n_images, t);
  const ImageDesc* D = &w.images[im];
  const int lt = t - D->t_base;
  const int tyi = lt / D->tiles_x;
  const int ox = (lt - tyi * D->tiles_x) * 16 + (q & 1) * 8;
  const int oy = tyi * 16 + D->row0 + (q >> 1) * 8;
  if (ox >= D->out_w || oy - D->row0 >= D->out_h) return;   // quadrant past the output (uniform)
  stage_grad<8>(w, D, ox, oy, sgA, sgB);
  const int4* win = reinterpret_cast<const int4*>(w.records);   // f3 of each record
  int head = 0, pos = 0;
  // list entries pos .. pos + 31, loaded one top-up ahead of their window test
  uint32_t nid = lane < n ? __ldg(vals + range.x + lane) : 0xffffffffu;
  while (true) {
    // top up the queue to at least 32 ids (or the end of the list)
    while (head < 32 && pos < n) {
      const uint32_t gid = nid;
      pos += 32;
      nid = pos + lane < n ? __ldg(vals + range.x + pos + lane) : 0xffffffffu;
      bool meets = false;
      if (gid < (uint32_t)w.n) {
        const int4 b = __ldg(win + (int64_t)gid * kRecordF4 + 3);   // x0, x1, y0, y1 (image)
        meets = b.x <= ox + 7 && b.y >= ox && b.z <= oy + 7 && b.w >= oy;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, meets);
      if (meets) qids[head + __popc(m & ((1u << lane) - 1u))] = gid;
      head += __popc(m);
    }
    __syncwarp();
    if (head == 0) break;   // uniform: the list is exhausted
    const uint32_t gid = lane < head ? qids[lane] : 0xffffffffu;
    const uint32_t carry = lane + 32 < head ? qids[lane + 32] : 0u;
    __syncwarp();
    if (lane + 32 < head) qids[lane] = carry;   // the ids past this chunk move to the front
    head = head > 32 ? head - 32 : 0;
    __syncwarp();
    bwd_chunk<8>(w, gid, gid < (uint32_t)w.n, ox, oy, sgA, sgB);
  }
}

// Persistent: at most as many one-warp CTAs as are resident at once. CTA b
// takes tile b first; when there are more tiles than CTAs, each then takes
// the next tile from the workspace counter (reset by the forward's setup and
// by the chain rule after each adjoint) until the tiles run out, so that no
// partial last wave idles SMs. The counter is asked only after a tile is done,
// which spreads the (same-address) atomics over the launch. Registers capped
// at 64 for 32 resident CTAs per SM (no spills at tile 8, 16 or 32).
template <int TILE>
__global__ void __launch_bounds__(32, 32) k_raster_bwd_tile(Ws w, const uint32_t* vals) {
  griddep_release();
  griddep_wait();
  __shared__ float4 sgA[TILE * TILE / 2];
  __shared__ float2 sgB[TILE * TILE / 2];
  const uint32_t tiles = (uint32_t)w.tiles;
  const bool more = gridDim.x < tiles;   // uniform over the grid
  uint32_t cur = blockIdx.x;
  while (cur < tiles) {
    bwd_one_tile<TILE>(w, vals, (int)cur, sgA, sgB);
    if (!more) break;
    uint32_t nx = 0;
    if (threadIdx.x == 0) nx = gridDim.x + atomicAdd(&w.hdr->bwd_counter, 1u);
    cur = __shfl_sync(0xffffffffu, nx, 0);
    __syncwarp();   // every lane is done with the staged gradient before the next tile's
  }
}

// The same over the 8 x 8 quadrants of 16 x 16 tiles: unit u is quadrant
// u % 4 of tile u / 4, so the four quadrants of a tile run side by side.
__global__ void __launch_bounds__(32) k_raster_bwd_quad(Ws w, const uint32_t* vals) {
  griddep_release();
  griddep_wait();
  __shared__ float4 sgA[32];
  __shared__ float2 sgB[32];
  __shared__ uint32_t qids[64];
  const uint32_t units = 4u * (uint32_t)w.tiles;
  const bool more = gridDim.x < units;   // uniform over the grid
  uint32_t cur = blockIdx.x;
  while (cur < units) {
    bwd_one_quadrant(w, vals, (int)(cur >> 2), (int)(cur & 3u), sgA, sgB, qids);
    if (!more) break;
    uint32_t nx = 0;
    if (threadIdx.x == 0) nx = gridDim.x + atomicAdd(&w.hdr->bwd_counter, 1u);
    cur = __shfl_sync(0xffffffffu, nx, 0);
    __syncwarp();   // every lane is done with the staged gradient and the queue
  }
}

}  // namespace

cudaError_t launch_raster_bwd_tile(const Ws& w, const uint32_t* lists, bool quadrants,
                                   cudaStream_t s) {
  if (w.tiles == 0) return cudaSuccess;
  LaunchScope ls(kKRasterBwd, s);
  const dim3 block(32);
  if (quadrants) {   // tile 16 (the caller checks)
    const dim3 grid(resident_grid((const void*)k_raster_bwd_quad, 32, 4 * (int64_t)w.tiles));
    return launch_chain(k_raster_bwd_quad, grid, block, 0, s, w, lists);
  }
  switch (w.tile) {
    case 8: {
      const dim3 grid(resident_grid((const void*)k_raster_bwd_tile<8>, 32, w.tiles));
      return launch_chain(k_raster_bwd_tile<8>, grid, block, 0, s, w, lists);
    }
    case 32: {
      const dim3 grid(resident_grid((const void*)k_raster_bwd_tile<32>, 32, w.tiles));
      return launch_chain(k_raster_bwd_tile<32>, grid, block, 0, s, w, lists);
    }
    default: {
      const dim3 grid(resident_grid((const void*)k_raster_bwd_tile<16>, 32, w.tiles));
      return launch_chain(k_raster_bwd_tile<16>, grid, block, 0, s, w, lists);
    }
  }
}

}  // namespace gs
