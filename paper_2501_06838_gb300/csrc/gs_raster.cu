// Tile rasterizer of the scale-aware 2D Gaussian splatting render (GSASR,
// arXiv 2501.06838, Eq. 4 with the Algorithm-1 window) and its adjoint.
//
// One CTA renders one TILE x TILE tile of HR pixels. Thread (col, rg) owns the
// BY pixels of column `col`, rows [rg*BY, rg*BY + BY) of the tile. The tile's
// Gaussians (a contiguous run of the sorted pair list) are staged through
// shared memory in batches:
//   stage 1: one thread per Gaussian gathers its 64-byte record and moves its
//            centre into tile-local coordinates (cx - x_tile, small numbers, so
//            X = x - cx keeps full float32 precision even at x ~ 5760);
//   stage 2: per (Gaussian, tile row) the row terms of the exponent
//              e = -(sA X - sK Y)^2 + g Y^2 + l        (log2 units)
//            rowK = sK*Y, rowG = g*Y^2 + l   (rowG = -inf outside the window rows)
//   stage 3: per Gaussian each thread forms Xs = sA*(col - cxl) (+inf outside
//            the window columns) and, per pixel,
//              d = Xs - rowK, e = -d*d + rowG, w = 2^e (MUFU.EX2), out += c*w,
//            i.e. 1 FADD + 1 FFMA + 1 MUFU + 3 FFMA per (Gaussian, pixel) pair.
// The window masks are folded into the exponent: -inf rows and +inf columns
// both give e = -inf and w = +0, so masked pairs cost no branch. The completed
// square has no cancellation for any |rho| < 1 (the Y term is the marginal).
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr float kInf = __builtin_huge_valf();

template <int TILE>
__device__ __forceinline__ void tile_origin(const Ws& w, int t, const ImageDesc*& D, int& ox,
                                            int& oy) {
  const int im = image_of_tile(w.images, w.n_images, t);
  D = &w.images[im];
  const int lt = t - D->t_base;
  const int ty = lt / D->tiles_x;
  const int tx = lt - ty * D->tiles_x;
  ox = tx * TILE;
  oy = ty * TILE;
}

// Stage 1: gather records of the batch into tile-local form.
//   gA = (cxl, sA, lx0, lx1)   gB = (cyl, sK, g, l)   gC = (r, g, b, ly0 | ly1 << 16)
template <int TILE, int NT>
__device__ __forceinline__ void stage_records(const Ws& w, const uint32_t* vals, int bs, int nb,
                                              int ox, int oy, float4* gA, float4* gB, float4* gC,
                                              uint32_t* gid_out) {
  for (int i = threadIdx.x; i < nb; i += NT) {
    const uint32_t gid = __ldg(vals + bs + i);
    const float4* rec = w.records + (int64_t)gid * kRecordF4;
    const float4 f0 = __ldg(rec), f1 = __ldg(rec + 1), f2 = __ldg(rec + 2), f3 = __ldg(rec + 3);
    const float cxl = __fadd_rn(__fsub_rn(f0.x, (float)ox), f0.y);
    const float cyl = __fadd_rn(__fsub_rn(f0.z, (float)oy), f0.w);
    const int lx0 = max(__float_as_int(f3.x) - ox, 0), lx1 = min(__float_as_int(f3.y) - ox, TILE - 1);
    const int ly0 = max(__float_as_int(f3.z) - oy, 0), ly1 = min(__float_as_int(f3.w) - oy, TILE - 1);
    gA[i] = make_float4(cxl, f1.x, (float)lx0, (float)lx1);
    gB[i] = make_float4(cyl, f1.y, f1.z, f1.w);
    gC[i] = make_float4(f2.x, f2.y, f2.z, __int_as_float(ly0 | (ly1 << 16)));
    if (gid_out) gid_out[i] = gid;
  }
}

template <int TILE, int BY>
__global__ void __launch_bounds__(TILE * TILE / BY) k_raster_fwd(Ws w, const uint32_t* vals,
                                                                 int batch) {
  constexpr int NT = TILE * TILE / BY;
  constexpr int NW = (NT + 31) / 32;
  extern __shared__ float4 smem[];
  float4* gA = smem;
  float4* gB = gA + batch;
  float4* gC = gB + batch;
  float2* rows = reinterpret_cast<float2*>(gC + batch);

  const ImageDesc* D;
  int ox, oy;
  tile_origin<TILE>(w, blockIdx.x, D, ox, oy);
  const uint2 range = w.ranges[blockIdx.x];
  const int col = threadIdx.x % TILE;
  const int row0 = (threadIdx.x / TILE) * BY;
  const float fcol = (float)col;
  // rows covered by this warp (used to skip Gaussians that miss them)
  const int wrow0 = ((threadIdx.x & ~31) / TILE) * BY;
  const int wrow1 = min(TILE - 1, (((threadIdx.x | 31) / TILE) + 1) * BY - 1);

  float acc[BY][3];
#pragma unroll
  for (int k = 0; k < BY; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0f;

  for (int bs = (int)range.x; bs < (int)range.y; bs += batch) {
    const int nb = min(batch, (int)range.y - bs);
    stage_records<TILE, NT>(w, vals, bs, nb, ox, oy, gA, gB, gC, nullptr);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * TILE; idx += NT) {
      const int i = idx / TILE, r = idx - i * TILE;
      const float4 b = gB[i];
      const int pk = __float_as_int(gC[i].w);
      const float Y = (float)r - b.x;
      float rowG = fmaf(b.z * Y, Y, b.w);
      if (r < (pk & 0xffff) || r > (pk >> 16)) rowG = -kInf;
      rows[i * TILE + r] = make_float2(b.y * Y, rowG);
    }
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      const float4 c = gC[i];
      if (NW > 1) {
        const int pk = __float_as_int(c.w);
        if ((pk >> 16) < wrow0 || (pk & 0xffff) > wrow1) continue;  // warp-uniform
      }
      const float4 a = gA[i];
      float Xs = a.y * (fcol - a.x);
      if (fcol < a.z || fcol > a.w) Xs = kInf;
      const float4* rr = reinterpret_cast<const float4*>(rows + i * TILE + row0);
#pragma unroll
      for (int k = 0; k < BY; k += 2) {
        const float4 q = rr[k / 2];
        const float d0 = Xs - q.x;
        const float w0 = ex2_approx(fmaf(-d0, d0, q.y));
        const float d1 = Xs - q.z;
        const float w1 = ex2_approx(fmaf(-d1, d1, q.w));
        acc[k][0] = fmaf(c.x, w0, acc[k][0]);
        acc[k][1] = fmaf(c.y, w0, acc[k][1]);
        acc[k][2] = fmaf(c.z, w0, acc[k][2]);
        acc[k + 1][0] = fmaf(c.x, w1, acc[k + 1][0]);
        acc[k + 1][1] = fmaf(c.y, w1, acc[k + 1][1]);
        acc[k + 1][2] = fmaf(c.z, w1, acc[k + 1][2]);
      }
    }
    __syncthreads();
  }

  const int H = D->out_h, W = D->out_w;
  const int x = ox + col;
  if (x < W) {
    float* out = D->out;
    const int64_t plane = (int64_t)H * W;
#pragma unroll
    for (int k = 0; k < BY; ++k) {
      const int y = oy + row0 + k;
      if (y < H) {
        const int64_t o = (int64_t)y * W + x;
        out[o] = acc[k][0];
        out[plane + o] = acc[k][1];
        out[2 * plane + o] = acc[k][2];
      }
    }
  }
}

// Adjoint. Each thread holds dL/dI of its pixels; per staged Gaussian it
// accumulates, over its pixels, Gw = (g . c) 2^e and the moments
//   S0 = sum Gw, SY = sum Gw Y, SYY = sum Gw Y^2, C_k = sum g_k 2^e,
// then (its X is fixed) SX = X S0, SXX = X SX, SXY = X SY. The nine values are
// summed over the warp with shuffles, over warps through shared memory, and
// added to the Gaussian's record-space accumulator with one atomic per
// (tile, Gaussian, value).
template <int TILE, int BY>
__global__ void __launch_bounds__(TILE * TILE / BY) k_raster_bwd(Ws w, const uint32_t* vals,
                                                                 int batch) {
  constexpr int NT = TILE * TILE / BY;
  constexpr int NW = (NT + 31) / 32;
  extern __shared__ float4 smem[];
  float4* gA = smem;
  float4* gB = gA + batch;
  float4* gC = gB + batch;
  float4* rows = gC + batch;                                          // [batch][TILE]
  float* part = reinterpret_cast<float*>(rows + (size_t)batch * TILE);  // [batch][NW][9]
  uint32_t* gids = reinterpret_cast<uint32_t*>(part + (size_t)batch * NW * 9);

  const ImageDesc* D;
  int ox, oy;
  tile_origin<TILE>(w, blockIdx.x, D, ox, oy);
  const uint2 range = w.ranges[blockIdx.x];
  if (range.y <= range.x) return;
  const int col = threadIdx.x % TILE;
  const int row0 = (threadIdx.x / TILE) * BY;
  const float fcol = (float)col;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wrow0 = ((threadIdx.x & ~31) / TILE) * BY;
  const int wrow1 = min(TILE - 1, (((threadIdx.x | 31) / TILE) + 1) * BY - 1);

  float g[BY][3];
  {
    const int H = D->out_h, W = D->out_w;
    const int x = ox + col;
    const int64_t plane = (int64_t)H * W;
#pragma unroll
    for (int k = 0; k < BY; ++k) {
      const int y = oy + row0 + k;
      const bool in = x < W && y < H;
      const int64_t o = (int64_t)y * W + x;
      g[k][0] = in ? __ldg(D->grad_out + o) : 0.0f;
      g[k][1] = in ? __ldg(D->grad_out + plane + o) : 0.0f;
      g[k][2] = in ? __ldg(D->grad_out + 2 * plane + o) : 0.0f;
    }
  }

  for (int bs = (int)range.x; bs < (int)range.y; bs += batch) {
    const int nb = min(batch, (int)range.y - bs);
    stage_records<TILE, NT>(w, vals, bs, nb, ox, oy, gA, gB, gC, gids);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * TILE; idx += NT) {
      const int i = idx / TILE, r = idx - i * TILE;
      const float4 b = gB[i];
      const int pk = __float_as_int(gC[i].w);
      const float Y = (float)r - b.x;
      float rowG = fmaf(b.z * Y, Y, b.w);
      if (r < (pk & 0xffff) || r > (pk >> 16)) rowG = -kInf;
      rows[i * TILE + r] = make_float4(b.y * Y, rowG, Y, 0.0f);
    }
    __syncthreads();
    for (int i = 0; i < nb; ++i) {
      const float4 c = gC[i];
      float* pw = part + ((size_t)i * NW + warp) * 9;
      if (NW > 1) {
        const int pk = __float_as_int(c.w);
        if ((pk >> 16) < wrow0 || (pk & 0xffff) > wrow1) {
          if (lane < 9) pw[lane] = 0.0f;
          continue;
        }
      }
      const float4 a = gA[i];
      const float Xr = fcol - a.x;
      const float Xs = (fcol < a.z || fcol > a.w) ? kInf : a.y * Xr;
      const float4* rr = rows + i * TILE + row0;
      float S0 = 0.f, SY = 0.f, SYY = 0.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
#pragma unroll
      for (int k = 0; k < BY; ++k) {
        const float4 q = rr[k];
        const float dd = Xs - q.x;
        const float wv = ex2_approx(fmaf(-dd, dd, q.y));
        const float G = fmaf(g[k][2], c.z, fmaf(g[k][1], c.y, g[k][0] * c.x));
        const float Gw = G * wv;
        const float GwY = Gw * q.z;
        S0 += Gw;
        SY += GwY;
        SYY = fmaf(GwY, q.z, SYY);
        Cr = fmaf(g[k][0], wv, Cr);
        Cg = fmaf(g[k][1], wv, Cg);
        Cb = fmaf(g[k][2], wv, Cb);
      }
      float v[9];
      v[0] = S0;
      v[1] = Xr * S0;
      v[2] = SY;
      v[3] = Xr * v[1];
      v[4] = Xr * SY;
      v[5] = SYY;
      v[6] = Cr;
      v[7] = Cg;
      v[8] = Cb;
#pragma unroll
      for (int f = 0; f < 9; ++f) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[f] += __shfl_xor_sync(0xffffffffu, v[f], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int f = 0; f < 9; ++f) pw[f] = v[f];
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * 9; idx += NT) {
      const int i = idx / 9, f = idx - i * 9;
      float s = 0.0f;
#pragma unroll
      for (int q = 0; q < NW; ++q) s += part[((size_t)i * NW + q) * 9 + f];
      if (s != 0.0f) atomicAdd(w.grec + (int64_t)gids[i] * 12 + f, s);
    }
    __syncthreads();
  }
}

template <int TILE, int BY>
size_t fwd_smem(int batch) {
  return (size_t)batch * (3 * sizeof(float4) + TILE * sizeof(float2));
}

template <int TILE, int BY>
size_t bwd_smem(int batch) {
  constexpr int NW = (TILE * TILE / BY + 31) / 32;
  return (size_t)batch * (3 * sizeof(float4) + TILE * sizeof(float4) + NW * 9 * sizeof(float) +
                          sizeof(uint32_t));
}

template <class K>
cudaError_t ensure_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int TILE, int BY>
cudaError_t run_fwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  const size_t sm = fwd_smem<TILE, BY>(batch);
  cudaError_t e = ensure_smem(k_raster_fwd<TILE, BY>, sm);
  if (e != cudaSuccess) return e;
  LaunchScope ls(kKRasterFwd, s);
  k_raster_fwd<TILE, BY><<<w.tiles, TILE * TILE / BY, sm, s>>>(w, vals, batch);
  return cudaGetLastError();
}

template <int TILE, int BY>
cudaError_t run_bwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  const size_t sm = bwd_smem<TILE, BY>(batch);
  cudaError_t e = ensure_smem(k_raster_bwd<TILE, BY>, sm);
  if (e != cudaSuccess) return e;
  LaunchScope ls(kKRasterBwd, s);
  k_raster_bwd<TILE, BY><<<w.tiles, TILE * TILE / BY, sm, s>>>(w, vals, batch);
  return cudaGetLastError();
}

}  // namespace

size_t raster_smem_bytes(int tile, int batch, int bwd) {
  switch (tile) {
    case 8: return bwd ? bwd_smem<8, 2>(batch) : fwd_smem<8, 2>(batch);
    case 32: return bwd ? bwd_smem<32, 16>(batch) : fwd_smem<32, 16>(batch);
    default: return bwd ? bwd_smem<16, 8>(batch) : fwd_smem<16, 8>(batch);
  }
}

cudaError_t launch_raster_fwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  if (w.tiles == 0) return cudaSuccess;
  switch (w.tile) {
    case 8: return run_fwd<8, 2>(w, vals, batch, s);
    case 32: return run_fwd<32, 16>(w, vals, batch, s);
    default: return run_fwd<16, 8>(w, vals, batch, s);
  }
}

cudaError_t launch_raster_bwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  if (w.tiles == 0) return cudaSuccess;
  switch (w.tile) {
    case 8: return run_bwd<8, 2>(w, vals, batch, s);
    case 32: return run_bwd<32, 16>(w, vals, batch, s);
    default: return run_bwd<16, 8>(w, vals, batch, s);
  }
}

}  // namespace gs
