// Tile rasterizer of the scale-aware 2D Gaussian splatting render (GSASR,
// arXiv 2501.06838, Eq. 4 with the Algorithm-1 window) and its adjoint.
//
// One CTA of NT = TILE*TILE/BY threads renders one TILE x TILE tile of HR
// pixels; thread t owns column t % TILE and the BY consecutive rows
// [(t / TILE) * BY, + BY). The tile's Gaussians (a contiguous run of the sorted
// pair list) go through shared memory in batches of NT * PF, double buffered:
//   copy:    each thread cp.async-copies the 64-byte records of its Gaussians
//            of the NEXT batch into a raw buffer while the CTA computes this
//            batch (their ids are loaded one batch earlier still);
//   stage 1: one thread per Gaussian moves its centre into tile-local
//            coordinates (cx - x_tile: small numbers, so X = x - cx keeps full
//            float32 precision even at x ~ 5760) and clips its window;
//   stage 2: per (Gaussian, tile row) the row terms of the exponent
//              e = -(sA X - sK Y)^2 + g Y^2 + l        (log2 units)
//            rowK = sK*Y, rowG = g*Y^2 + l  (rowG = -inf outside the window rows);
//   compute: per Gaussian each thread forms Xs = sA*(col - cxl) (+inf outside
//            the window columns) and, per owned pixel,
//              d = Xs - rowK, e = -d*d + rowG, w = 2^e (MUFU.EX2), out += c*w,
//            i.e. 1 FADD + 1 FFMA + 1 MUFU + 3 FFMA per (Gaussian, pixel) pair.
//            The next Gaussian's shared-memory operands are loaded while the
//            current one is computed.
// The window masks are folded into the exponent: -inf rows and +inf columns
// both give e = -inf and w = +0, so masked pairs cost no branch. The completed
// square has no cancellation for any |rho| < 1 (the Y term is the marginal).
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr float kInf = __builtin_huge_valf();

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

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

// Copy the records of batch entries t, t + NT, ... (ids in gid[]) to raw.
template <int NT, int PF>
__device__ __forceinline__ void issue_records(const Ws& w, const uint32_t (&gid)[PF], int nb,
                                              float4* raw) {
#pragma unroll
  for (int j = 0; j < PF; ++j) {
    const int i = j * NT + threadIdx.x;
    if (i < nb) {
      const float4* rec = w.records + (int64_t)gid[j] * kRecordF4;
#pragma unroll
      for (int q = 0; q < kRecordF4; ++q) cp_async16(raw + i * kRecordF4 + q, rec + q);
    }
  }
  cp_async_commit();
}

template <int NT, int PF>
__device__ __forceinline__ void load_ids(const uint32_t* vals, int bs, int nb, uint32_t (&gid)[PF]) {
#pragma unroll
  for (int j = 0; j < PF; ++j) {
    const int i = j * NT + threadIdx.x;
    gid[j] = i < nb ? __ldg(vals + bs + i) : 0u;
  }
}

// Stage 1 from the raw records:
//   gA = (cxl, sA, lx0, lx1)   gB = (cyl, sK, g, l)   gC = (r, g, b, ly0 | ly1 << 16)
template <int TILE, int NT>
__device__ __forceinline__ void stage_records(const float4* raw, int nb, int ox, int oy,
                                              float4* gA, float4* gB, float4* gC) {
  for (int i = threadIdx.x; i < nb; i += NT) {
    const float4 f0 = raw[i * kRecordF4], f1 = raw[i * kRecordF4 + 1];
    const float4 f2 = raw[i * kRecordF4 + 2], f3 = raw[i * kRecordF4 + 3];
    const float cxl = __fadd_rn(__fsub_rn(f0.x, (float)ox), f0.y);
    const float cyl = __fadd_rn(__fsub_rn(f0.z, (float)oy), f0.w);
    const int lx0 = max(__float_as_int(f3.x) - ox, 0), lx1 = min(__float_as_int(f3.y) - ox, TILE - 1);
    const int ly0 = max(__float_as_int(f3.z) - oy, 0), ly1 = min(__float_as_int(f3.w) - oy, TILE - 1);
    gA[i] = make_float4(cxl, f1.x, (float)lx0, (float)lx1);
    gB[i] = make_float4(cyl, f1.y, f1.z, f1.w);
    gC[i] = make_float4(f2.x, f2.y, f2.z, __int_as_float(ly0 | (ly1 << 16)));
  }
}

// Stage 2: row terms (rowK, rowG[, Y]) of every staged Gaussian and tile row.
template <int TILE, int NT, bool WITH_Y>
__device__ __forceinline__ void stage_rows(int nb, const float4* gB, const float4* gC, void* rows) {
  for (int idx = threadIdx.x; idx < nb * TILE; idx += NT) {
    const int i = idx / TILE, r = idx - i * TILE;
    const float4 b = gB[i];
    const int pk = __float_as_int(gC[i].w);
    const float Y = (float)r - b.x;
    float rowG = fmaf(b.z * Y, Y, b.w);
    if (r < (pk & 0xffff) || r > (pk >> 16)) rowG = -kInf;
    if (WITH_Y) {
      reinterpret_cast<float4*>(rows)[idx] = make_float4(b.y * Y, rowG, Y, 0.0f);
    } else {
      reinterpret_cast<float2*>(rows)[idx] = make_float2(b.y * Y, rowG);
    }
  }
}

template <int TILE, int BY, int PF>
__global__ void __launch_bounds__(TILE * TILE / BY) k_raster_fwd(Ws w, const uint32_t* vals) {
  constexpr int NT = TILE * TILE / BY, BATCH = NT * PF, NQ = BY / 2;
  __shared__ __align__(16) float4 raw[2][BATCH * kRecordF4];
  __shared__ float4 gA[BATCH], gB[BATCH], gC[BATCH];
  __shared__ __align__(16) float2 rows[BATCH * TILE];

  const ImageDesc* D;
  int ox, oy;
  tile_origin<TILE>(w, blockIdx.x, D, ox, oy);
  const uint2 range = w.ranges[blockIdx.x];
  const int col = threadIdx.x % TILE;
  const int row0 = (threadIdx.x / TILE) * BY;
  const float fcol = (float)col;

  float acc[BY][3];
#pragma unroll
  for (int k = 0; k < BY; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.0f;

  const int start = (int)range.x, total = (int)range.y - start;
  const int nbat = (total + BATCH - 1) / BATCH;
  uint32_t gid[PF];
  if (nbat > 0) {
    load_ids<NT, PF>(vals, start, min(BATCH, total), gid);
    issue_records<NT, PF>(w, gid, min(BATCH, total), raw[0]);
    if (nbat > 1) load_ids<NT, PF>(vals, start + BATCH, min(BATCH, total - BATCH), gid);
  }
  for (int b = 0; b < nbat; ++b) {
    const int nb = min(BATCH, total - b * BATCH);
    cp_async_wait_all();
    __syncthreads();
    stage_records<TILE, NT>(raw[b & 1], nb, ox, oy, gA, gB, gC);
    __syncthreads();
    stage_rows<TILE, NT, false>(nb, gB, gC, rows);
    __syncthreads();
    if (b + 1 < nbat) {
      issue_records<NT, PF>(w, gid, min(BATCH, total - (b + 1) * BATCH), raw[(b + 1) & 1]);
      if (b + 2 < nbat)
        load_ids<NT, PF>(vals, start + (b + 2) * BATCH, min(BATCH, total - (b + 2) * BATCH), gid);
    }
    // software pipeline: operands of Gaussian i + 1 load while i computes
    float4 a = gA[0], c = gC[0];
    float4 q[NQ];
    {
      const float4* rr = reinterpret_cast<const float4*>(rows + row0);
#pragma unroll
      for (int j = 0; j < NQ; ++j) q[j] = rr[j];
    }
    for (int i = 0; i < nb; ++i) {
      const int inext = min(i + 1, nb - 1);
      const float4 an = gA[inext], cn = gC[inext];
      float4 qn[NQ];
      const float4* rr = reinterpret_cast<const float4*>(rows + inext * TILE + row0);
#pragma unroll
      for (int j = 0; j < NQ; ++j) qn[j] = rr[j];
      float Xs = a.y * (fcol - a.x);
      if (fcol < a.z || fcol > a.w) Xs = kInf;
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        const float d0 = Xs - q[j].x;
        const float w0 = ex2_approx(fmaf(-d0, d0, q[j].y));
        const float d1 = Xs - q[j].z;
        const float w1 = ex2_approx(fmaf(-d1, d1, q[j].w));
        acc[2 * j][0] = fmaf(c.x, w0, acc[2 * j][0]);
        acc[2 * j][1] = fmaf(c.y, w0, acc[2 * j][1]);
        acc[2 * j][2] = fmaf(c.z, w0, acc[2 * j][2]);
        acc[2 * j + 1][0] = fmaf(c.x, w1, acc[2 * j + 1][0]);
        acc[2 * j + 1][1] = fmaf(c.y, w1, acc[2 * j + 1][1]);
        acc[2 * j + 1][2] = fmaf(c.z, w1, acc[2 * j + 1][2]);
      }
      a = an;
      c = cn;
#pragma unroll
      for (int j = 0; j < NQ; ++j) q[j] = qn[j];
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
// then (its X is fixed) SX = X S0, SXX = X SX, SXY = X SY.
// Reduction over each warp's 32 lanes, batched over kRB Gaussians: lanes store
// their nine values transposed in shared memory (row (g, f) holds the 32 lane
// values, padded to 33 floats so that no two lanes read one bank), then lane j
// sums rows j, j + 32, ... and adds each total to the Gaussian's record-space
// accumulator: one atomic per (tile, Gaussian, value) and warp.
constexpr int kRB = 8;            // Gaussians per reduction round
constexpr int kRedRow = 33;       // padded row of 32 lane values

template <int TILE, int BY, int PF>
__global__ void __launch_bounds__(TILE * TILE / BY) k_raster_bwd(Ws w, const uint32_t* vals) {
  constexpr int NT = TILE * TILE / BY, NW = NT / 32, BATCH = NT * PF;
  __shared__ __align__(16) float4 raw[2][BATCH * kRecordF4];
  __shared__ float4 gA[BATCH], gB[BATCH], gC[BATCH];
  __shared__ __align__(16) float4 rows[BATCH * TILE];
  __shared__ float red[NW][kRB * 9 * kRedRow];
  __shared__ uint32_t gids[2][BATCH];

  const ImageDesc* D;
  int ox, oy;
  tile_origin<TILE>(w, blockIdx.x, D, ox, oy);
  const uint2 range = w.ranges[blockIdx.x];
  if (range.y <= range.x) return;
  const int col = threadIdx.x % TILE;
  const int row0 = (threadIdx.x / TILE) * BY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float fcol = (float)col;
  float* wred = red[warp];
  // rows covered by this warp, for skipping Gaussians that miss them (NW > 1)
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

  const int start = (int)range.x, total = (int)range.y - start;
  const int nbat = (total + BATCH - 1) / BATCH;
  uint32_t gid[PF];
  load_ids<NT, PF>(vals, start, min(BATCH, total), gid);
#pragma unroll
  for (int j = 0; j < PF; ++j) gids[0][j * NT + threadIdx.x] = gid[j];
  issue_records<NT, PF>(w, gid, min(BATCH, total), raw[0]);
  if (nbat > 1) load_ids<NT, PF>(vals, start + BATCH, min(BATCH, total - BATCH), gid);

  for (int b = 0; b < nbat; ++b) {
    const int nb = min(BATCH, total - b * BATCH);
    cp_async_wait_all();
    __syncthreads();
    stage_records<TILE, NT>(raw[b & 1], nb, ox, oy, gA, gB, gC);
    __syncthreads();
    stage_rows<TILE, NT, true>(nb, gB, gC, rows);
    __syncthreads();
    if (b + 1 < nbat) {
#pragma unroll
      for (int j = 0; j < PF; ++j) gids[(b + 1) & 1][j * NT + threadIdx.x] = gid[j];
      issue_records<NT, PF>(w, gid, min(BATCH, total - (b + 1) * BATCH), raw[(b + 1) & 1]);
      if (b + 2 < nbat)
        load_ids<NT, PF>(vals, start + (b + 2) * BATCH, min(BATCH, total - (b + 2) * BATCH), gid);
    }
    const uint32_t* bgid = gids[b & 1];
    for (int i = 0; i < nb; ++i) {
      const float4 c = gC[i];
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const int pk = __float_as_int(c.w);
      if (NW == 1 || ((pk >> 16) >= wrow0 && (pk & 0xffff) <= wrow1)) {   // warp-uniform
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
        v[0] = S0;
        v[1] = Xr * S0;
        v[2] = SY;
        v[3] = Xr * v[1];
        v[4] = Xr * SY;
        v[5] = SYY;
        v[6] = Cr;
        v[7] = Cg;
        v[8] = Cb;
      }
      const int slot = i % kRB;
#pragma unroll
      for (int f = 0; f < 9; ++f) wred[(slot * 9 + f) * kRedRow + lane] = v[f];
      if (slot == kRB - 1 || i == nb - 1) {   // block-uniform
        __syncwarp();
        const int rows_used = (slot + 1) * 9;
        for (int rix = lane; rix < rows_used; rix += 32) {
          const float* src = wred + rix * kRedRow;
          float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
          for (int l = 0; l < 32; l += 4) {
            s0 += src[l];
            s1 += src[l + 1];
            s2 += src[l + 2];
            s3 += src[l + 3];
          }
          const float s = (s0 + s1) + (s2 + s3);
          const int gi = i - slot + rix / 9;
          if (s != 0.0f) atomicAdd(w.grec + (int64_t)bgid[gi] * 12 + (rix % 9), s);
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

template <int TILE, int BY, int PF>
cudaError_t run(const Ws& w, const uint32_t* vals, bool bwd, cudaStream_t s) {
  constexpr int NT = TILE * TILE / BY;
  if (bwd) {
    LaunchScope ls(kKRasterBwd, s);
    k_raster_bwd<TILE, BY, PF><<<w.tiles, NT, 0, s>>>(w, vals);
  } else {
    LaunchScope ls(kKRasterFwd, s);
    k_raster_fwd<TILE, BY, PF><<<w.tiles, NT, 0, s>>>(w, vals);
  }
  return cudaGetLastError();
}

// Launch configurations: tile edge -> rows per thread (threads = TILE^2 / BY);
// batch = Gaussians staged per round = threads * PF, PF in {1, 2}.
cudaError_t dispatch(const Ws& w, const uint32_t* vals, int batch, bool bwd, cudaStream_t s) {
  if (w.tiles == 0) return cudaSuccess;
  switch (w.tile) {
    case 8:   // 32 threads
      return batch >= 64 ? run<8, 2, 2>(w, vals, bwd, s) : run<8, 2, 1>(w, vals, bwd, s);
    case 32:  // 64 threads
      return batch >= 128 ? run<32, 16, 2>(w, vals, bwd, s) : run<32, 16, 1>(w, vals, bwd, s);
    default:  // 32 threads
      return batch >= 64 ? run<16, 8, 2>(w, vals, bwd, s) : run<16, 8, 1>(w, vals, bwd, s);
  }
}

}  // namespace

cudaError_t launch_raster_fwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  return dispatch(w, vals, batch, false, s);
}

cudaError_t launch_raster_bwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  return dispatch(w, vals, batch, true, s);
}

}  // namespace gs
