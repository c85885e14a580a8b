// Gaussian-warp adjoint of the scale-aware rasterizer (GSASR, arXiv 2501.06838,
// Eq. 4 with the Algorithm-1 window): one warp per Gaussian walks the pixels of
// its own window R_i, so every moment is summed by one warp in a fixed order
// and written once, with no atomics (deterministic bit for bit).
//
// Per Gaussian the warp needs, over its window, with G = sum_k g_k c_k,
// w = 2^e and the record's exponent e = -d^2 + g Y^2 + l in the completed
// square's coordinates d = sA X - sK Y, Y = y - cy (HR px):
//   Sd = sum G w d, SY = sum G w Y, Sdd = sum G w d^2, SdY = sum G w d Y,
//   SYY = sum G w Y^2, C_k = sum g_k w,
// the same eight moments the tile adjoint leaves (k_preprocess_bwd turns them
// into parameter gradients).
//
// Layout of the walk:
//   - the window's rows go through a per-warp row table in shared memory,
//     (Y, Y, R, R) with R = g Y^2 + l the row part of the exponent, filled 64
//     rows at a time;
//   - each lane owns a pair of adjacent columns (x, x + 1): the grad_out loads
//     are float2 (8-byte aligned when the row width is even) and all FP32 work
//     is packed two-wide (FFMA2 etc.), one instruction for both columns;
//   - columns go in chunks of up to 32 pairs; a narrow chunk (< 17 pairs)
//     gives the spare lanes further rows, so a warp covers 32/cw rows of cw
//     column pairs per step and few lanes idle.
// Masked columns (outside [x0, x1], or lanes past the chunk) take sA X = 1e18,
// so d stays finite, e = -1e36 and w = +0 with no branch.
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr int kGwWarps = 8;    // Gaussians (warps) per CTA
constexpr int kGwRows = 64;    // rows per row-table block
constexpr float kFarGw = 1e18f;   // masked column: w = +0, every moment product 0

__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }

// Sum of v[0..7] over the warp's 32 lanes by recursive halving: afterwards
// lane l holds the total of value (l >> 2) & 7. Fixed order: deterministic.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float u[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b4 ? v[i] : v[i + 4];
    const float keep = b4 ? v[i + 4] : v[i];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float t[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b3 ? u[i] : u[i + 2];
    const float keep = b3 ? u[i + 2] : u[i];
    t[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? t[0] : t[1];
  float s = (b2 ? t[1] : t[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  return s;
}

struct GwAcc {
  float2 C[3], SY, SYY, Sd, Sdd, SdY;
};

// One step: the lane's column pair on table row `q` (Y, Y, R, R), loads at
// element offset `off` (second column at `off2` when the row is not 8-byte
// aligned).
template <bool ALIGNED>
__device__ __forceinline__ void gw_pixel_pair(GwAcc& a, const float* __restrict__ g0,
                                              const float* __restrict__ g1,
                                              const float* __restrict__ g2, int64_t off,
                                              int64_t off2, const float4 q, float2 Xs, float2 nsK,
                                              float2 cr, float2 cg, float2 cb) {
  float2 gr, gg, gb;
  if (ALIGNED) {
    gr = __ldg(reinterpret_cast<const float2*>(g0 + off));
    gg = __ldg(reinterpret_cast<const float2*>(g1 + off));
    gb = __ldg(reinterpret_cast<const float2*>(g2 + off));
  } else {
    gr = p2(__ldg(g0 + off), __ldg(g0 + off2));
    gg = p2(__ldg(g1 + off), __ldg(g1 + off2));
    gb = p2(__ldg(g2 + off), __ldg(g2 + off2));
  }
  const float2 Y = p2(q.x, q.y);
  const float2 d = __ffma2_rn(nsK, Y, Xs);                       // sA X - sK Y
  const float2 e = __ffma2_rn(p2(-d.x, -d.y), d, p2(q.z, q.w));  // R - d^2
  const float2 wv = p2(ex2_approx(e.x), ex2_approx(e.y));
  const float2 G = __ffma2_rn(gb, cb, __ffma2_rn(gg, cg, __fmul2_rn(gr, cr)));
  const float2 Gw = __fmul2_rn(G, wv);
  const float2 GwY = __fmul2_rn(Gw, Y);
  const float2 Gwd = __fmul2_rn(Gw, d);
  a.SY = __fadd2_rn(a.SY, GwY);
  a.SYY = __ffma2_rn(GwY, Y, a.SYY);
  a.Sd = __fadd2_rn(a.Sd, Gwd);
  a.Sdd = __ffma2_rn(Gwd, d, a.Sdd);
  a.SdY = __ffma2_rn(Gwd, Y, a.SdY);
  a.C[0] = __ffma2_rn(gr, wv, a.C[0]);
  a.C[1] = __ffma2_rn(gg, wv, a.C[1]);
  a.C[2] = __ffma2_rn(gb, wv, a.C[2]);
}

template <bool ALIGNED>
__device__ __forceinline__ void gw_walk(const float* __restrict__ go, int64_t plane, int W, int x0,
                                        int x1, int y0, int y1, const float4 f0, const float4 f1,
                                        const float4 f2, float4* rt, int lane, float (&v)[8]) {
  const float cxh = f0.x, cxl = f0.y, cyh = f0.z, cyl = f0.w;
  const float sA = f1.x, gq = f1.z, l = f1.w;
  const float2 nsK = p2(-f1.y, -f1.y);
  const float2 cr = p2(f2.x, f2.x), cg = p2(f2.y, f2.y), cb = p2(f2.z, f2.z);
  const float* g0 = go;
  const float* g1 = go + plane;
  const float* g2 = go + 2 * plane;
  const int xs = x0 & ~1;
  const int np = ((x1 - xs) >> 1) + 1;   // column pairs covering [xs, x1]
  float2 tSd = p2(0.f, 0.f), tSdd = tSd, tSdY = tSd, tSY = tSd, tSYY = tSd;
  float2 tC0 = tSd, tC1 = tSd, tC2 = tSd;

  for (int rb = y0; rb <= y1; rb += kGwRows) {
    const int nr = min(kGwRows, y1 - rb + 1);
    __syncwarp();
    for (int t = lane; t < nr; t += 32) {
      const float Y = __fsub_rn(__fsub_rn((float)(rb + t), cyh), cyl);
      const float R = fmaf(gq * Y, Y, l);
      rt[t] = make_float4(Y, Y, R, R);
    }
    __syncwarp();
    for (int c0 = 0; c0 < np; c0 += 32) {
      const int cp = min(32, np - c0);
      const int lcw = cp > 16 ? 5 : cp > 8 ? 4 : cp > 4 ? 3 : cp > 2 ? 2 : cp > 1 ? 1 : 0;
      const int rpi = 32 >> lcw;
      const int lc = lane & ((1 << lcw) - 1), lr = lane >> lcw;
      const bool live = lc < cp;
      const int xp = xs + 2 * (c0 + (live ? lc : 0));
      const float2 X = p2(__fsub_rn(__fsub_rn((float)xp, cxh), cxl),
                          __fsub_rn(__fsub_rn((float)(xp + 1), cxh), cxl));
      float2 Xs = p2(sA * X.x, sA * X.y);
      if (!live || xp < x0) Xs.x = kFarGw;
      if (!live || xp + 1 > x1) Xs.y = kFarGw;
      const int xq = min(xp + 1, W - 1);
      GwAcc a;
      a.C[0] = a.C[1] = a.C[2] = a.SY = a.SYY = a.Sd = a.Sdd = a.SdY = p2(0.f, 0.f);
      int r = lr;
      for (; r + rpi < nr; r += 2 * rpi) {
        const int64_t ya = (int64_t)(rb + r) * W, yb = ya + (int64_t)rpi * W;
        const float4 qa = rt[r], qb = rt[r + rpi];
        gw_pixel_pair<ALIGNED>(a, g0, g1, g2, ya + xp, ya + xq, qa, Xs, nsK, cr, cg, cb);
        gw_pixel_pair<ALIGNED>(a, g0, g1, g2, yb + xp, yb + xq, qb, Xs, nsK, cr, cg, cb);
      }
      if (r < nr) {
        const int64_t ya = (int64_t)(rb + r) * W;
        gw_pixel_pair<ALIGNED>(a, g0, g1, g2, ya + xp, ya + xq, rt[r], Xs, nsK, cr, cg, cb);
      }
      tSd = __fadd2_rn(tSd, a.Sd);
      tSdd = __fadd2_rn(tSdd, a.Sdd);
      tSdY = __fadd2_rn(tSdY, a.SdY);
      tSY = __fadd2_rn(tSY, a.SY);
      tSYY = __fadd2_rn(tSYY, a.SYY);
      tC0 = __fadd2_rn(tC0, a.C[0]);
      tC1 = __fadd2_rn(tC1, a.C[1]);
      tC2 = __fadd2_rn(tC2, a.C[2]);
    }
  }
  v[0] = tSd.x + tSd.y;
  v[1] = tSY.x + tSY.y;
  v[2] = tSdd.x + tSdd.y;
  v[3] = tSdY.x + tSdY.y;
  v[4] = tSYY.x + tSYY.y;
  v[5] = tC0.x + tC0.y;
  v[6] = tC1.x + tC1.y;
  v[7] = tC2.x + tC2.y;
}

__global__ void __launch_bounds__(kGwWarps * 32) k_raster_bwd_gw(Ws w) {
  griddep_release();
  griddep_wait();
  __shared__ float4 rt[kGwWarps][kGwRows];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t gi = (int64_t)blockIdx.x * kGwWarps + wp;
  if (gi >= w.n) return;   // whole warp; no block-wide barrier follows
  const float4* rec = w.records + gi * kRecordF4;
  const float4 f3 = rec[3];
  const int x0 = __float_as_int(f3.x), x1 = __float_as_int(f3.y);
  const int y0 = __float_as_int(f3.z), y1 = __float_as_int(f3.w);
  float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (x0 <= x1 && y0 <= y1) {   // warp-uniform
    const ImageDesc& D = w.images[image_of_gaussian(w.images, w.n_images, gi)];
    const int W = D.out_w;
    const int64_t plane = (int64_t)D.out_h * W;
    // rows are image rows; the upstream gradient holds rows row0 .. row0 + out_h - 1
    const float* go = (w.direct ? w.grad_out0 : D.grad_out) - (int64_t)D.row0 * W;
    const bool aligned = (W & 1) == 0 && (reinterpret_cast<uintptr_t>(go) & 7) == 0;
    if (aligned)
      gw_walk<true>(go, plane, W, x0, x1, y0, y1, rec[0], rec[1], rec[2], rt[wp], lane, v);
    else
      gw_walk<false>(go, plane, W, x0, x1, y0, y1, rec[0], rec[1], rec[2], rt[wp], lane, v);
  }
  const float s = warp_sum8(v, lane);
  if ((lane & 3) == 0) w.grec[gi * 12 + (lane >> 2)] = s;
}

}  // namespace

cudaError_t launch_raster_bwd_gw(const Ws& w, cudaStream_t s) {
  if (w.n == 0) return cudaSuccess;
  LaunchScope ls(kKRasterBwdGw, s);
  const int64_t blocks = (w.n + kGwWarps - 1) / kGwWarps;
  return launch_chain(k_raster_bwd_gw, dim3((unsigned)blocks), dim3(kGwWarps * 32), 0, s, w);
}

}  // namespace gs
