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
#include <atomic>
#include <climits>
#include <type_traits>

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
// SMEM: the three planes are a staged copy in shared memory (always aligned).
template <bool ALIGNED, bool SMEM, typename Off>
__device__ __forceinline__ void gw_pixel_pair(GwAcc& a, const float* __restrict__ g0,
                                              const float* __restrict__ g1,
                                              const float* __restrict__ g2, Off off,
                                              Off off2, const float4 q, float2 Xs, float2 nsK,
                                              float2 cr, float2 cg, float2 cb) {
  float2 gr, gg, gb;
  if (SMEM) {
    gr = *reinterpret_cast<const float2*>(g0 + off);
    gg = *reinterpret_cast<const float2*>(g1 + off);
    gb = *reinterpret_cast<const float2*>(g2 + off);
  } else if (ALIGNED) {
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

// The walk over the window [x0, x1] x [y0, y1] (image coordinates). Pixel
// (x, y) of the upstream gradient sits at go[(y - oy) * W + (x - ox)] of each
// plane: the caller's image (ox = 0, oy = row0, W the output width) or a
// staged region (its first column ox even and W even when SMEM).
template <bool ALIGNED, bool SMEM>
__device__ __forceinline__ void gw_walk(const float* __restrict__ go, int64_t plane, int W, int ox,
                                        int oy, int x0, int x1, int y0, int y1, const float4 f0,
                                        const float4 f1, const float4 f2, float4* rt, int lane,
                                        float (&v)[8]) {
  using Off = typename std::conditional<SMEM, int, int64_t>::type;
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
      const int xl = xp - ox, xq = min(xp + 1, ox + W - 1) - ox;   // columns in go
      GwAcc a;
      a.C[0] = a.C[1] = a.C[2] = a.SY = a.SYY = a.Sd = a.Sdd = a.SdY = p2(0.f, 0.f);
      int r = lr;
      for (; r + rpi < nr; r += 2 * rpi) {
        // 32-bit offsets within a staged region, 64-bit within an image
        const Off ya = (Off)(rb + r - oy) * W, yb = ya + (Off)rpi * W;
        const float4 qa = rt[r], qb = rt[r + rpi];
        gw_pixel_pair<ALIGNED, SMEM>(a, g0, g1, g2, ya + xl, ya + xq, qa, Xs, nsK, cr, cg, cb);
        gw_pixel_pair<ALIGNED, SMEM>(a, g0, g1, g2, yb + xl, yb + xq, qb, Xs, nsK, cr, cg, cb);
      }
      if (r < nr) {
        const Off ya = (Off)(rb + r - oy) * W;
        gw_pixel_pair<ALIGNED, SMEM>(a, g0, g1, g2, ya + xl, ya + xq, rt[r], Xs, nsK, cr, cg, cb);
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
    const float* go = w.direct ? w.grad_out0 : D.grad_out;
    const bool aligned = (W & 1) == 0 && (reinterpret_cast<uintptr_t>(go) & 7) == 0;
    if (aligned)
      gw_walk<true, false>(go, plane, W, 0, D.row0, x0, x1, y0, y1, rec[0], rec[1], rec[2], rt[wp],
                           lane, v);
    else
      gw_walk<false, false>(go, plane, W, 0, D.row0, x0, x1, y0, y1, rec[0], rec[1], rec[2],
                            rt[wp], lane, v);
  }
  const float s = warp_sum8(v, lane);
  if ((lane & 3) == 0) w.grec[gi * 12 + (lane >> 2)] = s;
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  // 4-byte asynchronous copy; bytes past src_bytes (0 or 4) are filled with zeros
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async16z(void* smem, const void* gmem, int src_bytes) {
  // 16-byte asynchronous copy; bytes past src_bytes (0 or 16) are filled with zeros
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}

// Block form, for Gaussians on a reference grid (m > 0): one CTA per block of
// kGbCellsX x kGbCellsY LR cells of an image. The CTA first forms the union box
// of its Gaussians' windows and, when the box fits kGbFloats, copies the
// upstream gradient over it into shared memory once (three planes, the first
// column even and the width even); its warps then walk their Gaussians (the
// k-th of the block goes to warp k % kGbWarps) exactly as the one-warp form
// does, reading the gradient from shared memory instead of L1/L2. A block
// whose box does not fit walks the gradient in global memory. Each Gaussian's
// sums keep the one-warp form's order, so the moments are the same bits.
constexpr int kGbWarps = 8;
constexpr int kGbFloats = 24 * 1024;   // 96 KB of staged gradient at most

__device__ __forceinline__ int image_of_gblock(const ImageDesc* im, int n_images, int b) {
  int lo = 0, hi = n_images - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (im[mid].b_base <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kGbWarps * 32) k_raster_bwd_gblock(Ws w) {
  griddep_release();
  griddep_wait();
  extern __shared__ float4 gstage4[];   // [3][RH][RW] floats (float4 for 16-byte alignment)
  float* gstage = reinterpret_cast<float*>(gstage4);
  __shared__ float4 rt[kGbWarps][kGwRows];
  __shared__ float4 srec[kGbCellsX * kGbCellsY * kRecordF4];   // the records when m = 1
  __shared__ int sbox[4];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int im = image_of_gblock(w.images, w.n_images, (int)blockIdx.x);
  const ImageDesc& D = w.images[im];
  const int bxs = (D.lr_w + kGbCellsX - 1) / kGbCellsX;
  const int lb = (int)blockIdx.x - D.b_base;
  const int by = lb / bxs, bx = lb - by * bxs;
  const int j0 = bx * kGbCellsX, i0 = by * kGbCellsY;
  const int cw = min(kGbCellsX, D.lr_w - j0), ch = min(kGbCellsY, D.lr_h - i0);
  const int m = D.m;
  const int ng = cw * ch * m;
  // global id of the block's k-th Gaussian (cells row by row, m per cell)
  auto gid_of = [&](int k) -> int64_t {
    const int c = k / m, sub = k - c * m;
    const int ci = c / cw, cj = c - ci * cw;
    return D.g_base + ((int64_t)(i0 + ci) * D.lr_w + (j0 + cj)) * m + sub;
  };

  // the union box of the live windows
  if (threadIdx.x == 0) {
    sbox[0] = INT_MAX; sbox[1] = INT_MIN; sbox[2] = INT_MAX; sbox[3] = INT_MIN;
  }
  __syncthreads();
  {
    int bx0 = INT_MAX, bx1 = INT_MIN, by0 = INT_MAX, by1 = INT_MIN;
    for (int k = threadIdx.x; k < ng; k += blockDim.x) {
      const float4* rec = w.records + gid_of(k) * kRecordF4;
      const float4 f3 = rec[3];
      if (m == 1) {   // one Gaussian per cell: the warps read the records from shared memory
        srec[k * kRecordF4] = rec[0];
        srec[k * kRecordF4 + 1] = rec[1];
        srec[k * kRecordF4 + 2] = rec[2];
        srec[k * kRecordF4 + 3] = f3;
      }
      const int x0 = __float_as_int(f3.x), x1 = __float_as_int(f3.y);
      const int y0 = __float_as_int(f3.z), y1 = __float_as_int(f3.w);
      if (x0 <= x1 && y0 <= y1) {
        bx0 = min(bx0, x0); bx1 = max(bx1, x1); by0 = min(by0, y0); by1 = max(by1, y1);
      }
    }
    bx0 = __reduce_min_sync(0xffffffffu, bx0);
    bx1 = __reduce_max_sync(0xffffffffu, bx1);
    by0 = __reduce_min_sync(0xffffffffu, by0);
    by1 = __reduce_max_sync(0xffffffffu, by1);
    if (lane == 0) {
      atomicMin(&sbox[0], bx0); atomicMax(&sbox[1], bx1);
      atomicMin(&sbox[2], by0); atomicMax(&sbox[3], by1);
    }
  }
  __syncthreads();
  const int W = D.out_w;
  const float* go = w.direct ? w.grad_out0 : D.grad_out;
  // 16-byte copies when the output's rows allow them: the box then starts on
  // a multiple of 4 columns and spans a multiple of 4 (else of 2)
  const bool vec4 = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(go) & 15) == 0;
  const int al = vec4 ? 3 : 1;
  const int rx0 = sbox[0] & ~al, rx1 = sbox[1], ry0 = sbox[2], ry1 = sbox[3];
  const bool any = rx0 <= rx1 && ry0 <= ry1;
  const int RW = any ? ((rx1 - rx0 + 1 + al) & ~al) : 0, RH = any ? ry1 - ry0 + 1 : 0;
  const int64_t rplane = (int64_t)RW * RH;
  const bool staged = any && 3 * rplane <= kGbFloats;   // uniform over the CTA
  const int64_t plane = (int64_t)D.out_h * W;
  if (staged && vec4) {
    const int RW4 = RW >> 2;
    for (int r = wp; r < RH; r += kGbWarps) {
      const float* src = go + (int64_t)(ry0 + r - D.row0) * W;   // output row (inside the output)
      float* dst = gstage + r * RW;
      for (int x4 = lane; x4 < RW4; x4 += 32) {
        const int gx = rx0 + 4 * x4;
        const bool in = gx < W;      // all four columns or none (W a multiple of 4)
        const int o = in ? gx : 0;   // always a valid address
        const int nb = in ? 16 : 0;
        cp_async16z(dst + 4 * x4, src + o, nb);
        cp_async16z(dst + rplane + 4 * x4, src + plane + o, nb);
        cp_async16z(dst + 2 * rplane + 4 * x4, src + 2 * plane + o, nb);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  } else if (staged) {
    // one warp per row of the box, its lanes along the row (coalesced), as
    // asynchronous copies so that all of a thread's loads are in flight at once
    // (columns past the output's edge are filled with zeros)
    for (int r = wp; r < RH; r += kGbWarps) {
      const float* src = go + (int64_t)(ry0 + r - D.row0) * W;   // output row (inside the output)
      float* dst = gstage + r * RW;
      for (int x = lane; x < RW; x += 32) {
        const int gx = rx0 + x;
        const bool in = gx < W;
        const int o = in ? gx : 0;   // always a valid address
        const int nb = in ? 4 : 0;
        cp_async4(dst + x, src + o, nb);
        cp_async4(dst + rplane + x, src + plane + o, nb);
        cp_async4(dst + 2 * rplane + x, src + 2 * plane + o, nb);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();
  const bool aligned = (W & 1) == 0 && (reinterpret_cast<uintptr_t>(go) & 7) == 0;
  for (int k = wp; k < ng; k += kGbWarps) {
    const int64_t gi = gid_of(k);
    const float4* rec = m == 1 ? srec + k * kRecordF4 : w.records + gi * kRecordF4;
    const float4 f3 = rec[3];
    const int x0 = __float_as_int(f3.x), x1 = __float_as_int(f3.y);
    const int y0 = __float_as_int(f3.z), y1 = __float_as_int(f3.w);
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (x0 <= x1 && y0 <= y1) {   // warp-uniform
      if (staged)
        gw_walk<true, true>(gstage, rplane, RW, rx0, ry0, x0, x1, y0, y1, rec[0], rec[1], rec[2],
                            rt[wp], lane, v);
      else if (aligned)
        gw_walk<true, false>(go, plane, W, 0, D.row0, x0, x1, y0, y1, rec[0], rec[1], rec[2],
                             rt[wp], lane, v);
      else
        gw_walk<false, false>(go, plane, W, 0, D.row0, x0, x1, y0, y1, rec[0], rec[1], rec[2],
                              rt[wp], lane, v);
    }
    const float sum = warp_sum8(v, lane);
    if ((lane & 3) == 0) w.grec[gi * 12 + (lane >> 2)] = sum;
  }
}

}  // namespace

cudaError_t launch_raster_bwd_gblock(const Ws& w, cudaStream_t s) {
  if (w.n == 0 || w.n_gblocks == 0) return cudaSuccess;
  static std::atomic<int> configured_device{-1};
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device.load() != dev) {
    const cudaError_t e = cudaFuncSetAttribute(k_raster_bwd_gblock,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(kGbFloats * sizeof(float)));
    if (e != cudaSuccess) return e;
    configured_device.store(dev);
  }
  LaunchScope ls(kKRasterBwdGw, s);
  return launch_chain(k_raster_bwd_gblock, dim3((unsigned)w.n_gblocks), dim3(kGbWarps * 32),
                      kGbFloats * sizeof(float), s, w);
}

cudaError_t launch_raster_bwd_gw(const Ws& w, cudaStream_t s) {
  if (w.n == 0) return cudaSuccess;
  LaunchScope ls(kKRasterBwdGw, s);
  const int64_t blocks = (w.n + kGwWarps - 1) / kGwWarps;
  return launch_chain(k_raster_bwd_gw, dim3((unsigned)blocks), dim3(kGwWarps * 32), 0, s, w);
}

}  // namespace gs
