// Per-Gaussian passes of the scale-aware rasterizer (GSASR, arXiv 2501.06838):
//   k_setup           copies the image table into the workspace, resets counters
//   k_preprocess      footprint pass: parameters -> record, window R_i, tile count
//   k_preprocess_bwd  record-space gradient moments -> parameter gradients
// Both read the parameters through load_gaussian, which applies the fused
// Gaussian head (Sec. 3.2) when the arrays hold raw head outputs.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr float kLog2E = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kLog2TwoPi = 2.6514961294723187f;

__global__ void k_setup(SetupChunk c, Ws w) {
  griddep_release();
  griddep_wait();
  const int t = threadIdx.x;
  if (c.reset && w.grid)   // clear the per-tile pair counts of grid binning
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + t; i < w.tiles; i += (int64_t)gridDim.x * blockDim.x)
      w.tcount[i] = 0u;
  if (blockIdx.x != 0) return;
  if (t < c.count) w.images[c.first + t] = c.d[t];
  if (t < c.count && c.reset_ext) w.ext[c.first + t] = make_int4(0, 0, 0, 0);
  if (c.reset && t == 0) {
    Header* h = w.hdr;
    h->status = 0u;
    h->pairs = 0ull;
    h->pixel_pairs = 0ull;
    h->capacity = (unsigned long long)w.capacity;
    h->work_counter = 0u;
    h->bwd_counter = 0u;
    h->list_cursor = 0ull;
    h->reserved[0] = (unsigned long long)w.n;
    h->reserved[1] = (unsigned long long)w.tiles;
    h->reserved[2] = (unsigned long long)w.pair;
    h->reserved[3] = (unsigned long long)w.adjoint;
  }
}

// Integer window edge on one axis, in float32 with round-to-nearest and no
// contraction (the __f*_rn intrinsics are never fused), c the float32 HR
// centre:
//   k-sigma box (Algorithm 1 with a 3-sigma footprint), closed:
//     r = (s * k) * sigma, lo = ceil(c - r), hi = floor(c + r);
//   ratio box (Algorithm 1's rasterization ratio, extent L = lr_w or lr_h), open:
//     r = (s * k) * L, lo = floor(c - r) + 1, hi = ceil(c + r) - 1;
// lo clamped to >= first, hi to <= last (the rendered rows or columns);
// empty -> lo = 1, hi = 0 (relative to first).
__device__ __forceinline__ void window_axis(float c, float sig, int lr_extent, float s, float k,
                                            bool ratio, int first, int last_i, int& lo, int& hi) {
  float sk = __fmul_rn(s, k);
  float r = __fmul_rn(sk, ratio ? (float)lr_extent : sig);
  float a = __fsub_rn(c, r), b = __fadd_rn(c, r);
  float flo = ratio ? __fadd_rn(floorf(a), 1.0f) : ceilf(a);
  float fhi = ratio ? __fsub_rn(ceilf(b), 1.0f) : floorf(b);
  const float f0 = (float)first, last = (float)last_i;
  if (!(flo >= f0)) flo = f0;
  if (!(fhi <= last)) fhi = last;
  if (flo > last || fhi < f0 || flo > fhi) { lo = first + 1; hi = first; return; }
  lo = (int)flo;
  hi = (int)fhi;
}

// One Gaussian's parameters, physical: read as stored, or mapped from raw head
// outputs (Sec. 3.2, Gaussian Primary Head) when the image has a fused head.
// raw[] keeps the stored values for the head's derivatives.
struct Phys {
  float ox, oy, sx, sy, rho, cr, cg, cb, al;
  float D;   // (1 - rho)(1 + rho), formed without cancellation as |rho| -> 1
};

__device__ __forceinline__ Phys load_gaussian(const ImageDesc& D, int64_t li, float (&raw)[9]) {
  const int dt = D.dtype;
  raw[0] = load_param(D.off, 2 * li, dt);
  raw[1] = load_param(D.off, 2 * li + 1, dt);
  raw[2] = load_param(D.sig, 2 * li, dt);
  raw[3] = load_param(D.sig, 2 * li + 1, dt);
  raw[4] = load_param(D.rho, li, dt);
  raw[5] = load_param(D.rgb, 3 * li, dt);
  raw[6] = load_param(D.rgb, 3 * li + 1, dt);
  raw[7] = load_param(D.rgb, 3 * li + 2, dt);
  raw[8] = load_param(D.alpha, li, dt);
  Phys p;
  if (D.flags & kFlagHead) {
    const bool ot = (D.flags & kFlagOffsetTanh) != 0;
    p.ox = __fmul_rn(D.h_offset_scale, ot ? tanh_seq(raw[0]) : raw[0]);
    p.oy = __fmul_rn(D.h_offset_scale, ot ? tanh_seq(raw[1]) : raw[1]);
    p.sx = __fadd_rn(D.h_sigma_lo, __fmul_rn(D.h_sigma_span, sigmoid_seq(raw[2])));
    p.sy = __fadd_rn(D.h_sigma_lo, __fmul_rn(D.h_sigma_span, sigmoid_seq(raw[3])));
    // rho = k tanh(x); 1 - rho^2 = (1 - k^2) + k^2 sech^2(x) with
    // sech^2(x) = 4 e / (1 + e)^2, e = exp(-2|x|): no cancellation near |rho| = 1
    {
      const float e = exp_seq(__fmul_rn(-2.0f, fabsf(raw[4])));
      const float t = __fdiv_rn(__fsub_rn(1.0f, e), __fadd_rn(1.0f, e));
      const float k = D.h_rho_scale;
      const float ope = __fadd_rn(1.0f, e);
      const float sech2 = __fdiv_rn(4.0f * e, __fmul_rn(ope, ope));
      p.rho = k * (raw[4] < 0.0f ? -t : t);
      p.D = fmaf(k * k, sech2, (1.0f - k) * (1.0f + k));
    }
    p.cr = sigmoid_seq(raw[5]);
    p.cg = sigmoid_seq(raw[6]);
    p.cb = sigmoid_seq(raw[7]);
    p.al = sigmoid_seq(raw[8]);
  } else {
    p.ox = raw[0]; p.oy = raw[1]; p.sx = raw[2]; p.sy = raw[3]; p.rho = raw[4];
    p.cr = raw[5]; p.cg = raw[6]; p.cb = raw[7]; p.al = raw[8];
    p.D = __fmul_rn(__fsub_rn(1.0f, p.rho), __fadd_rn(1.0f, p.rho));
  }
  return p;
}

// d(physical)/d(raw) of the fused head, in the gradient order
// (o_x, o_y, sigma_x, sigma_y, rho, r, g, b, alpha).
__device__ __forceinline__ void head_jacobian(const ImageDesc& D, const float (&raw)[9], const Phys& p,
                                              float (&J)[9]) {
  const bool ot = (D.flags & kFlagOffsetTanh) != 0;
  for (int k = 0; k < 2; ++k) {
    const float t = ot ? tanh_seq(raw[k]) : 0.0f;
    J[k] = ot ? D.h_offset_scale * (1.0f - t * t) : D.h_offset_scale;
    const float sv = sigmoid_seq(raw[2 + k]);
    J[2 + k] = D.h_sigma_span * sv * (1.0f - sv);
  }
  const float e = exp_seq(__fmul_rn(-2.0f, fabsf(raw[4])));
  const float ope = __fadd_rn(1.0f, e);
  J[4] = D.h_rho_scale * __fdiv_rn(4.0f * e, __fmul_rn(ope, ope));   // k sech^2(x)
  J[5] = p.cr * (1.0f - p.cr);
  J[6] = p.cg * (1.0f - p.cg);
  J[7] = p.cb * (1.0f - p.cb);
  J[8] = p.al * (1.0f - p.al);
}

constexpr int kCountBand = 512;   // entries of a warp's tile-count table (grid binning)

__device__ __forceinline__ int grid_root(int m) { return m == 1 ? 1 : m == 4 ? 2 : m == 9 ? 3 : 4; }

__global__ void __launch_bounds__(kFootprintBlock) k_preprocess(Ws w) {
  griddep_wait();
  __shared__ unsigned long long sw[kFootprintBlock / 32 + 1];
  __shared__ int band[kFootprintBlock / 32][kCountBand];   // grid binning: per-warp count table
  // Sorted binning: clear the tile ranges (grid-stride) so empty tiles read
  // (0, 0). Grid binning: the forward raster writes every tile's range.
  if (!w.grid)
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < w.tiles;
         t += (int64_t)gridDim.x * blockDim.x)
      w.ranges[t] = make_uint2(0u, 0u);

  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long pix = 0ull;
  uint32_t cnt = 0u;
  int4 reach = make_int4(0, 0, 0, 0);   // grid mode: window reach past the LR cell
  int rim = -1;                          // image of `reach` (-1: none)
  uint4 trk = make_uint4(0u, 0u, 0u, 0u);  // tile rectangle, for the per-tile counts
  uint32_t tcol0 = 0u;                     // its first tile column in the image
  int tim = -1, tty0 = 0, tty1 = -1;       // its image and tile rows
  if (gi < w.n) {
    const int im = image_of_gaussian(w.images, w.n_images, gi);
    const ImageDesc& D = w.images[im];
    const int64_t li = gi - D.g_base;
    float raw[9];
    const Phys P = load_gaussian(D, li, raw);
    const float ox = P.ox, oy = P.oy, sx = P.sx, sy = P.sy, rho = P.rho;
    const float cr = P.cr, cg = P.cg, cb = P.cb, al = P.al;
    const bool ok = isfinite(ox) && isfinite(oy) && isfinite(cr) && isfinite(cg) && isfinite(cb) &&
                    isfinite(al) && sx > 0.0f && sy > 0.0f && isfinite(sx) && isfinite(sy) &&
                    rho >= -1.0f && rho <= 1.0f && P.D > 0.0f && isfinite(P.D);
    const float s = D.scale;

    // Reference position p (float32) and the two centres: mu32 = fl(p + o) for
    // the window, and s * (p + o) as an exact float pair (hi + lo) for the
    // exponent (TwoSum of p + o, then TwoProduct of s times its head).
    float px = 0.0f, py = 0.0f;
    if (D.m > 0) {
      const int n = grid_root(D.m);
      const int64_t cell = li / D.m;
      const int sub = (int)(li - cell * D.m);
      const int64_t i = cell / D.lr_w, j = cell - i * D.lr_w;
      const int a = sub % n, b = sub / n;
      const float da = __fdiv_rn((float)(2 * a + 1 - n), (float)(2 * n));
      const float db = __fdiv_rn((float)(2 * b + 1 - n), (float)(2 * n));
      px = __fadd_rn((float)j, da);
      py = __fadd_rn((float)i, db);
    }
    float mux, muy, ex, ey;
    if (D.m > 0) {
      mux = __fadd_rn(px, ox);
      float bb = __fsub_rn(mux, px);
      ex = __fadd_rn(__fsub_rn(px, __fsub_rn(mux, bb)), __fsub_rn(ox, bb));
      muy = __fadd_rn(py, oy);
      bb = __fsub_rn(muy, py);
      ey = __fadd_rn(__fsub_rn(py, __fsub_rn(muy, bb)), __fsub_rn(oy, bb));
    } else {
      mux = ox; muy = oy; ex = 0.0f; ey = 0.0f;
    }
    float cx_hi = __fmul_rn(s, mux);
    float cx_lo = __fadd_rn(__fmaf_rn(s, mux, -cx_hi), __fmul_rn(s, ex));
    float cy_hi = __fmul_rn(s, muy);
    float cy_lo = __fadd_rn(__fmaf_rn(s, muy, -cy_hi), __fmul_rn(s, ey));
    // Half-pixel alignment: HR pixel x samples (x + 1/2)/s - 1/2, i.e. the HR
    // centre moves by h = s/2 - 1/2 (exact in float32 for s < 2^23). The window
    // uses fl(fl(s mu) + h); the exponent's pair absorbs h by TwoSum.
    float wcx = cx_hi, wcy = cy_hi;
    if (D.flags & kFlagHalf) {
      const float h = __fsub_rn(0.5f * s, 0.5f);
      wcx = __fadd_rn(cx_hi, h);
      wcy = __fadd_rn(cy_hi, h);
      float bb = __fsub_rn(wcx, cx_hi);
      float e = __fadd_rn(__fsub_rn(cx_hi, __fsub_rn(wcx, bb)), __fsub_rn(h, bb));
      cx_hi = wcx;
      cx_lo = __fadd_rn(cx_lo, e);
      bb = __fsub_rn(wcy, cy_hi);
      e = __fadd_rn(__fsub_rn(cy_hi, __fsub_rn(wcy, bb)), __fsub_rn(h, bb));
      cy_hi = wcy;
      cy_lo = __fadd_rn(cy_lo, e);
    }

    // the window in image coordinates, clamped to the rendered rows
    // row0 .. row0 + out_h - 1 (a band of the image, or all of it)
    int x0 = 1, x1 = 0, y0 = D.row0 + 1, y1 = D.row0;
    if (ok) {
      if (D.trunc_k > 0.0f) {
        const bool ratio = (D.flags & kFlagRatio) != 0;
        window_axis(wcx, sx, D.lr_w, s, D.trunc_k, ratio, 0, D.out_w - 1, x0, x1);
        window_axis(wcy, sy, D.lr_h, s, D.trunc_k, ratio, D.row0, D.row0 + D.out_h - 1, y0, y1);
      } else {
        x0 = 0; x1 = D.out_w - 1; y0 = D.row0; y1 = D.row0 + D.out_h - 1;
      }
    }
    // Records and compact windows stay in image coordinates; tiles are the
    // output's (rows from row0).

    // Exponent in HR pixels and log2 units: -q/2 of Eq. 2 times log2(e), with
    // u = X/s, v = Y/s, written with the square completed in X so that no
    // cancellation occurs however close |rho| is to 1:
    //   e = -(sA X - sK Y)^2 + g Y^2 + l,
    //   sA = r / (s sx), sK = rho r / (s sy), r = sqrt(log2(e) / (2 D)),
    //   g = -log2(e) / (2 s^2 sy^2)   (the Y marginal),  D = (1 - rho)(1 + rho).
    const float Dr = P.D;
    const float isx = __frcp_rn(__fmul_rn(s, sx)), isy = __frcp_rn(__fmul_rn(s, sy));
    const float r = sqrtf(__fdiv_rn(0.5f * kLog2E, Dr));
    const float sA = r * isx;
    const float sK = rho * r * isy;
    const float gY = -0.5f * kLog2E * isy * isy;
    // Eq. 2 normalisation 1 / (2 pi sx sy sqrt(D)), or 1 for the peak reading.
    const float l = (D.flags & kFlagPeak) == 0 ? -(kLog2TwoPi + log2f(sx) + log2f(sy) + 0.5f * log2f(Dr)) : 0.0f;

    float4* rec = w.records + gi * kRecordF4;
    // the adjoint's record-space accumulators start at zero (the tile adjoint
    // adds to them; the chain rule clears them again after reading them)
    // (whole 48-byte rows: a warp's stores then cover whole sectors)
    float4* acc = reinterpret_cast<float4*>(w.grec + gi * 12);
    acc[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    acc[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    acc[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    rec[0] = make_float4(cx_hi, cx_lo, cy_hi, cy_lo);
    rec[1] = make_float4(sA, sK, gY, l);
    rec[2] = make_float4(al * cr, al * cg, al * cb, 0.0f);
    rec[3] = make_float4(__int_as_float(x0), __int_as_float(x1), __int_as_float(y0), __int_as_float(y1));

    if (w.grid) {
      // compact window for the tile test, and how far it reaches past the
      // Gaussian's LR cell (i, j): DL = s j - x0, DR = x1 - s j (rows alike),
      // rounded up, plus one pixel of margin for the float32 rounding of s j
      const bool live = x0 <= x1 && y0 <= y1;
      w.win[gi] = live ? make_short4((short)x0, (short)x1, (short)y0, (short)y1)
                       : make_short4(32767, -32768, 32767, -32768);
      if (live) {
        const int64_t cell = li / D.m;
        const float sj = s * (float)(cell % D.lr_w), si = s * (float)(cell / D.lr_w);
        reach.x = max(0, (int)ceilf(sj - (float)x0) + 1);
        reach.y = max(0, (int)ceilf((float)x1 - sj) + 1);
        reach.z = max(0, (int)ceilf(si - (float)y0) + 1);
        reach.w = max(0, (int)ceilf((float)y1 - si) + 1);
        rim = im;
      }
    }
    uint4 tr = make_uint4(0u, 0u, 0u, 0u);
    if (x0 <= x1 && y0 <= y1) {
      const int tx0 = x0 >> w.tile_shift, tx1 = x1 >> w.tile_shift;
      const int ty0 = (y0 - D.row0) >> w.tile_shift, ty1 = (y1 - D.row0) >> w.tile_shift;
      const uint32_t tw = (uint32_t)(tx1 - tx0 + 1), th = (uint32_t)(ty1 - ty0 + 1);
      cnt = tw * th;
      tr = make_uint4((uint32_t)(D.t_base + ty0 * D.tiles_x + tx0), (uint32_t)D.tiles_x, tw, th);
      tcol0 = (uint32_t)tx0;
      tim = im;
      tty0 = ty0;
      tty1 = ty1;
      pix = (unsigned long long)(x1 - x0 + 1) * (unsigned long long)(y1 - y0 + 1);
    }
    w.trect[gi] = tr;
    w.counts[gi] = cnt;
    trk = tr;
    if (!ok) atomicOr(&w.hdr->status, kStInvalid);
  }
  if (w.grid) {
    // pairs per tile, as per-row differences: +1 at the rectangle's first
    // tile of each of its rows, -1 just past its last (a tile's count is the
    // sum along its row up to it; the raster forms it).
    const int lane = threadIdx.x & 31;
    const bool act = cnt != 0u;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    const int lead = am ? __ffs(am) - 1 : 0;
    const int imL = __shfl_sync(0xffffffffu, tim, lead);
    const bool same = __all_sync(0xffffffffu, !act || tim == imL);
    // The warp's tile band (rows RY0..RY1, columns CX0..CX1, the -1 entries
    // included): when the whole warp is on one image and the band fits, the
    // differences are first summed in a per-warp shared-memory table and each
    // nonzero entry is added once; otherwise lanes on the same entry combine
    // by warp match.
    const int tilesx = (int)__shfl_sync(0xffffffffu, trk.y, lead);
    const int lastc = act ? (int)(tcol0 + trk.z) : 0;        // column just past the rectangle
    const int RY0 = __reduce_min_sync(0xffffffffu, act ? tty0 : 0x7fffffff);
    const int RY1 = __reduce_max_sync(0xffffffffu, act ? tty1 : -1);
    const int CX0 = __reduce_min_sync(0xffffffffu, act ? (int)tcol0 : 0x7fffffff);
    const int CX1 = __reduce_max_sync(0xffffffffu, act ? min(lastc, tilesx - 1) : -1);
    const int bw = CX1 - CX0 + 1, bh = RY1 - RY0 + 1;
    if (am != 0u && same && bw > 0 && bh > 0 && bw * bh <= kCountBand) {
      int* h = band[threadIdx.x >> 5];
      const int span = bw * bh;
      for (int e = lane; e < span; e += 32) h[e] = 0;
      __syncwarp();
      if (act) {
        const int c0 = (int)tcol0 - CX0, c1 = lastc - CX0;
        const bool endin = lastc < tilesx;
        for (int r = tty0 - RY0; r <= tty1 - RY0; ++r) {
          atomicAdd(h + r * bw + c0, 1);
          if (endin) atomicSub(h + r * bw + c1, 1);
        }
      }
      __syncwarp();
      const int64_t base = w.images[imL].t_base + (int64_t)RY0 * tilesx + CX0;
      for (int e = lane; e < span; e += 32) {
        const int v = h[e];
        if (v != 0) {
          const int rr = e / bw;
          atomicAdd(w.tcount + base + (int64_t)rr * tilesx + (e - rr * bw), (uint32_t)v);
        }
      }
    } else if (am != 0u) {
      const uint32_t rows = cnt ? trk.w : 0u;
      const uint32_t last = tcol0 + trk.z;   // column just past the rectangle
      for (uint32_t k = 0;; ++k) {
        const bool on = k < rows;
        if (!__any_sync(0xffffffffu, on)) break;
        const uint32_t a = on ? trk.x + k * trk.y : 0xffffffffu;
        const unsigned ga = __match_any_sync(0xffffffffu, a);
        if (on && (__ffs(ga) - 1) == lane) atomicAdd(w.tcount + a, (uint32_t)__popc(ga));
        const bool endin = on && last < trk.y;
        const uint32_t b = endin ? a + trk.z : 0xffffffffu;
        const unsigned gb = __match_any_sync(0xffffffffu, b);
        if (endin && (__ffs(gb) - 1) == lane) atomicSub(w.tcount + b, (uint32_t)__popc(gb));
      }
    }
    // the per-image reach: warp maxima when the whole warp is on one image,
    // else per lane; an atomic only where the stored maximum is exceeded
    // (every warp would otherwise queue on the same four words)
    auto raise = [&](int im, int4 r) {
      int* e = reinterpret_cast<int*>(w.ext + im);
      const int4 cur = __ldcg(w.ext + im);
      if (r.x > cur.x) atomicMax(e, r.x);
      if (r.y > cur.y) atomicMax(e + 1, r.y);
      if (r.z > cur.z) atomicMax(e + 2, r.z);
      if (r.w > cur.w) atomicMax(e + 3, r.w);
    };
    const int im0 = __shfl_sync(0xffffffffu, rim, 0);
    if (__all_sync(0xffffffffu, rim == im0 || rim < 0) && im0 >= 0) {
      const int4 r = make_int4(__reduce_max_sync(0xffffffffu, reach.x),
                               __reduce_max_sync(0xffffffffu, reach.y),
                               __reduce_max_sync(0xffffffffu, reach.z),
                               __reduce_max_sync(0xffffffffu, reach.w));
      if ((threadIdx.x & 31) == 0) raise(im0, r);
    } else if (rim >= 0) {
      raise(rim, reach);
    }
  }
  // this block's pair count, scanned over blocks by k_scan_top (sorted
  // binning); grid binning adds the block total to P directly
  unsigned long long tot;
  block_exclusive_scan<unsigned long long, kFootprintBlock>(cnt, sw, tot);
  if (threadIdx.x == 0) {
    if (w.grid) {
      if (tot) atomicAdd(&w.hdr->pairs, tot);
    } else if (blockIdx.x < w.scan_parts) {
      w.parts[blockIdx.x] = tot;
    }
  }
  // block sum of the window areas, one atomic per block
  for (int o = 16; o > 0; o >>= 1) pix += __shfl_xor_sync(0xffffffffu, pix, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = pix;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sp = 0ull;
    for (int k = 0; k < kFootprintBlock / 32; ++k) sp += sw[k];
    if (sp) atomicAdd(&w.hdr->pixel_pairs, sp);
  }
}

// Chain rule from the record space to the parameters. The raster adjoint left,
// per Gaussian, the moments over its window of Gw = (sum_k g_k c_k) 2^e in the
// exponent's completed-square coordinates,
//   m = (Sd, SY, Sdd, SdY, SYY, Cr, Cg, Cb),  S_ab = sum Gw d^a Y^b,
//   C_k = sum g_k 2^e, and S0 = sum Gw = c . C,
// with e = -d^2 + g Y^2 + l, d = sA X - sK Y, X = x - cx, Y = y - cy, and
// out_k += c_k 2^e (c the record colour alpha * rgb). Since dL/de = ln2 Gw:
//   dL/dcx = 2 ln2 sA Sd,            dL/dcy = -2 ln2 (sK Sd + g SY),
//   dL/dsA = -2 ln2 (Sdd + sK SdY) / sA   (X = (d + sK Y) / sA),
//   dL/dsK = 2 ln2 SdY,  dL/dg = ln2 SYY,  dL/dl = ln2 S0.
// With sA = r / (s sx), sK = rho r / (s sy), g = -L2 / (2 s^2 sy^2),
// r = sqrt(L2 / (2 D)), D = (1 - rho)(1 + rho), L2 = log2 e, and
// l = -log2(2 pi sx sy sqrt D) (density; 0 for the peak reading):
//   dL/dsx  = (2 ln2 (Sdd + sK SdY) - S0) / sx
//   dL/dsy  = (-2 ln2 (sK SdY + g SYY) - S0) / sy
//   dL/drho = rho (S0 - 2 ln2 Sdd) / D + 2 ln2 SdY r / (s sy)
// (the S0 terms only with the density normalisation; dsA/drho = sA rho / D,
// dsK/drho = r / (s sy D), dl/drho = rho / (D ln2)), and cx = s mu_x.
// No term cancels at order 1/D^2 as |rho| -> 1, which the same chain rule in
// the moments of X would.
__global__ void __launch_bounds__(256) k_preprocess_bwd(Ws w) {
  griddep_release();
  griddep_wait();
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi == 0) w.hdr->bwd_counter = 0u;   // the next adjoint of this forward starts at tile 0
  if (gi >= w.n) return;
  const int im = image_of_gaussian(w.images, w.n_images, gi);
  const ImageDesc& D = w.images[im];
  const int64_t li = gi - D.g_base;
  float* out = (w.direct ? w.grads0 : D.grads) + li * 9;
  const float4* rec = w.records + gi * kRecordF4;
  // every load that does not depend on the image table, issued together
  float4* gm = reinterpret_cast<float4*>(w.grec + gi * 12);
  const float4 r3 = rec[3], rc = rec[2], m0 = gm[0], m1 = gm[1];
  const bool live = __float_as_int(r3.x) <= __float_as_int(r3.y) &&
                    __float_as_int(r3.z) <= __float_as_int(r3.w);
  if (!live) {
    for (int k = 0; k < 9; ++k) out[k] = 0.0f;
    return;
  }
  float raw[9];
  const Phys P = load_gaussian(D, li, raw);
  const float sx = P.sx, sy = P.sy, rho = P.rho;
  const float cr = P.cr, cg = P.cg, cb = P.cb, al = P.al;
  const float s = D.scale;
  const float Dr = P.D;
  const float isx = __frcp_rn(__fmul_rn(s, sx)), isy = __frcp_rn(__fmul_rn(s, sy));
  // the record's exponent constants, as the footprint pass forms them
  const float r = sqrtf(__fdiv_rn(0.5f * kLog2E, Dr));
  const float sA = r * isx;
  const float sK = rho * r * isy;
  const float gY = -0.5f * kLog2E * isy * isy;
  const float Sd = m0.x, SY = m0.y, Sdd = m0.z, SdY = m0.w, SYY = m1.x;
  const float Cr = m1.y, Cg = m1.z, Cb = m1.w;
  const float S0 = fmaf(rc.z, Cb, fmaf(rc.y, Cg, rc.x * Cr));

  const float two_ln2 = 2.0f * kLn2;
  const float dcx = two_ln2 * sA * Sd;
  const float dcy = -two_ln2 * fmaf(sK, Sd, gY * SY);
  const float dens = (D.flags & kFlagPeak) == 0 ? 1.0f : 0.0f;
  const float dsx = (two_ln2 * fmaf(sK, SdY, Sdd) - dens * S0) / sx;
  const float dsy = (-two_ln2 * fmaf(sK, SdY, gY * SYY) - dens * S0) / sy;
  const float drho = rho * fmaf(-two_ln2, Sdd, dens * S0) / Dr + two_ln2 * SdY * r * isy;
  float gr[9] = {s * dcx, s * dcy, dsx, dsy, drho, al * Cr, al * Cg, al * Cb,
                 cr * Cr + cg * Cg + cb * Cb};
  if (D.flags & kFlagHead) {   // chain rule through the head's activations
    float J[9];
    head_jacobian(D, raw, P, J);
    for (int k = 0; k < 9; ++k) gr[k] *= J[k];
  }
  for (int k = 0; k < 9; ++k) out[k] = gr[k];
  // cleared for the next adjoint of the same forward (the tile adjoint adds);
  // last, so that no load waits behind these stores, and whole 48-byte rows
  gm[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  gm[1] = make_float4(0.f, 0.f, 0.f, 0.f);
  gm[2] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

cudaError_t launch_setup(const SetupChunk& c, const Ws& w, cudaStream_t s) {
  LaunchScope ls(kKSetup, s);
  int blocks = 1;
  if (c.reset && w.grid) blocks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, ((int64_t)w.tiles + 255) / 256));
  return launch_chain(k_setup, dim3(blocks), dim3(256), 0, s, c, w);
}

cudaError_t launch_preprocess(const Ws& w, cudaStream_t s) {
  int64_t work = w.n > (int64_t)w.tiles ? w.n : (int64_t)w.tiles;
  int blocks = (int)((work + kFootprintBlock - 1) / kFootprintBlock);
  if (blocks < 1) blocks = 1;
  LaunchScope ls(kKPreprocess, s);
  return launch_chain(k_preprocess, dim3(blocks), dim3(kFootprintBlock), 0, s, w);
}

cudaError_t launch_preprocess_bwd(const Ws& w, cudaStream_t s) {
  if (w.n == 0) return cudaSuccess;
  int blocks = (int)((w.n + 255) / 256);
  LaunchScope ls(kKPreprocessBwd, s);
  return launch_chain(k_preprocess_bwd, dim3(blocks), dim3(256), 0, s, w);
}

}  // namespace gs
