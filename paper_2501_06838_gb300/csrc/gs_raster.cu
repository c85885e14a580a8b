// Tile rasterizer of the scale-aware 2D Gaussian splatting render (GSASR,
// arXiv 2501.06838, Eq. 4 with the Algorithm-1 window): the forward. (The
// adjoint, one lane per Gaussian over a tile's pixels, is gs_adjoint_tile.cu.)
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
//   stage 2: per (Gaussian, pair of tile rows) the row terms of the exponent
//              e = -(sA X - sK Y)^2 + g Y^2 + l        (log2 units)
//            as one float4 (-K(r), -K(r+1), R(r), R(r+1)), with K = sK*Y and
//            R = g*Y^2 + l (R = -inf outside the window rows);
//   compute: per Gaussian each thread forms Xs = sA*(col - cxl) (+inf outside
//            the window columns) and, for each of its row pairs, in packed
//            FP32x2 arithmetic (one instruction for both rows),
//              d = Xs - K, e = R - d*d, w = 2^e (MUFU.EX2, one per pixel),
//              out += c*w  (three FFMA2 for the three channels),
//            i.e. per pixel 2.5 FP32 instructions + 1 MUFU. The next
//            Gaussian's shared-memory operands load while the current one
//            is computed.
// The window masks are folded into the exponent: -inf rows and +inf columns
// both give e = -inf and w = +0, so masked pairs cost no branch. The completed
// square has no cancellation for any |rho| < 1 (the Y term is the marginal).
#include <type_traits>

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
  oy = ty * TILE + D->row0;   // image rows (the output holds rows row0 ..)
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

// Where a tile's Gaussian ids come from, one batch at a time (ids ascending,
// so both sources give a tile the same Gaussians in the same order and the
// forward the same bits).
//
// SortedSource: the tile's run [start, end) of the radix-sorted pair list.
template <int NT, int PF>
struct SortedSource {
  const uint32_t* vals;
  int pos, end;
  __device__ __forceinline__ int next(uint32_t (&gid)[PF]) {
    const int nb = max(0, min(NT * PF, end - pos));
    load_ids<NT, PF>(vals, pos, nb, gid);
    pos += nb;
    return nb;
  }
};

// GridSource (grid-implicit binning): with centres mu = p + o on the reference
// grid, a Gaussian of LR cell (i, j) has its window within
// [s j - DL, s j + DR] x [s i - DT, s i + DB], the per-image reach measured by
// the footprint pass. So the tile's candidates are the Gaussians of a box of
// LR cells: rows i0..i1, each a contiguous run of gids. Every candidate's
// window is tested against the tile (the same test that puts a pair into the
// sorted list); the survivors go through a shared-memory queue in gid order.
// All warps run the enumeration (the same loads and ballots); warp 0 writes.
template <int NT, int PF>
struct GridSource {
  static constexpr int BATCH = NT * PF;
  static constexpr int KR = 4;                          // candidates per lane per round
  static constexpr int QCAP = BATCH + 32 * KR <= 256 ? 256 : 512;
  const short4* win;
  uint32_t* q;           // shared [QCAP]
  int64_t rb0, rstride;  // gid of the first candidate of row r: rb0 + r * rstride
  int L, total, cur;     // candidates per row, in all, next to test
  int head, tail;        // queue positions (monotonic)
  int X0, X1, Y0, Y1;    // tile pixel bounds

  __device__ __forceinline__ void sync() {
    if (NT == 32) __syncwarp(); else __syncthreads();
  }
  float invL;            // 1 / L, for the row of a candidate index
  __device__ __forceinline__ uint32_t gid_of(int c) const {
    // r = c / L by a float reciprocal, corrected to the exact quotient
    int r = __float2int_rz(__fmul_rn((float)c + 0.5f, invL));
    r -= (r * L > c) ? 1 : 0;
    r += ((r + 1) * L <= c) ? 1 : 0;
    return (uint32_t)(rb0 + (int64_t)r * rstride + (c - r * L));
  }
  __device__ __forceinline__ int next(uint32_t (&gid)[PF]) {
    const int lane = threadIdx.x & 31;
    while (tail - head < BATCH && cur < total) {   // uniform over the CTA
      // KR independent window loads per lane, then the ballots in candidate order
      uint32_t g[KR];
      short4 v[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const int c = cur + 32 * k + lane;
        g[k] = c < total ? gid_of(c) : 0u;
        v[k] = c < total ? win[g[k]] : make_short4(32767, -32768, 32767, -32768);
      }
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const bool hit = v[k].x <= X1 && v[k].y >= X0 && v[k].z <= Y1 && v[k].w >= Y0;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (threadIdx.x < 32 && hit)
          q[(tail + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1)] = g[k];
        tail += __popc(bal);
      }
      cur += 32 * KR;
    }
    sync();
    const int nb = min(BATCH, tail - head);
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      const int i = j * NT + threadIdx.x;
      gid[j] = i < nb ? q[(head + i) & (QCAP - 1)] : 0u;
    }
    head += nb;
    return nb;
  }
};

// Candidate box of a tile in grid mode (see GridSource).
template <int TILE, int NT, int PF>
__device__ __forceinline__ void grid_source_init(const Ws& w, const ImageDesc* D, int ox, int oy,
                                                 uint32_t* q, GridSource<NT, PF>& g) {
  const int4 e = w.ext[D - w.images];   // (DL, DR, DT, DB), HR px
  const float s = D->scale;
  g.win = w.win;
  g.q = q;
  g.X0 = ox; g.X1 = ox + TILE - 1; g.Y0 = oy; g.Y1 = oy + TILE - 1;
  // A Gaussian of column j meets the tile only if s j - DL < x0 <= X1 and
  // s j + DR > x1 >= X0; the reach carries a pixel of margin, far more than the
  // float32 rounding of these quotients, so floor/ceil bound the cells exactly.
  const int j0 = max(0, (int)ceilf(__fdiv_rn((float)(g.X0 - e.y), s)));
  const int j1 = min(D->lr_w - 1, (int)floorf(__fdiv_rn((float)(g.X1 + e.x), s)));
  const int i0 = max(0, (int)ceilf(__fdiv_rn((float)(g.Y0 - e.w), s)));
  const int i1 = min(D->lr_h - 1, (int)floorf(__fdiv_rn((float)(g.Y1 + e.z), s)));
  g.rstride = (int64_t)D->lr_w * D->m;
  g.rb0 = D->g_base + ((int64_t)i0 * D->lr_w + j0) * D->m;
  g.L = (j1 - j0 + 1) * D->m;
  g.invL = g.L > 0 ? __frcp_rn((float)g.L) : 0.0f;
  g.total = (j0 <= j1 && i0 <= i1) ? (i1 - i0 + 1) * g.L : 0;
  g.cur = 0;
  g.head = g.tail = 0;
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

// Stage 2: row terms (-K(2p), -K(2p+1), R(2p), R(2p+1)) of every staged
// Gaussian and pair of tile rows; the packed window rows come from gC[i].w.
template <int TILE, int NT>
__device__ __forceinline__ void stage_rowpairs(int nb, const float4* gB, const float4* gC,
                                               float4* rq) {
  constexpr int HP = TILE / 2;
  for (int idx = threadIdx.x; idx < nb * HP; idx += NT) {
    const int i = idx / HP, p = idx - i * HP;
    const float4 b = gB[i];
    const int pk = __float_as_int(gC[i].w);
    const int ly0 = pk & 0xffff, ly1 = pk >> 16;
    const int r0 = 2 * p, r1 = 2 * p + 1;
    const float Y0 = (float)r0 - b.x, Y1 = (float)r1 - b.x;
    float R0 = fmaf(b.z * Y0, Y0, b.w), R1 = fmaf(b.z * Y1, Y1, b.w);
    if (r0 < ly0 || r0 > ly1) R0 = -kInf;
    if (r1 < ly0 || r1 > ly1) R1 = -kInf;
    rq[idx] = make_float4(-b.y * Y0, -b.y * Y1, R0, R1);
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Shared-memory operands of one Gaussian for one thread: gA, gC and the row
// terms of its NQ = BY / 2 row pairs.
template <int NQ>
struct FwdOps {
  float4 a, c, q[NQ];
  __device__ __forceinline__ void load(const float4* gA, const float4* gC, const float4* rq,
                                       int i, int hp, int pair0) {
    a = gA[i];
    c = gC[i];
    const float4* rr = rq + i * hp + pair0;
#pragma unroll
    for (int j = 0; j < NQ; ++j) q[j] = rr[j];
  }
};

template <int NQ>
__device__ __forceinline__ void fwd_gaussian(float2 (&acc)[NQ][3], const FwdOps<NQ>& o, float fcol) {
  float Xs = o.a.y * (fcol - o.a.x);
  if (fcol < o.a.z || fcol > o.a.w) Xs = kInf;
  const float2 X2 = f2(Xs, Xs);
  const float2 c0 = f2(o.c.x, o.c.x), c1 = f2(o.c.y, o.c.y), c2 = f2(o.c.z, o.c.z);
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const float2 d = __fadd2_rn(X2, f2(o.q[j].x, o.q[j].y));
    const float2 e = __ffma2_rn(f2(-d.x, -d.y), d, f2(o.q[j].z, o.q[j].w));
    const float2 wv = f2(ex2_approx(e.x), ex2_approx(e.y));
    acc[j][0] = __ffma2_rn(c0, wv, acc[j][0]);
    acc[j][1] = __ffma2_rn(c1, wv, acc[j][1]);
    acc[j][2] = __ffma2_rn(c2, wv, acc[j][2]);
  }
}

template <int TILE, int BY, int PF, bool GRID>
__global__ void __launch_bounds__(TILE * TILE / BY) k_raster_fwd(Ws w, const uint32_t* vals) {
  griddep_release();
  griddep_wait();
  constexpr int NT = TILE * TILE / BY, BATCH = NT * PF, NQ = BY / 2, HP = TILE / 2;
  __shared__ __align__(16) float4 raw[2][BATCH * kRecordF4];
  __shared__ float4 gA[BATCH], gB[BATCH], gC[BATCH];
  __shared__ float4 rq[BATCH * HP];
  __shared__ uint32_t qbuf[GRID ? GridSource<NT, PF>::QCAP : 1];

  const ImageDesc* D;
  int ox, oy;
  tile_origin<TILE>(w, blockIdx.x, D, ox, oy);
  const int col = threadIdx.x % TILE;
  const int row0 = (threadIdx.x / TILE) * BY;
  const int pair0 = row0 / 2;
  const float fcol = (float)col;

  float2 acc[NQ][3];
#pragma unroll
  for (int j = 0; j < NQ; ++j) acc[j][0] = acc[j][1] = acc[j][2] = f2(0.0f, 0.0f);

  typename std::conditional<GRID, GridSource<NT, PF>, SortedSource<NT, PF>>::type src;
  // grid mode: the tile's slice [lbase, lbase + lcount) of the pair list, where
  // the forward leaves its Gaussian ids (ascending) for the adjoint
  __shared__ int sl_base;
  int lbase = 0, lcount = 0, lpos = 0;
  bool lok = false;
  if constexpr (GRID) {
    grid_source_init<TILE, NT, PF>(w, D, ox, oy, qbuf, src);
    {
      // the tile's pair count: the prefix, along its tile row, of the
      // footprint pass's per-row differences
      const int lane = threadIdx.x & 31;
      const int lt = blockIdx.x - D->t_base;
      const int tyl = lt / D->tiles_x, txl = lt - tyl * D->tiles_x;
      const uint32_t* row = w.tcount + D->t_base + (int64_t)tyl * D->tiles_x;
      uint32_t acc = 0u;
      for (int x = lane; x <= txl; x += 32) acc += row[x];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      lcount = (int)acc;
    }
    if (threadIdx.x == 0) {
      const unsigned long long b = atomicAdd(&w.hdr->list_cursor, (unsigned long long)lcount);
      const bool fits = b + (unsigned long long)lcount <= (unsigned long long)w.capacity;
      sl_base = fits ? (int)b : -1;
      w.ranges[blockIdx.x] = fits ? make_uint2((uint32_t)b, (uint32_t)(b + lcount)) : make_uint2(0u, 0u);
      if (!fits && lcount > 0) atomicOr(&w.hdr->status, kStCapacity);
    }
    __syncthreads();
    lbase = sl_base;
    lok = lbase >= 0;
  } else {
    const uint2 range = w.ranges[blockIdx.x];
    src.vals = vals;
    src.pos = (int)range.x;
    src.end = (int)range.y;
  }
  // grid mode: append a batch of ids to the tile's slice of the list
  auto keep = [&](const uint32_t (&ids)[PF], int n) {
    if constexpr (GRID) {
      if (lpos + n > lcount) {   // the footprint count and the tile test disagree
        if (threadIdx.x == 0) atomicOr(&w.hdr->status, kStInternal);
        lok = false;
      }
      if (lok) {
#pragma unroll
        for (int j = 0; j < PF; ++j) {
          const int i = j * NT + threadIdx.x;
          if (i < n) w.vals[0][lbase + lpos + i] = ids[j];
        }
      }
      lpos += n;
    }
  };
  // batches of the tile's `total` Gaussians (grid mode: the footprint count)
  int total;
  if constexpr (GRID) total = lcount; else total = src.end - src.pos;
  const int nbat = (total + BATCH - 1) / BATCH;
  uint32_t gid[PF];
  if (nbat > 0) {
    keep(gid, src.next(gid));                              // batch 0
    issue_records<NT, PF>(w, gid, min(BATCH, total), raw[0]);
    if (nbat > 1) keep(gid, src.next(gid));                // batch 1
  }
  for (int b = 0; b < nbat; ++b) {
    const int nb = min(BATCH, total - b * BATCH);
    cp_async_wait_all();
    __syncthreads();
    stage_records<TILE, NT>(raw[b & 1], nb, ox, oy, gA, gB, gC);
    __syncthreads();
    stage_rowpairs<TILE, NT>(nb, gB, gC, rq);
    __syncthreads();
    if (b + 1 < nbat) {
      issue_records<NT, PF>(w, gid, min(BATCH, total - (b + 1) * BATCH), raw[(b + 1) & 1]);
      if (b + 2 < nbat) keep(gid, src.next(gid));          // batch b + 2
    }
    // Two operand sets in registers: Gaussian i + 1's loads overlap i's math.
    FwdOps<NQ> A, B;
    A.load(gA, gC, rq, 0, HP, pair0);
    for (int i = 0; i < nb; i += 2) {
      if (i + 1 < nb) B.load(gA, gC, rq, i + 1, HP, pair0);
      fwd_gaussian<NQ>(acc, A, fcol);
      if (i + 1 >= nb) break;
      if (i + 2 < nb) A.load(gA, gC, rq, i + 2, HP, pair0);
      fwd_gaussian<NQ>(acc, B, fcol);
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
      const int y = oy - D->row0 + row0 + k;   // output row
      if (y < H) {
        const int64_t o = (int64_t)y * W + x;
        const int j = k / 2;
        out[o] = (k & 1) ? acc[j][0].y : acc[j][0].x;
        out[plane + o] = (k & 1) ? acc[j][1].y : acc[j][1].x;
        out[2 * plane + o] = (k & 1) ? acc[j][2].y : acc[j][2].x;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Forward over a pair of horizontally adjacent 16 x 16 tiles (grid-implicit
// binning, tile 16): one warp renders a 32 x 16 region; lane l owns columns
// c = l % 16 (tile A) and c + 16 (tile B), rows (l / 16) * 8 .. + 8. The pair's
// candidates are enumerated once; each kept Gaussian carries whether its
// window meets tile A, tile B or both, and each half is computed only for the
// Gaussians that meet it (a warp-uniform test), so the evaluated pixels are
// those of 16 x 16 tiles while the per-Gaussian work (staging, operand loads,
// loop) is shared by up to 16 pixels per lane. The two tiles' lists are left
// for the adjoint exactly as the single-tile forward leaves them (same
// Gaussians, ascending ids), and every pixel sums its Gaussians in the same
// order, so the image is bitwise the single-tile forward's.
// ---------------------------------------------------------------------------
template <int PF>
struct PairSource {
  static constexpr int NT = 32, BATCH = NT * PF, KR = 4;
  static constexpr int QCAP = BATCH + 32 * KR <= 256 ? 256 : 512;
  const short4* win;
  uint32_t* q;           // shared [QCAP] ids
  uint8_t* qf;           // shared [QCAP] hit flags: 1 tile A, 2 tile B
  int64_t rb0, rstride;
  int L, total, cur, head, tail;
  int X0, XM, X1, Y0, Y1;   // tile A [X0, XM - 1], tile B [XM, X1], rows [Y0, Y1]
  float invL;
  __device__ __forceinline__ uint32_t gid_of(int c) const {
    int r = __float2int_rz(__fmul_rn((float)c + 0.5f, invL));
    r -= (r * L > c) ? 1 : 0;
    r += ((r + 1) * L <= c) ? 1 : 0;
    return (uint32_t)(rb0 + (int64_t)r * rstride + (c - r * L));
  }
  // the next batch: ids and flags of up to BATCH kept candidates, gid order
  __device__ __forceinline__ int next(uint32_t (&gid)[PF], uint32_t (&fl)[PF]) {
    const int lane = threadIdx.x & 31;
    while (tail - head < BATCH && cur < total) {
      uint32_t g[KR];
      short4 v[KR];
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const int c = cur + 32 * k + lane;
        g[k] = c < total ? gid_of(c) : 0u;
        v[k] = c < total ? win[g[k]] : make_short4(32767, -32768, 32767, -32768);
      }
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const bool rows = v[k].z <= Y1 && v[k].w >= Y0;
        const bool ha = rows && v[k].x <= XM - 1 && v[k].y >= X0;
        const bool hb = rows && v[k].x <= X1 && v[k].y >= XM;
        const bool hit = ha || hb;
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int at = (tail + __popc(bal & ((1u << lane) - 1u))) & (QCAP - 1);
          q[at] = g[k];
          qf[at] = (uint8_t)((ha ? 1 : 0) | (hb ? 2 : 0));
        }
        tail += __popc(bal);
      }
      cur += 32 * KR;
    }
    __syncwarp();
    const int nb = min(BATCH, tail - head);
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      const int i = j * NT + lane;
      const int at = (head + i) & (QCAP - 1);
      gid[j] = i < nb ? q[at] : 0u;
      fl[j] = i < nb ? (uint32_t)qf[at] : 0u;
    }
    head += nb;
    __syncwarp();
    return nb;
  }
};

// Stage 1 for a pair, each half exactly as the single-tile forward stages it
// for that tile (so the image is bitwise the same):
//   gA = (cxl_a, sA, lx0_a, lx1_a)   gD = (cxl_b, lx0_b, lx1_b, 0)
//   gB = (cyl, sK, g, l)             gC = (r, g, b, ly0 | ly1 << 16)
// with cxl_h the centre relative to half h's first column and [lx0_h, lx1_h]
// the window's columns in that half (empty when lx0_h > lx1_h).
template <int NT>
__device__ __forceinline__ void stage_pair_records(const float4* raw, int nb, int ox, int oy,
                                                   float4* gA, float4* gB, float4* gC,
                                                   float4* gD) {
  for (int i = threadIdx.x; i < nb; i += NT) {
    const float4 f0 = raw[i * kRecordF4], f1 = raw[i * kRecordF4 + 1];
    const float4 f2 = raw[i * kRecordF4 + 2], f3 = raw[i * kRecordF4 + 3];
    const int ob = ox + 16;
    const float cxa = __fadd_rn(__fsub_rn(f0.x, (float)ox), f0.y);
    const float cxb = __fadd_rn(__fsub_rn(f0.x, (float)ob), f0.y);
    const float cyl = __fadd_rn(__fsub_rn(f0.z, (float)oy), f0.w);
    const int x0 = __float_as_int(f3.x), x1 = __float_as_int(f3.y);
    const int ly0 = max(__float_as_int(f3.z) - oy, 0), ly1 = min(__float_as_int(f3.w) - oy, 15);
    gA[i] = make_float4(cxa, f1.x, (float)max(x0 - ox, 0), (float)min(x1 - ox, 15));
    gD[i] = make_float4(cxb, (float)max(x0 - ob, 0), (float)min(x1 - ob, 15), 0.0f);
    gB[i] = make_float4(cyl, f1.y, f1.z, f1.w);
    gC[i] = make_float4(f2.x, f2.y, f2.z, __int_as_float(ly0 | (ly1 << 16)));
  }
}

// Operands of one Gaussian for one lane of the pair kernel.
struct PairOps {
  float4 a, d, c, q[4];
  __device__ __forceinline__ void load(const float4* gA, const float4* gD, const float4* gC,
                                       const float4* rq, int i, int pair0) {
    a = gA[i];
    d = gD[i];
    c = gC[i];
    const float4* rr = rq + i * 8 + pair0;
#pragma unroll
    for (int j = 0; j < 4; ++j) q[j] = rr[j];
  }
};

// One Gaussian on one 16-column half: centre cxl, window columns [lo, hi].
__device__ __forceinline__ void fwd_half(float2 (&acc)[4][3], const float4 (&q)[4], float sA,
                                         float cxl, float lo, float hi, float fcol, float2 c0,
                                         float2 c1, float2 c2) {
  float Xs = sA * (fcol - cxl);
  if (fcol < lo || fcol > hi) Xs = kInf;
  const float2 X2 = f2(Xs, Xs);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 d = __fadd2_rn(X2, f2(q[j].x, q[j].y));
    const float2 e = __ffma2_rn(f2(-d.x, -d.y), d, f2(q[j].z, q[j].w));
    const float2 wv = f2(ex2_approx(e.x), ex2_approx(e.y));
    acc[j][0] = __ffma2_rn(c0, wv, acc[j][0]);
    acc[j][1] = __ffma2_rn(c1, wv, acc[j][1]);
    acc[j][2] = __ffma2_rn(c2, wv, acc[j][2]);
  }
}

// Both halves at once: the two halves' eight row-pair chains interleave.
__device__ __forceinline__ void fwd_both(float2 (&accA)[4][3], float2 (&accB)[4][3],
                                         const PairOps& o, float fcol, float2 c0, float2 c1,
                                         float2 c2) {
  float XsA = o.a.y * (fcol - o.a.x);
  if (fcol < o.a.z || fcol > o.a.w) XsA = kInf;
  float XsB = o.a.y * (fcol - o.d.x);
  if (fcol < o.d.y || fcol > o.d.z) XsB = kInf;
  const float2 XA = f2(XsA, XsA), XB = f2(XsB, XsB);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 nK = f2(o.q[j].x, o.q[j].y), R = f2(o.q[j].z, o.q[j].w);
    const float2 da = __fadd2_rn(XA, nK), db = __fadd2_rn(XB, nK);
    const float2 ea = __ffma2_rn(f2(-da.x, -da.y), da, R);
    const float2 eb = __ffma2_rn(f2(-db.x, -db.y), db, R);
    const float2 wa = f2(ex2_approx(ea.x), ex2_approx(ea.y));
    const float2 wb = f2(ex2_approx(eb.x), ex2_approx(eb.y));
    accA[j][0] = __ffma2_rn(c0, wa, accA[j][0]);
    accB[j][0] = __ffma2_rn(c0, wb, accB[j][0]);
    accA[j][1] = __ffma2_rn(c1, wa, accA[j][1]);
    accB[j][1] = __ffma2_rn(c1, wb, accB[j][1]);
    accA[j][2] = __ffma2_rn(c2, wa, accA[j][2]);
    accB[j][2] = __ffma2_rn(c2, wb, accB[j][2]);
  }
}

__device__ __forceinline__ void fwd_pair_gaussian(float2 (&accA)[4][3], float2 (&accB)[4][3],
                                                  const PairOps& o, float fcol) {
  const float2 c0 = f2(o.c.x, o.c.x), c1 = f2(o.c.y, o.c.y), c2 = f2(o.c.z, o.c.z);
  const bool ha = o.a.z <= o.a.w, hb = o.d.y <= o.d.z;   // meets tile A / B (warp-uniform)
  if (ha && hb)
    fwd_both(accA, accB, o, fcol, c0, c1, c2);
  else if (ha)
    fwd_half(accA, o.q, o.a.y, o.a.x, o.a.z, o.a.w, fcol, c0, c1, c2);
  else
    fwd_half(accB, o.q, o.a.y, o.d.x, o.d.y, o.d.z, fcol, c0, c1, c2);
}

// PF = 1: 18 resident CTAs per SM (shared memory allows 18); the cap takes it
// from 110 to 93 registers with no spills. PF = 2 is held to 9 by shared memory.
template <int PF>
__global__ void __launch_bounds__(32, PF == 1 ? 18 : 1) k_raster_fwd_pair(Ws w) {
  griddep_release();
  griddep_wait();
  constexpr int NT = 32, BATCH = NT * PF;
  using Src = PairSource<PF>;
  __shared__ __align__(16) float4 raw[2][BATCH * kRecordF4];
  __shared__ float4 gA[BATCH], gB[BATCH], gC[BATCH], gD[BATCH];
  __shared__ float4 rq[BATCH * 8];
  __shared__ uint32_t qbuf[Src::QCAP];
  __shared__ uint8_t qflg[Src::QCAP];
  __shared__ int sbase;

  const int lane = threadIdx.x;
  // the pair: image, tile row, tile A's column (tile B = A + 1 when it exists)
  int im = 0;
  {
    int lo = 0, hi = w.n_images - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (w.images[mid].p_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    im = lo;
  }
  const ImageDesc* D = &w.images[im];
  const int pairs_x = (D->tiles_x + 1) >> 1;
  const int lp = blockIdx.x - D->p_base;
  const int ty = lp / pairs_x;
  const int txa = 2 * (lp - ty * pairs_x);
  const bool has_b = txa + 1 < D->tiles_x;
  const int ox = txa * 16, oy = ty * 16 + D->row0;   // image rows (a band's start at row0)
  const int ta = D->t_base + ty * D->tiles_x + txa;

  // pair counts of tiles A and B: prefixes, along their tile row, of the
  // footprint pass's per-row differences
  int na, nb_ = 0;
  {
    const uint32_t* row = w.tcount + D->t_base + (int64_t)ty * D->tiles_x;
    uint32_t s = 0u;
    for (int x = lane; x <= txa; x += 32) s += row[x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    na = (int)s;
    if (has_b) nb_ = na + (int)row[txa + 1];
  }
  // the two tiles' slices of the pair list: A at [base, base + na), B after it
  if (lane == 0) {
    const unsigned long long tot = (unsigned long long)(na + nb_);
    const unsigned long long b = atomicAdd(&w.hdr->list_cursor, tot);
    const bool fits = b + tot <= (unsigned long long)w.capacity;
    sbase = fits ? (int)b : -1;
    w.ranges[ta] = fits ? make_uint2((uint32_t)b, (uint32_t)(b + na)) : make_uint2(0u, 0u);
    if (has_b)
      w.ranges[ta + 1] = fits ? make_uint2((uint32_t)(b + na), (uint32_t)(b + na + nb_))
                              : make_uint2(0u, 0u);
    if (!fits && tot > 0) atomicOr(&w.hdr->status, kStCapacity);
  }
  __syncwarp();
  const int lbase = sbase;
  bool lok = lbase >= 0;
  int pos_a = 0, pos_b = 0;

  // candidate cells of the pair region (the per-image reach of the windows)
  Src src;
  {
    const int4 e = w.ext[im];
    const float s = D->scale;
    src.win = w.win;
    src.q = qbuf;
    src.qf = qflg;
    src.X0 = ox;
    src.XM = ox + 16;
    src.X1 = ox + (has_b ? 31 : 15);
    src.Y0 = oy;
    src.Y1 = oy + 15;
    const int j0 = max(0, (int)ceilf(__fdiv_rn((float)(src.X0 - e.y), s)));
    const int j1 = min(D->lr_w - 1, (int)floorf(__fdiv_rn((float)(src.X1 + e.x), s)));
    const int i0 = max(0, (int)ceilf(__fdiv_rn((float)(src.Y0 - e.w), s)));
    const int i1 = min(D->lr_h - 1, (int)floorf(__fdiv_rn((float)(src.Y1 + e.z), s)));
    src.rstride = (int64_t)D->lr_w * D->m;
    src.rb0 = D->g_base + ((int64_t)i0 * D->lr_w + j0) * D->m;
    src.L = (j1 - j0 + 1) * D->m;
    src.invL = src.L > 0 ? __frcp_rn((float)src.L) : 0.0f;
    src.total = (j0 <= j1 && i0 <= i1) ? (i1 - i0 + 1) * src.L : 0;
    src.cur = 0;
    src.head = src.tail = 0;
  }
  // append a batch to the two tiles' lists (each in id order), checking the
  // footprint pass's counts against the tile tests
  auto keep = [&](const uint32_t (&ids)[PF], const uint32_t (&fl)[PF], int n) {
#pragma unroll
    for (int j = 0; j < PF; ++j) {
      const int i = j * NT + lane;
      const bool fa = i < n && (fl[j] & 1u), fb = i < n && (fl[j] & 2u);
      const unsigned ba = __ballot_sync(0xffffffffu, fa), bb = __ballot_sync(0xffffffffu, fb);
      const unsigned lt = (1u << lane) - 1u;
      const int at = pos_a + __popc(ba & lt), bt = pos_b + __popc(bb & lt);
      if (lok && fa && at < na) w.vals[0][lbase + at] = ids[j];
      if (lok && fb && bt < nb_) w.vals[0][lbase + na + bt] = ids[j];
      pos_a += __popc(ba);
      pos_b += __popc(bb);
    }
    if (pos_a > na || pos_b > nb_) {
      if (lane == 0) atomicOr(&w.hdr->status, kStInternal);
      lok = false;
    }
  };

  const int c = lane & 15;
  const int pair0 = (lane >> 4) * 4;
  const float fcol = (float)c;
  float2 accA[4][3], accB[4][3];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) accA[j][k] = accB[j][k] = f2(0.0f, 0.0f);

  uint32_t gid[PF], fl[PF];
  int nb0 = src.next(gid, fl);   // batch 0
  keep(gid, fl, nb0);
  int nb1 = 0;
  if (nb0 > 0) {
    issue_records<NT, PF>(w, gid, nb0, raw[0]);
    nb1 = src.next(gid, fl);      // batch 1
    keep(gid, fl, nb1);
  }
  for (int b = 0; nb0 > 0; ++b) {
    cp_async_wait_all();
    __syncwarp();
    stage_pair_records<NT>(raw[b & 1], nb0, ox, oy, gA, gB, gC, gD);
    __syncwarp();
    stage_rowpairs<16, NT>(nb0, gB, gC, rq);
    __syncwarp();
    int nb2 = 0;
    if (nb1 > 0) {
      issue_records<NT, PF>(w, gid, nb1, raw[(b + 1) & 1]);
      nb2 = src.next(gid, fl);    // batch b + 2
      keep(gid, fl, nb2);
    }
    // One operand set in registers (a second one for overlapping the next
    // Gaussian's loads measured slower: the registers cost more warps)
    for (int i = 0; i < nb0; ++i) {
      PairOps A;
      A.load(gA, gD, gC, rq, i, pair0);
      fwd_pair_gaussian(accA, accB, A, fcol);
    }
    __syncwarp();
    nb0 = nb1;
    nb1 = nb2;
  }
  if (pos_a != na || pos_b != nb_) {   // fewer kept than counted: stale list entries
    if (lane == 0) atomicOr(&w.hdr->status, kStInternal);
  }

  const int H = D->out_h, W = D->out_w;
  float* out = D->out;
  const int64_t plane = (int64_t)H * W;
  auto store = [&](const float2 (&acc)[4][3], int x) {
    if (x >= W) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int y = oy - D->row0 + pair0 * 2 + k;   // output row
      if (y < H) {
        const int64_t o = (int64_t)y * W + x;
        out[o] = (k & 1) ? acc[k / 2][0].y : acc[k / 2][0].x;
        out[plane + o] = (k & 1) ? acc[k / 2][1].y : acc[k / 2][1].x;
        out[2 * plane + o] = (k & 1) ? acc[k / 2][2].y : acc[k / 2][2].x;
      }
    }
  };
  store(accA, ox + c);
  store(accB, ox + 16 + c);
}

template <int TILE, int BY, int PF>
cudaError_t run(const Ws& w, const uint32_t* vals, cudaStream_t s) {
  constexpr int NT = TILE * TILE / BY;
  LaunchScope ls(kKRasterFwd, s);
  if (w.grid) return launch_chain(k_raster_fwd<TILE, BY, PF, true>, dim3(w.tiles), dim3(NT), 0, s, w, vals);
  return launch_chain(k_raster_fwd<TILE, BY, PF, false>, dim3(w.tiles), dim3(NT), 0, s, w, vals);
}

// Launch configurations: tile edge -> rows per thread (threads = TILE^2 / BY);
// batch = Gaussians staged per round = threads * PF, PF in {1, 2} (the host
// accepts only these batches; 0 selects PF = 1).
cudaError_t dispatch(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  if (w.tiles == 0) return cudaSuccess;
  if (w.pair) {   // grid binning, tile 16: one warp per horizontal pair of tiles
    LaunchScope ls(kKRasterFwd, s);
    if (batch >= 64)
      return launch_chain(k_raster_fwd_pair<2>, dim3(w.n_pairs), dim3(32), 0, s, w);
    return launch_chain(k_raster_fwd_pair<1>, dim3(w.n_pairs), dim3(32), 0, s, w);
  }
  switch (w.tile) {
    case 8:   // 32 threads
      return batch >= 64 ? run<8, 2, 2>(w, vals, s) : run<8, 2, 1>(w, vals, s);
    case 32:  // 64 threads
      return batch >= 128 ? run<32, 16, 2>(w, vals, s) : run<32, 16, 1>(w, vals, s);
    default:  // 32 threads
      return batch >= 64 ? run<16, 8, 2>(w, vals, s) : run<16, 8, 1>(w, vals, s);
  }
}

}  // namespace

cudaError_t launch_raster_fwd(const Ws& w, const uint32_t* vals, int batch, cudaStream_t s) {
  return dispatch(w, vals, batch, s);
}

}  // namespace gs
