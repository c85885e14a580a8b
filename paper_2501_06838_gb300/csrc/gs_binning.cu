// Binning of (tile, Gaussian) pairs for the tile rasterizer:
//   prefix sum of per-Gaussian tile counts -> emit (tile key, Gaussian id) pairs
//   in Gaussian-major order -> stable LSD radix sort by tile key -> per-tile
//   [start, end) ranges. A stable sort keeps the Gaussian ids of each tile in
//   ascending order, so every tile accumulates its Gaussians in a fixed order
//   and the forward is bitwise reproducible.
// Algorithm 1 of GSASR (arXiv 2501.06838) touches, per Gaussian, only the HR
// pixels of its window; binning the windows to screen tiles lets each tile
// visit only the Gaussians whose window meets it.
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr int kTopThreads = 1024;

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                           // per thread
constexpr int kSortBlock = kSortThreads * kSortItems;    // 4096 pairs per block
constexpr int kRadix = 256;

// Exclusive scan of the block partials in place (one block). In count mode the
// total is the pair count P: it is stored and checked against the capacity.
__global__ void __launch_bounds__(kTopThreads) k_scan_top(unsigned long long* parts, int nparts,
                                                          Header* hdr, int count_mode) {
  __shared__ unsigned long long sw[kTopThreads / 32 + 1];
  unsigned long long carry = 0ull;
  for (int c = 0; c < nparts; c += kTopThreads) {
    const int i = c + threadIdx.x;
    unsigned long long v = i < nparts ? parts[i] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_exclusive_scan<unsigned long long, kTopThreads>(v, sw, tot);
    if (i < nparts) parts[i] = carry + ex;
    carry += tot;
  }
  if (count_mode && threadIdx.x == 0) {
    hdr->pairs = carry;
    if (carry > hdr->capacity) atomicOr(&hdr->status, kStCapacity);
  }
}

// Block b handles the same 256 Gaussians as footprint block b: their pair
// offsets are the block's scanned partial plus an in-block exclusive scan of
// the counts. One lane per Gaussian gathers its tile rectangle; the warp then
// writes each of its 32 Gaussians' pairs cooperatively (coalesced stores).
__global__ void __launch_bounds__(kFootprintBlock) k_emit(Ws w) {
  __shared__ unsigned long long sw[kFootprintBlock / 32 + 1];
  const unsigned long long P = effective_pairs(w.hdr);
  if (P == 0ull) return;   // uniform over the grid
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t cnt = 0u;
  uint4 tr = make_uint4(0u, 0u, 1u, 1u);
  if (gi < w.n) {
    cnt = w.counts[gi];
    tr = w.trect[gi];
  }
  unsigned long long tot;
  const uint32_t off = (uint32_t)(block_exclusive_scan<unsigned long long, kFootprintBlock>(
                                      cnt, sw, tot) + w.parts[blockIdx.x]);
  const int64_t g0 = gi - lane;
  for (int j = 0; j < 32; ++j) {
    const uint32_t c = __shfl_sync(0xffffffffu, cnt, j);
    if (c == 0u) continue;
    const uint32_t o = __shfl_sync(0xffffffffu, off, j);
    const uint32_t key0 = __shfl_sync(0xffffffffu, tr.x, j);
    const uint32_t tx = __shfl_sync(0xffffffffu, tr.y, j);
    const uint32_t tw = __shfl_sync(0xffffffffu, tr.z, j);
    const uint32_t gid = (uint32_t)(g0 + j);
    for (uint32_t k = lane; k < c; k += 32u) {
      const uint32_t r = k / tw, q = k - r * tw;
      w.keys[0][o + k] = key0 + r * tx + q;
      w.vals[0][o + k] = gid;
    }
  }
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* keys, const Header* hdr,
                                                             int shift, uint32_t* hist, int nblk) {
  __shared__ uint32_t h[kSortWarps][kRadix];
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long P = effective_pairs(hdr);
  const int64_t base = blockIdx.x * (int64_t)kSortBlock;
  const int warp = threadIdx.x >> 5;
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + k * kSortThreads + threadIdx.x;
    if ((unsigned long long)i < P) atomicAdd(&h[warp][(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t s = 0u;
    for (int q = 0; q < kSortWarps; ++q) s += h[q][d];
    hist[(int64_t)d * nblk + blockIdx.x] = s;
  }
}

// Per-digit exclusive scan over blocks, in place: block d scans the row
// hist[d][0..nblk) and writes the row total to dtot[d].
__global__ void __launch_bounds__(kSortThreads) k_radix_rowscan(uint32_t* hist, int nblk,
                                                                uint32_t* dtot) {
  __shared__ unsigned long long sw[kSortThreads / 32 + 1];
  uint32_t* row = hist + (int64_t)blockIdx.x * nblk;
  unsigned long long carry = 0ull;
  for (int c = 0; c < nblk; c += kSortThreads) {
    const int i = c + threadIdx.x;
    const uint32_t v = i < nblk ? row[i] : 0u;
    unsigned long long tot;
    const unsigned long long ex =
        block_exclusive_scan<unsigned long long, kSortThreads>(v, sw, tot);
    if (i < nblk) row[i] = (uint32_t)(carry + ex);
    carry += tot;
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = (uint32_t)carry;
}

// Stable scatter of one radix pass. Warp q of block b owns the contiguous
// chunk [b*4096 + q*512, +512) and walks it 32 pairs at a time; a pair's rank
// among equal digits is (pairs of that digit earlier in the warp's chunk) +
// (lower lanes with that digit in the same step). Blocks then warps then lanes
// follow input order, which makes the pass stable.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* kin,
                                                                const uint32_t* vin, uint32_t* kout,
                                                                uint32_t* vout, const Header* hdr,
                                                                int shift, const uint32_t* hist,
                                                                const uint32_t* dtot, int nblk) {
  __shared__ uint32_t wc[kSortWarps][kRadix];
  __shared__ uint32_t dstart[kRadix];
  __shared__ unsigned long long sw[kSortThreads / 32 + 1];
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&wc[0][0])[i] = 0u;
  {
    // digit start = exclusive scan of the per-digit totals
    static_assert(kRadix == kSortThreads, "one thread per digit");
    unsigned long long tot;
    dstart[threadIdx.x] = (uint32_t)block_exclusive_scan<unsigned long long, kSortThreads>(
        dtot[threadIdx.x], sw, tot);
  }
  __syncthreads();
  const unsigned long long P = effective_pairs(hdr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = blockIdx.x * (int64_t)kSortBlock + warp * (32 * kSortItems);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const int64_t i = base + j * 32 + lane;
    const bool valid = (unsigned long long)i < P;
    key[j] = valid ? kin[i] : 0u;
    val[j] = valid ? vin[i] : 0u;
    const uint32_t d = (key[j] >> shift) & (kRadix - 1);
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    const uint32_t before = valid ? wc[warp][d] : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0u) wc[warp][d] = before + __popc(peers);
    __syncwarp();
    rank[j] = valid ? before + __popc(peers & lt_mask) : 0xffffffffu;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t run = dstart[d] + hist[(int64_t)d * nblk + blockIdx.x];
    for (int q = 0; q < kSortWarps; ++q) {
      const uint32_t t = wc[q][d];
      wc[q][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if (rank[j] == 0xffffffffu) continue;
    const uint32_t d = (key[j] >> shift) & (kRadix - 1);
    const uint32_t pos = wc[warp][d] + rank[j];
    kout[pos] = key[j];
    vout[pos] = val[j];
  }
}

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* keys, const Header* hdr,
                                                uint2* ranges) {
  const unsigned long long P = effective_pairs(hdr);
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if ((unsigned long long)i >= P) return;
  const uint32_t k = keys[i];
  if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
  if ((unsigned long long)(i + 1) == P || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
}

}  // namespace

int scan_parts_needed(int64_t n) { return (int)((n + kFootprintBlock - 1) / kFootprintBlock); }
int sort_blocks_needed(int64_t capacity) { return (int)((capacity + kSortBlock - 1) / kSortBlock); }

// Exclusive scan of the footprint pass's per-block pair counts; stores P.
cudaError_t launch_scan_counts(const Ws& w, cudaStream_t s) {
  const int parts = scan_parts_needed(w.n);
  LaunchScope ls(kKScanTop, s);
  k_scan_top<<<1, kTopThreads, 0, s>>>(w.parts, parts, w.hdr, 1);
  return cudaGetLastError();
}

cudaError_t launch_emit(const Ws& w, cudaStream_t s) {
  if (w.n == 0) return cudaSuccess;
  const int blocks = scan_parts_needed(w.n);
  LaunchScope ls(kKEmit, s);
  k_emit<<<blocks, kFootprintBlock, 0, s>>>(w);
  return cudaGetLastError();
}

cudaError_t launch_sort(const Ws& w, int passes, cudaStream_t s, int* final_buf) {
  int cur = 0;
  *final_buf = 0;
  if (w.sort_blocks == 0) return cudaSuccess;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    {
      LaunchScope ls(kKRadixHist, s);
      k_radix_hist<<<w.sort_blocks, kSortThreads, 0, s>>>(w.keys[cur], w.hdr, shift, w.hist,
                                                          w.sort_blocks);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(kKRadixRowscan, s);
      k_radix_rowscan<<<kRadix, kSortThreads, 0, s>>>(w.hist, w.sort_blocks, w.hscan);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
      LaunchScope ls(kKRadixScatter, s);
      k_radix_scatter<<<w.sort_blocks, kSortThreads, 0, s>>>(w.keys[cur], w.vals[cur],
                                                             w.keys[cur ^ 1], w.vals[cur ^ 1],
                                                             w.hdr, shift, w.hist, w.hscan,
                                                             w.sort_blocks);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  *final_buf = cur;
  return cudaSuccess;
}

cudaError_t launch_ranges(const Ws& w, const uint32_t* sorted_keys, cudaStream_t s) {
  if (w.capacity == 0) return cudaSuccess;
  const int blocks = (int)((w.capacity + 255) / 256);
  LaunchScope ls(kKRanges, s);
  k_ranges<<<blocks, 256, 0, s>>>(sorted_keys, w.hdr, w.ranges);
  return cudaGetLastError();
}

}  // namespace gs
