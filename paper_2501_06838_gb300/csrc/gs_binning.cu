// Binning of (tile, Gaussian) pairs for the tile rasterizer:
//   prefix sum of per-Gaussian tile counts -> emit (tile key, Gaussian id) pairs
//   in Gaussian-major order -> stable LSD radix sort by tile key -> per-tile
//   [start, end) ranges. A stable sort keeps the Gaussian ids of each tile in
//   ascending order, so every tile accumulates its Gaussians in a fixed order
//   and the forward is bitwise reproducible.
// Algorithm 1 of GSASR (arXiv 2501.06838) touches, per Gaussian, only the HR
// pixels of its window; binning the windows to screen tiles lets each tile
// visit only the Gaussians whose window meets it.
//
// Grid-implicit binning (the raster's GridSource) builds the same per-tile
// lists without a sort when every centre sits on the reference grid
// (mu = p + o, Sec. 3.2).
#include "gs_internal.cuh"

namespace gs {

namespace {

constexpr int kTopThreads = 1024;

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                            // per thread
constexpr int kSortBlock = kSortThreads * kSortItems;    // 2048 pairs per block

// Exclusive scan of the block partials in place (one block). In count mode the
// total is the pair count P: it is stored and checked against the capacity.
__global__ void __launch_bounds__(kTopThreads) k_scan_top(unsigned long long* parts, int nparts,
                                                          Header* hdr, int count_mode) {
  griddep_release();
  griddep_wait();
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
  griddep_release();
  griddep_wait();
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

template <int BITS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* keys, const Header* hdr,
                                                             int shift, uint32_t* hist, int nblk) {
  griddep_release();
  griddep_wait();
  constexpr int R = 1 << BITS;
  __shared__ uint32_t h[kSortWarps][R];
  for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) (&h[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long P = effective_pairs(hdr);
  const int64_t base = blockIdx.x * (int64_t)kSortBlock;
  const int warp = threadIdx.x >> 5;
  uint32_t kk[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {   // all loads in flight before any atomic
    const int64_t i = base + k * kSortThreads + threadIdx.x;
    kk[k] = (unsigned long long)i < P ? __ldg(keys + i) : 0xffffffffu;
  }
#pragma unroll
  for (int k = 0; k < kSortItems; ++k)
    if (kk[k] != 0xffffffffu) atomicAdd(&h[warp][(kk[k] >> shift) & (R - 1)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < R; d += kSortThreads) {
    uint32_t s = 0u;
    for (int q = 0; q < kSortWarps; ++q) s += h[q][d];
    hist[(int64_t)d * nblk + blockIdx.x] = s;
  }
}

// Per-digit exclusive scan over blocks, in place: block d scans the row
// hist[d][0..nblk) and writes the row total to dtot[d].
__global__ void __launch_bounds__(kSortThreads) k_radix_rowscan(uint32_t* hist, int nblk,
                                                                uint32_t* dtot) {
  griddep_release();
  griddep_wait();
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
// chunk [b*2048 + q*256, +256) and walks it 32 pairs at a time; a pair's rank
// among equal digits is (pairs of that digit earlier in the warp's chunk) +
// (lower lanes with that digit in the same step). Blocks, then warps, then
// lanes follow input order, which makes the pass stable. The block first
// places its pairs in shared memory in digit order, then writes each digit's
// run to its global position with consecutive threads on consecutive
// addresses (coalesced stores).
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* kin,
                                                                const uint32_t* vin, uint32_t* kout,
                                                                uint32_t* vout, const Header* hdr,
                                                                int shift, const uint32_t* hist,
                                                                const uint32_t* dtot, int nblk) {
  griddep_release();
  griddep_wait();
  constexpr int R = 1 << BITS;
  constexpr int DPT = R / kSortThreads;   // digits per thread in the digit scans
  extern __shared__ uint32_t sm[];
  uint32_t* wc = sm;                          // [kSortWarps][R]
  uint32_t* lstart = wc + kSortWarps * R;     // [R] block-local start of each digit
  uint32_t* gshift = lstart + R;              // [R] global start - local start
  uint32_t* skey = gshift + R;                // [kSortBlock]
  uint32_t* sval = skey + kSortBlock;         // [kSortBlock]
  __shared__ unsigned long long sw[kSortThreads / 32 + 1];

  for (int i = threadIdx.x; i < kSortWarps * R; i += kSortThreads) wc[i] = 0u;
  __syncthreads();
  const unsigned long long P = effective_pairs(hdr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t bbase = blockIdx.x * (int64_t)kSortBlock;
  const int64_t base = bbase + warp * (32 * kSortItems);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {   // all loads in flight before the ranking
    const int64_t i = base + j * 32 + lane;
    const bool valid = (unsigned long long)i < P;
    key[j] = valid ? __ldg(kin + i) : 0u;
    val[j] = valid ? __ldg(vin + i) : 0u;
    rank[j] = valid ? 0u : 0xffffffffu;
  }
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const bool valid = rank[j] == 0u;
    const uint32_t d = (key[j] >> shift) & (R - 1);
    // lanes holding the same digit (invalid lanes match nobody)
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : (0x80000000u | lane));
    const uint32_t before = valid ? wc[warp * R + d] : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0u) wc[warp * R + d] = before + __popc(peers);
    __syncwarp();
    rank[j] = valid ? before + __popc(peers & lt_mask) : 0xffffffffu;
  }
  __syncthreads();
  // block-local digit starts (exclusive scan over digits of the block counts);
  // per-warp prefixes within each digit; global shift per digit
  {
    uint32_t cnt[DPT];
    uint32_t tsum = 0u;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      uint32_t c = 0u;
      for (int w = 0; w < kSortWarps; ++w) c += wc[w * R + d];
      cnt[q] = c;
      tsum += c;
    }
    unsigned long long tot;
    uint32_t run = (uint32_t)block_exclusive_scan<unsigned long long, kSortThreads>(tsum, sw, tot);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      lstart[d] = run;
      uint32_t wrun = run;
      for (int w = 0; w < kSortWarps; ++w) {
        const uint32_t t = wc[w * R + d];
        wc[w * R + d] = wrun;
        wrun += t;
      }
      run += cnt[q];
    }
    // global start of digit d for this block: sum of all digits < d over all
    // blocks (exclusive scan of dtot) + this digit's count in earlier blocks
    uint32_t dsum = 0u;
    uint32_t dt[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      dt[q] = dtot[threadIdx.x * DPT + q];
      dsum += dt[q];
    }
    uint32_t drun = (uint32_t)block_exclusive_scan<unsigned long long, kSortThreads>(dsum, sw, tot);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = threadIdx.x * DPT + q;
      gshift[d] = drun + hist[(int64_t)d * nblk + blockIdx.x] - lstart[d];
      drun += dt[q];
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if (rank[j] == 0xffffffffu) continue;
    const uint32_t d = (key[j] >> shift) & (R - 1);
    const uint32_t lp = wc[warp * R + d] + rank[j];
    skey[lp] = key[j];
    sval[lp] = val[j];
  }
  __syncthreads();
  const int nvalid = (int)min((unsigned long long)kSortBlock,
                              P > (unsigned long long)bbase ? P - (unsigned long long)bbase : 0ull);
  for (int i = threadIdx.x; i < nvalid; i += kSortThreads) {
    const uint32_t k = skey[i];
    const uint32_t pos = gshift[(k >> shift) & (R - 1)] + (uint32_t)i;
    kout[pos] = k;
    vout[pos] = sval[i];
  }
}

template <int BITS>
size_t scatter_smem() {
  return sizeof(uint32_t) * ((size_t)(kSortWarps + 2) * (1 << BITS) + 2 * kSortBlock);
}

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* keys, const Header* hdr,
                                                uint2* ranges) {
  griddep_wait();
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
  return launch_chain(k_scan_top, dim3(1), dim3(kTopThreads), 0, s, w.parts, parts, w.hdr, 1);
}

cudaError_t launch_emit(const Ws& w, cudaStream_t s) {
  if (w.n == 0) return cudaSuccess;
  const int blocks = scan_parts_needed(w.n);
  LaunchScope ls(kKEmit, s);
  return launch_chain(k_emit, dim3(blocks), dim3(kFootprintBlock), 0, s, w);
}

template <int BITS>
cudaError_t sort_pass(const Ws& w, int shift, int cur, cudaStream_t s) {
  cudaError_t e0;
  {
    LaunchScope ls(kKRadixHist, s);
    e0 = launch_chain(k_radix_hist<BITS>, dim3(w.sort_blocks), dim3(kSortThreads), 0, s,
                      (const uint32_t*)w.keys[cur], (const Header*)w.hdr, shift, w.hist,
                      w.sort_blocks);
  }
  cudaError_t e = e0;
  if (e != cudaSuccess) return e;
  {
    LaunchScope ls(kKRadixRowscan, s);
    e = launch_chain(k_radix_rowscan, dim3(1 << BITS), dim3(kSortThreads), 0, s, w.hist,
                     w.sort_blocks, w.hscan);
  }
  if (e != cudaSuccess) return e;
  const size_t smem = scatter_smem<BITS>();
  static bool smem_set = false;   // opt in to > 48 KB once per process
  if (!smem_set) {
    e = cudaFuncSetAttribute(k_radix_scatter<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  {
    LaunchScope ls(kKRadixScatter, s);
    e = launch_chain(k_radix_scatter<BITS>, dim3(w.sort_blocks), dim3(kSortThreads), smem, s,
                     (const uint32_t*)w.keys[cur], (const uint32_t*)w.vals[cur], w.keys[cur ^ 1],
                     w.vals[cur ^ 1], (const Header*)w.hdr, shift, (const uint32_t*)w.hist,
                     (const uint32_t*)w.hscan, w.sort_blocks);
  }
  return e;
}

// Stable LSD sort of the tile keys: `bits` significant bits in passes of at
// most 9 bits (digit width ceil(bits / passes)).
cudaError_t launch_sort(const Ws& w, int bits, cudaStream_t s, int* final_buf) {
  int cur = 0;
  *final_buf = 0;
  if (w.sort_blocks == 0 || bits == 0) return cudaSuccess;
  const int passes = (bits + 8) / 9;
  const int width = (bits + passes - 1) / passes;   // <= 9
  for (int p = 0; p < passes; ++p) {
    const int shift = p * width;
    cudaError_t e = width > 8 ? sort_pass<9>(w, shift, cur, s) : sort_pass<8>(w, shift, cur, s);
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
  return launch_chain(k_ranges, dim3(blocks), dim3(256), 0, s, sorted_keys, (const Header*)w.hdr,
                      w.ranges);
}

}  // namespace gs
