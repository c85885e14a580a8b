// Internal definitions shared by the CUDA translation units of libgs.
// Not part of the public ABI (include/gs.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

// Status bits of the device status word (mapped to gs_status on the host).
enum : uint32_t { kStInvalid = 1u, kStCapacity = 2u, kStInternal = 4u, kStTimeout = 8u };

constexpr int kSetupChunk = 16;       // image descriptors per setup launch
constexpr int kFootprintBlock = 256;  // Gaussians per footprint / emit block
constexpr int kRecordF4 = 4;          // a record is 4 float4 = 64 B
constexpr int kGbCellsX = 8;          // LR cells per block of the block Gaussian-warp adjoint
constexpr int kGbCellsY = 8;

// Per-image descriptor, copied into the workspace at the start of each call.
struct ImageDesc {
  const void* off;
  const void* sig;
  const void* rho;
  const void* rgb;
  const void* alpha;
  float* out;
  const float* grad_out;
  float* grads;
  int64_t n;
  int64_t g_base;   // first global Gaussian index of this image
  int32_t dtype, m, lr_h, lr_w, out_h, out_w;
  float scale, trunc_k;
  int32_t flags, tiles_x, tiles_y, t_base;  // t_base: first global tile index
  // fused head (kFlagHead): sigma = h_sigma_lo + h_sigma_span sigmoid(raw),
  // rho = h_rho_scale tanh(raw), c = alpha = sigmoid(raw),
  // o = h_offset_scale raw (or tanh(raw) with kFlagOffsetTanh)
  float h_sigma_lo, h_sigma_span, h_rho_scale, h_offset_scale;
  int32_t row0;   // first image row of the output (a band; 0: the whole image)
  int32_t p_base; // grid binning, tile 16: first global index of this image's tile pairs
  int32_t b_base; // m > 0: first global index of this image's blocks of LR cells
  int32_t pad_;
};
// ImageDesc::flags
constexpr int32_t kFlagPeak = 1;   // Z = 1 instead of Eq. 2's normalisation
constexpr int32_t kFlagRatio = 2;  // Algorithm 1's ratio window instead of the k-sigma box
constexpr int32_t kFlagHalf = 4;   // HR pixel x samples (x + 1/2)/s - 1/2
constexpr int32_t kFlagHead = 8;   // the parameter arrays hold raw head outputs
constexpr int32_t kFlagOffsetTanh = 16;
static_assert(sizeof(ImageDesc) == 160, "ImageDesc layout");

struct SetupChunk {
  int32_t first, count, reset, reset_ext;   // reset: header (first chunk); reset_ext: reaches
  ImageDesc d[kSetupChunk];
};

// Workspace header (device).
struct Header {
  uint32_t status;
  uint32_t pad0;
  unsigned long long pairs;        // P, total (tile, Gaussian) pairs
  unsigned long long pixel_pairs;  // sum_i |R_i|
  unsigned long long capacity;
  uint32_t work_counter;            // next tile (or pair) for the forward raster's CTAs
  uint32_t bwd_counter;             // next tile for the tile adjoint's CTAs
  unsigned long long list_cursor;  // grid mode: pair-list slots handed out to tiles
  unsigned long long reserved[10];
};
static_assert(sizeof(Header) == 128, "Header layout");

// Per-Gaussian record written by the footprint pass (64 B):
//   f0 = (cx_hi, cx_lo, cy_hi, cy_lo)  HR-pixel centre s*mu as exact float pairs
//   f1 = (sA, sK, g, l)                exponent, log2 units, X = x - cx, Y = y - cy (HR px):
//                                      e = -(sA X - sK Y)^2 + g Y^2 + l
//                                        = A X^2 + B X Y + C Y^2 + l  (Eq. 2's quadratic
//                                      form completed in X: sA = sqrt(-A), sK = B/(2 sA),
//                                      g = C - B^2/(4A), the Y-marginal)
//   f2 = (alpha r, alpha g, alpha b, 0)
//   f3 = (x0, x1, y0, y1)              integer window R_i, inclusive (x0 > x1: empty)
// Tile rectangle of the same Gaussian (16 B, emit pass):
//   (first key, tiles_x of its image, tiles wide, tiles high); count = w * h.

// Device pointers into the caller's workspace, plus sizes.
struct Ws {
  Header* hdr;
  ImageDesc* images;
  float4* records;            // [N][4]
  uint4* trect;               // [N]
  uint32_t* counts;           // [N]
  unsigned long long* parts;  // per-footprint-block pair counts, scanned in place
  uint32_t* keys[2];          // [capacity]
  uint32_t* vals[2];          // [capacity]
  uint32_t* hist;             // [radix][sort_blocks], row-scanned in place
  uint32_t* hscan;            // [radix] per-digit totals
  uint2* ranges;              // [T]
  float* grec;                // [N][12] record-space gradient moments
  short4* win;                // [N] windows (x0, x1, y0, y1) for grid binning (empty: never meets a tile)
  int4* ext;                  // [n_images] reach (DL, DR, DT, DB) of the windows past their LR cell, HR px
  uint32_t* tcount;           // [T] grid mode: per-row differences of the (tile, Gaussian)
                              // pairs per tile (a tile's count is the prefix along its row)
  int64_t n;                  // total Gaussians
  int64_t capacity;           // pair capacity
  int32_t n_images;
  int32_t tiles;              // total tiles
  int32_t tile;               // tile edge (8, 16, 32)
  int32_t tile_shift;
  int32_t sort_blocks;
  int32_t scan_parts;         // size of `parts`
  int32_t grid;               // 1: grid-implicit binning (no pair list), 0: sorted pair list
  int32_t direct;             // 1: one image, its grad_out / grads pointers below (adjoint)
  int32_t n_pairs;            // grid binning, tile 16: horizontal tile pairs over all images
  int32_t pair;               // 1: the forward raster runs one warp per pair of tiles
  int32_t adjoint;            // the adjoint kernel of these views (gs_adjoint, resolved)
  int32_t n_gblocks;          // every image with m > 0: blocks of LR cells in all; else 0
  const float* grad_out0;     // direct: dL/dI of image 0
  float* grads0;              // direct: parameter gradients of image 0
};

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
  // MUFU.EX2 (2^x on the special-function unit), flush-to-zero; ex2(-inf) = +0.
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// e^x in float32 by Cody-Waite range reduction: x = n ln2 + r with ln 2 split
// into 0.693359375 (9 bits, so n * it is exact) and -2.12194442e-4, then the
// degree-7 Taylor polynomial of e^r (|r| <= ln2/2) in Horner form and the exact
// scaling by 2^n. Each operation rounds to nearest and none is fused, so the
// result is a fixed function of x (a few ulp from e^x): the fused head's window
// edges depend on it and must be reproducible.
__device__ __forceinline__ float exp_seq(float x) {
  x = fminf(fmaxf(x, -87.0f), 88.0f);
  const float n = rintf(__fmul_rn(x, 1.44269502162933349609375f));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(n, 0.693359375f)),
                            __fmul_rn(n, -2.12194441701285541057586669921875e-4f));
  float p = 1.9841270113829523324966431e-4f;
  p = __fadd_rn(__fmul_rn(p, r), 1.3888889225199818611145020e-3f);
  p = __fadd_rn(__fmul_rn(p, r), 8.3333337679505348205566406e-3f);
  p = __fadd_rn(__fmul_rn(p, r), 4.1666667908430099487304688e-2f);
  p = __fadd_rn(__fmul_rn(p, r), 0.16666667163372039794921875f);
  p = __fadd_rn(__fmul_rn(p, r), 0.5f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  return ldexpf(p, (int)n);
}
__device__ __forceinline__ float sigmoid_seq(float x) {
  return __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_seq(-x)));
}
__device__ __forceinline__ float tanh_seq(float x) {
  const float e = exp_seq(__fmul_rn(-2.0f, fabsf(x)));
  const float t = __fdiv_rn(__fsub_rn(1.0f, e), __fadd_rn(1.0f, e));
  return x < 0.0f ? -t : t;
}

__device__ __forceinline__ float load_param(const void* p, int64_t i, int dtype) {
  if (dtype == 0) return __ldg(reinterpret_cast<const float*>(p) + i);
  if (dtype == 1) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[i]);
  return __half2float(reinterpret_cast<const __half*>(p)[i]);
}

// Highest image index whose first Gaussian index is <= gi.
__device__ __forceinline__ int image_of_gaussian(const ImageDesc* im, int n_images, int64_t gi) {
  int lo = 0, hi = n_images - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (im[mid].g_base <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int image_of_tile(const ImageDesc* im, int n_images, int t) {
  int lo = 0, hi = n_images - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (im[mid].t_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive block scan; returns the exclusive prefix of v and the block total.
template <class T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T* smem_warp, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_inclusive_scan(v);
  if (lane == 31) smem_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T x = lane < NT / 32 ? smem_warp[lane] : T(0);
    T xi = warp_inclusive_scan(x);
    if (lane < NT / 32) smem_warp[lane] = xi - x;
    if (lane == NT / 32 - 1) smem_warp[NT / 32] = xi;
  }
  __syncthreads();
  T r = smem_warp[warp] + incl - v;
  total = smem_warp[NT / 32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ unsigned long long effective_pairs(const Header* h) {
  unsigned long long p = h->pairs;
  return p <= h->capacity ? p : 0ull;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one per translation unit), all asynchronous on stream.
// Each returns the cudaError_t of its launches.
// ---------------------------------------------------------------------------
cudaError_t launch_setup(const SetupChunk& c, const Ws& w, cudaStream_t s);
cudaError_t launch_preprocess(const Ws& w, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const Ws& w, cudaStream_t s);
cudaError_t launch_scan_counts(const Ws& w, cudaStream_t s);
cudaError_t launch_emit(const Ws& w, cudaStream_t s);
cudaError_t launch_sort(const Ws& w, int key_bits, cudaStream_t s, int* final_buf);
cudaError_t launch_ranges(const Ws& w, const uint32_t* sorted_keys, cudaStream_t s);
cudaError_t launch_raster_fwd(const Ws& w, const uint32_t* sorted_vals, int batch, cudaStream_t s);
cudaError_t launch_raster_bwd_gw(const Ws& w, cudaStream_t s);
cudaError_t launch_raster_bwd_gblock(const Ws& w, cudaStream_t s);   // needs w.n_gblocks > 0
// quadrants: walk the 8 x 8 quadrants of 16 x 16 tiles (tile 16 only), each
// with the Gaussians of the tile's list whose window meets it
cudaError_t launch_raster_bwd_tile(const Ws& w, const uint32_t* lists, bool quadrants,
                                   cudaStream_t s);

// Kernel ids for launch accounting / per-kernel timing.
enum KernelId {
  kKSetup = 0, kKPreprocess, kKReserved2, kKScanTop, kKRadixRowscan, kKEmit, kKRadixHist,
  kKRadixScatter, kKRanges, kKRasterFwd, kKRasterBwd, kKPreprocessBwd, kKReserved12, kKRasterBwdGw,
  kKNumKernels
};

// Launch bookkeeping implemented in gs_api.cu: every launch goes through
// begin/end so that the launch counter and the optional event timing see it.
void launch_begin(int kernel_id, cudaStream_t s);
void launch_end(int kernel_id, cudaStream_t s);

// Programmatic dependent launch. Every kernel of the render's launch chains
// starts with griddep_wait(): it waits until the kernel before it in the
// stream has completed and its memory is visible (the waiting is the
// hardware's; a kernel launched without the attribute passes straight
// through). A kernel whose successor is a short pass also starts with
// griddep_release(), which lets that successor be scheduled while this one
// drains; kernels followed by a raster pass leave the release to their exit,
// so that the raster's single wave of CTAs is spread over the SMs as usual.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
__device__ __forceinline__ void griddep_release() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

bool chain_overlap();   // false when the environment sets GS_NO_PDL (launch-mode comparisons)

// CTAs of `kernel` (blocks of `threads`) that are resident on the current
// device at once, at most `work`: the grid of a persistent launch whose CTAs
// take their tiles from a counter. `work` when the occupancy query fails.
int resident_grid(const void* kernel, int threads, int64_t work);

// Launch one kernel of a chain with programmatic stream serialization.
template <typename... P, typename... A>
cudaError_t launch_chain(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                         A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = chain_overlap() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

struct LaunchScope {
  int id;
  cudaStream_t s;
  LaunchScope(int id_, cudaStream_t s_) : id(id_), s(s_) { launch_begin(id, s); }
  ~LaunchScope() { launch_end(id, s); }
};

}  // namespace gs
