/*
 * gs.h -- C-ABI of the GB300 (sm_103a) scale-aware 2D Gaussian rasterizer.
 *
 * The library renders N image Gaussians into a super-resolved image at any
 * scale factor s and back-propagates through the render, as defined by GSASR
 * (arXiv 2501.06838):
 *   Sec. 3.1, Eq. 1   G(x, y) = alpha * c * f(x, y)
 *   Sec. 3.1, Eq. 2   f = (2 pi sx sy sqrt(1 - rho^2))^-1
 *                         * exp(-(dx^2/sx^2 - 2 rho dx dy/(sx sy) + dy^2/sy^2)
 *                                / (2 (1 - rho^2)))
 *   Sec. 3.1, Eq. 4   I_SR(x, y; s) = sum_i G_i(x / s, y / s)
 *   Algorithm 1       each Gaussian only touches the HR pixels of a box window
 *                     around its centre; here the box is the footprint
 *                     |x/s - mu_x| <= k sx, |y/s - mu_y| <= k sy (k = trunc_k),
 *                     taken as an integer pixel rectangle whose edges are the
 *                     float32 values ceil(s mu - (s k) sigma), floor(s mu + (s k) sigma)
 *                     (round to nearest, no fused multiply-add), clamped to the
 *                     image.
 *   Sec. 3.1, "Fast Rasterization", and Sec. 3.2, "Rendering": the render is
 *                     differentiable; gs_render_bwd gives the gradient of
 *                     L = sum grad_out * I with the windows held fixed.
 *   Sec. 3.2, Gaussian Primary Head / Gaussian Embedding: with ref_grid_m = m
 *                     > 0 the centre is mu = p + o, p on an equal-interval
 *                     sqrt(m) x sqrt(m) sub-grid of each LR pixel (index order
 *                     ((i * lr_w + j) * m + b * sqrt(m) + a), p = (j + d_a, i + d_b),
 *                     d_a = (2a + 1 - sqrt(m)) / (2 sqrt(m)) in float32).
 *
 * Coordinates: LR pixel (j, i) is centred at (j, i) (Eq. 3); HR pixel (x, y),
 * integers in [0, out_w) x [0, out_h), samples the LR point (x/s, y/s) (Eq. 4).
 * Images are planar float32 [3][out_h][out_w], row-major.
 *
 * Conventions for every entry point:
 *  - Every pointer inside gs_gaussians and every image / gradient pointer is a
 *    DEVICE pointer (current CUDA device) unless stated otherwise; the caller
 *    owns all memory. The library allocates no device memory: scratch lives in
 *    a caller-allocated workspace sized by gs_workspace_size.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All calls except gs_count_pairs, gs_sync_status and gs_read_stats are
 *    asynchronous on that stream and may be captured in a CUDA graph.
 *  - Return value: GS_OK, or a status detected on the host before anything was
 *    launched (invalid argument, too-small workspace, CUDA launch error); the
 *    message is available from gs_last_error() (thread-local). Problems found
 *    on the device while the kernels run (an invalid Gaussian parameter, a pair
 *    count above the workspace's capacity) are written to a status word in the
 *    workspace and returned by the next gs_sync_status / gs_read_stats.
 *  - Gradients are overwritten, never accumulated.
 *  - No call waits on another kernel through a spin loop; nothing here traps.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_INVALID = 1,      /* bad argument, or (device) a non-finite / out-of-range parameter */
  GS_ERR_CAPACITY = 2,     /* (device) more (tile, Gaussian) pairs than the workspace holds */
  GS_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed */
  GS_ERR_UNSUPPORTED = 4,  /* a valid request the library does not implement */
  GS_ERR_TIMEOUT = 5,      /* reserved: a bounded device-side wait gave up */
  GS_ERR_INTERNAL = 6      /* an internal consistency check failed */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

typedef enum {
  GS_NORM_DENSITY = 0,  /* Eq. 2 as printed: Z = 1 / (2 pi sx sy sqrt(1 - rho^2)) */
  GS_NORM_PEAK = 1      /* Z = 1: c is the colour at the centre (the "peak RGB" reading) */
} gs_norm;

/* The window R_i of Algorithm 1 over which a Gaussian is summed, as an integer
 * pixel rectangle clamped to the image (c = the HR centre, see gs_align):
 *   SIGMA: c - s k sigma <= x <= c + s k sigma per axis, k = trunc_k (3.0);
 *   RATIO: c - s r L < x < c + s r L per axis, r = trunc_k, L = lr_w for x and
 *          lr_h for y (Algorithm 1's rasterization ratio r, Sec. 3.1 "Fast
 *          Rasterization", read with the HR coordinate compared against the HR
 *          centre and the x half-width taken from the width).
 * Edges are computed in float32 (round to nearest, no fused multiply-add):
 * SIGMA lo = ceil(c - fl(fl(s k) sigma)), hi = floor(c + ...); RATIO
 * lo = floor(c - fl(fl(s r) L)) + 1, hi = ceil(c + ...) - 1. trunc_k <= 0
 * selects the whole image in either mode. */
typedef enum { GS_WINDOW_SIGMA = 0, GS_WINDOW_RATIO = 1 } gs_window;

/* Which LR point HR pixel x samples (Eq. 4):
 *   EQ4:  x / s, as printed; the HR centre is c = fl(s mu);
 *   HALF: (x + 1/2) / s - 1/2, pixel centres aligned across scales; the HR
 *         centre is c = fl(fl(s mu) + (s/2 - 1/2)). */
typedef enum { GS_ALIGN_EQ4 = 0, GS_ALIGN_HALF = 1 } gs_align;

/* How the adjoint sums each Gaussian's record-space moments over its window:
 *   TILE:     one warp per screen tile, one lane per Gaussian of the tile's
 *             list (the tile's upstream gradient read from shared memory by
 *             every lane at once); each (tile, Gaussian) sum is added with
 *             atomics (summation order varies run to run);
 *   GAUSSIAN: one warp per Gaussian over its own window, one fixed summation
 *             order, no atomics: bitwise deterministic (when every image has
 *             ref_grid_m > 0 the warps work in CTAs over 8 x 8 blocks of LR
 *             cells, with the upstream gradient under the block staged in
 *             shared memory; the sums are the same);
 *   QUADRANT: TILE over the 8 x 8 quadrants of 16 x 16 tiles: each quadrant's
 *             warp keeps, from the tile's list, the Gaussians whose window
 *             meets the quadrant, so small windows waste fewer pixel
 *             evaluations at tile edges. Needs tile 16 (GS_ERR_UNSUPPORTED
 *             otherwise);
 *   AUTO:     QUADRANT at tile 16 when every view uses the SIGMA window with
 *             trunc_k > 0 at scale < 6 (small windows, where it measured
 *             faster), else TILE
 *             (GAUSSIAN re-reads grad_out once per (Gaussian, pixel) pair
 *             instead of once per (tile, pixel) and measured slower).
 * All compute the same derivative (Eq. 4 with the windows held fixed). */
typedef enum {
  GS_ADJOINT_AUTO = 0,
  GS_ADJOINT_TILE = 1,
  GS_ADJOINT_GAUSSIAN = 2,
  GS_ADJOINT_QUADRANT = 3
} gs_adjoint;

/* How each screen tile finds the Gaussians whose window meets it:
 *   SORT: every (tile, Gaussian) pair is emitted, radix-sorted by tile and cut
 *         into per-tile runs (needs pair capacity in the workspace);
 *   GRID: grid-implicit binning. A Gaussian's centre is mu = p + o with p on
 *         the reference grid (Sec. 3.2), so the footprint pass records how far
 *         any window reaches past its LR cell (and counts the pairs of every
 *         tile), and each tile enumerates the Gaussians of the LR cells within
 *         that reach and tests their windows. No sort: the forward leaves each
 *         tile's list in the workspace for the adjoint (one 4-byte array of
 *         pair capacity instead of four). Needs ref_grid_m > 0 for every image
 *         and outputs of at most 32767 px a side (GS_ERR_UNSUPPORTED otherwise);
 *   AUTO: GRID where it applies, else SORT.
 * Both give every tile the same Gaussians in the same (ascending id) order, so
 * the forward is bitwise the same. */
typedef enum { GS_BINNING_AUTO = 0, GS_BINNING_SORT = 1, GS_BINNING_GRID = 2 } gs_binning;

/* How the forward raster lays its warps over the screen tiles (a launch
 * parameter: the image is the same bit for bit):
 *   TILE: one warp per tile (tile 16: each thread one column, eight rows);
 *   PAIR: one warp per horizontal pair of 16 x 16 tiles, each thread one
 *         column of each tile: the per-Gaussian work (shared-memory staging,
 *         operand loads) is shared by the two tiles, and each tile is computed
 *         only for the Gaussians whose window meets it. Needs GRID binning and
 *         tile 16 (GS_ERR_UNSUPPORTED otherwise);
 *   AUTO: PAIR with GRID binning at tile 16 when every view uses the SIGMA
 *         window and some view's scale is >= 6 (large windows, where it
 *         measured faster), else TILE. */
typedef enum { GS_RASTER_AUTO = 0, GS_RASTER_TILE = 1, GS_RASTER_PAIR = 2 } gs_raster;

/* The Gaussian primary head's activations (Sec. 3.2, "Gaussian Primary Head"),
 * fused into the render: with a head the five arrays of gs_gaussians hold raw
 * head outputs, mapped per Gaussian to the physical parameters
 *   sigma = sigma_lo + sigma_span * sigmoid(raw)   (sigma_lo >= 0, sigma_span > 0)
 *   rho   = rho_scale * tanh(raw)                  (|rho_scale| <= 1)
 *   c     = sigmoid(raw),  alpha = sigmoid(raw)
 *   o     = offset_scale * raw, or offset_scale * tanh(raw) with offset_tanh = 1
 * (the paper's head: 0, 1, 1, 1, 0). The adjoint then returns dL/d(raw). The
 * window uses sigma and o from a fixed float32 sequence (e^x by Cody-Waite
 * reduction, ln 2 = 0.693359375 - 2.12194442e-4, and the degree-7 Taylor
 * polynomial in Horner form; sigmoid = 1 / (1 + e^-x); tanh = (1 - e^-2|x|) /
 * (1 + e^-2|x|) with the sign of x; every operation rounded to nearest, none
 * fused), so that its integer edges can be reproduced exactly. */
typedef struct gs_head {
  float sigma_lo, sigma_span, rho_scale, offset_scale;
  int32_t offset_tanh;   /* 0 or 1 */
  int32_t reserved[3];   /* must be 0 */
} gs_head;

/* Parameters of n Gaussians, structure of arrays, contiguous, all of element
 * type `dtype`: physical (post-activation) values, or raw head outputs when
 * `head` is set. Device pointers, caller-owned. */
typedef struct gs_gaussians {
  const void* offset; /* [n][2] o (ref_grid_m > 0) or absolute mu (ref_grid_m == 0), LR px */
  const void* sigma;  /* [n][2] (sigma_x, sigma_y) > 0, LR px */
  const void* rho;    /* [n]    correlation, |rho| < 1 */
  const void* rgb;    /* [n][3] colour c */
  const void* alpha;  /* [n]    opacity */
  int64_t n;          /* number of Gaussians; must equal m * lr_h * lr_w when ref_grid_m > 0 */
  int32_t dtype;      /* gs_dtype of all five arrays */
  int32_t ref_grid_m; /* 0, 1, 4, 9 or 16 */
  const gs_head* head; /* host pointer, read during the call; NULL: physical parameters */
} gs_gaussians;

/* One output request. tile and batch are launch parameters (0 = defaults);
 * every view of one batched call must use the same tile. */
typedef struct gs_view {
  int32_t lr_h, lr_w;   /* LR grid (used by the reference grid and for validation) */
  int32_t out_h, out_w; /* HR output size, 1 <= out <= floor(s * lr) + 1 */
  float scale;          /* s > 0 */
  float trunc_k;        /* window parameter (gs_window): k in sigma (3.0) or the ratio r;
                           <= 0: whole image */
  int32_t norm;         /* gs_norm */
  int32_t tile;         /* screen tile edge in HR px: 8, 16 or 32 (0 = 16) */
  int32_t batch;        /* Gaussians staged in shared memory per round of the raster: 0
                           (default: the smaller), 32 or 64 at tile 8 and 16, 64 or 128 at
                           tile 32 (one or two per thread); other values are GS_ERR_INVALID */
  int32_t window;       /* gs_window */
  int32_t align;        /* gs_align */
  int32_t adjoint;      /* gs_adjoint; every view of one batched call must agree */
  int32_t binning;      /* gs_binning; every view of one batched call must agree */
  int32_t row0;         /* first image row this view renders (0: the whole image). The output
                           holds rows row0 .. row0 + out_h - 1 of the image: a horizontal band,
                           with row0 + out_h <= floor(s * lr_h) + 1. Windows and exponents are
                           those of the whole image, so a band renders the image's rows (bit for
                           bit when row0 is a multiple of the tile, else to float32 rounding),
                           and the adjoints of the bands of a partition sum to the whole image's
                           (the row split of one image over several devices, one sum of the
                           gradients). */
  int32_t raster;       /* gs_raster; every view of one batched call must agree */
} gs_view;

/* Counters of the last forward call on a workspace. */
typedef struct gs_stats {
  int64_t tile_pairs;   /* P: (tile, Gaussian) pairs emitted for binning */
  int64_t pixel_pairs;  /* sum_i |R_i|: (Gaussian, HR pixel) pairs inside the windows */
  int64_t capacity;     /* pair capacity of the workspace */
  int64_t n_gaussians;  /* total Gaussians over all images */
  int32_t n_tiles;      /* screen tiles over all images */
  int32_t status;       /* device status word (gs_status) */
  int32_t raster;       /* the forward raster's layout that ran (GS_RASTER_TILE or _PAIR) */
  int32_t adjoint;      /* the adjoint kernel an adjoint with the same views runs
                           (GS_ADJOINT_TILE, _GAUSSIAN or _QUADRANT) */
} gs_stats;

/* Bytes of workspace for rendering n_images images (arrays of n_images entries,
 * host memory) with room for `pair_capacity` (tile, Gaussian) pairs. Returns 0
 * when the arguments are invalid (see gs_last_error). Host-only, no CUDA call. */
size_t gs_workspace_size(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                         int64_t pair_capacity);

/* Exact number of (tile, Gaussian) pairs the render of these images emits.
 * Runs the per-Gaussian footprint pass and the prefix sum on `stream` inside
 * `ws` (which needs capacity >= 0 only), then SYNCHRONISES the stream and
 * writes the count to *pairs_out (host pointer). Device status problems are
 * returned directly. */
gs_status gs_count_pairs(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                         void* ws, size_t ws_bytes, void* stream, int64_t* pairs_out);

/* Forward render of one image (Eq. 4 with the Algorithm-1 window) into `out`
 * (device, float32 [3][out_h][out_w], fully overwritten). `ws` (device,
 * ws_bytes >= gs_workspace_size(1, g, v, cap)) keeps the binned state that
 * gs_render_bwd needs; do not modify it in between. */
gs_status gs_render_fwd(const gs_gaussians* g, const gs_view* v, float* out, void* ws,
                        size_t ws_bytes, void* stream);

/* Adjoint of the last gs_render_fwd on `ws` (same g and v, unchanged values).
 * grad_out: device float32 [3][out_h][out_w], dL/dI. grads: device float32
 * [n][9] = dL/d(o_x, o_y, sigma_x, sigma_y, rho, r, g, b, alpha), overwritten
 * (dL/do = dL/dmu). The windows R_i are held fixed (Eq. 4's sum over a fixed
 * set of pixels per Gaussian). */
gs_status gs_render_bwd(const gs_gaussians* g, const gs_view* v, const float* grad_out,
                        float* grads, void* ws, size_t ws_bytes, void* stream);

/* The forward render (Eq. 4 with the Algorithm-1 window) of n_images
 * independent images, each with its own Gaussians, LR size, output size, scale
 * factor and view options (GSASR's training draws the scale factor at random
 * from [1, 4], Sec. 4.1; a batch may mix scales and sizes),
 * in one chain of launches over a global tile index space: one kernel per
 * stage, whatever the number of images.
 *   g, v, outs: host arrays of n_images entries, read during the call; outs[i]
 *     is device float32 [3][v[i].out_h][v[i].out_w], fully overwritten.
 *   All views must agree on tile, batch, binning and adjoint.
 *   ws: as for gs_render_fwd, sized by gs_workspace_size(n_images, g, v, cap);
 *     it keeps the state gs_render_batched_bwd needs.
 * Errors: invalid arguments return GS_ERR_INVALID before any launch (message
 * in gs_last_error); invalid parameter values and pair-capacity overflow are
 * flagged in the workspace status word (gs_sync_status). Capture-safe: no
 * host synchronisation, no allocation. */
gs_status gs_render_batched(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                            float* const* outs, void* ws, size_t ws_bytes, void* stream);

/* Adjoint of the last gs_render_batched on `ws` (same g and v, unchanged
 * values), windows held fixed as in gs_render_bwd. grad_outs, grads: host
 * arrays of n_images device pointers; grad_outs[i] is float32
 * [3][out_h][out_w] (dL/dI of image i), grads[i] is float32 [n_i][9] in the
 * order of gs_render_bwd, overwritten. Errors as for gs_render_batched.
 * Capture-safe. */
gs_status gs_render_batched_bwd(int32_t n_images, const gs_gaussians* g, const gs_view* v,
                                const float* const* grad_outs, float* const* grads, void* ws,
                                size_t ws_bytes, void* stream);

/* Forward render like gs_render_fwd, for callers that cannot allocate device
 * memory and so cannot supply a workspace: a plugin whose host framework owns
 * all device memory and passes it only input and output pointers, or a
 * real-time loop that must not call cudaMalloc. The GSASR paper has no
 * counterpart to this call; it only changes where the scratch lives.
 *   - Scratch: one static 64 MiB array in device memory (held by every device
 *     that loads libgs.so until the process exits). Renders that need more,
 *     for the per-Gaussian state (about 130 bytes per Gaussian) or for the
 *     (tile, Gaussian) pairs (16 bytes each), are rejected with
 *     GS_ERR_UNSUPPORTED and a message saying how much they need.
 *   - Every call looks up the array's device address in the current device's
 *     context (cudaGetSymbolAddress).
 *   - Each call counts the pairs first, synchronising `stream`, then launches
 *     the render asynchronously on `stream`. Because of that synchronisation
 *     the call can never be made while `stream` is being captured into a
 *     CUDA graph.
 *   - All calls share the one array and each leaves its state there: calls
 *     that overlap on the GPU (other streams, other host threads) race and
 *     give wrong images. gs_render_bwd cannot follow this call.
 *   - Problems the kernels find while they run (an internal check, a count
 *     above the capacity) are left in the array's status word: read them with
 *     gs_noalloc_sync_status after the call.
 * g, v, out: as for gs_render_fwd (device parameters, device output). */
gs_status gs_render_fwd_noalloc(const gs_gaussians* g, const gs_view* v, float* out,
                                void* stream);

/* The device status of the last gs_render_fwd_noalloc, for callers without a
 * workspace pointer: synchronises `stream`, returns the static scratch's status
 * word as gs_sync_status does for a workspace, and resets it to GS_OK. Like the
 * call it follows, it has no counterpart in the paper. */
gs_status gs_noalloc_sync_status(void* stream);

/* Synchronises `stream`, returns the workspace's device status word and resets
 * it to GS_OK. */
gs_status gs_sync_status(void* ws, void* stream);

/* Synchronises `stream` and copies the counters of the last forward on `ws`
 * into *out (host). Does not reset the status. */
gs_status gs_read_stats(void* ws, void* stream, gs_stats* out);

/* Thread-local text of the last host-side error ("" when none). */
const char* gs_last_error(void);

/* Static name of a status code. */
const char* gs_status_string(int32_t status);

/* Number of kernels this library has launched in this process. */
int64_t gs_launch_count(void);

/* Per-kernel timing with CUDA events recorded around each launch on the
 * launching stream (off by default). kernel_mask: bit k times kernel id k (see
 * gs_kernel_name); 0 turns timing off, -1 times every kernel. gs_timing_read
 * synchronises the recorded events, adds each kernel's time since the last
 * read into ms_out[k] and its launches into count_out[k] for k < n, returns
 * the number of kernel ids, and clears the record. Launches made under stream
 * capture record their events as the graph's event-record nodes: every replay
 * records them again, gs_timing_read adds the last replay's times (none before
 * the first replay) and keeps them for the next read, and gs_timing_release
 * drops them (call it before destroying the graph). */
gs_status gs_timing_enable(int32_t kernel_mask);
int32_t gs_timing_read(double* ms_out, int64_t* count_out, int32_t n);
gs_status gs_timing_release(void);
/* Static name of kernel id `id` ("raster_fwd", "raster_bwd", ...); "" for an
 * id out of range. */
const char* gs_kernel_name(int32_t id);

/* Measured throughputs of the units that bound the raster kernels. */
typedef struct gs_peaks {
  double ffma_per_s;              /* scalar FP32 FMA lane-operations per second */
  double ffma2_lane_ops_per_s;    /* FP32 FMA lane-operations per second, packed two-wide */
  double ex2_per_s;               /* MUFU.EX2 lane-operations per second */
  double fwd_pairs_scalar_per_s;  /* forward (Gaussian, pixel) pair mix, scalar FP32 */
  double fwd_pairs_packed_per_s;  /* the same mix in packed FP32x2 */
  int32_t sm_count;
  int32_t reserved;
} gs_peaks;

/* Runs five short throughput kernels on the current device (about 50 ms in
 * total) and fills *out (host). scratch: device buffer of at least
 * 6 * SM count * 256 floats, used only to keep results alive. Synchronous.
 * Not part of the method: it supplies the ALU roofline's denominators. */
gs_status gs_probe_peaks(void* scratch, size_t scratch_bytes, void* stream, gs_peaks* out);

/* Launch parameters picked by gs_tune for one workload. */
typedef struct gs_tuning {
  int32_t tile, batch, binning, adjoint;  /* values for the gs_view fields of the same names */
  float ms;                               /* median time of one call (forward + adjoint if timed) */
  int32_t from_cache;                     /* 1: read from the cache file, nothing was timed */
  int32_t n_timed;                        /* candidates timed */
  int32_t raster;                         /* value for gs_view.raster */
} gs_tuning;

/* Autotuner for the launch parameters (not part of the method: they change the
 * speed, not the result). Times the render of these images, forward and, when
 * grad_outs and grads are non-NULL, the adjoint, on `stream` for each
 * candidate: tile 16, 8 and 32 with batch 32 and 64 (64 and 128 at tile 32),
 * each with SORT binning and, where it applies, GRID binning (raster TILE), and
 * at tile 16 GRID binning with raster PAIR; all with adjoint TILE and, when
 * the adjoint is timed, those at tile 16 also with adjoint QUADRANT; then the
 * fastest of these with adjoint GAUSSIAN.
 * Every candidate runs twice untimed, then `reps` times (1..100) between CUDA
 * events; the median decides. The fastest is returned in *best (host). A
 * candidate whose pairs do not fit the workspace is skipped: size `ws` with
 * gs_workspace_size(..., cap) for cap = gs_count_pairs at tile 8 (the most
 * pairs). outs / grads are overwritten by the timed calls. Synchronous.
 *
 * cache_path (may be NULL): a JSON-lines file, one object per tuned workload,
 *   {"signature": "...", "tile": T, "batch": B, "binning": N, "adjoint": A, "raster": R, "ms": t},
 * the signature being the device name, parameter dtype, fwd or fwd+bwd, and
 * the log2 size classes of the HR pixels, the images and the pairs per pixel.
 * A matching line is returned without timing (from_cache = 1); a new result is
 * appended. g, v, outs, grad_outs, grads: as for gs_render_batched /
 * gs_render_batched_bwd (the views' own tile, batch, binning, adjoint and
 * raster are ignored). */
gs_status gs_tune(int32_t n_images, const gs_gaussians* g, const gs_view* v, float* const* outs,
                  const float* const* grad_outs, float* const* grads, void* ws, size_t ws_bytes,
                  void* stream, int32_t reps, const char* cache_path, gs_tuning* best);

/* Library build identity, e.g. "gs 0.1 sm_103a". */
const char* gs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
