// Throughput probes of the GB300 units that bound the raster kernels: FP32
// FFMA (scalar and packed two-wide), MUFU.EX2, and the forward's per-pair
// instruction mix (scalar and packed). Each kernel runs independent chains in
// registers long enough to hide latency; results go to a caller buffer only to
// keep the work alive.
#include <cuda_runtime.h>

#include "../../include/gs.h"
#include "gs_internal.cuh"

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) p_ffma(float* out, int iters) {
  float a[8];
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 1e-3f + j;
  const float b = 1.0000001f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.f;
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) p_ffma2(float* out, int iters) {
  float2 a[8];
  for (int j = 0; j < 8; ++j) a[j] = make_float2(threadIdx.x * 1e-3f + j, j * 0.5f);
  const float2 b = make_float2(1.0000001f, 0.9999999f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = __ffma2_rn(a[j], b, c);
  }
  float s = 0.f;
  for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) p_ex2(float* out, int iters) {
  float a[8];
  for (int j = 0; j < 8; ++j) a[j] = (threadIdx.x & 7) * 0.1f + j * 0.01f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = gs::ex2_approx(-a[j]);
  }
  float s = 0.f;
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Forward pair mix: d = X - K, w = 2^(R - d^2), acc += c w (3 channels).
__global__ void __launch_bounds__(kThreads) p_mix(float* out, int iters) {
  float X = 0.001f * threadIdx.x, cr = 0.3f, cg = 0.4f, cb = 0.5f;
  float acc[8][3], K[8], R[8];
  for (int j = 0; j < 8; ++j) {
    acc[j][0] = acc[j][1] = acc[j][2] = 0.f;
    K[j] = 0.1f * j;
    R[j] = -0.2f * j;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float d = X - K[j];
      const float w = gs::ex2_approx(fmaf(-d, d, R[j]));
      acc[j][0] = fmaf(cr, w, acc[j][0]);
      acc[j][1] = fmaf(cg, w, acc[j][1]);
      acc[j][2] = fmaf(cb, w, acc[j][2]);
    }
    X += 1e-6f;
    cr += 1e-7f;
  }
  float s = 0.f;
  for (int j = 0; j < 8; ++j) s += acc[j][0] + acc[j][1] + acc[j][2];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) p_mix2(float* out, int iters) {
  float X = 0.001f * threadIdx.x, cr = 0.3f, cg = 0.4f, cb = 0.5f;
  float2 acc[4][3], nK[4], R[4];
  for (int j = 0; j < 4; ++j) {
    acc[j][0] = acc[j][1] = acc[j][2] = make_float2(0.f, 0.f);
    nK[j] = make_float2(-0.1f * j, -0.1f * j - 0.05f);
    R[j] = make_float2(-0.2f * j, -0.2f * j - 0.1f);
  }
  for (int i = 0; i < iters; ++i) {
    const float2 X2 = make_float2(X, X);
    const float2 c0 = make_float2(cr, cr), c1 = make_float2(cg, cg), c2 = make_float2(cb, cb);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 d = __fadd2_rn(X2, nK[j]);
      const float2 e = __ffma2_rn(make_float2(-d.x, -d.y), d, R[j]);
      const float2 w = make_float2(gs::ex2_approx(e.x), gs::ex2_approx(e.y));
      acc[j][0] = __ffma2_rn(c0, w, acc[j][0]);
      acc[j][1] = __ffma2_rn(c1, w, acc[j][1]);
      acc[j][2] = __ffma2_rn(c2, w, acc[j][2]);
    }
    X += 1e-6f;
    cr += 1e-7f;
  }
  float s = 0.f;
  for (int j = 0; j < 4; ++j)
    s += acc[j][0].x + acc[j][1].x + acc[j][2].x + acc[j][0].y + acc[j][1].y + acc[j][2].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class K>
double time_kernel(K kernel, int blocks, float* out, int iters, cudaStream_t s, cudaError_t* err) {
  cudaEvent_t a, b;
  if ((*err = cudaEventCreate(&a)) != cudaSuccess) return 0.0;
  if ((*err = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return 0.0; }
  kernel<<<blocks, kThreads, 0, s>>>(out, iters / 10);   // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(a, s);
    kernel<<<blocks, kThreads, 0, s>>>(out, iters);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  *err = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best * 1e-3;
}

}  // namespace

extern "C" gs_status gs_probe_peaks(void* scratch, size_t scratch_bytes, void* stream,
                                    gs_peaks* out) {
  if (!out) return GS_ERR_INVALID;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int blocks = sms * 6;
  if (!scratch || scratch_bytes < (size_t)blocks * kThreads * sizeof(float)) return GS_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* buf = static_cast<float*>(scratch);
  const double lanes = (double)blocks * kThreads;
  const int it = 20000;
  double t;
  t = time_kernel(p_ffma, blocks, buf, it, s, &e);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  out->ffma_per_s = lanes * 8 * it / t;
  t = time_kernel(p_ffma2, blocks, buf, it, s, &e);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  out->ffma2_lane_ops_per_s = lanes * 16 * it / t;
  t = time_kernel(p_ex2, blocks, buf, it, s, &e);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  out->ex2_per_s = lanes * 8 * it / t;
  t = time_kernel(p_mix, blocks, buf, it / 2, s, &e);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  out->fwd_pairs_scalar_per_s = lanes * 8 * (it / 2) / t;
  t = time_kernel(p_mix2, blocks, buf, it / 2, s, &e);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  out->fwd_pairs_packed_per_s = lanes * 8 * (it / 2) / t;
  out->sm_count = sms;
  return GS_OK;
}
