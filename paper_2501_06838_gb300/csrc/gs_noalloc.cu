// gs_render_fwd_noalloc: the forward render for callers that cannot allocate
// device memory. Examples: a plugin or operator that a host framework hands
// only input and output pointers, with every other byte of device memory owned
// by that framework's pre-reserved pool; a real-time loop where cudaMalloc
// (which can synchronise the whole device) is not allowed once the loop runs.
// Such callers cannot provide the workspace that gs_render_fwd needs, so this
// entry point keeps its scratch in one fixed array in device memory instead.
//
// The array is a file-scope __device__ variable of kNoallocScratchBytes. Every
// GPU that loads this module holds it until the process exits. Host code never
// dereferences or passes the symbol itself (on the host it is only a stand-in,
// not a device address): every call looks up the array's device address on the
// current device with cudaGetSymbolAddress, so that a context created again
// (after cudaDeviceReset, say) never leaves a stale address behind.
#include <cstdio>

#include "../../include/gs.h"
#include "gs_internal.cuh"

namespace gs {
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

gs_status noalloc_fail(gs_status st, const char* msg) {
  gs::set_last_error(msg);
  return st;
}

// Device address of the scratch array in the current device's context.
gs_status noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    char buf[256];
    std::snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the static scratch failed: %s",
                  cudaGetErrorString(e));
    return noalloc_fail(GS_ERR_CUDA, buf);
  }
  *out = p;
  return GS_OK;
}

}  // namespace

extern "C" gs_status gs_render_fwd_noalloc(const gs_gaussians* g, const gs_view* v, float* out,
                                           void* stream) {
  void* ws = nullptr;
  gs_status st = noalloc_scratch(&ws);
  if (st != GS_OK) return st;
  // Fixed part (per-Gaussian records, image table, tile ranges) must fit.
  const size_t fixed = gs_workspace_size(1, g, v, 0);
  if (fixed == 0) return GS_ERR_INVALID;   // message set by the validation
  char buf[320];
  if (fixed > kNoallocScratchBytes) {
    std::snprintf(buf, sizeof(buf),
                  "gs_render_fwd_noalloc: %lld Gaussians / %dx%d output need %zu bytes of scratch "
                  "before any pair; the static scratch holds %zu bytes",
                  (long long)g->n, v->out_w, v->out_h, fixed, kNoallocScratchBytes);
    return noalloc_fail(GS_ERR_UNSUPPORTED, buf);
  }
  // Count the (tile, Gaussian) pairs in the scratch (synchronises `stream`)
  // and reject the call if they do not fit, before anything is rendered.
  int64_t pairs = 0;
  st = gs_count_pairs(1, g, v, ws, kNoallocScratchBytes, stream, &pairs);
  if (st != GS_OK) return st;
  const size_t need = gs_workspace_size(1, g, v, pairs);
  if (need == 0 || need > kNoallocScratchBytes) {
    // the count itself flagged the overflow in the array's status word; the
    // refusal reports it, so clear it for the next status read
    gs_sync_status(ws, stream);
    std::snprintf(buf, sizeof(buf),
                  "gs_render_fwd_noalloc: %lld (tile, Gaussian) pairs need %zu bytes of scratch; "
                  "the static scratch holds %zu bytes",
                  (long long)pairs, need, kNoallocScratchBytes);
    return noalloc_fail(GS_ERR_UNSUPPORTED, buf);
  }
  // The render resets the scratch header itself and clears its tile ranges;
  // every other scratch byte is written before it is read.
  return gs_render_fwd(g, v, out, ws, kNoallocScratchBytes, stream);
}

// The status word the kernels of the last gs_render_fwd_noalloc left in the
// static scratch (a count above the capacity, an internal check): the caller
// has no workspace pointer to give gs_sync_status, so this reads the scratch's
// header through the same symbol lookup, then resets it.
extern "C" gs_status gs_noalloc_sync_status(void* stream) {
  void* ws = nullptr;
  const gs_status st = noalloc_scratch(&ws);
  if (st != GS_OK) return st;
  return gs_sync_status(ws, stream);
}
