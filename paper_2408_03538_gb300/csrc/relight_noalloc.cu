// Relight backward without any allocation or caller workspace.
//
// Some callers cannot hand us device memory for scratch: for example a renderer plugin or a
// serving process whose host application owns every device allocation through its own
// fixed pool, or a latency-critical loop where a cudaMalloc (which may synchronise the
// device) is not acceptable. For them this entry point keeps its scratch (the per-chunk
// partial sums of dL) in a fixed array in device global memory that is part of the library
// image: every GPU that loads the library holds it until the process exits.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr size_t kScratchFloats = size_t(1) << 18;  // 1 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_relight_scratch[kScratchFloats];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on first use.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_relight_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return PRTGS_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return PRTGS_OK;
}

}  // namespace

extern "C" {

size_t prtgs_relight_backward_noalloc_max_bytes(void) { return kScratchFloats * sizeof(float); }

int prtgs_relight_backward_noalloc(int64_t n, int32_t sh_order, const float* T, int32_t t_channels,
                                   const float* albedo, const float* L, int32_t k, const float* dcolors,
                                   float* d_albedo, float* dT, float* dL, prtgs_stream_t stream) {
  if (n < 0 || k < 0) return PRTGS_ERR_SHAPE;
  if (sh_order < 1 || sh_order > 3) return PRTGS_ERR_UNSUPPORTED;
  if (t_channels != 1 && t_channels != 3) return PRTGS_ERR_SHAPE;
  if (k == 0) return PRTGS_OK;
  if (!dL || (n > 0 && (!T || !albedo || !L || !dcolors || !d_albedo))) return PRTGS_ERR_INVALID_ARG;
  // the scratch holds ceil(n / 2048) * k * 3 * C partial sums
  if (prtgs::relight_backward_workspace(n, sh_order, k) > kScratchFloats * sizeof(float))
    return PRTGS_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != PRTGS_OK) return rc;
  rc = prtgs::relight_backward(n, sh_order, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, scratch,
                               reinterpret_cast<cudaStream_t>(stream));
  if (rc != PRTGS_OK) return rc;
  if (cudaPeekAtLastError() != cudaSuccess) {
    (void)cudaGetLastError();
    return PRTGS_ERR_CUDA;
  }
  return PRTGS_OK;
}

}  // extern "C"
