// Autotuning of launch variants: each tunable call has variants that give the same results
// (within the stated tolerances); prtgs_autotune times every variant on the caller's own inputs
// with CUDA events on the caller's stream and reports the times as JSON, so that a caller (the
// Python side keeps a cache keyed by device and shape bucket) can pass the fastest to later calls.
//
//   PRTGS_TUNE_TRANSFER   the walk of the transfer: warp packets with packet_dirs directions per
//                         work item (the work tile is 32 receivers x packet_dirs directions:
//                         1, 2, 4, 8, 16, 32), or one ray per lane (reported as 0)
//   PRTGS_TUNE_RELIGHT    relight precision among the FP32-accurate ones: FP32 CUDA cores or the
//                         3-term BF16 split on the tensor cores (where the shape fits them)
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace {

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Timer() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// Mean milliseconds of `repeats` runs of fn after one untimed run; negative on an error.
template <class F>
float time_variant(F fn, int repeats, cudaStream_t s, Timer& t, int* rc) {
  *rc = fn();
  if (*rc != PRTGS_OK) return -1.f;
  cudaEventRecord(t.e0, s);
  for (int r = 0; r < repeats; ++r) {
    *rc = fn();
    if (*rc != PRTGS_OK) return -1.f;
  }
  cudaEventRecord(t.e1, s);
  if (cudaEventSynchronize(t.e1) != cudaSuccess) {
    (void)cudaGetLastError();
    *rc = PRTGS_ERR_CUDA;
    return -1.f;
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, t.e0, t.e1);
  return ms / (float)repeats;
}

// Appends to the JSON buffer; false when it no longer fits.
bool put(char* buf, size_t cap, size_t& len, const char* fmt, double a = 0.0, double b = 0.0) {
  const int w = snprintf(buf + len, cap > len ? cap - len : 0, fmt, a, b);
  if (w < 0 || (size_t)w >= (cap > len ? cap - len : 0)) return false;
  len += (size_t)w;
  return true;
}

}  // namespace

extern "C" {

int prtgs_autotune(int32_t kernel_id, const void* args, int32_t repeats, prtgs_stream_t stream, int32_t* best,
                   char* out_json, size_t json_bytes) {
  if (!args || !best || !out_json || json_bytes < 64 || repeats < 1 || repeats > 1000) return PRTGS_ERR_INVALID_ARG;
  if (kernel_id != PRTGS_TUNE_TRANSFER && kernel_id != PRTGS_TUNE_RELIGHT) return PRTGS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Timer t;
  if (!t.e0 || !t.e1) return PRTGS_ERR_CUDA;
  size_t len = 0;
  out_json[0] = 0;
  int rc = PRTGS_OK;
  float best_ms = -1.f;
  if (kernel_id == PRTGS_TUNE_TRANSFER) {
    const prtgs_tune_transfer* a = static_cast<const prtgs_tune_transfer*>(args);
    if (!a->g || !a->bvh) return PRTGS_ERR_INVALID_ARG;
    prtgs_transfer_params p = a->params;
    if (!put(out_json, json_bytes, len,
             "{\"kernel\": \"transfer\", \"variant\": \"packet_dirs\", \"shape\": {\"n\": %.0f, \"n_dirs\": %.0f",
             (double)a->g->n, (double)p.n_dirs) ||
        !put(out_json, json_bytes, len, ", \"sh_order\": %.0f, \"flags\": %.0f}, \"ms\": {", (double)p.sh_order,
             (double)p.flags))
      return PRTGS_ERR_INVALID_ARG;
    const int dirs[] = {1, 2, 4, 8, 16, 32, 0};  // 0: the per-ray walk
    for (int v = 0; v < 7; ++v) {
      p.walk = dirs[v] == 0 ? 1 : 0;
      p.packet_dirs = dirs[v];
      const float ms = time_variant(
          [&]() {
            return prtgs_precompute_transfer(a->g, a->bvh, &p, a->P, a->T, a->idx, a->M, a->n_glossy, a->status,
                                             a->workspace, a->workspace_bytes, stream);
          },
          repeats, s, t, &rc);
      if (rc != PRTGS_OK) return rc;
      if (!put(out_json, json_bytes, len, v ? ", \"%.0f\": %.4f" : "\"%.0f\": %.4f", (double)dirs[v], (double)ms))
        return PRTGS_ERR_INVALID_ARG;
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        *best = dirs[v];
      }
    }
  } else if (kernel_id == PRTGS_TUNE_RELIGHT) {
    const prtgs_tune_relight* a = static_cast<const prtgs_tune_relight*>(args);
    if (!put(out_json, json_bytes, len,
             "{\"kernel\": \"relight\", \"variant\": \"precision\", \"shape\": {\"n\": %.0f, \"k\": %.0f", (double)a->n,
             (double)a->k) ||
        !put(out_json, json_bytes, len, ", \"t_channels\": %.0f, \"n_scenes\": %.0f}, \"ms\": {",
             (double)a->t_channels, (double)a->n_scenes))
      return PRTGS_ERR_INVALID_ARG;
    int precs[2] = {PRTGS_PREC_FP32, PRTGS_PREC_BF16X3};
    const int nv = prtgs::relight_tc_fits(a->sh_order, a->k, a->t_channels, PRTGS_PREC_BF16X3) ? 2 : 1;
    for (int v = 0; v < nv; ++v) {
      const float ms = time_variant(
          [&]() {
            return prtgs_relight_batched(a->n, a->sh_order, a->T, a->t_channels, a->albedo, a->scene_offsets,
                                         a->n_scenes, a->L, a->k, precs[v], a->colors, a->status,
                                         PRTGS_TC_WAIT_POLLS, stream);
          },
          repeats, s, t, &rc);
      if (rc != PRTGS_OK) return rc;
      if (!put(out_json, json_bytes, len, v ? ", \"%.0f\": %.4f" : "\"%.0f\": %.4f", (double)precs[v], (double)ms))
        return PRTGS_ERR_INVALID_ARG;
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        *best = precs[v];
      }
    }
  } else {
    return PRTGS_ERR_INVALID_ARG;
  }
  if (!put(out_json, json_bytes, len, "}, \"best\": %.0f}", (double)*best)) return PRTGS_ERR_INVALID_ARG;
  return PRTGS_OK;
}

}  // extern "C"
