// LBVH over the Gaussians' 3-sigma boxes (Sec. 4.4: ray tracing "constructed upon the BVH").
//
// Steps: per-scene centre bounds -> 30-bit Morton codes (FP32 quantisation with explicit
// round-to-nearest ops, so the integer result is reproducible) -> stable LSD radix sort ->
// Karras (2012) split search, one thread per internal node -> traversal records and leaf
// boxes (Eq. 2: Sigma = R S S^T R^T, half-extent_a = 3 sqrt(Sigma_aa)) -> bottom-up box
// refit with per-node arrival counters.
#include "common.cuh"
#include "internal.h"

namespace prtgs {

size_t bvh_bytes(int64_t n, int32_t n_scenes) {
  int64_t ni = n > 1 ? n - 1 : 1;
  return align_up(sizeof(uint64_t) * n) + align_up(sizeof(int32_t) * n) + align_up(sizeof(float) * 16 * ni) +
         align_up(sizeof(float) * 16 * n) + align_up(sizeof(int32_t) * n) + align_up(sizeof(int32_t) * n_scenes);
}

int bvh_layout(void* buffer, int64_t n, int32_t n_scenes, const int64_t* scene_offsets, prtgs_bvh* out) {
  int64_t ni = n > 1 ? n - 1 : 1;
  Carver c(buffer);
  out->n = n;
  out->n_scenes = n_scenes;
  out->reserved = 0;
  out->keys = c.take<uint64_t>(n);
  out->order = c.take<int32_t>(n);
  out->nodes = c.take<float>(16 * ni);
  out->records = c.take<float>(16 * n);
  out->leaf_parent = c.take<int32_t>(n);
  out->roots = c.take<int32_t>(n_scenes);
  out->scene_offsets = scene_offsets;
  return PRTGS_OK;
}

static int scene_bits(int32_t n_scenes) {
  int b = 0;
  while ((1 << b) < n_scenes) ++b;
  return b;
}

size_t build_bvh_workspace(int64_t n, int32_t n_scenes) {
  int64_t ni = n > 1 ? n - 1 : 1;
  return align_up(sizeof(uint32_t) * 6 * n_scenes) + 2 * align_up(sizeof(uint64_t) * n) +
         2 * align_up(sizeof(int32_t) * n) + align_up(sizeof(uint32_t) * ni) + radix_sort_workspace(n);
}

// ---- bounds --------------------------------------------------------------------------------
constexpr int kBoundsThreads = 256;
constexpr int kBoundsItems = 8;

__global__ void k_bounds_init(uint32_t* bounds, int n_scenes) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_scenes * 6) bounds[i] = (i % 6) < 3 ? 0xffffffffu : 0u;  // lo as ordered max, hi as 0
}

__global__ void k_bounds(const float* __restrict__ means, int64_t n, const int64_t* __restrict__ offsets,
                         int n_scenes, uint32_t* __restrict__ bounds) {
  __shared__ uint32_t red[6][kBoundsThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kBoundsThreads * kBoundsItems;
  if (base >= n) return;
  int64_t last = base + kBoundsThreads * kBoundsItems - 1;
  if (last >= n) last = n - 1;
  int b0 = find_scene(offsets, n_scenes, base);
  bool uniform = find_scene(offsets, n_scenes, last) == b0;
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int k = 0; k < kBoundsItems; ++k) {
    int64_t i = base + (int64_t)k * kBoundsThreads + threadIdx.x;
    if (i >= n) break;
    int b = uniform ? b0 : find_scene(offsets, n_scenes, i);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      uint32_t u = float_to_ordered(means[3 * i + a]);
      if (uniform) {
        lo[a] = min(lo[a], u);
        hi[a] = max(hi[a], u);
      } else {
        atomicMin(&bounds[6 * b + a], u);
        atomicMax(&bounds[6 * b + 3 + a], u);
      }
    }
  }
  if (!uniform) return;  // uniform over the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    for (int off = 16; off > 0; off >>= 1) {
      lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
      hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
    }
    if (lane == 0) {
      red[a][warp] = lo[a];
      red[3 + a][warp] = hi[a];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    int a = threadIdx.x;
    uint32_t v = red[a][0];
    for (int w = 1; w < kBoundsThreads / 32; ++w) v = a < 3 ? min(v, red[a][w]) : max(v, red[a][w]);
    if (a < 3) atomicMin(&bounds[6 * b0 + a], v); else atomicMax(&bounds[6 * b0 + a], v);
  }
}

// ---- Morton keys ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(const float* __restrict__ means, int64_t n, const int64_t* __restrict__ offsets,
                         int n_scenes, const uint32_t* __restrict__ bounds, uint64_t* __restrict__ keys,
                         int32_t* __restrict__ vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = find_scene(offsets, n_scenes, i);
  uint32_t q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float lo = ordered_to_float(bounds[6 * b + a]);
    float hi = ordered_to_float(bounds[6 * b + 3 + a]);
    float ext = __fsub_rn(hi, lo);
    float sc = ext > 0.0f ? __fdiv_rn(1024.0f, ext) : 0.0f;
    float m = __fmul_rn(__fsub_rn(means[3 * i + a], lo), sc);
    float f = floorf(m);
    int v = (int)f;
    v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
    q[a] = (uint32_t)v;
  }
  uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
  keys[i] = ((uint64_t)b << kSceneShift) | ((uint64_t)code << kCodeShift) | (uint64_t)(i - offsets[b]);
  vals[i] = (int32_t)i;
}

// ---- Karras split search -------------------------------------------------------------------
__device__ __forceinline__ int key_delta(const uint64_t* __restrict__ keys, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  return __clzll(keys[i] ^ keys[j]);
}

__device__ __forceinline__ void node_set_int(float* nodes, int64_t node, int slot, int32_t v) {
  nodes[16 * node + slot] = __int_as_float(v);
}

__global__ void k_karras(const uint64_t* __restrict__ keys, int64_t n, const int64_t* __restrict__ offsets,
                         int n_scenes, float* __restrict__ nodes, int32_t* __restrict__ leaf_parent,
                         int32_t* __restrict__ roots) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (key_delta(keys, n, i, i + 1) - key_delta(keys, n, i, i - 1)) > 0 ? 1 : -1;
  int dmin = key_delta(keys, n, i, i - d);
  int64_t lmax = 2;
  while (key_delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (key_delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = key_delta(keys, n, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (key_delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  int32_t left = (lo == gamma) ? ~(int32_t)gamma : (int32_t)gamma;
  int32_t right = (hi == gamma + 1) ? ~(int32_t)(gamma + 1) : (int32_t)(gamma + 1);
  if (gamma < 0 || gamma + 1 >= n) return;  // cannot happen for unique sorted keys
  node_set_int(nodes, i, 12, left);
  node_set_int(nodes, i, 13, right);
  if (left >= 0) node_set_int(nodes, left, 14, (int32_t)i); else leaf_parent[gamma] = (int32_t)i;
  if (right >= 0) node_set_int(nodes, right, 14, (int32_t)i); else leaf_parent[gamma + 1] = (int32_t)i;
  if (i == 0) node_set_int(nodes, 0, 14, -1);
  int b = find_scene(offsets, n_scenes, lo);
  if (offsets[b] == lo && offsets[b + 1] - 1 == hi) roots[b] = (int32_t)i;
}

__global__ void k_small_scene_roots(const int64_t* __restrict__ offsets, int n_scenes, int64_t n,
                                    int32_t* __restrict__ roots, int32_t* __restrict__ leaf_parent) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_scenes) return;
  int64_t s0 = offsets[b], s1 = offsets[b + 1];
  if (s1 - s0 == 1) roots[b] = ~(int32_t)s0;
  else if (s1 == s0) roots[b] = INT32_MIN;
  if (n == 1 && b == 0) leaf_parent[0] = -1;
}

// ---- records, leaf boxes and refit ---------------------------------------------------------
__global__ void k_pack_refit(const float* __restrict__ means, const float* __restrict__ scales,
                             const float* __restrict__ quats, const float* __restrict__ opacity,
                             const float* __restrict__ normals, int64_t n, const int32_t* __restrict__ order,
                             float* __restrict__ records, float* nodes, const int32_t* __restrict__ leaf_parent,
                             uint32_t* counters, int32_t* status) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t g = order[p];
  float mx = means[3 * g], my = means[3 * g + 1], mz = means[3 * g + 2];
  float s0 = scales[3 * g], s1 = scales[3 * g + 1], s2 = scales[3 * g + 2];
  float qw = quats[4 * g], qx = quats[4 * g + 1], qy = quats[4 * g + 2], qz = quats[4 * g + 3];
  float op = opacity[g];
  float nx = normals[3 * g], ny = normals[3 * g + 1], nz = normals[3 * g + 2];
  float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  bool ok = isfinite(mx) && isfinite(my) && isfinite(mz) && s0 > 0.f && s1 > 0.f && s2 > 0.f && isfinite(s0) &&
            isfinite(s1) && isfinite(s2) && op >= 0.f && op < 1.f && qn > 0.f && isfinite(qn) && isfinite(nx) &&
            isfinite(ny) && isfinite(nz);
  if (!ok) {
    set_status(status, PRTGS_STATUS_NONFINITE);
    // keep the tree well formed: a tiny transparent Gaussian at a finite place
    mx = isfinite(mx) ? mx : 0.f; my = isfinite(my) ? my : 0.f; mz = isfinite(mz) ? mz : 0.f;
    s0 = s1 = s2 = 1e-6f; op = 0.f; qw = 1.f; qx = qy = qz = 0.f; qn = 1.f;
  }
  qw /= qn; qx /= qn; qy /= qn; qz /= qn;
  // R(q), Eq. 2
  float R[3][3];
  R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); R[0][1] = 2.f * (qx * qy - qw * qz); R[0][2] = 2.f * (qx * qz + qw * qy);
  R[1][0] = 2.f * (qx * qy + qw * qz); R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); R[1][2] = 2.f * (qy * qz - qw * qx);
  R[2][0] = 2.f * (qx * qz - qw * qy); R[2][1] = 2.f * (qy * qz + qw * qx); R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
  float inv[3] = {1.f / s0, 1.f / s1, 1.f / s2};
  float s2v[3] = {s0 * s0, s1 * s1, s2 * s2};
  // whitening A = diag(1/s) R^T: row k = (column k of R) / s_k
  float A[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[3 * k + j] = R[j][k] * inv[k];
  float4* rec = reinterpret_cast<float4*>(records) + 4 * p;
  rec[0] = make_float4(mx, my, mz, op);
  rec[1] = make_float4(A[0], A[1], A[2], A[3]);
  rec[2] = make_float4(A[4], A[5], A[6], A[7]);
  rec[3] = make_float4(A[8], nx, ny, nz);
  // 3-sigma box, padded so that FP32 rounding can only enlarge it
  float bx[6];
  float pad_abs = 1e-5f * (fabsf(mx) + fabsf(my) + fabsf(mz)) + 1e-7f;
  float m3[3] = {mx, my, mz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float var = R[a][0] * R[a][0] * s2v[0] + R[a][1] * R[a][1] * s2v[1] + R[a][2] * R[a][2] * s2v[2];
    float h = 3.0f * sqrtf(var) * 1.0001f + pad_abs;
    bx[a] = m3[a] - h;
    bx[3 + a] = m3[a] + h;
  }
  // bottom-up refit: the second child to arrive at a node writes the union into its parent
  int32_t parent = leaf_parent[p];
  int32_t child = ~(int32_t)p;
  for (int level = 0; parent >= 0; ++level) {
    if ((int64_t)parent >= n - 1 || level > 2 * kStackDepth) {  // never for a well-formed tree
      set_status(status, PRTGS_STATUS_BAD_INDEX);
      return;
    }
    float* pn = nodes + 16 * (int64_t)parent;
    int slot = (__float_as_int(__ldcg(pn + 12)) == child) ? 0 : 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) __stcg(pn + slot + k, bx[k]);
    __threadfence();
    uint32_t prev = atomicAdd(&counters[parent], 1u);
    if (prev == 0) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      bx[k] = fminf(__ldcg(pn + k), __ldcg(pn + 6 + k));
      bx[3 + k] = fmaxf(__ldcg(pn + 3 + k), __ldcg(pn + 9 + k));
    }
    child = parent;
    parent = __float_as_int(__ldcg(pn + 14));
  }
}

int build_bvh(const prtgs_gaussians* g, prtgs_bvh* bvh, int32_t* status, void* ws, cudaStream_t stream) {
  const int64_t n = g->n;
  const int nsc = bvh->n_scenes;
  if (n == 0) return PRTGS_OK;
  Carver c(ws);
  uint32_t* bounds = c.take<uint32_t>(6 * (size_t)nsc);
  uint64_t* keys_x = c.take<uint64_t>(n);
  uint64_t* keys_y = c.take<uint64_t>(n);
  int32_t* vals_x = c.take<int32_t>(n);
  int32_t* vals_y = c.take<int32_t>(n);
  int64_t ni = n > 1 ? n - 1 : 1;
  uint32_t* counters = c.take<uint32_t>(ni);
  void* sort_ws = c.take<char>(radix_sort_workspace(n));

  k_bounds_init<<<(6 * nsc + 255) / 256, 256, 0, counted(stream)>>>(bounds, nsc);
  int64_t nb = (n + kBoundsThreads * kBoundsItems - 1) / (kBoundsThreads * kBoundsItems);
  k_bounds<<<(unsigned)nb, kBoundsThreads, 0, counted(stream)>>>(g->means, n, bvh->scene_offsets, nsc, bounds);
  k_morton<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(g->means, n, bvh->scene_offsets, nsc, bounds, keys_x,
                                                           vals_x);
  PRTGS_CHECK_LAUNCH();
  // the low 27 bits (index within the scene) are already in order: sort the code and scene bits
  int rc = radix_sort_pairs(keys_x, vals_x, bvh->keys, bvh->order, keys_y, vals_y, n, nullptr, kCodeShift,
                            kSceneShift + scene_bits(nsc), sort_ws, stream);
  if (rc != PRTGS_OK) return rc;
  if (n > 1)
    k_karras<<<(unsigned)((n - 1 + 255) / 256), 256, 0, counted(stream)>>>(bvh->keys, n, bvh->scene_offsets, nsc,
                                                                   bvh->nodes, bvh->leaf_parent, bvh->roots);
  k_small_scene_roots<<<(nsc + 127) / 128, 128, 0, counted(stream)>>>(bvh->scene_offsets, nsc, n, bvh->roots,
                                                              bvh->leaf_parent);
  cudaMemsetAsync(counters, 0, sizeof(uint32_t) * ni, stream);
  k_pack_refit<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(g->means, g->scales, g->quats, g->opacity,
                                                               g->normals, n, bvh->order, bvh->records, bvh->nodes,
                                                               bvh->leaf_parent, counters, status);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

}  // namespace prtgs
