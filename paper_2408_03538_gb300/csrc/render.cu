// Tile-binned splat rasteriser (Sec. 3.1: Eq. 2 covariance, Eq. 3 EWA projection, Eq. 4
// front-to-back alpha blending) with the 3DGS conventions the paper builds on, and its
// backward pass.
//
// Forward: k_preprocess (one thread per Gaussian) -> inclusive scan of the touched-tile
// counts -> k_duplicate writes (tile << 32 | depth bits, Gaussian) pairs -> radix sort on
// the device-side pair count -> k_ranges -> k_composite (one 16x16-pixel tile per block,
// Gaussians staged through shared memory in batches of 256, evaluated once for a group of
// up to 8 light colour sets).
// Backward: k_composite_bwd walks each pixel's list back to front from its last
// contributor, reduces per-Gaussian gradients across the warp and then the block in shared
// memory before one global atomic per Gaussian and batch; k_preprocess_bwd maps the 2D
// gradients to means, scales and rotations.
#include "common.cuh"
#include "internal.h"

namespace prtgs {

constexpr int kTile = 16;
constexpr int kTileThreads = kTile * kTile;
constexpr float kNear = 0.2f;
constexpr float kDilation = 0.3f;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

struct Cam {
  float r[9], t[3];
  float fx, fy, cx, cy;
  int W, H, gx, gy;
  float near_plane;
  float limx, limy;
};

static Cam make_cam(const prtgs_camera* c) {
  Cam k;
  for (int i = 0; i < 9; ++i) k.r[i] = c->rot[i];
  for (int i = 0; i < 3; ++i) k.t[i] = c->trans[i];
  k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy;
  k.W = c->width; k.H = c->height;
  k.gx = (c->width + kTile - 1) / kTile;
  k.gy = (c->height + kTile - 1) / kTile;
  k.near_plane = c->near_plane > 0.f ? c->near_plane : kNear;
  k.limx = 1.3f * (0.5f * (float)c->width / c->fx);
  k.limy = 1.3f * (0.5f * (float)c->height / c->fy);
  return k;
}

// Where each Gaussian's camera, colours and image live. OneView: a single scene (colours
// [k][n][3], image [k][3][H][W]). ManyViews: scene b holds Gaussians offs[b] .. offs[b+1], has its
// own camera (every camera has the same image size), its colours are the [k][n_b][3] block at
// 3 k offs[b] (the layout of prtgs_relight_batched) and its images the [k][3][H][W] block b. The
// cameras travel by value in the kernel parameters (no device copy, graph-capturable).
struct OneView {
  Cam c;
  __device__ __forceinline__ int scene_of(int64_t) const { return 0; }
  __device__ __forceinline__ const Cam& cam(int) const { return c; }
  __device__ __forceinline__ int64_t first(int) const { return 0; }
  __device__ __forceinline__ int64_t count(int, int64_t n) const { return n; }
};

struct ManyViews {
  Cam c[kMaxScenes];
  const int64_t* offs;
  int B;
  __device__ __forceinline__ int scene_of(int64_t i) const { return find_scene(offs, B, i); }
  __device__ __forceinline__ const Cam& cam(int b) const { return c[b]; }
  __device__ __forceinline__ int64_t first(int b) const { return offs[b]; }
  __device__ __forceinline__ int64_t count(int b, int64_t) const { return offs[b + 1] - offs[b]; }
};

// Colour of light l, channel ch of Gaussian g (in scene b).
template <class V>
__device__ __forceinline__ int64_t color_at(const V& v, int b, int64_t g, int l, int k, int64_t n) {
  const int64_t o = v.first(b);
  return 3 * (int64_t)k * o + ((int64_t)l * v.count(b, n) + (g - o)) * 3;
}

size_t render_state_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  return render_state_bytes_batched(n, 1, width, height, max_pairs);
}

int render_state_layout(void* buffer, int64_t n, int32_t width, int32_t height, int64_t max_pairs,
                        prtgs_render_state* out) {
  return render_state_layout_batched(buffer, n, 1, width, height, max_pairs, out);
}

// B scenes of one image size: tile ranges, final transmittance and contributor counts per scene.
size_t render_state_bytes_batched(int64_t n, int32_t B, int32_t width, int32_t height, int64_t max_pairs) {
  int64_t tiles = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile) * B;
  int64_t px = (int64_t)width * height * B;
  return align_up(sizeof(float) * 2 * n) + align_up(sizeof(float) * 4 * n) + align_up(sizeof(float) * n) +
         align_up(sizeof(int32_t) * n) + align_up(sizeof(uint32_t) * n) + align_up(sizeof(uint64_t) * max_pairs) +
         align_up(sizeof(int32_t) * max_pairs) + align_up(sizeof(uint32_t) * 2 * tiles) +
         align_up(sizeof(float) * px) + align_up(sizeof(int32_t) * px) + align_up(sizeof(uint32_t));
}

int render_state_layout_batched(void* buffer, int64_t n, int32_t B, int32_t width, int32_t height,
                                int64_t max_pairs, prtgs_render_state* out) {
  int64_t tiles = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile) * B;
  int64_t px = (int64_t)width * height * B;
  Carver c(buffer);
  out->n_scenes = B;
  out->n = n;
  out->max_pairs = max_pairs;
  out->width = width;
  out->height = height;
  out->tiles_x = (width + kTile - 1) / kTile;
  out->tiles_y = (height + kTile - 1) / kTile;
  out->mean2d = c.take<float>(2 * n);
  out->conic_op = c.take<float>(4 * n);
  out->depth = c.take<float>(n);
  out->radius = c.take<int32_t>(n);
  out->tiles_touched = c.take<uint32_t>(n);
  out->pair_keys = c.take<uint64_t>(max_pairs);
  out->pair_ids = c.take<int32_t>(max_pairs);
  out->ranges = c.take<uint32_t>(2 * tiles);
  out->final_T = c.take<float>(px);
  out->n_contrib = c.take<int32_t>(px);
  out->n_pairs = c.take<uint32_t>(1);
  return PRTGS_OK;
}

size_t render_workspace(int64_t n, int32_t, int32_t, int64_t max_pairs) {
  return scan_workspace(n) + 2 * align_up(sizeof(uint64_t) * max_pairs) + 2 * align_up(sizeof(int32_t) * max_pairs) +
         radix_sort_workspace(max_pairs);
}

__device__ __forceinline__ void quat_rot(float qw, float qx, float qy, float qz, float R[3][3]) {
  float n = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= n; qx *= n; qy *= n; qz *= n;
  R[0][0] = 1.f - 2.f * (qy * qy + qz * qz); R[0][1] = 2.f * (qx * qy - qw * qz); R[0][2] = 2.f * (qx * qz + qw * qy);
  R[1][0] = 2.f * (qx * qy + qw * qz); R[1][1] = 1.f - 2.f * (qx * qx + qz * qz); R[1][2] = 2.f * (qy * qz - qw * qx);
  R[2][0] = 2.f * (qx * qz - qw * qy); R[2][1] = 2.f * (qy * qz + qw * qx); R[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
}

// Sigma = R diag(s^2) R^T (Eq. 2), upper triangle (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ void covariance3d(const float R[3][3], float s0, float s1, float s2, float S[6]) {
  float d[3] = {s0 * s0, s1 * s1, s2 * s2};
  S[0] = R[0][0] * R[0][0] * d[0] + R[0][1] * R[0][1] * d[1] + R[0][2] * R[0][2] * d[2];
  S[1] = R[0][0] * R[1][0] * d[0] + R[0][1] * R[1][1] * d[1] + R[0][2] * R[1][2] * d[2];
  S[2] = R[0][0] * R[2][0] * d[0] + R[0][1] * R[2][1] * d[1] + R[0][2] * R[2][2] * d[2];
  S[3] = R[1][0] * R[1][0] * d[0] + R[1][1] * R[1][1] * d[1] + R[1][2] * R[1][2] * d[2];
  S[4] = R[1][0] * R[2][0] * d[0] + R[1][1] * R[2][1] * d[1] + R[1][2] * R[2][2] * d[2];
  S[5] = R[2][0] * R[2][0] * d[0] + R[2][1] * R[2][1] * d[1] + R[2][2] * R[2][2] * d[2];
}

__device__ __forceinline__ void tile_rect(float mx, float my, int r, const Cam& c, int& x0, int& y0, int& x1,
                                          int& y1) {
  const float fr = (float)r;
  x0 = min(max((int)floorf((mx - fr) / kTile), 0), c.gx);
  x1 = min(max((int)floorf((mx + fr) / kTile) + 1, 0), c.gx);
  y0 = min(max((int)floorf((my - fr) / kTile), 0), c.gy);
  y1 = min(max((int)floorf((my + fr) / kTile) + 1, 0), c.gy);
}

template <class V>
__global__ void k_preprocess(int64_t n, const float* __restrict__ means, const float* __restrict__ scales,
                             const float* __restrict__ quats, const float* __restrict__ opacity, V v,
                             float* __restrict__ mean2d, float4* __restrict__ conic_op, float* __restrict__ depth,
                             int32_t* __restrict__ radius, uint32_t* __restrict__ touched) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Cam& c = v.cam(v.scene_of(i));
  radius[i] = 0;
  touched[i] = 0;
  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  const float x = c.r[0] * mx + c.r[1] * my + c.r[2] * mz + c.t[0];
  const float y = c.r[3] * mx + c.r[4] * my + c.r[5] * mz + c.t[1];
  const float z = c.r[6] * mx + c.r[7] * my + c.r[8] * mz + c.t[2];
  depth[i] = z;
  if (!(z > c.near_plane)) return;
  float R[3][3];
  quat_rot(quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3], R);
  float S[6];
  covariance3d(R, scales[3 * i], scales[3 * i + 1], scales[3 * i + 2], S);
  const float iz = 1.0f / z;
  const float tx = fminf(c.limx, fmaxf(-c.limx, x * iz)) * z;
  const float ty = fminf(c.limy, fmaxf(-c.limy, y * iz)) * z;
  // J (2x3) = [[fx/z, 0, -fx tx/z^2], [0, fy/z, -fy ty/z^2]]; M = J W
  const float j00 = c.fx * iz, j02 = -c.fx * tx * iz * iz, j11 = c.fy * iz, j12 = -c.fy * ty * iz * iz;
  float m0[3], m1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    m0[k] = j00 * c.r[k] + j02 * c.r[6 + k];
    m1[k] = j11 * c.r[3 + k] + j12 * c.r[6 + k];
  }
  // cov2 = M Sigma M^T
  float s0[3] = {S[0] * m0[0] + S[1] * m0[1] + S[2] * m0[2], S[1] * m0[0] + S[3] * m0[1] + S[4] * m0[2],
                 S[2] * m0[0] + S[4] * m0[1] + S[5] * m0[2]};
  float s1[3] = {S[0] * m1[0] + S[1] * m1[1] + S[2] * m1[2], S[1] * m1[0] + S[3] * m1[1] + S[4] * m1[2],
                 S[2] * m1[0] + S[4] * m1[1] + S[5] * m1[2]};
  const float a = m0[0] * s0[0] + m0[1] * s0[1] + m0[2] * s0[2] + kDilation;
  const float b = m0[0] * s1[0] + m0[1] * s1[1] + m0[2] * s1[2];
  const float cc = m1[0] * s1[0] + m1[1] * s1[1] + m1[2] * s1[2] + kDilation;
  const float det = a * cc - b * b;
  if (!(det > 0.f)) return;
  const float idet = 1.0f / det;
  const float mid = 0.5f * (a + cc);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
  const int r = (int)ceilf(3.0f * sqrtf(lam));
  const float px = c.fx * x * iz + c.cx, py = c.fy * y * iz + c.cy;
  int x0, y0, x1, y1;
  tile_rect(px, py, r, c, x0, y0, x1, y1);
  const uint32_t cnt = (uint32_t)((x1 - x0) * (y1 - y0));
  if (r <= 0 || cnt == 0) return;
  mean2d[2 * i] = px;
  mean2d[2 * i + 1] = py;
  conic_op[i] = make_float4(cc * idet, -b * idet, a * idet, opacity[i]);
  radius[i] = r;
  touched[i] = cnt;
}

template <class V>
__global__ void k_duplicate(int64_t n, V v, const float* __restrict__ mean2d, const float* __restrict__ depth,
                            const int32_t* __restrict__ radius, const uint32_t* __restrict__ incl,
                            int64_t max_pairs, uint64_t* __restrict__ keys, int32_t* __restrict__ ids,
                            int32_t* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = radius[i];
  if (r <= 0) return;
  const int b = v.scene_of(i);
  const Cam& c = v.cam(b);
  const uint64_t tile0 = (uint64_t)b * (uint64_t)(c.gx * c.gy);  // the scene's first tile
  int x0, y0, x1, y1;
  tile_rect(mean2d[2 * i], mean2d[2 * i + 1], r, c, x0, y0, x1, y1);
  const uint32_t end = incl[i];
  int64_t p = (int64_t)end - (int64_t)((x1 - x0) * (y1 - y0));
  if ((int64_t)end > max_pairs) set_status(status, PRTGS_STATUS_CAPACITY);
  const uint64_t dbits = (uint64_t)__float_as_uint(depth[i]);
  for (int ty = y0; ty < y1; ++ty)
    for (int tx = x0; tx < x1; ++tx, ++p) {
      if (p >= max_pairs) return;
      keys[p] = ((tile0 + (uint64_t)(ty * c.gx + tx)) << 32) | dbits;
      ids[p] = (int32_t)i;
    }
}

__global__ void k_clamp_count(uint32_t* count, int64_t max_pairs) {
  if (*count > (uint64_t)max_pairs) *count = (uint32_t)max_pairs;
}

__global__ void k_ranges(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ count, int64_t tiles,
                         uint32_t* __restrict__ ranges) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = *count;
  if (p >= n) return;
  uint32_t tile = (uint32_t)(keys[p] >> 32);
  if ((int64_t)tile >= tiles) return;
  if (p == 0 || (uint32_t)(keys[p - 1] >> 32) != tile) ranges[2 * tile] = (uint32_t)p;
  if (p == n - 1 || (uint32_t)(keys[p + 1] >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(p + 1);
}

template <int KG, class V>
__global__ void __launch_bounds__(kTileThreads) k_composite(V v, const uint32_t* __restrict__ ranges,
                                                            const int32_t* __restrict__ ids,
                                                            const float* __restrict__ mean2d,
                                                            const float4* __restrict__ conic_op,
                                                            const float* __restrict__ colors, int64_t n, int k,
                                                            const float* __restrict__ bg, float* __restrict__ image,
                                                            float* __restrict__ final_T, int32_t* __restrict__ n_contrib) {
  __shared__ float2 s_xy[kTileThreads];
  __shared__ float4 s_co[kTileThreads];
  __shared__ float s_col[kTileThreads][3 * KG];
  const int gtile = blockIdx.x;  // scene-major tile index
  const Cam& c = v.cam(0);
  const int per_scene = c.gx * c.gy;
  const int b = gtile / per_scene, tile = gtile % per_scene;
  const int l0 = blockIdx.y * KG;
  const int nl = min(KG, k - l0);
  const int tx = tile % c.gx, ty = tile / c.gx;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const uint32_t start = ranges[2 * gtile], end = ranges[2 * gtile + 1];
  float T = 1.0f;
  float acc[KG][3];
#pragma unroll
  for (int l = 0; l < KG; ++l) acc[l][0] = acc[l][1] = acc[l][2] = 0.f;
  bool done = !inside;
  uint32_t contributor = 0, last = 0;
  const float fpx = (float)px, fpy = (float)py;
  for (uint32_t bt = start; bt < end; bt += kTileThreads) {
    if (__syncthreads_count(done) == kTileThreads) break;
    uint32_t e = bt + threadIdx.x;
    if (e < end) {
      int g = ids[e];
      s_xy[threadIdx.x] = make_float2(mean2d[2 * g], mean2d[2 * g + 1]);
      s_co[threadIdx.x] = conic_op[g];
#pragma unroll
      for (int l = 0; l < KG; ++l)
        if (l < nl) {
          const float* cp = colors + color_at(v, b, g, l0 + l, k, n);
          s_col[threadIdx.x][3 * l] = cp[0];
          s_col[threadIdx.x][3 * l + 1] = cp[1];
          s_col[threadIdx.x][3 * l + 2] = cp[2];
        }
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kTileThreads, end - bt);
    for (int j = 0; j < cnt && !done; ++j) {
      ++contributor;
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      const float dx = xy.x - fpx, dy = xy.y - fpy;
      const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
      if (power > 0.f) continue;
      const float alpha = fminf(kAlphaMax, co.w * __expf(power));
      if (alpha < kAlphaMin) continue;
      const float test_T = T * (1.0f - alpha);
      if (test_T < kTStop) {
        done = true;
        continue;
      }
      const float wgt = alpha * T;
#pragma unroll
      for (int l = 0; l < KG; ++l) {
        acc[l][0] = fmaf(s_col[j][3 * l], wgt, acc[l][0]);
        acc[l][1] = fmaf(s_col[j][3 * l + 1], wgt, acc[l][1]);
        acc[l][2] = fmaf(s_col[j][3 * l + 2], wgt, acc[l][2]);
      }
      T = test_T;
      last = contributor;
    }
  }
  if (!inside) return;
  const int64_t HW = (int64_t)c.W * c.H;
  const int64_t pix = (int64_t)py * c.W + px;
  if (blockIdx.y == 0) {
    final_T[b * HW + pix] = T;
    n_contrib[b * HW + pix] = (int32_t)last;
  }
  float* img = image + (int64_t)b * k * 3 * HW;
#pragma unroll
  for (int l = 0; l < KG; ++l)
    if (l < nl)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) img[((int64_t)(l0 + l) * 3 + ch) * HW + pix] = acc[l][ch] + T * bg[ch];
}

// Forward pass for B scenes of one image size (B = 1 with OneView): tiles are numbered
// scene-major, so one sort and one composite launch cover every scene.
template <class V>
static int render_views(const prtgs_gaussians* g, const float* colors, int32_t k, const V& v, const Cam& c, int B,
                        const float* bg, float* image, prtgs_render_state* st, int32_t* status, void* ws,
                        cudaStream_t stream) {
  const int64_t n = g->n;
  const int64_t tiles = (int64_t)c.gx * c.gy * B;
  Carver cv(ws);
  void* scan_ws = cv.take<char>(scan_workspace(n));
  uint64_t* keys_x = cv.take<uint64_t>(st->max_pairs);
  uint64_t* keys_y = cv.take<uint64_t>(st->max_pairs);
  int32_t* ids_x = cv.take<int32_t>(st->max_pairs);
  int32_t* ids_y = cv.take<int32_t>(st->max_pairs);
  void* sort_ws = cv.take<char>(radix_sort_workspace(st->max_pairs));
  cudaMemsetAsync(st->ranges, 0, sizeof(uint32_t) * 2 * tiles, stream);
  cudaMemsetAsync(st->n_pairs, 0, sizeof(uint32_t), stream);
  if (n > 0) {
    k_preprocess<V><<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(
        n, g->means, g->scales, g->quats, g->opacity, v, st->mean2d, reinterpret_cast<float4*>(st->conic_op),
        st->depth, st->radius, st->tiles_touched);
    PRTGS_CHECK_LAUNCH();
    int rc = scan_u32(st->tiles_touched, st->tiles_touched, n, false, st->n_pairs, scan_ws, stream);
    if (rc != PRTGS_OK) return rc;
    k_duplicate<V><<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, v, st->mean2d, st->depth, st->radius,
                                                                   st->tiles_touched, st->max_pairs, keys_x, ids_x,
                                                                   status);
    k_clamp_count<<<1, 1, 0, counted(stream)>>>(st->n_pairs, st->max_pairs);
    PRTGS_CHECK_LAUNCH();
    int tile_bits = 0;
    while ((int64_t(1) << tile_bits) < tiles) ++tile_bits;
    rc = radix_sort_pairs(keys_x, ids_x, st->pair_keys, st->pair_ids, keys_y, ids_y, st->max_pairs, st->n_pairs, 0,
                          32 + tile_bits, sort_ws, stream);
    if (rc != PRTGS_OK) return rc;
    k_ranges<<<(unsigned)((st->max_pairs + 255) / 256), 256, 0, counted(stream)>>>(st->pair_keys, st->n_pairs, tiles,
                                                                            st->ranges);
    PRTGS_CHECK_LAUNCH();
  }
  const int kg = k <= 1 ? 1 : (k <= 4 ? 4 : 8);
  dim3 grid((unsigned)tiles, (unsigned)((k + kg - 1) / kg));
  const float4* co = reinterpret_cast<const float4*>(st->conic_op);
  if (kg == 1)
    k_composite<1, V><<<grid, kTileThreads, 0, counted(stream)>>>(v, st->ranges, st->pair_ids, st->mean2d, co, colors, n, k,
                                                         bg, image, st->final_T, st->n_contrib);
  else if (kg == 4)
    k_composite<4, V><<<grid, kTileThreads, 0, counted(stream)>>>(v, st->ranges, st->pair_ids, st->mean2d, co, colors, n, k,
                                                         bg, image, st->final_T, st->n_contrib);
  else
    k_composite<8, V><<<grid, kTileThreads, 0, counted(stream)>>>(v, st->ranges, st->pair_ids, st->mean2d, co, colors, n, k,
                                                         bg, image, st->final_T, st->n_contrib);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int render(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam, const float* bg,
           float* image, prtgs_render_state* st, int32_t* status, void* ws, cudaStream_t stream) {
  OneView v{make_cam(cam)};
  return render_views(g, colors, k, v, v.c, 1, bg, image, st, status, ws, stream);
}

static int many_views(const prtgs_camera* cams, int32_t B, const int64_t* offsets, ManyViews& v) {
  if (B < 1 || B > kMaxScenes) return PRTGS_ERR_UNSUPPORTED;
  for (int b = 0; b < B; ++b) {
    v.c[b] = make_cam(cams + b);
    if (cams[b].width != cams[0].width || cams[b].height != cams[0].height) return PRTGS_ERR_SHAPE;
  }
  v.offs = offsets;
  v.B = B;
  return PRTGS_OK;
}

int render_batched(const prtgs_gaussians* g, const int64_t* offsets, int32_t B, const float* colors, int32_t k,
                   const prtgs_camera* cams, const float* bg, float* images, prtgs_render_state* st, int32_t* status,
                   void* ws, cudaStream_t stream) {
  static_assert(sizeof(ManyViews) < 30000, "the cameras must fit the kernel parameter space");
  ManyViews v;
  const int rc = many_views(cams, B, offsets, v);
  if (rc != PRTGS_OK) return rc;
  return render_views(g, colors, k, v, v.c[0], B, bg, images, st, status, ws, stream);
}

// ---- backward ------------------------------------------------------------------------------
template <int KG, class V>
__global__ void __launch_bounds__(kTileThreads) k_composite_bwd(
    V v, const uint32_t* __restrict__ ranges, const int32_t* __restrict__ ids, const float* __restrict__ mean2d,
    const float4* __restrict__ conic_op, const float* __restrict__ colors, int64_t n, int k,
    const float* __restrict__ bg, const float* __restrict__ final_T, const int32_t* __restrict__ n_contrib,
    const float* __restrict__ dimage, float* __restrict__ d_mean2d, float* __restrict__ d_conic,
    float* __restrict__ d_opacity, float* __restrict__ d_colors) {
  constexpr int NV = 6 + 3 * KG;  // mean2d(2) conic(3) opacity(1) colours(3 KG)
  __shared__ float2 s_xy[kTileThreads];
  __shared__ float4 s_co[kTileThreads];
  __shared__ float s_col[kTileThreads][3 * KG];
  __shared__ int s_id[kTileThreads];
  __shared__ float s_acc[kTileThreads][NV];
  const int gtile = blockIdx.x;  // scene-major tile index
  const Cam& c = v.cam(0);
  const int per_scene = c.gx * c.gy;
  const int b = gtile / per_scene, tile = gtile % per_scene;
  const int l0 = blockIdx.y * KG;
  const int nl = min(KG, k - l0);
  const int tx = tile % c.gx, ty = tile / c.gx;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const int lane = threadIdx.x & 31;
  const uint32_t start = ranges[2 * gtile], end = ranges[2 * gtile + 1];
  const int64_t HW = (int64_t)c.W * c.H;
  const int64_t pix = (int64_t)py * c.W + px;
  const float T_final = inside ? final_T[b * HW + pix] : 0.f;
  float T = T_final;
  const uint32_t last = inside ? (uint32_t)n_contrib[b * HW + pix] : 0u;
  const float* dimg = dimage + (int64_t)b * k * 3 * HW;
  float dpix[KG][3], accum[KG][3], last_col[KG][3];
  float bg_dot = 0.f;
#pragma unroll
  for (int l = 0; l < KG; ++l)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      dpix[l][ch] = (inside && l < nl) ? dimg[((int64_t)(l0 + l) * 3 + ch) * HW + pix] : 0.f;
      accum[l][ch] = 0.f;
      last_col[l][ch] = 0.f;
      bg_dot += bg[ch] * dpix[l][ch];
    }
  float last_alpha = 0.f;
  const float fpx = (float)px, fpy = (float)py;
  const uint32_t count = end - start;
  // walk batches from the back of the list
  for (uint32_t done_cnt = 0; done_cnt < count; done_cnt += kTileThreads) {
    const uint32_t bsize = min((uint32_t)kTileThreads, count - done_cnt);
    const uint32_t bstart = end - done_cnt - bsize;  // list position of s_*[0]
    __syncthreads();
    {
      uint32_t t = threadIdx.x;
      if (t < bsize) {
        int g = ids[bstart + t];
        s_id[t] = g;
        s_xy[t] = make_float2(mean2d[2 * g], mean2d[2 * g + 1]);
        s_co[t] = conic_op[g];
#pragma unroll
        for (int l = 0; l < KG; ++l)
          if (l < nl) {
            const float* cp = colors + color_at(v, b, g, l0 + l, k, n);
            s_col[t][3 * l] = cp[0];
            s_col[t][3 * l + 1] = cp[1];
            s_col[t][3 * l + 2] = cp[2];
          }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) s_acc[threadIdx.x][v] = 0.f;
    }
    __syncthreads();
    for (int j = (int)bsize - 1; j >= 0; --j) {
      const uint32_t pos = bstart + j - start + 1;  // 1-based position in the tile list
      float gv[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) gv[v] = 0.f;
      bool contrib = false;
      if (inside && pos <= last) {
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        const float dx = xy.x - fpx, dy = xy.y - fpy;
        const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
        if (power <= 0.f) {
          const float G = __expf(power);
          const float raw = co.w * G;
          const float alpha = fminf(kAlphaMax, raw);
          if (alpha >= kAlphaMin) {
            contrib = true;
            T = T / (1.0f - alpha);
            const float wgt = alpha * T;
            float dL_dalpha = 0.f;
#pragma unroll
            for (int l = 0; l < KG; ++l)
#pragma unroll
              for (int ch = 0; ch < 3; ++ch) {
                const float col = s_col[j][3 * l + ch];
                accum[l][ch] = last_alpha * last_col[l][ch] + (1.0f - last_alpha) * accum[l][ch];
                last_col[l][ch] = col;
                dL_dalpha += (col - accum[l][ch]) * dpix[l][ch];
                gv[6 + 3 * l + ch] = wgt * dpix[l][ch];
              }
            dL_dalpha *= T;
            last_alpha = alpha;
            dL_dalpha += (-T_final / (1.0f - alpha)) * bg_dot;
            if (raw < kAlphaMax) {
              const float dL_dG = co.w * dL_dalpha;
              const float gdx = G * dx, gdy = G * dy;
              gv[0] = dL_dG * (-gdx * co.x - gdy * co.y);
              gv[1] = dL_dG * (-gdy * co.z - gdx * co.y);
              gv[2] = -0.5f * gdx * dx * dL_dG;
              gv[3] = -gdx * dy * dL_dG;
              gv[4] = -0.5f * gdy * dy * dL_dG;
              gv[5] = G * dL_dalpha;
            }
          }
        }
      }
      // warp reduction, then shared-memory accumulation for this batch entry
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float x = warp_sum(gv[v]);
          if (lane == 0) atomicAdd(&s_acc[j][v], x);
        }
      }
    }
    __syncthreads();
    {
      uint32_t t = threadIdx.x;
      if (t < bsize) {
        const int g = s_id[t];
        const float* a = s_acc[t];
        if (a[0] != 0.f || a[1] != 0.f) {
          atomicAdd(&d_mean2d[2 * g], a[0]);
          atomicAdd(&d_mean2d[2 * g + 1], a[1]);
        }
        if (a[2] != 0.f || a[3] != 0.f || a[4] != 0.f) {
          atomicAdd(&d_conic[3 * g], a[2]);
          atomicAdd(&d_conic[3 * g + 1], a[3]);
          atomicAdd(&d_conic[3 * g + 2], a[4]);
        }
        if (a[5] != 0.f) atomicAdd(&d_opacity[g], a[5]);
#pragma unroll
        for (int l = 0; l < KG; ++l)
          if (l < nl)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
              const float gc = a[6 + 3 * l + ch];
              if (gc != 0.f) atomicAdd(&d_colors[color_at(v, b, g, l0 + l, k, n) + ch], gc);
            }
      }
    }
  }
}

// 2D gradients -> means, scales, rotations (chain rule through Eq. 3 and Eq. 2).
template <class V>
__global__ void k_preprocess_bwd(int64_t n, const float* __restrict__ means, const float* __restrict__ scales,
                                 const float* __restrict__ quats, V v, const int32_t* __restrict__ radius,
                                 const float* __restrict__ d_mean2d, const float* __restrict__ d_conic,
                                 float* __restrict__ d_means, float* __restrict__ d_scales,
                                 float* __restrict__ d_quats) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Cam& c = v.cam(v.scene_of(i));
  float gm[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  if (radius[i] > 0) {
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
    const float x = c.r[0] * mx + c.r[1] * my + c.r[2] * mz + c.t[0];
    const float y = c.r[3] * mx + c.r[4] * my + c.r[5] * mz + c.t[1];
    const float z = c.r[6] * mx + c.r[7] * my + c.r[8] * mz + c.t[2];
    const float qw0 = quats[4 * i], qx0 = quats[4 * i + 1], qy0 = quats[4 * i + 2], qz0 = quats[4 * i + 3];
    const float qn = sqrtf(qw0 * qw0 + qx0 * qx0 + qy0 * qy0 + qz0 * qz0);
    const float qw = qw0 / qn, qx = qx0 / qn, qy = qy0 / qn, qz = qz0 / qn;
    float R[3][3];
    quat_rot(qw, qx, qy, qz, R);
    const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    float S[6];
    covariance3d(R, s[0], s[1], s[2], S);
    const float Sm[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
    const float iz = 1.0f / z;
    const float xz = x * iz, yz = y * iz;
    const bool clx = xz < -c.limx || xz > c.limx, cly = yz < -c.limy || yz > c.limy;
    const float cxz = fminf(c.limx, fmaxf(-c.limx, xz)), cyz = fminf(c.limy, fmaxf(-c.limy, yz));
    // J = [[fx/z, 0, -fx cxz / z], [0, fy/z, -fy cyz / z]]
    const float J[2][3] = {{c.fx * iz, 0.f, -c.fx * cxz * iz}, {0.f, c.fy * iz, -c.fy * cyz * iz}};
    const float W[3][3] = {{c.r[0], c.r[1], c.r[2]}, {c.r[3], c.r[4], c.r[5]}, {c.r[6], c.r[7], c.r[8]}};
    float M[2][3];
    for (int a = 0; a < 2; ++a)
      for (int k2 = 0; k2 < 3; ++k2) M[a][k2] = J[a][0] * W[0][k2] + J[a][1] * W[1][k2] + J[a][2] * W[2][k2];
    float cov[2][2];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        float acc = 0.f;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) acc += M[a][p] * Sm[p][q] * M[b][q];
        cov[a][b] = acc;
      }
    const float A = cov[0][0] + kDilation, B = cov[0][1], Cc = cov[1][1] + kDilation;
    const float det = A * Cc - B * B;
    const float id2 = 1.0f / (det * det);
    const float gA = d_conic[3 * i], gB = d_conic[3 * i + 1], gC = d_conic[3 * i + 2];
    // conic = (C/det, -B/det, A/det)
    const float dA = id2 * (-Cc * Cc * gA + B * Cc * gB - B * B * gC);
    const float dC = id2 * (-B * B * gA + A * B * gB - A * A * gC);
    const float dB = id2 * (2.f * B * Cc * gA - (det + 2.f * B * B) * gB + 2.f * A * B * gC);
    // symmetric gradient of cov2 (B is read from the 01 entry once)
    const float G2[2][2] = {{dA, 0.5f * dB}, {0.5f * dB, dC}};
    // dSigma = M^T G2 M
    float dS[3][3];
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        float acc = 0.f;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) acc += M[a][p] * G2[a][b] * M[b][q];
        dS[p][q] = acc;
      }
    // dM = 2 G2 M Sigma ; dJ = dM W^T
    float dM[2][3];
    for (int a = 0; a < 2; ++a)
      for (int q = 0; q < 3; ++q) {
        float acc = 0.f;
        for (int b = 0; b < 2; ++b)
          for (int p = 0; p < 3; ++p) acc += G2[a][b] * M[b][p] * Sm[p][q];
        dM[a][q] = 2.f * acc;
      }
    float dJ[2][3];
    for (int a = 0; a < 2; ++a)
      for (int k2 = 0; k2 < 3; ++k2) dJ[a][k2] = dM[a][0] * W[k2][0] + dM[a][1] * W[k2][1] + dM[a][2] * W[k2][2];
    // camera-space gradient from J(x,y,z) and from mean2d = (fx x/z + cx, fy y/z + cy)
    const float gmx = d_mean2d[2 * i], gmy = d_mean2d[2 * i + 1];
    float gx = gmx * c.fx * iz;
    float gy = gmy * c.fy * iz;
    float gz = -gmx * c.fx * x * iz * iz - gmy * c.fy * y * iz * iz;
    gz += dJ[0][0] * (-c.fx * iz * iz) + dJ[1][1] * (-c.fy * iz * iz);
    // J02 = -fx cxz / z, cxz = clamp(x/z)
    if (!clx) {
      gx += dJ[0][2] * (-c.fx * iz * iz);
      gz += dJ[0][2] * (2.f * c.fx * x * iz * iz * iz);
    } else {
      gz += dJ[0][2] * (c.fx * cxz * iz * iz);
    }
    if (!cly) {
      gy += dJ[1][2] * (-c.fy * iz * iz);
      gz += dJ[1][2] * (2.f * c.fy * y * iz * iz * iz);
    } else {
      gz += dJ[1][2] * (c.fy * cyz * iz * iz);
    }
    // world-space: p = W mu + t
    for (int k2 = 0; k2 < 3; ++k2) gm[k2] = W[0][k2] * gx + W[1][k2] * gy + W[2][k2] * gz;
    // Sigma = R diag(s^2) R^T
    const float D[3] = {s[0] * s[0], s[1] * s[1], s[2] * s[2]};
    float gR[3][3];
    for (int a = 0; a < 3; ++a)
      for (int k2 = 0; k2 < 3; ++k2) {
        float acc = 0.f;
        for (int j = 0; j < 3; ++j) acc += (dS[a][j] + dS[j][a]) * R[j][k2];
        gR[a][k2] = acc * D[k2];
      }
    for (int k2 = 0; k2 < 3; ++k2) {
      float acc = 0.f;
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) acc += dS[a][j] * R[a][k2] * R[j][k2];
      gs[k2] = acc * 2.f * s[k2];
    }
    // R(q) with q normalised
    const float gw = 2.f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] +
                            qx * gR[2][1]);
    const float gxq = 2.f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.f * qx * gR[1][1] - qw * gR[1][2] +
                             qz * gR[2][0] + qw * gR[2][1] - 2.f * qx * gR[2][2]);
    const float gyq = 2.f * (-2.f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] + qz * gR[1][2] -
                             qw * gR[2][0] + qz * gR[2][1] - 2.f * qy * gR[2][2]);
    const float gzq = 2.f * (-2.f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] -
                             2.f * qz * gR[1][1] + qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
    const float dot = qw * gw + qx * gxq + qy * gyq + qz * gzq;
    gq[0] = (gw - qw * dot) / qn;
    gq[1] = (gxq - qx * dot) / qn;
    gq[2] = (gyq - qy * dot) / qn;
    gq[3] = (gzq - qz * dot) / qn;
  }
  for (int k2 = 0; k2 < 3; ++k2) {
    d_means[3 * i + k2] = gm[k2];
    d_scales[3 * i + k2] = gs[k2];
  }
  for (int k2 = 0; k2 < 4; ++k2) d_quats[4 * i + k2] = gq[k2];
}

// ---- depth and normal maps (Eq. 23, Eq. 25): the composite of d_i and n_i -------------------------
// Features for render() with two "lights": light 0 carries (d_i, 0, 0), d_i the view-space
// depth of the splat's mean; light 1 carries the raw normal n_i.
__global__ void k_geometry_features(int64_t n, Cam c, const float* __restrict__ means,
                                    const float* __restrict__ normals, float* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = means[3 * i], y = means[3 * i + 1], z = means[3 * i + 2];
  const float d = fmaf(c.r[6], x, fmaf(c.r[7], y, fmaf(c.r[8], z, c.t[2])));
  F[3 * i] = d;
  F[3 * i + 1] = 0.f;
  F[3 * i + 2] = 0.f;
  float* Fn = F + 3 * n;
#pragma unroll
  for (int k = 0; k < 3; ++k) Fn[3 * i + k] = normals[3 * i + k];
}

size_t render_geometry_workspace(int64_t n, int32_t width, int32_t height, int64_t max_pairs) {
  return align_up(sizeof(float) * 6 * (size_t)n) + align_up(sizeof(float) * 6 * (size_t)width * height) +
         align_up(sizeof(float) * 4) + render_workspace(n, width, height, max_pairs);
}

int render_geometry(const prtgs_gaussians* g, const prtgs_camera* cam, float* depth, float* normal,
                    prtgs_render_state* st, int32_t* status, void* ws, cudaStream_t stream) {
  const int64_t n = g->n;
  const int64_t n_pix = (int64_t)cam->width * cam->height;
  Carver cv(ws);
  float* F = cv.take<float>(6 * (size_t)n);
  float* img = cv.take<float>(6 * (size_t)n_pix);
  float* zero = cv.take<float>(4);
  void* rws = static_cast<char*>(ws) + cv.off;
  cudaMemsetAsync(zero, 0, sizeof(float) * 4, stream);
  if (n > 0) {
    k_geometry_features<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, make_cam(cam), g->means, g->normals, F);
    PRTGS_CHECK_LAUNCH();
  }
  const int rc = render(g, F, 2, cam, zero, img, st, status, rws, stream);
  if (rc != PRTGS_OK) return rc;
  // image [2][3][H][W]: depth is light 0's first channel, the normal light 1's three channels
  cudaMemcpyAsync(depth, img, sizeof(float) * n_pix, cudaMemcpyDeviceToDevice, stream);
  cudaMemcpyAsync(normal, img + 3 * n_pix, sizeof(float) * 3 * n_pix, cudaMemcpyDeviceToDevice, stream);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

size_t render_backward_workspace(int64_t n, int32_t) {
  return align_up(sizeof(float) * 2 * n) + align_up(sizeof(float) * 3 * n);
}

template <class V>
static int render_backward_views(const prtgs_gaussians* g, const float* colors, int32_t k, const V& v, const Cam& c,
                                 int B, const float* bg, const prtgs_render_state* st, const float* dimage,
                                 float* d_means, float* d_scales, float* d_quats, float* d_opacity, float* d_colors,
                                 void* ws, cudaStream_t stream) {
  const int64_t n = g->n;
  if (n == 0) return PRTGS_OK;
  const int64_t tiles = (int64_t)c.gx * c.gy * B;
  Carver cv(ws);
  float* dm2 = cv.take<float>(2 * n);
  float* dcon = cv.take<float>(3 * n);
  cudaMemsetAsync(dm2, 0, sizeof(float) * 2 * n, stream);
  cudaMemsetAsync(dcon, 0, sizeof(float) * 3 * n, stream);
  cudaMemsetAsync(d_opacity, 0, sizeof(float) * n, stream);
  cudaMemsetAsync(d_colors, 0, sizeof(float) * 3 * n * k, stream);
  // groups of up to 4 light colour sets per pass (shared memory bound)
  const int kg = k <= 1 ? 1 : 4;
  dim3 grid((unsigned)tiles, (unsigned)((k + kg - 1) / kg));
  const float4* co = reinterpret_cast<const float4*>(st->conic_op);
  if (kg == 1)
    k_composite_bwd<1, V><<<grid, kTileThreads, 0, counted(stream)>>>(v, st->ranges, st->pair_ids, st->mean2d, co, colors, n,
                                                             k, bg, st->final_T, st->n_contrib, dimage, dm2, dcon,
                                                             d_opacity, d_colors);
  else
    k_composite_bwd<4, V><<<grid, kTileThreads, 0, counted(stream)>>>(v, st->ranges, st->pair_ids, st->mean2d, co, colors, n,
                                                             k, bg, st->final_T, st->n_contrib, dimage, dm2, dcon,
                                                             d_opacity, d_colors);
  PRTGS_CHECK_LAUNCH();
  k_preprocess_bwd<V><<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, g->means, g->scales, g->quats, v,
                                                                      st->radius, dm2, dcon, d_means, d_scales,
                                                                      d_quats);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int render_backward(const prtgs_gaussians* g, const float* colors, int32_t k, const prtgs_camera* cam,
                    const float* bg, const prtgs_render_state* st, const float* dimage, float* d_means,
                    float* d_scales, float* d_quats, float* d_opacity, float* d_colors, void* ws,
                    cudaStream_t stream) {
  OneView v{make_cam(cam)};
  return render_backward_views(g, colors, k, v, v.c, 1, bg, st, dimage, d_means, d_scales, d_quats, d_opacity,
                               d_colors, ws, stream);
}

int render_backward_batched(const prtgs_gaussians* g, const int64_t* offsets, int32_t B, const float* colors,
                            int32_t k, const prtgs_camera* cams, const float* bg, const prtgs_render_state* st,
                            const float* dimages, float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                            float* d_colors, void* ws, cudaStream_t stream) {
  ManyViews v;
  const int rc = many_views(cams, B, offsets, v);
  if (rc != PRTGS_OK) return rc;
  return render_backward_views(g, colors, k, v, v.c[0], B, bg, st, dimages, d_means, d_scales, d_quats, d_opacity,
                               d_colors, ws, stream);
}

// ---- L2 loss ---------------------------------------------------------------------------------
constexpr int kLossThreads = 256;
constexpr int kLossItems = 16;

__global__ void k_l2_partial(const float* __restrict__ a, const float* __restrict__ b, int64_t count, float scale,
                             float* __restrict__ grad, float* __restrict__ partial) {
  __shared__ float sw[kLossThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kLossThreads * kLossItems;
  float s = 0.f;
  for (int q = 0; q < kLossItems; ++q) {
    int64_t i = base + (int64_t)q * kLossThreads + threadIdx.x;
    if (i < count) {
      float d = a[i] - b[i];
      grad[i] = scale * d;
      s = fmaf(d, d, s);
    }
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kLossThreads / 32; ++w) t += sw[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_l2_final(const float* __restrict__ partial, int64_t nb, float inv_count, float* __restrict__ loss) {
  __shared__ double sd[256];
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += (double)partial[b];
  sd[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sd[threadIdx.x] += sd[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(sd[0] * (double)inv_count);
}

// Per-scene losses of B images of `count` elements each: loss[b] = mean over scene b, dimage =
// 2 (image - target) / count. Blocks never straddle scenes (grid.y = scene).
__global__ void k_l2_partial_batched(const float* __restrict__ a, const float* __restrict__ t, int64_t count,
                                     float scale, float* __restrict__ grad, float* __restrict__ partial) {
  __shared__ float sw[kLossThreads / 32];
  const int64_t off = (int64_t)blockIdx.y * count;
  const int64_t base = (int64_t)blockIdx.x * kLossThreads * kLossItems;
  float s = 0.f;
  for (int q = 0; q < kLossItems; ++q) {
    const int64_t i = base + (int64_t)q * kLossThreads + threadIdx.x;
    if (i < count) {
      const float d = a[off + i] - t[off + i];
      grad[off + i] = scale * d;
      s = fmaf(d, d, s);
    }
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float u = 0.f;
    for (int w = 0; w < kLossThreads / 32; ++w) u += sw[w];
    partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = u;
  }
}

__global__ void k_l2_final_batched(const float* __restrict__ partial, int64_t nb, float inv_count,
                                   float* __restrict__ loss) {
  __shared__ double sd[256];
  const float* p = partial + (int64_t)blockIdx.x * nb;
  double s = 0.0;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += (double)p[b];
  sd[threadIdx.x] = s;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) sd[threadIdx.x] += sd[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[blockIdx.x] = (float)(sd[0] * (double)inv_count);
}

size_t l2_loss_batched_workspace(int64_t count, int32_t n_scenes) {
  const int64_t nb = (count + kLossThreads * kLossItems - 1) / (kLossThreads * kLossItems);
  return align_up(sizeof(float) * (size_t)(nb > 0 ? nb : 1) * (n_scenes > 0 ? n_scenes : 1));
}

int l2_loss_batched(const float* images, const float* targets, int64_t count, int32_t n_scenes, float* losses,
                    float* dimages, void* ws, cudaStream_t stream) {
  if (count <= 0 || n_scenes <= 0) return PRTGS_ERR_INVALID_ARG;
  const int64_t nb = (count + kLossThreads * kLossItems - 1) / (kLossThreads * kLossItems);
  float* partial = static_cast<float*>(ws);
  k_l2_partial_batched<<<dim3((unsigned)nb, (unsigned)n_scenes), kLossThreads, 0, counted(stream)>>>(
      images, targets, count, 2.0f / (float)count, dimages, partial);
  k_l2_final_batched<<<(unsigned)n_scenes, 256, 0, counted(stream)>>>(partial, nb, 1.0f / (float)count, losses);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

size_t l2_loss_workspace(int64_t count) {
  int64_t nb = (count + kLossThreads * kLossItems - 1) / (kLossThreads * kLossItems);
  return align_up(sizeof(float) * (size_t)(nb > 0 ? nb : 1));
}

int l2_loss(const float* image, const float* target, int64_t count, float* loss, float* dimage, void* ws,
            cudaStream_t stream) {
  if (count <= 0) return PRTGS_ERR_INVALID_ARG;
  int64_t nb = (count + kLossThreads * kLossItems - 1) / (kLossThreads * kLossItems);
  float* partial = static_cast<float*>(ws);
  k_l2_partial<<<(unsigned)nb, kLossThreads, 0, counted(stream)>>>(image, target, count, 2.0f / (float)count, dimage, partial);
  k_l2_final<<<1, 256, 0, counted(stream)>>>(partial, nb, 1.0f / (float)count, loss);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

}  // namespace prtgs
