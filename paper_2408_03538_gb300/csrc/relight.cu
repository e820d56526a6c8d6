// Relight contraction (Eq. 14; glossy splats Eq. 41) and its backward pass.
//
// colors[k,i,c] = (rho_i[c] / pi) * sum_m T_i[c or 0][m] L[k,c,m]
#include "common.cuh"
#include "internal.h"

namespace prtgs {

constexpr int kRelightThreads = 256;
constexpr int kMaxLightsSmem = 256;

// One thread per Gaussian; the lights sit in shared memory. (Staging each warp's 384-byte
// rows through shared memory for 16-byte stores measured slower here: L2 merges the
// 12-byte-stride stores.)
template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight(int64_t n, const float* __restrict__ T,
                                                             const float* __restrict__ albedo,
                                                             const float* __restrict__ L, int k,
                                                             float* __restrict__ colors) {
  extern __shared__ float sL[];  // [k][3][C]
  for (int e = threadIdx.x; e < k * 3 * C; e += blockDim.x) sL[e] = L[e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float t[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) t[c][m] = __ldg(T + (i * TCH + c) * C + m);
  const float r0 = __ldg(albedo + 3 * i) * (1.0f / kPi);
  const float r1 = __ldg(albedo + 3 * i + 1) * (1.0f / kPi);
  const float r2 = __ldg(albedo + 3 * i + 2) * (1.0f / kPi);
  for (int l = 0; l < k; ++l) {
    const float* Ll = sL + l * 3 * C;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int m = 0; m < C; ++m) {
      d0 = fmaf(t[0][m], Ll[m], d0);
      d1 = fmaf(t[TCH > 1 ? 1 : 0][m], Ll[C + m], d1);
      d2 = fmaf(t[TCH > 1 ? 2 : 0][m], Ll[2 * C + m], d2);
    }
    float* out = colors + ((int64_t)l * n + i) * 3;
    out[0] = r0 * d0;
    out[1] = r1 * d1;
    out[2] = r2 * d2;
  }
}

// Glossy splats: t_eff[a] = sum_b M[a,b] Y_b(v), v = normalize(cam - mu) (Eq. 41).
template <int ORDER>
__global__ void __launch_bounds__(kRelightThreads) k_relight_glossy(int64_t n, int64_t n_glossy,
                                                                    const int32_t* __restrict__ ids,
                                                                    const float* __restrict__ M,
                                                                    const float* __restrict__ means,
                                                                    const float* __restrict__ cam,
                                                                    const float* __restrict__ albedo,
                                                                    const float* __restrict__ L, int k,
                                                                    float* __restrict__ colors) {
  constexpr int C = (ORDER + 1) * (ORDER + 1);
  extern __shared__ float sL[];
  for (int e = threadIdx.x; e < k * 3 * C; e += blockDim.x) sL[e] = L[e];
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_glossy) return;
  const int64_t i = ids[g];
  float vx = cam[0] - means[3 * i], vy = cam[1] - means[3 * i + 1], vz = cam[2] - means[3 * i + 2];
  float rn = rsqrtf(vx * vx + vy * vy + vz * vz);
  float Y[C];
  sh_eval_any<ORDER>(vx * rn, vy * rn, vz * rn, Y);
  float te[C];
#pragma unroll
  for (int a = 0; a < C; ++a) {
    float acc = 0.f;
#pragma unroll
    for (int b = 0; b < C; ++b) acc = fmaf(__ldg(M + (g * C + a) * C + b), Y[b], acc);
    te[a] = acc;
  }
  const float r0 = albedo[3 * i] * (1.0f / kPi), r1 = albedo[3 * i + 1] * (1.0f / kPi),
              r2 = albedo[3 * i + 2] * (1.0f / kPi);
  for (int l = 0; l < k; ++l) {
    const float* Ll = sL + l * 3 * C;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int m = 0; m < C; ++m) {
      d0 = fmaf(te[m], Ll[m], d0);
      d1 = fmaf(te[m], Ll[C + m], d1);
      d2 = fmaf(te[m], Ll[2 * C + m], d2);
    }
    float* out = colors + ((int64_t)l * n + i) * 3;
    out[0] = r0 * d0;
    out[1] = r1 * d1;
    out[2] = r2 * d2;
  }
}

// Orders 4-6 (25-49 coefficients): one thread per Gaussian, the transfer row and the lights read
// through the cache instead of held in registers.
__global__ void __launch_bounds__(kRelightThreads) k_relight_any(int64_t n, int C, int tch, const float* __restrict__ T,
                                                                 const float* __restrict__ albedo,
                                                                 const float* __restrict__ L, int k,
                                                                 float* __restrict__ colors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) r[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
  for (int l = 0; l < k; ++l) {
    float* out = colors + ((int64_t)l * n + i) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* t = T + (i * tch + (tch > 1 ? c : 0)) * C;
      const float* Ll = L + ((int64_t)l * 3 + c) * C;
      float d = 0.f;
      for (int m = 0; m < C; ++m) d = fmaf(__ldg(t + m), __ldg(Ll + m), d);
      out[c] = r[c] * d;
    }
  }
}

size_t relight_workspace(int64_t, int32_t, int32_t, int32_t) { return 0; }

template <int ORDER>
static void launch_relight_glossy(int64_t n, int64_t n_glossy, const int32_t* ids, const float* M, const float* means,
                                  const float* cam, const float* albedo, const float* L, int k, float* colors,
                                  cudaStream_t stream) {
  constexpr int C = (ORDER + 1) * (ORDER + 1);
  const size_t smem = sizeof(float) * k * 3 * C;
  cudaFuncSetAttribute(k_relight_glossy<ORDER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned grid = (unsigned)((n_glossy + kRelightThreads - 1) / kRelightThreads);
  k_relight_glossy<ORDER><<<grid, kRelightThreads, smem, counted(stream)>>>(n, n_glossy, ids, M, means, cam, albedo, L, k,
                                                                            colors);
}

template <int C>
static void launch_relight_c(int64_t n, const float* T, int tch, const float* albedo, const float* L, int k,
                             float* colors, cudaStream_t stream) {
  size_t smem = sizeof(float) * k * 3 * C;
  unsigned grid = (unsigned)((n + kRelightThreads - 1) / kRelightThreads);
  if (tch == 3) {
    cudaFuncSetAttribute(k_relight<C, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_relight<C, 3><<<grid, kRelightThreads, smem, counted(stream)>>>(n, T, albedo, L, k, colors);
  } else {
    cudaFuncSetAttribute(k_relight<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_relight<C, 1><<<grid, kRelightThreads, smem, counted(stream)>>>(n, T, albedo, L, k, colors);
  }
}

int relight(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo, int64_t n_glossy,
            const int32_t* glossy_ids, const float* M, const float* means, const float* cam_pos, const float* L,
            int32_t k, int32_t precision, float* colors, int32_t* status, unsigned tc_wait_polls, void* ws,
            cudaStream_t stream) {
  if (n == 0 || k == 0) return PRTGS_OK;
  if (k > kMaxLightsSmem) return PRTGS_ERR_UNSUPPORTED;
  if (precision != PRTGS_PREC_FP32) {
    // every row on the tensor cores; glossy rows are then rewritten by the glossy kernel
    const int rc = relight_tc(n, order, T, t_channels, albedo, L, k, precision, nullptr, 1, colors, status,
                              tc_wait_polls, stream);
    if (rc != PRTGS_OK) return rc;
  } else {
    switch (order) {
      case 1: launch_relight_c<4>(n, T, t_channels, albedo, L, k, colors, stream); break;
      case 2: launch_relight_c<9>(n, T, t_channels, albedo, L, k, colors, stream); break;
      case 3: launch_relight_c<16>(n, T, t_channels, albedo, L, k, colors, stream); break;
      case 4:
      case 5:
      case 6:
        k_relight_any<<<(unsigned)((n + kRelightThreads - 1) / kRelightThreads), kRelightThreads, 0, counted(stream)>>>(
            n, sh_count(order), t_channels, T, albedo, L, k, colors);
        break;
      default: return PRTGS_ERR_UNSUPPORTED;
    }
    PRTGS_CHECK_LAUNCH();
  }
  if (n_glossy > 0) {
    switch (order) {
      case 1: launch_relight_glossy<1>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      case 2: launch_relight_glossy<2>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      case 3: launch_relight_glossy<3>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      case 4: launch_relight_glossy<4>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      case 5: launch_relight_glossy<5>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      case 6: launch_relight_glossy<6>(n, n_glossy, glossy_ids, M, means, cam_pos, albedo, L, k, colors, stream); break;
      default: return PRTGS_ERR_UNSUPPORTED;
    }
    PRTGS_CHECK_LAUNCH();
  }
  return PRTGS_OK;
}

// ---- pixel-space relight of many lights (composite once, contract per pixel) ------------------
// The composite is linear in the splat colours: with colours (rho_i/pi) (T_i . L_l) every
// light's image is sum_m TI[m,c,p] L[l,c,m] + bg[c] final_T[p], TI the composite of the
// features F[m,i,c] = (rho_i[c]/pi) T_i[c][m] (glossy splats: t_eff = M_i Y(v_i), Eq. 41).
template <int TCH>
__global__ void k_transfer_features(int64_t n, int C, const float* __restrict__ T, const float* __restrict__ albedo,
                                    float* __restrict__ F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) r[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
  for (int m = 0; m < C; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c) F[((int64_t)m * n + i) * 3 + c] = r[c] * __ldg(T + (i * TCH + (TCH > 1 ? c : 0)) * C + m);
}

template <int ORDER>
__global__ void k_glossy_features(int64_t n, int64_t n_glossy, const int32_t* __restrict__ ids,
                                  const float* __restrict__ M, const float* __restrict__ means, float cx, float cy,
                                  float cz, const float* __restrict__ albedo, float* __restrict__ F) {
  constexpr int C = (ORDER + 1) * (ORDER + 1);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_glossy) return;
  const int64_t i = ids[g];
  const float vx = cx - means[3 * i], vy = cy - means[3 * i + 1], vz = cz - means[3 * i + 2];
  const float rn = rsqrtf(vx * vx + vy * vy + vz * vz);
  float Y[C];
  sh_eval_any<ORDER>(vx * rn, vy * rn, vz * rn, Y);
  float r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) r[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
#pragma unroll
  for (int a = 0; a < C; ++a) {
    float te = 0.f;
#pragma unroll
    for (int b = 0; b < C; ++b) te = fmaf(__ldg(M + (g * C + a) * C + b), Y[b], te);
#pragma unroll
    for (int c = 0; c < 3; ++c) F[((int64_t)a * n + i) * 3 + c] = r[c] * te;
  }
}

// FP32 form: one thread per pixel, the lights in shared memory.
template <int C>
__global__ void __launch_bounds__(kRelightThreads) k_pixel_relight(int64_t n_pix, const float* __restrict__ TI,
                                                                   const float* __restrict__ final_T,
                                                                   const float* __restrict__ bg,
                                                                   const float* __restrict__ L, int k,
                                                                   float* __restrict__ image) {
  extern __shared__ float sL[];  // [k][3][C]
  for (int e = threadIdx.x; e < k * 3 * C; e += blockDim.x) sL[e] = L[e];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  float t[3][C];
#pragma unroll
  for (int m = 0; m < C; ++m)
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c][m] = __ldg(TI + ((int64_t)m * 3 + c) * n_pix + p);
  const float ft = __ldg(final_T + p);
  float b[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c] = bg[c] * ft;
  for (int l = 0; l < k; ++l) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* Ll = sL + (l * 3 + c) * C;
      float d = b[c];
#pragma unroll
      for (int m = 0; m < C; ++m) d = fmaf(t[c][m], Ll[m], d);
      image[((int64_t)l * 3 + c) * n_pix + p] = d;
    }
  }
}

// Orders 4-6: one thread per pixel, one channel at a time (its C coefficients in registers), the
// lights in shared memory.
template <int C>
__global__ void __launch_bounds__(kRelightThreads) k_pixel_relight_hi(int64_t n_pix, const float* __restrict__ TI,
                                                                      const float* __restrict__ final_T,
                                                                      const float* __restrict__ bg,
                                                                      const float* __restrict__ L, int k,
                                                                      float* __restrict__ image) {
  extern __shared__ float sL[];  // [k][3][C]
  for (int e = threadIdx.x; e < k * 3 * C; e += blockDim.x) sL[e] = L[e];
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  const float ft = __ldg(final_T + p);
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    float t[C];
#pragma unroll
    for (int m = 0; m < C; ++m) t[m] = __ldg(TI + ((int64_t)m * 3 + c) * n_pix + p);
    const float b = bg[c] * ft;
    for (int l = 0; l < k; ++l) {
      const float* Ll = sL + (l * 3 + c) * C;
      float d = b;
#pragma unroll
      for (int m = 0; m < C; ++m) d = fmaf(t[m], Ll[m], d);
      image[((int64_t)l * 3 + c) * n_pix + p] = d;
    }
  }
}

template <int C>
static void launch_pixel_relight_hi(int64_t n_pix, const float* TI, const float* final_T, const float* bg,
                                    const float* L, int k, float* image, cudaStream_t stream) {
  const size_t smem = sizeof(float) * k * 3 * C;
  cudaFuncSetAttribute(k_pixel_relight_hi<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned blocks = (unsigned)((n_pix + kRelightThreads - 1) / kRelightThreads);
  k_pixel_relight_hi<C><<<blocks, kRelightThreads, smem, counted(stream)>>>(n_pix, TI, final_T, bg, L, k, image);
}

size_t render_relit_workspace(int64_t n, int32_t order, int32_t width, int32_t height, int64_t max_pairs) {
  const int C = sh_count(order);
  const int64_t n_pix = (int64_t)width * height;
  return align_up(sizeof(float) * (size_t)C * n * 3) + align_up(sizeof(float) * (size_t)C * 3 * n_pix) +
         align_up(sizeof(float) * 4) + render_workspace(n, width, height, max_pairs);
}

int render_relit(const prtgs_gaussians* g, int32_t order, const float* T, int32_t t_channels, int64_t n_glossy,
                 const int32_t* glossy_ids, const float* M, const float* L, int32_t k, int32_t precision,
                 const prtgs_camera* cam, const float* bg, float* image, prtgs_render_state* st, int32_t* status,
                 unsigned tc_wait_polls, void* ws, cudaStream_t stream) {
  const int64_t n = g->n;
  const int C = sh_count(order);
  const int64_t n_pix = (int64_t)cam->width * cam->height;
  Carver cv(ws);
  float* F = cv.take<float>((size_t)C * n * 3);
  float* TI = cv.take<float>((size_t)C * 3 * n_pix);
  float* zero = cv.take<float>(4);
  void* rws = static_cast<char*>(ws) + cv.off;
  cudaMemsetAsync(zero, 0, sizeof(float) * 4, stream);
  if (n > 0) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (t_channels == 3) k_transfer_features<3><<<blocks, 256, 0, counted(stream)>>>(n, C, T, g->albedo, F);
    else k_transfer_features<1><<<blocks, 256, 0, counted(stream)>>>(n, C, T, g->albedo, F);
    if (n_glossy > 0) {
      const unsigned gb = (unsigned)((n_glossy + 255) / 256);
      const float px = cam->pos[0], py = cam->pos[1], pz = cam->pos[2];
#define PRTGS_GF(O) k_glossy_features<O><<<gb, 256, 0, counted(stream)>>>(n, n_glossy, glossy_ids, M, g->means, px, py, pz, \
                                                                         g->albedo, F)
      switch (order) {
        case 1: PRTGS_GF(1); break;
        case 2: PRTGS_GF(2); break;
        case 3: PRTGS_GF(3); break;
        case 4: PRTGS_GF(4); break;
        case 5: PRTGS_GF(5); break;
        default: PRTGS_GF(6); break;
      }
#undef PRTGS_GF
    }
    PRTGS_CHECK_LAUNCH();
  }
  int rc = render(g, F, C, cam, zero, TI, st, status, rws, stream);
  if (rc != PRTGS_OK) return rc;
  if (precision != PRTGS_PREC_FP32)
    return relight_tc_pixels(n_pix, order, TI, st->final_T, bg, L, k, precision, image, status, tc_wait_polls,
                             stream);
  const size_t smem = sizeof(float) * k * 3 * C;
  const unsigned blocks = (unsigned)((n_pix + kRelightThreads - 1) / kRelightThreads);
  switch (order) {
    case 1: k_pixel_relight<4><<<blocks, kRelightThreads, smem, counted(stream)>>>(n_pix, TI, st->final_T, bg, L, k, image); break;
    case 2: k_pixel_relight<9><<<blocks, kRelightThreads, smem, counted(stream)>>>(n_pix, TI, st->final_T, bg, L, k, image); break;
    case 3: k_pixel_relight<16><<<blocks, kRelightThreads, smem, counted(stream)>>>(n_pix, TI, st->final_T, bg, L, k, image); break;
    case 4: launch_pixel_relight_hi<25>(n_pix, TI, st->final_T, bg, L, k, image, stream); break;
    case 5: launch_pixel_relight_hi<36>(n_pix, TI, st->final_T, bg, L, k, image, stream); break;
    default: launch_pixel_relight_hi<49>(n_pix, TI, st->final_T, bg, L, k, image, stream); break;
  }
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// ---- many scenes in one launch: scene b (Gaussians offsets[b] .. offsets[b+1]) has its own
// k lights L[b] --------------------------------------------------------------------------------
template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight_batched(int64_t n, const float* __restrict__ T,
                                                                     const float* __restrict__ albedo,
                                                                     const int64_t* __restrict__ offsets,
                                                                     int n_scenes, const float* __restrict__ L, int k,
                                                                     float* __restrict__ colors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_scene(offsets, n_scenes, i);
  const float* Lb = L + (int64_t)b * k * 3 * C;
  const int64_t ob = offsets[b], nb = offsets[b + 1] - ob;
  float* cb = colors + 3 * (int64_t)k * ob;  // this scene's [k, n_b, 3] block
  float t[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) t[c][m] = __ldg(T + (i * TCH + c) * C + m);
  const float r0 = __ldg(albedo + 3 * i) * (1.0f / kPi);
  const float r1 = __ldg(albedo + 3 * i + 1) * (1.0f / kPi);
  const float r2 = __ldg(albedo + 3 * i + 2) * (1.0f / kPi);
  for (int l = 0; l < k; ++l) {
    const float* Ll = Lb + l * 3 * C;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int m = 0; m < C; ++m) {
      d0 = fmaf(t[0][m], __ldg(Ll + m), d0);
      d1 = fmaf(t[TCH > 1 ? 1 : 0][m], __ldg(Ll + C + m), d1);
      d2 = fmaf(t[TCH > 1 ? 2 : 0][m], __ldg(Ll + 2 * C + m), d2);
    }
    float* out = cb + ((int64_t)l * nb + (i - ob)) * 3;
    out[0] = r0 * d0;
    out[1] = r1 * d1;
    out[2] = r2 * d2;
  }
}

// Orders 4-6, many scenes: as k_relight_any, scene b's lights L[b] and colour block [k, n_b, 3].
__global__ void __launch_bounds__(kRelightThreads) k_relight_any_batched(int64_t n, int C, int tch,
                                                                         const float* __restrict__ T,
                                                                         const float* __restrict__ albedo,
                                                                         const int64_t* __restrict__ offsets,
                                                                         int n_scenes, const float* __restrict__ L,
                                                                         int k, float* __restrict__ colors) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_scene(offsets, n_scenes, i);
  const int64_t ob = offsets[b], nb = offsets[b + 1] - ob;
  const float* Lb = L + (int64_t)b * k * 3 * C;
  float* cb = colors + 3 * (int64_t)k * ob;
  float r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) r[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
  for (int l = 0; l < k; ++l) {
    float* out = cb + ((int64_t)l * nb + (i - ob)) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* t = T + (i * tch + (tch > 1 ? c : 0)) * C;
      const float* Ll = Lb + ((int64_t)l * 3 + c) * C;
      float d = 0.f;
      for (int m = 0; m < C; ++m) d = fmaf(__ldg(t + m), __ldg(Ll + m), d);
      out[c] = r[c] * d;
    }
  }
}

// Orders 4-6 backward, per Gaussian and one channel at a time: with G[c][m] = sum_k dc[k,i,c]
// L_k[c][m] (C registers), d_albedo[c] = (T_i[c] . G[c]) / pi and dT[c][m] = (rho[c]/pi) G[c][m]
// (summed over c for a one-channel T): the same sums as k_relight_bwd_local, reassociated so that
// only C accumulators (2 C for a one-channel T) are live instead of 2 x 3 C.
template <int C, bool BATCHED>
__global__ void __launch_bounds__(kRelightThreads) k_relight_bwd_local_hi(
    int64_t n, int tch, const float* __restrict__ T, const float* __restrict__ albedo,
    const int64_t* __restrict__ offs, int B, const float* __restrict__ L, int k, const float* __restrict__ dcol,
    float* __restrict__ d_albedo, float* __restrict__ dT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = 0;
  int64_t o = 0, nb = n;
  if (BATCHED) {
    b = find_scene(offs, B, i);
    o = offs[b];
    nb = offs[b + 1] - o;
  }
  const float* Lb = L + (int64_t)b * k * 3 * C;
  const float* dc = dcol + 3 * (int64_t)k * o;
  float acc[C];
#pragma unroll
  for (int m = 0; m < C; ++m) acc[m] = 0.f;
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    float G[C];
#pragma unroll
    for (int m = 0; m < C; ++m) G[m] = 0.f;
    for (int l = 0; l < k; ++l) {
      const float g = __ldg(dc + ((int64_t)l * nb + (i - o)) * 3 + c);
      const float* Ll = Lb + ((int64_t)l * 3 + c) * C;
#pragma unroll
      for (int m = 0; m < C; ++m) G[m] = fmaf(g, __ldg(Ll + m), G[m]);
    }
    const float* t = T + (i * tch + (tch > 1 ? c : 0)) * C;
    float da = 0.f;
#pragma unroll
    for (int m = 0; m < C; ++m) da = fmaf(__ldg(t + m), G[m], da);
    d_albedo[3 * i + c] = da * (1.0f / kPi);
    const float rho = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
    if (dT) {
      if (tch > 1) {
#pragma unroll
        for (int m = 0; m < C; ++m) dT[(i * 3 + c) * C + m] = rho * G[m];
      } else {
#pragma unroll
        for (int m = 0; m < C; ++m) acc[m] = fmaf(rho, G[m], acc[m]);
      }
    }
  }
  if (dT && tch == 1) {
#pragma unroll
    for (int m = 0; m < C; ++m) dT[i * C + m] = acc[m];
  }
}

template <int C>
static void launch_relight_batched_c(int64_t n, const float* T, int tch, const float* albedo,
                                     const int64_t* offsets, int n_scenes, const float* L, int k, float* colors,
                                     cudaStream_t stream) {
  unsigned grid = (unsigned)((n + kRelightThreads - 1) / kRelightThreads);
  if (tch == 3)
    k_relight_batched<C, 3><<<grid, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, offsets, n_scenes, L, k, colors);
  else
    k_relight_batched<C, 1><<<grid, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, offsets, n_scenes, L, k, colors);
}

int relight_batched(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                    const int64_t* offsets, int32_t n_scenes, const float* L, int32_t k, int32_t precision,
                    float* colors, int32_t* status, unsigned tc_wait_polls, cudaStream_t stream) {
  if (n == 0 || k == 0) return PRTGS_OK;
  if (precision != PRTGS_PREC_FP32)
    return relight_tc(n, order, T, t_channels, albedo, L, k, precision, offsets, n_scenes, colors, status,
                      tc_wait_polls, stream);
  switch (order) {
    case 1: launch_relight_batched_c<4>(n, T, t_channels, albedo, offsets, n_scenes, L, k, colors, stream); break;
    case 2: launch_relight_batched_c<9>(n, T, t_channels, albedo, offsets, n_scenes, L, k, colors, stream); break;
    case 3: launch_relight_batched_c<16>(n, T, t_channels, albedo, offsets, n_scenes, L, k, colors, stream); break;
    case 4:
    case 5:
    case 6:
      k_relight_any_batched<<<(unsigned)((n + kRelightThreads - 1) / kRelightThreads), kRelightThreads, 0,
                              counted(stream)>>>(n, sh_count(order), t_channels, T, albedo, offsets, n_scenes, L, k,
                                                 colors);
      break;
    default: return PRTGS_ERR_UNSUPPORTED;
  }
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// ---- backward ------------------------------------------------------------------------------
// Per Gaussian: d_albedo[c] = sum_k dc[k,i,c] (T_i[c].L_k[c]) / pi and
// dT[c][m] = sum_k dc[k,i,c] (rho[c]/pi) L_k[c][m] (summed over c when T has one channel).
template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight_bwd_local(int64_t n, const float* __restrict__ T,
                                                                       const float* __restrict__ albedo,
                                                                       const float* __restrict__ L, int k,
                                                                       const float* __restrict__ dcol,
                                                                       float* __restrict__ d_albedo,
                                                                       float* __restrict__ dT) {
  extern __shared__ float sL[];
  for (int e = threadIdx.x; e < k * 3 * C; e += blockDim.x) sL[e] = L[e];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float t[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) t[c][m] = __ldg(T + (i * TCH + c) * C + m);
  float rho[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) rho[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
  float da[3] = {0.f, 0.f, 0.f};
  float gT[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) gT[c][m] = 0.f;
  for (int l = 0; l < k; ++l) {
    const float* Ll = sL + l * 3 * C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float g = __ldg(dcol + ((int64_t)l * n + i) * 3 + c);
      float dot = 0.f;
#pragma unroll
      for (int m = 0; m < C; ++m) {
        dot = fmaf(t[TCH > 1 ? c : 0][m], Ll[c * C + m], dot);
        gT[TCH > 1 ? c : 0][m] = fmaf(g * rho[c], Ll[c * C + m], gT[TCH > 1 ? c : 0][m]);
      }
      da[c] = fmaf(g, dot, da[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) d_albedo[3 * i + c] = da[c] * (1.0f / kPi);
  if (dT) {
#pragma unroll
    for (int c = 0; c < TCH; ++c)
#pragma unroll
      for (int m = 0; m < C; ++m) dT[(i * TCH + c) * C + m] = gT[c][m];
  }
}

// dL[k,c,m] = sum_i dc[k,i,c] (rho_i[c]/pi) T_i[c][m]: per-chunk partial sums (each block walks
// its chunk of Gaussians in order), then a fixed-order sum of the partials: deterministic.
constexpr int kDLChunk = 2048;
constexpr int kDLBatch = 32;

template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight_dL_partial(int64_t n, const float* __restrict__ T,
                                                                        const float* __restrict__ albedo, int k,
                                                                        const float* __restrict__ dcol,
                                                                        float* __restrict__ partial) {
  __shared__ float sT[kDLBatch][TCH * C];
  __shared__ float sW[kDLBatch][3 * 8];  // dc * rho / pi for up to 8 lights per pass
  const int outs_per_light = 3 * C;
  const int64_t i0 = (int64_t)blockIdx.x * kDLChunk;
  constexpr int LPP = 512 / (3 * C) < 8 ? 512 / (3 * C) : 8;  // lights per pass: <= 512 outputs
  for (int l0 = 0; l0 < k; l0 += LPP) {
    const int nl = min(LPP, k - l0);
    const int nout = nl * outs_per_light;
    float acc[2] = {0.f, 0.f};  // outputs tid and tid + 256 (nout <= 512)
    for (int64_t b = i0; b < i0 + kDLChunk && b < n; b += kDLBatch) {
      __syncthreads();
      for (int e = threadIdx.x; e < kDLBatch * TCH * C; e += blockDim.x) {
        int j = e / (TCH * C), r = e % (TCH * C);
        int64_t i = b + j;
        sT[j][r] = i < n ? T[i * TCH * C + r] : 0.f;
      }
      for (int e = threadIdx.x; e < kDLBatch * 3 * nl; e += blockDim.x) {
        int j = e / (3 * nl), r = e % (3 * nl);
        int l = r / 3, c = r % 3;
        int64_t i = b + j;
        sW[j][r] = i < n ? dcol[((int64_t)(l0 + l) * n + i) * 3 + c] * albedo[3 * i + c] * (1.0f / kPi) : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        int o = threadIdx.x + q * kRelightThreads;
        if (o < nout) {
          int l = o / outs_per_light, r = o % outs_per_light;
          int c = r / C, m = r % C;
          float a = acc[q];
          for (int j = 0; j < kDLBatch; ++j) a = fmaf(sW[j][3 * l + c], sT[j][(TCH > 1 ? c : 0) * C + m], a);
          acc[q] = a;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int o = threadIdx.x + q * kRelightThreads;
      if (o < nout) partial[(int64_t)blockIdx.x * k * outs_per_light + (int64_t)l0 * outs_per_light + o] = acc[q];
    }
  }
}

__global__ void k_sum_partials(const float* __restrict__ partial, int64_t nblocks, int nout, float* __restrict__ out) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  float s = 0.f, c = 0.f;
  for (int64_t b = 0; b < nblocks; ++b) {
    float t, e;
    two_sum(s, partial[b * nout + o], t, e);
    s = t;
    c += e;
  }
  out[o] = s + c;
}

size_t relight_backward_workspace(int64_t n, int32_t order, int32_t k) {
  int64_t nb = (n + kDLChunk - 1) / kDLChunk;
  return align_up(sizeof(float) * (size_t)(nb > 0 ? nb : 1) * k * 3 * sh_count(order));
}

template <int C>
static void launch_relight_bwd(int64_t n, const float* T, int tch, const float* albedo, const float* L, int k,
                               const float* dcol, float* d_albedo, float* dT, float* dL, float* partial,
                               cudaStream_t stream) {
  size_t smem = sizeof(float) * k * 3 * C;
  unsigned grid = (unsigned)((n + kRelightThreads - 1) / kRelightThreads);
  int64_t nb = (n + kDLChunk - 1) / kDLChunk;
  if constexpr (C > kMaxC)
    k_relight_bwd_local_hi<C, false><<<grid, kRelightThreads, 0, counted(stream)>>>(n, tch, T, albedo, nullptr, 1, L, k,
                                                                                   dcol, d_albedo, dT);
  else if (tch == 3)
    k_relight_bwd_local<C, 3><<<grid, kRelightThreads, smem, counted(stream)>>>(n, T, albedo, L, k, dcol, d_albedo, dT);
  else
    k_relight_bwd_local<C, 1><<<grid, kRelightThreads, smem, counted(stream)>>>(n, T, albedo, L, k, dcol, d_albedo, dT);
  if (tch == 3)
    k_relight_dL_partial<C, 3><<<(unsigned)nb, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, k, dcol, partial);
  else
    k_relight_dL_partial<C, 1><<<(unsigned)nb, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, k, dcol, partial);
  int nout = k * 3 * C;
  k_sum_partials<<<(nout + 255) / 256, 256, 0, counted(stream)>>>(partial, nb, nout, dL);
}

// ---- relight backward of many scenes (the layout of prtgs_relight_batched) -------------------
// Scene b holds Gaussians offs[b] .. offs[b+1], lights L[b] ([k,3,C]) and the colour block
// dcol + 3 k offs[b] ([k, n_b, 3]).
template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight_bwd_local_batched(
    int64_t n, const float* __restrict__ T, const float* __restrict__ albedo, const int64_t* __restrict__ offs,
    int B, const float* __restrict__ L, int k, const float* __restrict__ dcol, float* __restrict__ d_albedo,
    float* __restrict__ dT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = find_scene(offs, B, i);
  const int64_t o = offs[b], nb = offs[b + 1] - o;
  const float* Lb = L + (int64_t)b * k * 3 * C;
  const float* dc = dcol + 3 * (int64_t)k * o;
  float t[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) t[c][m] = __ldg(T + (i * TCH + c) * C + m);
  float rho[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) rho[c] = __ldg(albedo + 3 * i + c) * (1.0f / kPi);
  float da[3] = {0.f, 0.f, 0.f};
  float gT[TCH][C];
#pragma unroll
  for (int c = 0; c < TCH; ++c)
#pragma unroll
    for (int m = 0; m < C; ++m) gT[c][m] = 0.f;
  for (int l = 0; l < k; ++l) {
    const float* Ll = Lb + l * 3 * C;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float g = __ldg(dc + ((int64_t)l * nb + (i - o)) * 3 + c);
      float dot = 0.f;
#pragma unroll
      for (int m = 0; m < C; ++m) {
        const float lv = __ldg(Ll + c * C + m);
        dot = fmaf(t[TCH > 1 ? c : 0][m], lv, dot);
        gT[TCH > 1 ? c : 0][m] = fmaf(g * rho[c], lv, gT[TCH > 1 ? c : 0][m]);
      }
      da[c] = fmaf(g, dot, da[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) d_albedo[3 * i + c] = da[c] * (1.0f / kPi);
  if (dT) {
#pragma unroll
    for (int c = 0; c < TCH; ++c)
#pragma unroll
      for (int m = 0; m < C; ++m) dT[(i * TCH + c) * C + m] = gT[c][m];
  }
}

// Partial sums of dL over chunk x of scene y (blockIdx), written to slot offs[y] / kDLChunk + y + x
// (the slots of a scene are consecutive and disjoint from the other scenes').
template <int C, int TCH>
__global__ void __launch_bounds__(kRelightThreads) k_relight_dL_partial_batched(
    const int64_t* __restrict__ offs, const float* __restrict__ T, const float* __restrict__ albedo, int k,
    const float* __restrict__ dcol, float* __restrict__ partial) {
  __shared__ float sT[kDLBatch][TCH * C];
  __shared__ float sW[kDLBatch][3 * 8];
  const int b = blockIdx.y;
  const int64_t o = offs[b], nb = offs[b + 1] - o;
  const int64_t i0 = o + (int64_t)blockIdx.x * kDLChunk;
  if ((int64_t)blockIdx.x * kDLChunk >= nb) return;  // uniform: past the scene's chunks
  const int64_t i1 = min(o + nb, i0 + kDLChunk);
  const float* dc = dcol + 3 * (int64_t)k * o;
  const int outs_per_light = 3 * C;
  const int64_t slot = o / kDLChunk + b + blockIdx.x;
  constexpr int LPP = 512 / (3 * C) < 8 ? 512 / (3 * C) : 8;  // lights per pass: <= 512 outputs
  for (int l0 = 0; l0 < k; l0 += LPP) {
    const int nl = min(LPP, k - l0);
    const int nout = nl * outs_per_light;
    float acc[2] = {0.f, 0.f};
    for (int64_t bb = i0; bb < i1; bb += kDLBatch) {
      __syncthreads();
      for (int e = threadIdx.x; e < kDLBatch * TCH * C; e += blockDim.x) {
        const int j = e / (TCH * C), r = e % (TCH * C);
        const int64_t i = bb + j;
        sT[j][r] = i < i1 ? T[i * TCH * C + r] : 0.f;
      }
      for (int e = threadIdx.x; e < kDLBatch * 3 * nl; e += blockDim.x) {
        const int j = e / (3 * nl), r = e % (3 * nl);
        const int l = r / 3, c = r % 3;
        const int64_t i = bb + j;
        sW[j][r] = i < i1 ? dc[((int64_t)(l0 + l) * nb + (i - o)) * 3 + c] * albedo[3 * i + c] * (1.0f / kPi) : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int ot = threadIdx.x + q * kRelightThreads;
        if (ot < nout) {
          const int l = ot / outs_per_light, r = ot % outs_per_light;
          const int c = r / C, m = r % C;
          float a = acc[q];
          for (int j = 0; j < kDLBatch; ++j) a = fmaf(sW[j][3 * l + c], sT[j][(TCH > 1 ? c : 0) * C + m], a);
          acc[q] = a;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ot = threadIdx.x + q * kRelightThreads;
      if (ot < nout) partial[slot * k * outs_per_light + (int64_t)l0 * outs_per_light + ot] = acc[q];
    }
  }
}

// dL[b] = the scene's partial sums in chunk order (compensated): deterministic.
__global__ void k_sum_partials_batched(const float* __restrict__ partial, const int64_t* __restrict__ offs, int nout,
                                       float* __restrict__ dL) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (o >= nout) return;
  const int64_t nb = offs[b + 1] - offs[b];
  const int64_t chunks = (nb + kDLChunk - 1) / kDLChunk;
  const int64_t slot0 = offs[b] / kDLChunk + b;
  float s = 0.f, c = 0.f;
  for (int64_t x = 0; x < chunks; ++x) {
    float t, e;
    two_sum(s, partial[(slot0 + x) * nout + o], t, e);
    s = t;
    c += e;
  }
  dL[(int64_t)b * nout + o] = s + c;
}

size_t relight_backward_batched_workspace(int64_t n, int32_t n_scenes, int32_t order, int32_t k) {
  const int64_t slots = n / kDLChunk + 2 * (int64_t)n_scenes + 1;
  return align_up(sizeof(float) * (size_t)slots * k * 3 * sh_count(order));
}

template <int C>
static void launch_relight_bwd_batched(int64_t n, const float* T, int tch, const float* albedo, const int64_t* offs,
                                       int B, const float* L, int k, const float* dcol, float* d_albedo, float* dT,
                                       float* dL, float* partial, cudaStream_t stream) {
  const unsigned grid = (unsigned)((n + kRelightThreads - 1) / kRelightThreads);
  const dim3 pgrid((unsigned)((n + kDLChunk - 1) / kDLChunk), (unsigned)B);
  if constexpr (C > kMaxC)
    k_relight_bwd_local_hi<C, true><<<grid, kRelightThreads, 0, counted(stream)>>>(n, tch, T, albedo, offs, B, L, k,
                                                                                  dcol, d_albedo, dT);
  else if (tch == 3)
    k_relight_bwd_local_batched<C, 3><<<grid, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, offs, B, L, k, dcol,
                                                                                    d_albedo, dT);
  else
    k_relight_bwd_local_batched<C, 1><<<grid, kRelightThreads, 0, counted(stream)>>>(n, T, albedo, offs, B, L, k, dcol,
                                                                                    d_albedo, dT);
  if (tch == 3)
    k_relight_dL_partial_batched<C, 3><<<pgrid, kRelightThreads, 0, counted(stream)>>>(offs, T, albedo, k, dcol, partial);
  else
    k_relight_dL_partial_batched<C, 1><<<pgrid, kRelightThreads, 0, counted(stream)>>>(offs, T, albedo, k, dcol, partial);
  const int nout = k * 3 * C;
  k_sum_partials_batched<<<dim3((unsigned)((nout + 255) / 256), (unsigned)B), 256, 0, counted(stream)>>>(partial, offs, nout,
                                                                                                 dL);
}

int relight_backward_batched(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                             const int64_t* offsets, int32_t n_scenes, const float* L, int32_t k,
                             const float* dcolors, float* d_albedo, float* dT, float* dL, void* ws,
                             cudaStream_t stream) {
  if (k == 0) return PRTGS_OK;
  if (n == 0) {
    cudaMemsetAsync(dL, 0, sizeof(float) * n_scenes * k * 3 * sh_count(order), stream);
    return PRTGS_OK;
  }
  float* partial = static_cast<float*>(ws);
  switch (order) {
    case 1: launch_relight_bwd_batched<4>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 2: launch_relight_bwd_batched<9>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 3: launch_relight_bwd_batched<16>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 4: launch_relight_bwd_batched<25>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 5: launch_relight_bwd_batched<36>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 6: launch_relight_bwd_batched<49>(n, T, t_channels, albedo, offsets, n_scenes, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    default: return PRTGS_ERR_UNSUPPORTED;
  }
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int relight_backward(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo,
                     const float* L, int32_t k, const float* dcolors, float* d_albedo, float* dT, float* dL,
                     void* ws, cudaStream_t stream) {
  if (k == 0) return PRTGS_OK;
  if (k > kMaxLightsSmem) return PRTGS_ERR_UNSUPPORTED;
  if (n == 0) {
    cudaMemsetAsync(dL, 0, sizeof(float) * k * 3 * sh_count(order), stream);
    return PRTGS_OK;
  }
  float* partial = static_cast<float*>(ws);
  switch (order) {
    case 1: launch_relight_bwd<4>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 2: launch_relight_bwd<9>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 3: launch_relight_bwd<16>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 4: launch_relight_bwd<25>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 5: launch_relight_bwd<36>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    case 6: launch_relight_bwd<49>(n, T, t_channels, albedo, L, k, dcolors, d_albedo, dT, dL, partial, stream); break;
    default: return PRTGS_ERR_UNSUPPORTED;
  }
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

}  // namespace prtgs
