// Training-stage kernels (Sec. 4.3, Sec. 4.5).
//
//  k_training_transfer  the transfer vector for one known view (Eq. 28): for every Gaussian i
//                       and the direction v_i from its mean to the camera,
//                         t_i[c] = sum_s w k_i(w_s, v_i) (n_i.w_s)^+ V_is Y_c(w_s),  w = 4 pi / S,
//                       with the glossy BRDF kernel k = (1-m) + pi f_s (Eq. 15 times pi) and the
//                       visibility V cached from a prtgs_precompute_visibility call (geometry is
//                       frozen after the ray tracing, Sec. 4.4). One warp per Gaussian: the lanes
//                       stride the directions (V rows read coalesced), Y comes from a shared-memory
//                       table, and the C partial sums are reduced across the warp at the end. Its
//                       backward gives d/d roughness and d/d metallic from dL/dt with the same walk.
//  k_pseudo_normal      the pseudo-normal of the depth map (Eq. 24): one thread per pixel, the
//                       normal of the back-projected central differences in a closed form that
//                       needs no subtraction of nearby 3D points.
//  k_nl_*               the normal loss ||N - N'|| (Eq. 25) over the pixels where N' is defined, a
//                       fixed-grid (deterministic) reduction, and its gradient (N - N') / L.
#include "brdf.cuh"
#include "internal.h"

namespace prtgs {

constexpr int kTTThreads = 256;
constexpr int kTTWarps = kTTThreads / 32;

struct TTArgs {
  int64_t n;
  int S;
  const float* dirs;
  const float* Ytab;    // [S, C]
  const float* V;       // [n, S]
  const float* means;
  const float* normals;
  const float* rough;
  const float* metal;
  float cam[3];
  const float* dt;      // [n, C] (backward)
  float* t;             // [n, C] (forward)
  float* d_rough;       // [n] (backward)
  float* d_metal;       // [n] (backward)
};

// The live terms of one receiver (n.w_s > 0 and V > 0; about a third of the directions) are
// compacted through a per-warp queue of 64 entries, and the BRDF is evaluated 32 queued terms at
// a time, so that every lane works on a live term instead of idling on the dead ones.
constexpr int kTTQueue = 64;

// Warp sum of N <= 32 per-lane values v[0..N) by recursive halving (a reduce-scatter): at the
// step with xor offset o (16, 8, ...) a lane keeps the half of its values selected by its bit o
// and adds its partner's copy of that half, so each step halves the values held; when one value
// is left, the remaining offsets add it across the lanes that hold the same coefficient. Returns
// the sum of coefficient k (set on every lane; k = -1 on lanes that duplicate another's k) with
// log2(P) + (5 - log2(P)) shuffles in all, P the power of two >= N, instead of 5 N.
template <int N>
__device__ __forceinline__ float reduce_scatter(float* v, int lane, int& k) {
  constexpr int P = N <= 1 ? 1 : (N <= 2 ? 2 : (N <= 4 ? 4 : (N <= 8 ? 8 : (N <= 16 ? 16 : 32))));
  float w[P];
#pragma unroll
  for (int j = 0; j < P; ++j) w[j] = j < N ? v[j] : 0.0f;
  int idx = 0;
  int off = 16;
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1, off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = upper ? w[j] : w[j + h];
      const float keep = upper ? w[j + h] : w[j];
      w[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
    if (upper) idx += h;
  }
  float x = w[0];
  for (; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  // lanes that differ only in the bits below the last halving offset hold the same coefficient
  const int dup_mask = (32 / P) - 1;
  k = (lane & dup_mask) == 0 ? idx : -1;
  return x;
}

template <int ORDER, bool BACKWARD>
__global__ void __launch_bounds__(kTTThreads, ORDER <= 3 ? 4 : 2) k_training_transfer(TTArgs a) {
  constexpr int C = (ORDER + 1) * (ORDER + 1);
  extern __shared__ float sm[];
  const int S = a.S;
  float* sdir = sm;              // [3S]
  float* sY = sdir + 3 * S;      // [C][S]: coefficient-major, so that the lanes (consecutive
                                 // directions) read consecutive words, free of bank conflicts
  float* sdt = sY + S * C;       // [warps][C] (backward)
  __shared__ int qs_all[kTTWarps][kTTQueue];    // queued direction
  __shared__ float qw_all[kTTWarps][kTTQueue];  // its (n.w_s) V_s
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) sdir[i] = a.dirs[i];
  for (int i = threadIdx.x; i < S * C; i += blockDim.x) sY[i] = a.Ytab[(i % S) * C + i / S];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  int* qs = qs_all[warp];
  float* qw = qw_all[warp];
  const float wq = 4.0f * kPi / (float)S;
  for (int64_t i = (int64_t)blockIdx.x * kTTWarps + warp; i < a.n; i += (int64_t)gridDim.x * kTTWarps) {
    const float nx = __ldg(a.normals + 3 * i), ny = __ldg(a.normals + 3 * i + 1), nz = __ldg(a.normals + 3 * i + 2);
    float v[3] = {a.cam[0] - __ldg(a.means + 3 * i), a.cam[1] - __ldg(a.means + 3 * i + 1),
                  a.cam[2] - __ldg(a.means + 3 * i + 2)};
    const float il = 1.0f / sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
    v[0] *= il;
    v[1] *= il;
    v[2] *= il;
    const float no = fmaf(nx, v[0], fmaf(ny, v[1], nz * v[2]));
    const float r = __ldg(a.rough + i), m = __ldg(a.metal + i);
    const float alpha = r * r;
    const bool front = no > 0.0f;  // k = 0 for a view below the splat's horizon
    const float* Vi = a.V + i * S;
    float acc[BACKWARD ? 1 : C];
#pragma unroll
    for (int k = 0; k < (BACKWARD ? 1 : C); ++k) acc[k] = 0.0f;
    float gr = 0.0f, gm = 0.0f;
    float* dts = sdt + warp * C;
    if (BACKWARD) {
      for (int k = lane; k < C; k += 32) dts[k] = __ldg(a.dt + i * C + k);
      __syncwarp();
    }
    // one live term (direction s, cv = (n.w_s) V_s) on this lane
    auto term = [&](int s, float cv) {
      const float* d = sdir + 3 * s;
      if (!BACKWARD) {
        const float c = fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2]));  // > 0 for a queued term
        const float f = wq * brdf_kernel(nx, ny, nz, d, v, c, no, alpha, m) * cv;
#pragma unroll
        for (int k = 0; k < (BACKWARD ? 1 : C); ++k) acc[k] = fmaf(f, sY[k * S + s], acc[k]);
      } else {
        float q = 0.0f;
#pragma unroll
        for (int k = 0; k < C; ++k) q = fmaf(dts[k], sY[k * S + s], q);
        float kv;
        const float dk = brdf_kernel_dr(nx, ny, nz, d, v, fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2])), no, r, m, kv);
        const float f = wq * cv * q;
        gr = fmaf(f, dk, gr);
        gm -= f;  // dk/dm = -1
      }
    };
    if (front) {
      int qn = 0;  // warp-uniform queue length, < 32 between chunks
      for (int base = 0; base < S; base += 32) {
        const int s = base + lane;
        float cv = 0.0f;
        if (s < S) {
          const float* d = sdir + 3 * s;
          const float c = fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2]));
          if (c > 0.0f) cv = c * __ldg(Vi + s);
        }
        const bool live = cv != 0.0f;  // a NaN visibility stays live and reaches the output
        const unsigned mask = __ballot_sync(0xffffffffu, live);
        if (live) {
          const int pos = qn + __popc(mask & lt_mask);
          qs[pos] = s;
          qw[pos] = cv;
        }
        qn += __popc(mask);
        __syncwarp();
        if (qn >= 32) {  // 32 live terms: one per lane
          term(qs[lane], qw[lane]);
          const int rest = qn - 32;
          int ts = 0;
          float tw = 0.0f;
          if (lane < rest) {
            ts = qs[32 + lane];
            tw = qw[32 + lane];
          }
          __syncwarp();
          if (lane < rest) {
            qs[lane] = ts;
            qw[lane] = tw;
          }
          qn = rest;
          __syncwarp();
        }
      }
      if (lane < qn) term(qs[lane], qw[lane]);
      __syncwarp();
    }
    if (!BACKWARD) {
      float* ti = a.t + i * C;
      if (C <= 32) {
        int k;
        const float val = reduce_scatter<(BACKWARD ? 1 : C)>(acc, lane, k);
        if (k >= 0 && k < C) ti[k] = val;
      } else {
        float out0 = 0.0f, out1 = 0.0f;
#pragma unroll
        for (int k = 0; k < (BACKWARD ? 1 : C); ++k) {
          const float val = warp_sum(acc[k]);
          if ((k & 31) == lane) {
            if (k < 32) out0 = val;
            else out1 = val;
          }
        }
        if (lane < C) ti[lane] = out0;
        if (32 + lane < C) ti[32 + lane] = out1;
      }
    } else {
      gr = warp_sum(gr);
      gm = warp_sum(gm);
      if (lane == 0) {
        a.d_rough[i] = gr;
        a.d_metal[i] = gm;
      }
      __syncwarp();
    }
  }
}

template <int ORDER, bool BACKWARD>
static int launch_tt(const TTArgs& a, cudaStream_t stream) {
  constexpr int C = (ORDER + 1) * (ORDER + 1);
  const size_t smem = sizeof(float) * (3 * (size_t)a.S + (size_t)a.S * C + (BACKWARD ? kTTWarps * C : 0));
  cudaFuncSetAttribute(k_training_transfer<ORDER, BACKWARD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_training_transfer<ORDER, BACKWARD>, kTTThreads, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (a.n + kTTWarps - 1) / kTTWarps;
  if (blocks > need) blocks = need;
  k_training_transfer<ORDER, BACKWARD><<<(unsigned)blocks, kTTThreads, smem, counted(stream)>>>(a);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

size_t training_transfer_workspace(int32_t order, int32_t n_dirs) {
  return align_up(sizeof(float) * (size_t)n_dirs * sh_count(order));
}

int training_transfer(const prtgs_gaussians* g, int32_t order, int32_t S, const float* dirs, const float* V,
                      const float* cam_pos, const float* dt, float* t, float* d_roughness, float* d_metallic,
                      void* ws, cudaStream_t stream) {
  if (g->n == 0) return PRTGS_OK;
  float* Y = static_cast<float*>(ws);
  int rc = sh_table(S, order, dirs, Y, stream);
  if (rc != PRTGS_OK) return rc;
  TTArgs a;
  a.n = g->n;
  a.S = S;
  a.dirs = dirs;
  a.Ytab = Y;
  a.V = V;
  a.means = g->means;
  a.normals = g->normals;
  a.rough = g->roughness;
  a.metal = g->metallic;
  for (int k = 0; k < 3; ++k) a.cam[k] = cam_pos[k];
  a.dt = dt;
  a.t = t;
  a.d_rough = d_roughness;
  a.d_metal = d_metallic;
  const bool bwd = dt != nullptr;
  switch (order) {
    case 1: return bwd ? launch_tt<1, true>(a, stream) : launch_tt<1, false>(a, stream);
    case 2: return bwd ? launch_tt<2, true>(a, stream) : launch_tt<2, false>(a, stream);
    case 3: return bwd ? launch_tt<3, true>(a, stream) : launch_tt<3, false>(a, stream);
    case 4: return bwd ? launch_tt<4, true>(a, stream) : launch_tt<4, false>(a, stream);
    case 5: return bwd ? launch_tt<5, true>(a, stream) : launch_tt<5, false>(a, stream);
    case 6: return bwd ? launch_tt<6, true>(a, stream) : launch_tt<6, false>(a, stream);
    default: return PRTGS_ERR_UNSUPPORTED;
  }
}

// ---- pseudo-normal (Eq. 24) -----------------------------------------------------------------
// Pixel (x, y) at depth D is the camera-space point D (a, b, 1), a = (x - cx)/fx, b = (y - cy)/fy.
// With D+- the depths at x +- 1 (and y +- 1), du = D+ - D-, su = D+ + D- (dv, sv likewise), the
// central differences are X_u = (a du + su/fx, b du, du) and X_v = (a dv, b dv + sv/fy, dv), and
//   X_v x X_u = su sv / (fx fy) (p, q, -(a p + b q + 1)),  p = fx du / su,  q = fy dv / sv,
// so the normal facing the camera is R^T (p, q, -(a p + b q + 1)) normalised: du and dv are
// differences of the stored depths themselves, and no two nearly equal 3D points are subtracted.
struct PNCam {
  float r[9];
  float fx, fy, cx, cy;
  int W, H;
};

__global__ void k_pseudo_normal(PNCam c, const float* __restrict__ D, float* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= c.W || y >= c.H) return;
  const int64_t hw = (int64_t)c.W * c.H;
  const int64_t idx = (int64_t)y * c.W + x;
  float ox = 0.0f, oy = 0.0f, oz = 0.0f;
  if (x > 0 && y > 0 && x < c.W - 1 && y < c.H - 1) {
    const float d0 = D[idx], dl = D[idx - 1], dr = D[idx + 1], du = D[idx - c.W], dd = D[idx + c.W];
    if (d0 > 0.0f && dl > 0.0f && dr > 0.0f && du > 0.0f && dd > 0.0f) {
      const float p = c.fx * (dr - dl) / (dr + dl);
      const float q = c.fy * (dd - du) / (dd + du);
      const float a = ((float)x - c.cx) / c.fx, b = ((float)y - c.cy) / c.fy;
      const float pz = -fmaf(a, p, fmaf(b, q, 1.0f));
      const float wx = fmaf(c.r[0], p, fmaf(c.r[3], q, c.r[6] * pz));
      const float wy = fmaf(c.r[1], p, fmaf(c.r[4], q, c.r[7] * pz));
      const float wz = fmaf(c.r[2], p, fmaf(c.r[5], q, c.r[8] * pz));
      const float l2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
      if (l2 > 0.0f) {
        const float il = 1.0f / sqrtf(l2);
        ox = wx * il;
        oy = wy * il;
        oz = wz * il;
      }
    }
  }
  out[idx] = ox;
  out[hw + idx] = oy;
  out[2 * hw + idx] = oz;
}

int pseudo_normal(const prtgs_camera* cam, const float* depth, float* pseudo, cudaStream_t stream) {
  PNCam c;
  for (int k = 0; k < 9; ++k) c.r[k] = cam->rot[k];
  c.fx = cam->fx;
  c.fy = cam->fy;
  c.cx = cam->cx;
  c.cy = cam->cy;
  c.W = cam->width;
  c.H = cam->height;
  if (c.W <= 0 || c.H <= 0) return PRTGS_OK;
  const dim3 block(32, 8);
  const dim3 grid((unsigned)((c.W + 31) / 32), (unsigned)((c.H + 7) / 8));
  k_pseudo_normal<<<grid, block, 0, counted(stream)>>>(c, depth, pseudo);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// ---- normal loss (Eq. 25) -------------------------------------------------------------------
constexpr int kNLThreads = 256;
constexpr int kNLItems = 8;  // pixels per thread per grid pass

static int nl_blocks(int64_t hw) {
  const int64_t b = (hw + kNLThreads * kNLItems - 1) / (kNLThreads * kNLItems);
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

__device__ __forceinline__ bool nl_defined(const float* Np, int64_t hw, int64_t i) {
  return Np[i] != 0.0f || Np[hw + i] != 0.0f || Np[2 * hw + i] != 0.0f;
}

// Per-block sums of |N - N'|^2 over the defined pixels (a fixed grid, so the sum is deterministic).
__global__ void __launch_bounds__(kNLThreads) k_nl_partial(int64_t hw, const float* __restrict__ N,
                                                           const float* __restrict__ Np, double* __restrict__ part) {
  __shared__ double sw[kNLThreads / 32];
  float acc = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hw; i += (int64_t)gridDim.x * blockDim.x) {
    if (!nl_defined(Np, hw, i)) continue;
    const float e0 = N[i] - Np[i], e1 = N[hw + i] - Np[hw + i], e2 = N[2 * hw + i] - Np[2 * hw + i];
    acc = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, acc)));
  }
  double v = (double)acc;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sw[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNLThreads / 32; ++w) s += sw[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_nl_finish(int nb, const double* __restrict__ part, float* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  loss[0] = (float)sqrt(s);
}

__global__ void k_nl_grad(int64_t hw, const float* __restrict__ N, const float* __restrict__ Np,
                          const float* __restrict__ loss, float* __restrict__ dN) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hw) return;
  const float L = loss[0];
  const bool on = L > 0.0f && nl_defined(Np, hw, i);
  const float il = on ? 1.0f / L : 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) dN[k * hw + i] = on ? (N[k * hw + i] - Np[k * hw + i]) * il : 0.0f;
}

size_t normal_loss_workspace(int32_t width, int32_t height) {
  return align_up(sizeof(double) * (size_t)nl_blocks((int64_t)width * height));
}

int normal_loss(int32_t width, int32_t height, const float* normal, const float* pseudo, float* loss,
                float* d_normal, void* ws, cudaStream_t stream) {
  const int64_t hw = (int64_t)width * height;
  const int nb = nl_blocks(hw);
  double* part = static_cast<double*>(ws);
  k_nl_partial<<<nb, kNLThreads, 0, counted(stream)>>>(hw, normal, pseudo, part);
  k_nl_finish<<<1, 32, 0, counted(stream)>>>(nb, part, loss);
  if (d_normal && hw > 0)
    k_nl_grad<<<(unsigned)((hw + 255) / 256), 256, 0, counted(stream)>>>(hw, normal, pseudo, loss, d_normal);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

}  // namespace prtgs
