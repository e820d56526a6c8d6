// Radiance-transfer precompute for Gaussian splats (Sec. 4.4-4.5).
//
//  k_trace   one warp per receiver (persistent, work counter). The warp compacts the
//            directions with n.w > 0, then its lanes pull rays from that list and trace each
//            through the LBVH: visibility V = prod (1 - alpha_j) over the Gaussians whose
//            closest approach to the ray is inside their 3-sigma ellipsoid ahead of the
//            origin (Eq. 27 read as the Gaussian's maximum along the ray; Eq. 4 along a ray).
//            With the bounce flag the hits are visited in (t*, position) order through a
//            small sorted k-buffer, which gives the prefix transmittance of Eq. 26 and the
//            argmax weight of the index matrix (Sec. 4.4). Finally the warp projects
//            V (n.w)^+ onto the SH basis (Eq. 29 with Eq. 9, weight 4 pi / S) with a
//            compensated sum and a warp-shuffle reduction.
//  k_bounce  one warp per receiver: T = P + sum_s w (n.w_s)^+ (rho_j / pi) P_j (Eq. 33).
//  k_glossy  one block per glossy splat: M = sum_s sum_o w^2 Y(w_s) k(w_s,w_o) (n.w_s)^+ V_s
//            Y(w_o)^T (Eq. 40), factored as U^T B with B_s = sum_o k(s,o) Y(o).
#include <float.h>

#include "common.cuh"
#include "internal.h"

namespace prtgs {

constexpr int kTraceWarps = 4;
constexpr int kTraceThreads = 32 * kTraceWarps;
constexpr int kKBuf = 8;
constexpr int kMaxDirs = 1024;

struct TraceArgs {
  const float4* nodes;
  const float4* recs;
  const int32_t* order;
  const int32_t* roots;
  const int64_t* offsets;
  int n_scenes;
  int64_t n;
  const float* dirs;
  int S;
  int sh_order;
  float t_min;
  float filter_t;
  uint32_t flags;
  float* P;
  int32_t* idx;
  float* Vg;                 // [n_glossy, S] visibility of glossy receivers (nullable)
  const int32_t* glossy_slot; // [n] slot of each Gaussian in Vg, -1 if none (nullable)
  int32_t* status;
  unsigned int* work;
};

struct Ray {
  float ox, oy, oz, dx, dy, dz;
  float ix, iy, iz;     // 1/d (safe)
  float oix, oiy, oiz;  // o/d
};

__device__ __forceinline__ float safe_inv(float v) {
  const float tiny = 1e-20f;
  return 1.0f / (fabsf(v) > tiny ? v : copysignf(tiny, v));
}

__device__ __forceinline__ void make_ray(Ray& r, float ox, float oy, float oz, float dx, float dy, float dz) {
  r.ox = ox; r.oy = oy; r.oz = oz; r.dx = dx; r.dy = dy; r.dz = dz;
  r.ix = safe_inv(dx); r.iy = safe_inv(dy); r.iz = safe_inv(dz);
  r.oix = ox * r.ix; r.oiy = oy * r.iy; r.oiz = oz * r.iz;
}

// Slab test against [lo, hi]; returns the entry/exit parameters clipped to t >= 0.
__device__ __forceinline__ bool slab(const Ray& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                     float& tn, float& tf) {
  float t0x = fmaf(lx, r.ix, -r.oix), t1x = fmaf(hx, r.ix, -r.oix);
  float t0y = fmaf(ly, r.iy, -r.oiy), t1y = fmaf(hy, r.iy, -r.oiy);
  float t0z = fmaf(lz, r.iz, -r.oiz), t1z = fmaf(hz, r.iz, -r.oiz);
  tn = fmaxf(fmaxf(fminf(t0x, t1x), fminf(t0y, t1y)), fmaxf(fminf(t0z, t1z), 0.0f));
  tf = fminf(fminf(fmaxf(t0x, t1x), fmaxf(t0y, t1y)), fmaxf(t0z, t1z));
  return tn <= tf;
}

// Exact ray / Gaussian test (closest approach in the whitened frame A = diag(1/s) R^T).
// The offset of the closest point from the mean is formed with one fused multiply-add per
// component from the error-free difference o - mu, so D^2 carries no cancellation error from
// far-away Gaussians. Returns true for a hit (t* > 0, D^2 <= 9).
__device__ __forceinline__ bool gauss_hit(const float4* __restrict__ recs, int pos, const Ray& r, float& t_out,
                                          float& alpha_out, float& m_out) {
  const float4 q0 = __ldg(recs + 4 * pos);
  const float4 q1 = __ldg(recs + 4 * pos + 1);
  const float4 q2 = __ldg(recs + 4 * pos + 2);
  const float4 q3 = __ldg(recs + 4 * pos + 3);
  float ux, uy, uz, ex, ey, ez;
  two_sum(r.ox, -q0.x, ux, ex);
  two_sum(r.oy, -q0.y, uy, ey);
  two_sum(r.oz, -q0.z, uz, ez);
  // rows of A
  const float a00 = q1.x, a01 = q1.y, a02 = q1.z, a10 = q1.w, a11 = q2.x, a12 = q2.y, a20 = q2.z, a21 = q2.w,
              a22 = q3.x;
  float dax = fmaf(a00, r.dx, fmaf(a01, r.dy, a02 * r.dz));
  float day = fmaf(a10, r.dx, fmaf(a11, r.dy, a12 * r.dz));
  float daz = fmaf(a20, r.dx, fmaf(a21, r.dy, a22 * r.dz));
  float dd = fmaf(dax, dax, fmaf(day, day, daz * daz));
  float uax = fmaf(a00, ux, fmaf(a01, uy, a02 * uz));
  float uay = fmaf(a10, ux, fmaf(a11, uy, a12 * uz));
  float uaz = fmaf(a20, ux, fmaf(a21, uy, a22 * uz));
  float ud = fmaf(uax, dax, fmaf(uay, day, uaz * daz));
  float uu = fmaf(uax, uax, fmaf(uay, uay, uaz * uaz));
  float rdd = 1.0f / dd;
  float t0 = -ud * rdd;
  // cheap rejection with margins above the FP32 error of this first estimate
  float wx0 = fmaf(t0, dax, uax), wy0 = fmaf(t0, day, uay), wz0 = fmaf(t0, daz, uaz);
  float d2a = fmaf(wx0, wx0, fmaf(wy0, wy0, wz0 * wz0));
  float un = sqrtf(uu);
  if (d2a > 9.0f + 1e-3f + 5e-5f * un) return false;
  if (t0 < -(4e-6f * un * sqrtf(rdd) + 1e-30f)) return false;
  // refinement at t0: w = o + t0 d - mu, exact up to one rounding per component
  float wx = fmaf(t0, r.dx, ux) + ex;
  float wy = fmaf(t0, r.dy, uy) + ey;
  float wz = fmaf(t0, r.dz, uz) + ez;
  float wax = fmaf(a00, wx, fmaf(a01, wy, a02 * wz));
  float way = fmaf(a10, wx, fmaf(a11, wy, a12 * wz));
  float waz = fmaf(a20, wx, fmaf(a21, wy, a22 * wz));
  float wd = fmaf(wax, dax, fmaf(way, day, waz * daz));
  float dt = -wd * rdd;
  float ts = t0 + dt;
  float d2 = fmaxf(fmaf(wax, wax, fmaf(way, way, waz * waz)) + dt * wd, 0.0f);
  if (!(ts > 0.0f) || !(d2 <= 9.0f)) return false;
  t_out = ts;
  alpha_out = q0.w * expf(-0.5f * d2);
  m_out = fmaxf(-(r.dx * q3.y + r.dy * q3.z + r.dz * q3.w), 0.0f);
  return true;
}

// Children outside the tree are reported and dropped (a well-formed tree never has them).
__device__ __forceinline__ bool child_ok(int c, int64_t n, int32_t* status) {
  bool ok = c >= 0 ? (int64_t)c < n - 1 : (int64_t)(~c) < n;
  if (!ok) set_status(status, PRTGS_STATUS_BAD_INDEX);
  return ok;
}

__device__ __forceinline__ void load_node(const float4* __restrict__ nodes, int node, float4& n0, float4& n1,
                                          float4& n2, int& c0, int& c1) {
  n0 = __ldg(nodes + 4 * node);
  n1 = __ldg(nodes + 4 * node + 1);
  n2 = __ldg(nodes + 4 * node + 2);
  const float4 n3 = __ldg(nodes + 4 * node + 3);
  c0 = __float_as_int(n3.x);
  c1 = __float_as_int(n3.y);
}

// Unordered traversal: multiplies (1 - alpha) of every hit with key > (t_last, p_last) into
// T, stopping early once T < t_min. Returns T.
__device__ float trace_unordered(const TraceArgs& a, const Ray& r, int root, int self, float T, float t_last,
                                 int p_last) {
  float t, al, m;
  const float t_prune = t_last * (1.0f - 1e-5f) - 1e-6f;
  if (root < 0) {
    int pos = ~root;
    if (root != INT32_MIN && pos != self && gauss_hit(a.recs, pos, r, t, al, m) &&
        (t > t_last || (t == t_last && pos > p_last)))
      T *= 1.0f - al;
    return T;
  }
  int stack[kStackDepth];
  int sp = 0;
  int node = root;
  const int64_t max_visits = 2 * a.n + 64;
  for (int64_t visits = 0;; ++visits) {
    if (visits > max_visits) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      break;
    }
    float4 n0, n1, n2;
    int c0, c1;
    load_node(a.nodes, node, n0, n1, n2, c0, c1);
    float tn0, tf0, tn1, tf1;
    bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, tn0, tf0) && tf0 >= t_prune && child_ok(c0, a.n, a.status);
    bool h1 = slab(r, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, tn1, tf1) && tf1 >= t_prune && child_ok(c1, a.n, a.status);
    if (h0 && c0 < 0) {
      int pos = ~c0;
      if (pos != self && gauss_hit(a.recs, pos, r, t, al, m) && (t > t_last || (t == t_last && pos > p_last)))
        T *= 1.0f - al;
      h0 = false;
    }
    if (h1 && c1 < 0) {
      int pos = ~c1;
      if (pos != self && gauss_hit(a.recs, pos, r, t, al, m) && (t > t_last || (t == t_last && pos > p_last)))
        T *= 1.0f - al;
      h1 = false;
    }
    if (T < a.t_min) break;
    if (h0 && h1) {
      bool first0 = tn0 <= tn1;
      if (sp < kStackDepth) stack[sp++] = first0 ? c1 : c0;
      else set_status(a.status, PRTGS_STATUS_STACK_OVERFLOW);
      node = first0 ? c0 : c1;
    } else if (h0) {
      node = c0;
    } else if (h1) {
      node = c1;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
  return T;
}

// Sorted insertion of (t, pos, alpha, m) into the K-buffer; the largest entry drops out.
__device__ __forceinline__ void kbuf_insert(float (&bt)[kKBuf], int (&bp)[kKBuf], float (&ba)[kKBuf],
                                            float (&bm)[kKBuf], float t, int p, float al, float m) {
#pragma unroll
  for (int k = 0; k < kKBuf; ++k) {
    bool less = (t < bt[k]) || (t == bt[k] && p < bp[k]);
    if (less) {
      float tt = bt[k]; bt[k] = t; t = tt;
      int pp = bp[k]; bp[k] = p; p = pp;
      float aa = ba[k]; ba[k] = al; al = aa;
      float mm = bm[k]; bm[k] = m; m = mm;
    }
  }
}

// One ordered pass: the K nearest hits with key > (t_last, p_last).
__device__ void trace_kbuf(const TraceArgs& a, const Ray& r, int root, int self, float t_last, int p_last,
                           float (&bt)[kKBuf], int (&bp)[kKBuf], float (&ba)[kKBuf], float (&bm)[kKBuf]) {
#pragma unroll
  for (int k = 0; k < kKBuf; ++k) {
    bt[k] = FLT_MAX;
    bp[k] = INT32_MAX;
    ba[k] = 0.f;
    bm[k] = 0.f;
  }
  float t, al, m;
  const float t_lo = t_last * (1.0f - 1e-5f) - 1e-6f;
  if (root < 0) {
    int pos = ~root;
    if (root != INT32_MIN && pos != self && gauss_hit(a.recs, pos, r, t, al, m) &&
        (t > t_last || (t == t_last && pos > p_last)))
      kbuf_insert(bt, bp, ba, bm, t, pos, al, m);
    return;
  }
  int stack[kStackDepth];
  int sp = 0;
  int node = root;
  const int64_t max_visits = 2 * a.n + 64;
  for (int64_t visits = 0;; ++visits) {
    if (visits > max_visits) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      break;
    }
    float4 n0, n1, n2;
    int c0, c1;
    load_node(a.nodes, node, n0, n1, n2, c0, c1);
    const float t_hi = bt[kKBuf - 1] == FLT_MAX ? FLT_MAX : bt[kKBuf - 1] * (1.0f + 1e-5f) + 1e-6f;
    float tn0, tf0, tn1, tf1;
    bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, tn0, tf0) && tf0 >= t_lo && tn0 <= t_hi &&
              child_ok(c0, a.n, a.status);
    bool h1 = slab(r, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, tn1, tf1) && tf1 >= t_lo && tn1 <= t_hi &&
              child_ok(c1, a.n, a.status);
    if (h0 && c0 < 0) {
      int pos = ~c0;
      if (pos != self && gauss_hit(a.recs, pos, r, t, al, m) && (t > t_last || (t == t_last && pos > p_last)))
        kbuf_insert(bt, bp, ba, bm, t, pos, al, m);
      h0 = false;
    }
    if (h1 && c1 < 0) {
      int pos = ~c1;
      if (pos != self && gauss_hit(a.recs, pos, r, t, al, m) && (t > t_last || (t == t_last && pos > p_last)))
        kbuf_insert(bt, bp, ba, bm, t, pos, al, m);
      h1 = false;
    }
    if (h0 && h1) {
      bool first0 = tn0 <= tn1;
      if (sp < kStackDepth) stack[sp++] = first0 ? c1 : c0;
      else set_status(a.status, PRTGS_STATUS_STACK_OVERFLOW);
      node = first0 ? c0 : c1;
    } else if (h0) {
      node = c0;
    } else if (h1) {
      node = c1;
    } else {
      if (sp == 0) break;
      node = stack[--sp];
    }
  }
}

// Visibility and (optionally) the index-matrix entry of one ray.
template <bool BOUNCE>
__device__ float trace_ray(const TraceArgs& a, const Ray& r, int root, int self, int& best) {
  best = -1;
  if (!BOUNCE) return trace_unordered(a, r, root, self, 1.0f, -FLT_MAX, INT32_MIN);
  float T = 1.0f, wbest = 0.0f;
  float t_last = -FLT_MAX;
  int p_last = INT32_MIN;
  float bt[kKBuf], ba[kKBuf], bm[kKBuf];
  int bp[kKBuf];
  for (int64_t pass = 0;; ++pass) {
    if (pass > a.n / kKBuf + 1) {  // every pass consumes kKBuf hits
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      return T;
    }
    trace_kbuf(a, r, root, self, t_last, p_last, bt, bp, ba, bm);
#pragma unroll
    for (int k = 0; k < kKBuf; ++k) {
      if (bt[k] == FLT_MAX) break;
      float W = ba[k] * T * bm[k];
      if (T <= a.filter_t && W > wbest) {
        wbest = W;
        best = bp[k];
      }
      T *= 1.0f - ba[k];
    }
    if (bt[kKBuf - 1] == FLT_MAX) return T;  // every hit seen
    t_last = bt[kKBuf - 1];
    p_last = bp[kKBuf - 1];
    if (T < a.t_min) return T;
    if (T <= wbest) break;  // no later hit can outweigh the current best (W_later <= T)
  }
  return trace_unordered(a, r, root, self, T, t_last, p_last);
}

__device__ __forceinline__ float ray_cos(float nx, float ny, float nz, const float* d) {
  return fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2]));
}

template <bool BOUNCE>
__global__ void __launch_bounds__(kTraceThreads) k_trace(TraceArgs a) {
  extern __shared__ float smem[];
  float* sdir = smem;                                     // [S*3]
  float* svis = sdir + 3 * a.S;                           // [warps][S]
  unsigned short* slist = reinterpret_cast<unsigned short*>(svis + kTraceWarps * a.S);  // [warps][S]
  __shared__ unsigned int s_next[kTraceWarps];
  for (int i = threadIdx.x; i < 3 * a.S; i += blockDim.x) sdir[i] = a.dirs[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* vis = svis + warp * a.S;
  unsigned short* list = slist + warp * a.S;
  const int C = sh_count(a.sh_order);
  const float wq = 4.0f * kPi / (float)a.S;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (;;) {
    unsigned int w = 0;
    if (lane == 0) w = atomicAdd(a.work, 1u);
    w = __shfl_sync(0xffffffffu, w, 0);
    if ((int64_t)w >= a.n) break;
    const int self = (int)w;  // receivers are visited in sorted (Morton) order
    const float4 q0 = __ldg(a.recs + 4 * self);
    const float4 q3 = __ldg(a.recs + 4 * self + 3);
    const int gid = a.order[self];
    const int b = find_scene(a.offsets, a.n_scenes, gid);
    int root = a.roots[b];
    if (root != INT32_MIN && !child_ok(root, a.n, a.status)) root = INT32_MIN;
    // compact the directions of the upper hemisphere
    int cnt = 0;
    for (int base = 0; base < a.S; base += 32) {
      int s = base + lane;
      float c = s < a.S ? ray_cos(q3.y, q3.z, q3.w, sdir + 3 * s) : 0.0f;
      bool up = c > 0.0f;
      unsigned m = __ballot_sync(0xffffffffu, up);
      if (up) list[cnt + __popc(m & lt_mask)] = (unsigned short)s;
      if (s < a.S) vis[s] = 0.0f;
      if (BOUNCE && s < a.S && !up) a.idx[(int64_t)gid * a.S + s] = -1;
      cnt += __popc(m);
    }
    if (lane == 0) s_next[warp] = 0;
    __syncwarp();
    // lanes pull rays until the list is exhausted
    for (;;) {
      unsigned int t = atomicAdd(&s_next[warp], 1u);
      if ((int)t >= cnt) break;
      int s = list[t];
      Ray r;
      make_ray(r, q0.x, q0.y, q0.z, sdir[3 * s], sdir[3 * s + 1], sdir[3 * s + 2]);
      int best = -1;
      float V = 1.0f;
      if (a.flags & PRTGS_SHADOW) V = trace_ray<BOUNCE>(a, r, root, self, best);
      vis[s] = V;
      if (BOUNCE) a.idx[(int64_t)gid * a.S + s] = best >= 0 ? a.order[best] : -1;
    }
    __syncwarp();
    // SH projection of V (n.w)^+ with a compensated sum per lane, then across the warp
    float ps[kMaxC], pc[kMaxC];
#pragma unroll
    for (int k = 0; k < kMaxC; ++k) { ps[k] = 0.f; pc[k] = 0.f; }
    for (int s = lane; s < a.S; s += 32) {
      const float* d = sdir + 3 * s;
      float c = ray_cos(q3.y, q3.z, q3.w, d);
      if (!(c > 0.0f)) continue;
      float v = vis[s] * c * wq;
      float Y[kMaxC];
      sh_eval_dyn(a.sh_order, d[0], d[1], d[2], Y);
#pragma unroll
      for (int k = 0; k < kMaxC; ++k) {
        if (k < C) {
          float t, e;
          two_sum(ps[k], v * Y[k], t, e);
          ps[k] = t;
          pc[k] += e;
        }
      }
    }
    float mine = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxC; ++k) {
      if (k < C) {
        float val = warp_comp_sum(ps[k], pc[k]);
        if (lane == k) mine = val;
      }
    }
    if (lane < C) a.P[(int64_t)gid * C + lane] = mine;
    if (a.Vg) {
      int slot = a.glossy_slot[gid];
      if (slot >= 0)
        for (int s = lane; s < a.S; s += 32) a.Vg[(int64_t)slot * a.S + s] = vis[s];
    }
    __syncwarp();
  }
}

// ---- one-bounce self-transfer (Eq. 33) -------------------------------------------------------
__global__ void k_bounce(int64_t n, int C, int S, const float* __restrict__ dirs, const float* __restrict__ normals,
                         const float* __restrict__ albedo, const float* __restrict__ P,
                         const int32_t* __restrict__ idx, float* __restrict__ T, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int k = lane & 15, half = lane >> 4;
  const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
  const float wq = 4.0f * kPi / (float)S;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
  for (int base = 0; base < S; base += 32) {
    int s = base + lane;
    int jl = s < S ? idx[i * S + s] : -1;
    if (jl >= n) {
      set_status(status, PRTGS_STATUS_BAD_INDEX);
      jl = -1;
    }
    float cl = 0.f;
    if (jl >= 0) cl = fmaxf(fmaf(nx, dirs[3 * s], fmaf(ny, dirs[3 * s + 1], nz * dirs[3 * s + 2])), 0.f);
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      int src = 2 * q + half;
      int j = __shfl_sync(0xffffffffu, jl, src);
      float c = __shfl_sync(0xffffffffu, cl, src);
      if (j < 0) continue;
      float coef = wq * c * (1.0f / kPi);
      float pj = k < C ? __ldg(P + (int64_t)j * C + k) : 0.f;
      float cp = coef * pj;
      acc0 = fmaf(cp, __ldg(albedo + 3 * j), acc0);
      acc1 = fmaf(cp, __ldg(albedo + 3 * j + 1), acc1);
      acc2 = fmaf(cp, __ldg(albedo + 3 * j + 2), acc2);
    }
  }
  acc0 += __shfl_xor_sync(0xffffffffu, acc0, 16);
  acc1 += __shfl_xor_sync(0xffffffffu, acc1, 16);
  acc2 += __shfl_xor_sync(0xffffffffu, acc2, 16);
  if (half == 0 && k < C) {
    float p = P[i * C + k];
    T[(i * 3 + 0) * C + k] = p + acc0;
    T[(i * 3 + 1) * C + k] = p + acc1;
    T[(i * 3 + 2) * C + k] = p + acc2;
  }
}

// ---- glossy transfer matrices (Eq. 36-41) ---------------------------------------------------
constexpr int kGlossyThreads = 128;

// k(w_i, w_o) = (1 - m) + pi f_s, f_s = D F G / (4 (n.w_i)(n.w_o)); GGX D (alpha = r^2),
// Schlick F (F0 = 0.04, on w_o.h), Smith-Schlick G (k = alpha / 2). ni, no > 0.
__device__ __forceinline__ float brdf_kernel(float nx, float ny, float nz, const float* wi, const float* wo,
                                             float ni, float no, float alpha, float metal) {
  float hx = wi[0] + wo[0], hy = wi[1] + wo[1], hz = wi[2] + wo[2];
  float rh = rsqrtf(fmaf(hx, hx, fmaf(hy, hy, hz * hz)));
  float nh = fmaf(nx, hx, fmaf(ny, hy, nz * hz)) * rh;
  float oh = fminf(fmaxf(fmaf(wo[0], hx, fmaf(wo[1], hy, wo[2] * hz)) * rh, 0.f), 1.f);
  float a2 = alpha * alpha;
  float den = fmaf(nh * nh, a2 - 1.0f, 1.0f);
  float D = a2 / (kPi * den * den);
  float x = 1.0f - oh;
  float x2 = x * x;
  float F = fmaf(0.96f, x2 * x2 * x, 0.04f);
  float kk = 0.5f * alpha;
  float gi = 1.0f / fmaf(ni, 1.0f - kk, kk);
  float go = 1.0f / fmaf(no, 1.0f - kk, kk);
  return (1.0f - metal) + kPi * 0.25f * D * F * gi * go;
}

__global__ void __launch_bounds__(kGlossyThreads) k_glossy(int64_t n_glossy, const int32_t* __restrict__ glossy_ids,
                                                           int S, int order, const float* __restrict__ dirs,
                                                           const float* __restrict__ normals,
                                                           const float* __restrict__ roughness,
                                                           const float* __restrict__ metallic,
                                                           const float* __restrict__ Vg, float* __restrict__ M) {
  extern __shared__ float smem[];
  const int C = sh_count(order);
  float* sdir = smem;              // [S*3]
  float* sY = sdir + 3 * S;        // [S][C]
  float* sU = sY + S * C;          // [S][C]   w^2 (n.w_s)^+ V_s Y(w_s)
  float* sB = sU + S * C;          // [S][C]   sum_o k(s,o) Y(w_o)
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) sdir[i] = dirs[i];
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    float Y[kMaxC];
    sh_eval_dyn(order, sdir[3 * s], sdir[3 * s + 1], sdir[3 * s + 2], Y);
    for (int k = 0; k < C; ++k) sY[s * C + k] = Y[k];
  }
  __syncthreads();
  const float wq = 4.0f * kPi / (float)S;
  for (int64_t g = blockIdx.x; g < n_glossy; g += gridDim.x) {
    const int64_t i = glossy_ids[g];
    const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
    const float r = roughness[i];
    const float alpha = r * r, metal = metallic[i];
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      const float* wi = sdir + 3 * s;
      float ni = fmaf(nx, wi[0], fmaf(ny, wi[1], nz * wi[2]));
      float v = Vg[g * S + s];
      float Bs[kMaxC];
#pragma unroll
      for (int k = 0; k < kMaxC; ++k) Bs[k] = 0.f;
      float u = 0.f;
      if (ni > 0.0f && v > 0.0f) {
        u = wq * wq * ni * v;
        for (int o = 0; o < S; ++o) {
          const float* wo = sdir + 3 * o;
          float no = fmaf(nx, wo[0], fmaf(ny, wo[1], nz * wo[2]));
          if (!(no > 0.0f)) continue;
          float kv = brdf_kernel(nx, ny, nz, wi, wo, ni, no, alpha, metal);
#pragma unroll
          for (int k = 0; k < kMaxC; ++k)
            if (k < C) Bs[k] = fmaf(kv, sY[o * C + k], Bs[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < kMaxC; ++k) {
        if (k < C) {
          sB[s * C + k] = Bs[k];
          sU[s * C + k] = u * sY[s * C + k];
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
      int ra = e / C, cb = e % C;
      float acc = 0.f;
      for (int s = 0; s < S; ++s) acc = fmaf(sU[s * C + ra], sB[s * C + cb], acc);
      M[(g * C + ra) * C + cb] = acc;
    }
    __syncthreads();
  }
}

__global__ void k_glossy_slots(int64_t n, const uint8_t* __restrict__ mask, const uint32_t* __restrict__ incl,
                               int32_t* __restrict__ slot, int32_t* __restrict__ ids) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (mask[i]) {
    int32_t s = (int32_t)incl[i] - 1;
    slot[i] = s;
    ids[s] = (int32_t)i;
  } else {
    slot[i] = -1;
  }
}

__global__ void k_mask_u32(int64_t n, const uint8_t* __restrict__ mask, uint32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = mask[i] ? 1u : 0u;
}

static size_t trace_smem(int S) { return sizeof(float) * 3 * S + kTraceWarps * S * (sizeof(float) + 2); }
static size_t glossy_smem(int S, int C) { return sizeof(float) * (3 * S + 3 * (size_t)S * C); }

size_t transfer_workspace(int64_t n, int64_t n_glossy, const prtgs_transfer_params* p) {
  size_t b = align_up(sizeof(unsigned int));
  if (p->flags & PRTGS_GLOSSY) {
    b += 2 * align_up(sizeof(int32_t) * n) + align_up(sizeof(uint32_t) * n) + scan_workspace(n) +
         align_up(sizeof(uint32_t)) + align_up(sizeof(float) * (size_t)n_glossy * p->n_dirs);
  }
  return b;
}

static int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int precompute_transfer(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p, float* P,
                        float* T, int32_t* idx, float* M, int64_t n_glossy, int32_t* status, void* ws,
                        cudaStream_t stream) {
  const int64_t n = g->n;
  if (n == 0) return PRTGS_OK;
  const int S = p->n_dirs;
  const int C = sh_count(p->sh_order);
  const bool bounce = (p->flags & PRTGS_BOUNCE) != 0;
  const bool glossy = (p->flags & PRTGS_GLOSSY) != 0 && n_glossy > 0;
  Carver c(ws);
  unsigned int* work = c.take<unsigned int>(1);
  int32_t* slot = nullptr;
  int32_t* gids = nullptr;
  float* Vg = nullptr;
  if (p->flags & PRTGS_GLOSSY) {
    slot = c.take<int32_t>(n);
    gids = c.take<int32_t>(n);
    uint32_t* flags = c.take<uint32_t>(n);
    void* sws = c.take<char>(scan_workspace(n));
    uint32_t* total = c.take<uint32_t>(1);
    Vg = c.take<float>((size_t)n_glossy * S);
    k_mask_u32<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(n, g->glossy_mask, flags);
    int rc = scan_u32(flags, flags, n, false, total, sws, stream);
    if (rc != PRTGS_OK) return rc;
    k_glossy_slots<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(n, g->glossy_mask, flags, slot, gids);
  }
  cudaMemsetAsync(work, 0, sizeof(unsigned int), stream);
  TraceArgs a;
  a.nodes = reinterpret_cast<const float4*>(bvh->nodes);
  a.recs = reinterpret_cast<const float4*>(bvh->records);
  a.order = bvh->order;
  a.roots = bvh->roots;
  a.offsets = bvh->scene_offsets;
  a.n_scenes = bvh->n_scenes;
  a.n = n;
  a.dirs = p->dirs;
  a.S = S;
  a.sh_order = p->sh_order;
  a.t_min = p->t_min;
  a.filter_t = p->same_surface_t;
  a.flags = p->flags;
  a.P = P;
  a.idx = idx;
  a.Vg = glossy ? Vg : nullptr;
  a.glossy_slot = slot;
  a.status = status;
  a.work = work;
  size_t smem = trace_smem(S);
  int sms = device_sms();
  int per_sm = 0;
  if (bounce) {
    cudaFuncSetAttribute(k_trace<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<true>, kTraceThreads, smem);
    k_trace<true><<<sms * (per_sm > 0 ? per_sm : 1), kTraceThreads, smem, stream>>>(a);
  } else {
    cudaFuncSetAttribute(k_trace<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<false>, kTraceThreads, smem);
    k_trace<false><<<sms * (per_sm > 0 ? per_sm : 1), kTraceThreads, smem, stream>>>(a);
  }
  PRTGS_CHECK_LAUNCH();
  if (bounce) {
    k_bounce<<<(unsigned)((n + 7) / 8), 256, 0, stream>>>(n, C, S, p->dirs, g->normals, g->albedo, P, idx, T,
                                                         status);
    PRTGS_CHECK_LAUNCH();
  }
  if (glossy) {
    size_t gsm = glossy_smem(S, C);
    cudaFuncSetAttribute(k_glossy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    int gper = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gper, k_glossy, kGlossyThreads, gsm);
    int64_t blocks = (int64_t)sms * (gper > 0 ? gper : 1);
    if (blocks > n_glossy) blocks = n_glossy;
    k_glossy<<<(unsigned)blocks, kGlossyThreads, gsm, stream>>>(n_glossy, gids, S, p->sh_order, p->dirs, g->normals,
                                                               g->roughness, g->metallic, Vg, M);
    PRTGS_CHECK_LAUNCH();
  }
  return PRTGS_OK;
}

int transfer_check_dirs(int S) { return (S > 0 && S <= kMaxDirs) ? PRTGS_OK : PRTGS_ERR_UNSUPPORTED; }

}  // namespace prtgs
