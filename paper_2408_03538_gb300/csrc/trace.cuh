// Device-side pieces shared by the transfer kernels (per-ray walks in transfer.cu, warp-packet
// walks in packet.cu): kernel arguments, the ray / box / Gaussian tests, the per-ray visitors
// that turn hits into visibility, index-matrix candidates and prefix transmittances.
#pragma once

#include <float.h>

#include "common.cuh"
#include "internal.h"

namespace prtgs {

constexpr int kTraceWarps = 4;
// Resident 128-thread blocks per SM the kernels are compiled for (register caps chosen by
// measurement on the 100k surface workload: the visibility-only walk is fastest at 64
// registers; the bounce walk at 72 (7 blocks: 335 ms for the transfer against 345, 360 and 374 ms
// at 6, 5 and 4 blocks, 342 ms at 8); the later index rounds at 128).
constexpr int kShadowMinBlocks = 8;
#ifndef PRTGS_BOUNCE_MIN_BLOCKS
#define PRTGS_BOUNCE_MIN_BLOCKS 7
#endif
constexpr int kBounceMinBlocks = PRTGS_BOUNCE_MIN_BLOCKS;
constexpr int kRoundsMinBlocks = 4;
#ifndef PRTGS_PREFIX_MIN_BLOCKS
#define PRTGS_PREFIX_MIN_BLOCKS 8  // the first index round: 336 ms against 340 / 350 at 6 / 4
#endif
constexpr int kPrefixMinBlocks = PRTGS_PREFIX_MIN_BLOCKS;
#ifndef PRTGS_ROUND_HITS
#define PRTGS_ROUND_HITS 12
#endif
constexpr int kRoundHits = PRTGS_ROUND_HITS;  // hits per round in k_rounds (12: 296 ms, 8: 307, 16: 310)
constexpr int kTraceThreads = 32 * kTraceWarps;
constexpr int kDefaultIndexBuffer = 4;
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
  const float* Ytab;          // [S][C] SH of the directions for orders above 3 (else unused)
  float t_min;
  float filter_t;
  uint32_t flags;
  float* P;
  int32_t* idx;
  float* Vg;                 // [n_glossy, S] visibility of glossy receivers (nullable)
  const int32_t* glossy_slot; // [n] slot of each Gaussian in Vg, -1 if none (nullable)
  int32_t* status;
  unsigned int* work;
  unsigned long long* stats;  // nodes, leaves, hits, index rounds, traced rays (nullable)
  int64_t r0, r1;             // receivers [r0, r1) of this batch, in sorted (Morton) positions
  void* queue;                // [batch * S] per-ray candidate records, resolved by k_prefix / k_rounds
  uint32_t* pending;          // [batch * S] 1 = the ray has index-matrix candidates
  unsigned int* queue_count;
  int packet_dirs;            // directions per packet work item (0: chosen from the problem size)
};


__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned v) {
  unsigned long long x = v;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

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

// Exact ray / Gaussian test (closest approach in the whitened frame A = diag(1/s) R^T), in two
// parts: the terms that depend only on the Gaussian and the ray direction (shared by every ray of
// a packet, which all have the same direction) and the per-ray rest. The offset of the closest
// point from the mean is formed with one fused multiply-add per component from the error-free
// difference o - mu, so D^2 carries no cancellation error from far-away Gaussians.
struct DirTerms {
  float dax, day, daz;  // A d
  float rdd;            // 1 / |A d|^2
  float srdd;           // sqrt(rdd)
  float m;              // max(-d . n_j, 0), the facing term of Eq. 26
};

__device__ __forceinline__ DirTerms dir_terms(const float4& q1, const float4& q2, const float4& q3, float dx, float dy,
                                              float dz) {
  DirTerms t;
  t.dax = fmaf(q1.x, dx, fmaf(q1.y, dy, q1.z * dz));
  t.day = fmaf(q1.w, dx, fmaf(q2.x, dy, q2.y * dz));
  t.daz = fmaf(q2.z, dx, fmaf(q2.w, dy, q3.x * dz));
  const float dd = fmaf(t.dax, t.dax, fmaf(t.day, t.day, t.daz * t.daz));
  t.rdd = 1.0f / dd;
  t.srdd = sqrtf(t.rdd);
  t.m = fmaxf(-fmaf(dx, q3.y, fmaf(dy, q3.z, dz * q3.w)), 0.0f);
  return t;
}

// The per-ray part: q0 = (mu, opacity), q1, q2, a22 = rows of A. True for a hit (t* > 0, D^2 <= 9).
__device__ __forceinline__ bool hit_eval(const float4& q0, const float4& q1, const float4& q2, float a22,
                                         const DirTerms& dt, const Ray& r, float& t_out, float& alpha_out) {
  float ux, uy, uz, ex, ey, ez;
  two_sum(r.ox, -q0.x, ux, ex);
  two_sum(r.oy, -q0.y, uy, ey);
  two_sum(r.oz, -q0.z, uz, ez);
  const float a00 = q1.x, a01 = q1.y, a02 = q1.z, a10 = q1.w, a11 = q2.x, a12 = q2.y, a20 = q2.z, a21 = q2.w;
  const float uax = fmaf(a00, ux, fmaf(a01, uy, a02 * uz));
  const float uay = fmaf(a10, ux, fmaf(a11, uy, a12 * uz));
  const float uaz = fmaf(a20, ux, fmaf(a21, uy, a22 * uz));
  const float ud = fmaf(uax, dt.dax, fmaf(uay, dt.day, uaz * dt.daz));
  const float uu = fmaf(uax, uax, fmaf(uay, uay, uaz * uaz));
  const float t0 = -ud * dt.rdd;
  // cheap rejection with margins above the FP32 error of this first estimate
  const float wx0 = fmaf(t0, dt.dax, uax), wy0 = fmaf(t0, dt.day, uay), wz0 = fmaf(t0, dt.daz, uaz);
  const float d2a = fmaf(wx0, wx0, fmaf(wy0, wy0, wz0 * wz0));
  const float un = sqrtf(uu);
  if (d2a > 9.0f + 1e-3f + 5e-5f * un) return false;
  if (t0 < -(4e-6f * un * dt.srdd + 1e-30f)) return false;
  // refinement at t0: w = o + t0 d - mu, exact up to one rounding per component
  const float wx = fmaf(t0, r.dx, ux) + ex;
  const float wy = fmaf(t0, r.dy, uy) + ey;
  const float wz = fmaf(t0, r.dz, uz) + ez;
  const float wax = fmaf(a00, wx, fmaf(a01, wy, a02 * wz));
  const float way = fmaf(a10, wx, fmaf(a11, wy, a12 * wz));
  const float waz = fmaf(a20, wx, fmaf(a21, wy, a22 * wz));
  const float wd = fmaf(wax, dt.dax, fmaf(way, dt.day, waz * dt.daz));
  const float dtt = -wd * dt.rdd;
  const float ts = t0 + dtt;
  const float d2 = fmaxf(fmaf(wax, wax, fmaf(way, way, waz * waz)) + dtt * wd, 0.0f);
  if (!(ts > 0.0f) || !(d2 <= 9.0f)) return false;
  t_out = ts;
  alpha_out = q0.w * expf(-0.5f * d2);
  return true;
}

__device__ __forceinline__ bool gauss_hit(const float4* __restrict__ recs, int pos, const Ray& r, float& t_out,
                                          float& alpha_out, float& m_out) {
  const float4 q0 = __ldg(recs + 4 * pos);
  const float4 q1 = __ldg(recs + 4 * pos + 1);
  const float4 q2 = __ldg(recs + 4 * pos + 2);
  const float4 q3 = __ldg(recs + 4 * pos + 3);
  const DirTerms dt = dir_terms(q1, q2, q3, r.dx, r.dy, r.dz);
  if (!hit_eval(q0, q1, q2, q3.x, dt, r, t_out, alpha_out)) return false;
  m_out = dt.m;
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

// Per-ray work counters (only gathered when the caller asks for them).
struct RayStats {
  unsigned nodes, search_nodes, leaves, hits, rounds, entries;
};

__device__ __forceinline__ bool key_less(float t0, int p0, float t1, int p1) {
  return t0 < t1 || (t0 == t1 && p0 < p1);
}

// Depth-first traversal of one scene's subtree. Children are visited when the ray's slab
// interval overlaps [t_lo, vis.t_hi()]; leaves are handed to vis.leaf(pos); the walk ends
// when vis.stop() turns true. Leaf children are handled at their parent, so only internal
// nodes go on the stack.
template <class Vis>
__device__ __forceinline__ void traverse(const TraceArgs& a, const Ray& r, int root, float t_lo, Vis& vis,
                                         RayStats& st, unsigned& node_count) {
  if (root == INT32_MIN) return;
  if (root < 0) {
    vis.leaf(~root);
    return;
  }
  const float prune_lo = t_lo > 0.f ? t_lo * (1.0f - 1e-5f) - 1e-6f : -FLT_MAX;
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
    ++node_count;
    const float th = vis.t_hi();
    float tn0, tf0, tn1, tf1;
    bool h0 = slab(r, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, tn0, tf0) && tf0 >= prune_lo && tn0 <= th &&
              child_ok(c0, a.n, a.status);
    bool h1 = slab(r, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, tn1, tf1) && tf1 >= prune_lo && tn1 <= th &&
              child_ok(c1, a.n, a.status);
    if (h0 && c0 < 0) {
      vis.leaf(~c0);
      h0 = false;
    }
    if (h1 && c1 < 0) {
      vis.leaf(~c1);
      h1 = false;
    }
    if (vis.stop()) break;
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

// Visibility: product of (1 - alpha) over every hit, in any order; stops below t_min.
struct ShadowVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float T;
  __device__ float t_hi() const { return FLT_MAX; }
  __device__ bool stop() const { return T < a.t_min; }
  __device__ void hit(int, float, float al, float) { T *= 1.0f - al; }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (gauss_hit(a.recs, pos, r, t, al, m)) {
      ++st.hits;
      hit(pos, t, al, m);
    }
  }
};

// Sorted K-buffer of front-facing hits (max(-d.n_j, 0) > 0), keyed by (t*, position).
template <int KB>
struct FrontBuf {
  float bt[KB], ba[KB], bm[KB];
  int bp[KB];
  __device__ void clear() {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      bt[k] = FLT_MAX;
      bp[k] = INT32_MAX;
      ba[k] = 0.f;
      bm[k] = 0.f;
    }
  }
  __device__ float t_full() const { return bt[KB - 1]; }
  // Returns alpha * m of the entry that falls out (the new one if it is past the last slot;
  // 0 while the buffer is not full).
  __device__ float insert(float t, int p, float al, float m) {
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      if (key_less(t, p, bt[k], bp[k])) {
        float tt = bt[k]; bt[k] = t; t = tt;
        int pp = bp[k]; bp[k] = p; p = pp;
        float aa = ba[k]; ba[k] = al; al = aa;
        float mm = bm[k]; bm[k] = m; m = mm;
      }
    }
    return al * m;
  }
  __device__ int count() const {
    int nc = 0;
#pragma unroll
    for (int k = 0; k < KB; ++k) nc += bt[k] != FLT_MAX ? 1 : 0;
    return nc;
  }
};

// A ray whose visibility walk left index-matrix candidates: resolved by k_prefix / k_rounds.
template <int KB>
struct QueueRec {
  int self;
  int s;
  float t_hor;
  float amax;  // largest alpha_j max(-d.n_j, 0) of the front-facing hits past the KB in fb
  FrontBuf<KB> fb;
};

__device__ __forceinline__ float slack_hi(float t) { return t == FLT_MAX ? FLT_MAX : t * (1.0f + 1e-5f) + 1e-6f; }

// Visibility walk of the bounce mode. Until T < t_min it multiplies every hit into T (in
// any order, as ShadowVis) and keeps the KB nearest front-facing hits. At the cut-off it
// records the horizon: the largest t* met so far; every hit past it has a prefix
// transmittance below t_min, so it is no index-matrix candidate. The same walk then goes on,
// pruned to the horizon, so that the buffer ends up holding the KB nearest front-facing hits
// of the whole ray within the horizon and amax bounds alpha m of every one past them: a later
// candidate j has W_j <= amax T_j, which ends the search once the prefix drops below the best.
template <int KB>
struct ShadowFrontVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float T;
  float t_seen;
  float t_hor;
  float amax;
  FrontBuf<KB> fb;
  // pruned to the horizon only, so that amax covers every front-facing hit within it that
  // is not among the KB nearest (the candidates of the later rounds)
  __device__ float t_hi() const { return T < a.t_min ? slack_hi(t_hor) : FLT_MAX; }
  __device__ bool stop() const { return false; }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (!gauss_hit(a.recs, pos, r, t, al, m)) return;
    ++st.hits;
    hit(pos, t, al, m);
  }
  __device__ void hit(int pos, float t, float al, float m) {
    if (!(T < a.t_min)) {
      T *= 1.0f - al;
      t_seen = fmaxf(t_seen, t);
      if (T < a.t_min) t_hor = t_seen;
    } else if (t > t_hor) {
      return;
    }
    if (m > 0.f) amax = fmaxf(amax, fb.insert(t, pos, al, m));
  }
};

// Prefix walk of the index-matrix search (k_prefix): log prefix transmittance in front of each
// candidate, lt[j] += log(1 - alpha_k) for every hit k with previous-last < key_k < key_j.
template <int KB>
struct PrefixVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float t_last;
  int p_last;
  const FrontBuf<KB>& fb;
  int nc;
  float lt[KB];
  __device__ float t_hi() const { return slack_hi(fb.bt[nc - 1]); }
  __device__ bool stop() const { return false; }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (!gauss_hit(a.recs, pos, r, t, al, m)) return;
    ++st.hits;
    hit(pos, t, al, m);
  }
  __device__ void hit(int pos, float t, float al, float) {
    if (!key_less(t_last, p_last, t, pos)) return;
    const float l = log1pf(-al);
#pragma unroll
    for (int j = 0; j < KB; ++j)
      if (j < nc && key_less(t, pos, fb.bt[j], fb.bp[j])) lt[j] += l;
  }
};

__device__ __forceinline__ float ray_cos(float nx, float ny, float nz, const float* d) {
  return fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2]));
}

// State of a ray whose first index-matrix round did not settle the argmax.
struct RoundRec {
  int self;
  int s;
  float t_hor;
  float t_last;
  int p_last;
  float lt_base;
  int best;
  float lw_best;
  float lamax;  // log of the largest alpha m among the ray's front-facing hits (W_j <= amax T_j)
};

// Rounds over all hits: the KR nearest hits of any kind with key past the last processed one
// (and t* within the horizon), processed in key order -- one walk per round.
template <int KR>
struct AllHitsVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float t_last;
  int p_last;
  float t_hor;
  FrontBuf<KR> fb;  // here: every hit (ba = alpha, bm = max(-d.n, 0))
  __device__ float t_hi() const { return fminf(slack_hi(fb.t_full()), slack_hi(t_hor)); }
  __device__ bool stop() const { return false; }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (!gauss_hit(a.recs, pos, r, t, al, m)) return;
    ++st.hits;
    hit(pos, t, al, m);
  }
  __device__ void hit(int pos, float t, float al, float m) {
    if (!key_less(t_last, p_last, t, pos)) return;
    fb.insert(t, pos, al, m);
  }
};

}  // namespace prtgs
