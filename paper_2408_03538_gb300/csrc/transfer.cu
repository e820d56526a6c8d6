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
#include "brdf.cuh"
#include "trace.cuh"

namespace prtgs {


// Real SH up to order 6 of the direction set, one thread per direction, in double precision and
// rounded once: Y_l0 = K_l0 Q_l^0(z), Y_l(+-m) = sqrt2 K_lm Q_l^m(z) {Re, Im}(x + i y)^m, with
// Q_l^m = P_l^m / sin^m (Condon-Shortley phase) from Q_m^m = (-1)^m (2m-1)!!,
// Q_{m+1}^m = (2m+1) z Q_m^m, (l-m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m, and
// K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), index l*l+l+m as for orders <= 3.
__global__ void k_sh_table(int S, int order, const float* __restrict__ dirs, float* __restrict__ Y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double x = dirs[3 * s], y = dirs[3 * s + 1], z = dirs[3 * s + 2];
  const int C = (order + 1) * (order + 1);
  double re = 1.0, im = 0.0;  // (x + i y)^m
  double qmm = 1.0;           // Q_m^m
  for (int m = 0; m <= order; ++m) {
    if (m > 0) {
      const double r2 = re * x - im * y, i2 = re * y + im * x;
      re = r2;
      im = i2;
      qmm *= -(2.0 * m - 1.0);
    }
    double q2 = 0.0, q1 = qmm;  // Q_{l-2}^m, Q_{l-1}^m walking up in l
    for (int l = m; l <= order; ++l) {
      double q;
      if (l == m) q = qmm;
      else if (l == m + 1) q = (2.0 * m + 1.0) * z * qmm;
      else q = ((2.0 * l - 1.0) * z * q1 - (double)(l + m - 1) * q2) / (double)(l - m);
      if (l > m) {
        q2 = q1;
        q1 = q;
      }
      double ratio = 1.0;  // (l-m)! / (l+m)!
      for (int j = l - m + 1; j <= l + m; ++j) ratio /= (double)j;
      const double K = sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * ratio);
      if (m == 0) {
        Y[(int64_t)s * C + l * l + l] = (float)(K * q);
      } else {
        Y[(int64_t)s * C + l * l + l + m] = (float)(1.4142135623730951 * K * q * re);
        Y[(int64_t)s * C + l * l + l - m] = (float)(1.4142135623730951 * K * q * im);
      }
    }
  }
}

template <bool BOUNCE, int KB>
__global__ void __launch_bounds__(kTraceThreads, BOUNCE ? kBounceMinBlocks : kShadowMinBlocks) k_trace(TraceArgs a) {
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
    if ((int64_t)w >= a.r1 - a.r0) break;
    const int self = (int)(a.r0 + w);  // receivers are visited in sorted (Morton) order
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
      if (BOUNCE && s < a.S && !up) {
        a.idx[(int64_t)gid * a.S + s] = -1;
        a.pending[(int64_t)(self - a.r0) * a.S + s] = 0;
      }
      cnt += __popc(m);
    }
    if (lane == 0) s_next[warp] = 0;
    __syncwarp();
    // lanes pull rays until the list is exhausted
    RayStats rs{0u, 0u, 0u, 0u, 0u};
    for (;;) {
      unsigned int t = atomicAdd(&s_next[warp], 1u);
      if ((int)t >= cnt) break;
      int s = list[t];
      Ray r;
      make_ray(r, q0.x, q0.y, q0.z, sdir[3 * s], sdir[3 * s + 1], sdir[3 * s + 2]);
      float V = 1.0f;
      if (a.flags & PRTGS_SHADOW) {
        if (BOUNCE) {
          ShadowFrontVis<KB> sv{a, r, self, rs, 1.0f, 0.0f, FLT_MAX, 0.0f};
          sv.fb.clear();
          traverse(a, r, root, 0.0f, sv, rs, rs.nodes);
          V = sv.T;
          // the buffer holds the KB nearest front-facing hits within the horizon; rays with
          // candidates are listed for k_prefix (and, when needed, k_rounds)
          const int64_t slot = (int64_t)(self - a.r0) * a.S + s;
          if (sv.fb.count() == 0) {
            a.idx[(int64_t)gid * a.S + s] = -1;
            a.pending[slot] = 0;
          } else {
            QueueRec<KB>* q = static_cast<QueueRec<KB>*>(a.queue) + slot;
            q->self = self;
            q->s = s;
            q->t_hor = sv.t_hor;
            q->amax = sv.amax;
            q->fb = sv.fb;
            a.pending[slot] = 1;
          }
        } else {
          ShadowVis sv{a, r, self, rs, 1.0f};
          traverse(a, r, root, 0.0f, sv, rs, rs.nodes);
          V = sv.T;
        }
      } else if (BOUNCE) {
        a.idx[(int64_t)gid * a.S + s] = -1;
        a.pending[(int64_t)(self - a.r0) * a.S + s] = 0;
      }
      vis[s] = V;
    }
    __syncwarp();
    if (C > kMaxC) {
      // orders above 3: one lane per coefficient, compensated over the directions, the SH from
      // the table
      for (int k = lane; k < C; k += 32) {
        CompSum acc;
        for (int s = 0; s < a.S; ++s) {
          const float c = ray_cos(q3.y, q3.z, q3.w, sdir + 3 * s);
          if (!(c > 0.0f)) continue;
          acc.add(vis[s] * c * wq * __ldg(a.Ytab + (int64_t)s * C + k));
        }
        a.P[(int64_t)gid * C + k] = acc.value();
      }
    } else {
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
    }
    if (a.stats) {
      unsigned long long c0 = warp_sum_u64(rs.nodes), c1 = warp_sum_u64(rs.search_nodes),
                         c2 = warp_sum_u64(rs.leaves), c3 = warp_sum_u64(rs.hits), c4 = warp_sum_u64(rs.rounds);
      if (lane == 0) {
        atomicAdd(a.stats + 0, c0);
        atomicAdd(a.stats + 1, c1);
        atomicAdd(a.stats + 2, c2);
        atomicAdd(a.stats + 3, c3);
        atomicAdd(a.stats + 4, c4);
        atomicAdd(a.stats + 5, (unsigned long long)cnt);
      }
    }
    if (a.Vg) {
      int slot = a.glossy_slot[gid];
      if (slot >= 0)
        for (int s = lane; s < a.S; s += 32) a.Vg[(int64_t)slot * a.S + s] = vis[s];
    }
    __syncwarp();
  }
}

// First index-matrix round of the listed rays (one thread per ray): the prefix walk for the
// candidates found by the visibility walk and the decision. Rays that need more rounds go to
// a second queue for k_rounds.
template <int KB>
__global__ void __launch_bounds__(128, kPrefixMinBlocks) k_prefix(TraceArgs a, const uint32_t* __restrict__ list,
                                                                  RoundRec* __restrict__ more,
                                                                  unsigned int* __restrict__ more_count) {
  const unsigned count = *a.queue_count;
  const float lfilter = logf(a.filter_t);
  const float lmin = a.t_min > 0.f ? logf(a.t_min) : -FLT_MAX;
  RayStats rs{0u, 0u, 0u, 0u, 0u};
  unsigned n_first = 0, n_more = 0;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    ++n_first;
    const QueueRec<KB>& rec = static_cast<const QueueRec<KB>*>(a.queue)[list[q]];
    const int self = rec.self, s = rec.s;
    if (self < 0 || (int64_t)self >= a.n || s < 0 || s >= a.S) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      continue;
    }
    const float4 q0 = __ldg(a.recs + 4 * self);
    const int gid = a.order[self];
    int root = a.roots[find_scene(a.offsets, a.n_scenes, gid)];
    if (root != INT32_MIN && !child_ok(root, a.n, a.status)) root = INT32_MIN;
    Ray r;
    make_ray(r, q0.x, q0.y, q0.z, __ldg(a.dirs + 3 * s), __ldg(a.dirs + 3 * s + 1), __ldg(a.dirs + 3 * s + 2));
    FrontBuf<KB> fb;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      fb.bt[k] = rec.fb.bt[k];
      fb.bp[k] = rec.fb.bp[k];
    }
    const int nc = fb.count();
    PrefixVis<KB> pb{a, r, self, rs, -FLT_MAX, INT32_MIN, fb, nc};
#pragma unroll
    for (int k = 0; k < KB; ++k) pb.lt[k] = 0.f;
    traverse(a, r, root, 0.0f, pb, rs, rs.search_nodes);
    float lw_best = -FLT_MAX;
    int best = -1;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      if (k < nc && pb.lt[k] <= lfilter && pb.lt[k] >= lmin) {
        const float lw = logf(rec.fb.ba[k]) + pb.lt[k] + logf(rec.fb.bm[k]);
        if (lw > lw_best) {
          lw_best = lw;
          best = fb.bp[k];
        }
      }
    }
    bool settled = nc < KB;
    float lt_next = 0.f;
    const float lamax = logf(rec.amax);  // every candidate past the KB has W_j <= amax T_j
    if (!settled) {
      lt_next = pb.lt[KB - 1] + log1pf(-rec.fb.ba[KB - 1]);
      settled = lt_next + lamax <= lw_best || lt_next < lmin;
    }
    if (settled) {
      a.idx[(int64_t)gid * a.S + s] = best >= 0 ? a.order[best] : -1;
    } else {
      const unsigned m = atomicAdd(more_count, 1u);
      more[m] = RoundRec{self, s, rec.t_hor, fb.bt[KB - 1], fb.bp[KB - 1], lt_next, best, lw_best, lamax};
      ++n_more;
    }
  }
  if (a.stats) {
    unsigned long long c1 = warp_sum_u64(rs.search_nodes), c2 = warp_sum_u64(rs.leaves), c3 = warp_sum_u64(rs.hits),
                       c6 = warp_sum_u64(n_first), c7 = warp_sum_u64(n_more);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(a.stats + 1, c1);
      atomicAdd(a.stats + 2, c2);
      atomicAdd(a.stats + 3, c3);
      atomicAdd(a.stats + 6, c6);
      atomicAdd(a.stats + 7, c7);
    }
  }
}

template <int KR>
__device__ int index_search_all(const TraceArgs& a, const Ray& r, int root, int self, RayStats& st, float t_hor,
                                float t_last, int p_last, float lt, int best, float lw_best, float lamax) {
  const float lfilter = logf(a.filter_t);
  const float lmin = a.t_min > 0.f ? logf(a.t_min) : -FLT_MAX;
  for (int64_t round = 0;; ++round) {
    if (round > a.n / KR + 1) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      break;
    }
    if (lt < lmin || lt + lamax <= lw_best) break;  // later W_j <= amax T_j: none can do better
    ++st.rounds;
    AllHitsVis<KR> v{a, r, self, st, t_last, p_last, t_hor};
    v.fb.clear();
    traverse(a, r, root, t_last, v, st, st.search_nodes);
    const int nh = v.fb.count();
    bool decided = false;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      if (k < nh && !decided) {
        if (lt < lmin || lt + lamax <= lw_best) {
          decided = true;
        } else {
          if (v.fb.bm[k] > 0.f && lt <= lfilter) {
            const float lw = logf(v.fb.ba[k] * v.fb.bm[k]) + lt;
            if (lw > lw_best) {
              lw_best = lw;
              best = v.fb.bp[k];
            }
          }
          lt += log1pf(-v.fb.ba[k]);
        }
      }
    }
    if (decided || nh < KR) break;
    t_last = v.fb.bt[KR - 1];
    p_last = v.fb.bp[KR - 1];
  }
  return best;
}

// Further rounds for the rays k_prefix could not settle (one thread per ray).
template <int KB>
__global__ void __launch_bounds__(128, kRoundsMinBlocks) k_rounds(TraceArgs a, const RoundRec* __restrict__ more,
                                                                  const unsigned int* __restrict__ more_count) {
  const unsigned count = *more_count;
  RayStats rs{0u, 0u, 0u, 0u, 0u};
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x) {
    const RoundRec rec = more[q];
    const int self = rec.self, s = rec.s;
    if (self < 0 || (int64_t)self >= a.n || s < 0 || s >= a.S) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      continue;
    }
    const float4 q0 = __ldg(a.recs + 4 * self);
    const int gid = a.order[self];
    int root = a.roots[find_scene(a.offsets, a.n_scenes, gid)];
    if (root != INT32_MIN && !child_ok(root, a.n, a.status)) root = INT32_MIN;
    Ray r;
    make_ray(r, q0.x, q0.y, q0.z, __ldg(a.dirs + 3 * s), __ldg(a.dirs + 3 * s + 1), __ldg(a.dirs + 3 * s + 2));
    const int best = index_search_all<kRoundHits>(a, r, root, self, rs, rec.t_hor, rec.t_last, rec.p_last,
                                                  rec.lt_base, rec.best, rec.lw_best, rec.lamax);
    a.idx[(int64_t)gid * a.S + s] = best >= 0 ? a.order[best] : -1;
  }
  if (a.stats) {
    unsigned long long c1 = warp_sum_u64(rs.search_nodes), c2 = warp_sum_u64(rs.leaves),
                       c3 = warp_sum_u64(rs.hits), c4 = warp_sum_u64(rs.rounds);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(a.stats + 1, c1);
      atomicAdd(a.stats + 2, c2);
      atomicAdd(a.stats + 3, c3);
      atomicAdd(a.stats + 4, c4);
    }
  }
}

// Slots of the rays that still have candidates, compacted in (receiver, direction) order.
__global__ void k_compact_pending(int64_t count, const uint32_t* __restrict__ pending,
                                  const uint32_t* __restrict__ incl, uint32_t* __restrict__ list) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && pending[i]) list[incl[i] - 1] = (uint32_t)i;
}

static int device_sms();

// ---- transfer backward: dP -> the Gaussians (recomputed walks, no stored hit lists) ---------
// Geometry of a hit needed by the gradient: the closest-approach offset w = p - mu in world
// space and a = A w in the whitened frame (D^2 = |a|^2, stationary in t*).
struct HitGeom {
  float t, alpha, G;
  float w[3], a[3], A[9];
};

__device__ __forceinline__ bool gauss_hit_geom(const float4* __restrict__ recs, int pos, const Ray& r, HitGeom& h) {
  const float4 q0 = __ldg(recs + 4 * pos);
  const float4 q1 = __ldg(recs + 4 * pos + 1);
  const float4 q2 = __ldg(recs + 4 * pos + 2);
  const float4 q3 = __ldg(recs + 4 * pos + 3);
  float ux, uy, uz, ex, ey, ez;
  two_sum(r.ox, -q0.x, ux, ex);
  two_sum(r.oy, -q0.y, uy, ey);
  two_sum(r.oz, -q0.z, uz, ez);
  const float A[9] = {q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w, q3.x};
  float da[3], ua[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    da[k] = fmaf(A[3 * k], r.dx, fmaf(A[3 * k + 1], r.dy, A[3 * k + 2] * r.dz));
    ua[k] = fmaf(A[3 * k], ux, fmaf(A[3 * k + 1], uy, A[3 * k + 2] * uz));
  }
  const float dd = fmaf(da[0], da[0], fmaf(da[1], da[1], da[2] * da[2]));
  const float rdd = 1.0f / dd;
  const float t0 = -fmaf(ua[0], da[0], fmaf(ua[1], da[1], ua[2] * da[2])) * rdd;
  // the forward's cheap rejections (margins above the error of the first estimate)
  {
    const float wx0 = fmaf(t0, da[0], ua[0]), wy0 = fmaf(t0, da[1], ua[1]), wz0 = fmaf(t0, da[2], ua[2]);
    const float d2a = fmaf(wx0, wx0, fmaf(wy0, wy0, wz0 * wz0));
    const float un = sqrtf(fmaf(ua[0], ua[0], fmaf(ua[1], ua[1], ua[2] * ua[2])));
    if (d2a > 9.0f + 1e-3f + 5e-5f * un) return false;
    if (t0 < -(4e-6f * un * sqrtf(rdd) + 1e-30f)) return false;
  }
  const float w0[3] = {fmaf(t0, r.dx, ux) + ex, fmaf(t0, r.dy, uy) + ey, fmaf(t0, r.dz, uz) + ez};
  float wa[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) wa[k] = fmaf(A[3 * k], w0[0], fmaf(A[3 * k + 1], w0[1], A[3 * k + 2] * w0[2]));
  const float wd = fmaf(wa[0], da[0], fmaf(wa[1], da[1], wa[2] * da[2]));
  const float dt = -wd * rdd;
  const float ts = t0 + dt;
  // the same decision as gauss_hit: D^2 from the refined closest point
  const float d2 = fmaxf(fmaf(wa[0], wa[0], fmaf(wa[1], wa[1], wa[2] * wa[2])) + dt * wd, 0.0f);
  if (!(ts > 0.0f) || !(d2 <= 9.0f)) return false;
  h.t = ts;
  h.G = expf(-0.5f * d2);
  h.alpha = q0.w * h.G;
  // offset and whitened offset at the refined closest point
  h.w[0] = fmaf(dt, r.dx, w0[0]);
  h.w[1] = fmaf(dt, r.dy, w0[1]);
  h.w[2] = fmaf(dt, r.dz, w0[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    h.a[k] = fmaf(dt, da[k], wa[k]);
    h.A[3 * k] = A[3 * k];
    h.A[3 * k + 1] = A[3 * k + 1];
    h.A[3 * k + 2] = A[3 * k + 2];
  }
  return true;
}

struct GradArgs {
  const float* quats;
  const float* dP;  // [n,C], nullable (zero)
  const float* dV;  // [n,S] dLoss/dV of each ray beyond what P carries (the glossy matrices), nullable
  float* d_means;
  float* d_scales;
  float* d_quats;
  float* d_opacity;
  float* d_normals;
};

// Second walk of a ray: the same hits, in the same order and up to the same early exit as
// the visibility walk, each receiving dL/dalpha_j = g_V dV/dalpha_j = -g_V V / (1 - alpha_j).
struct BwdVis {
  const TraceArgs& a;
  const GradArgs& g;
  const Ray& r;
  int self;
  RayStats& st;
  float T;      // running product (replays the forward cut-off)
  float gVV;    // g_V * V
  float go[3];  // gradient with respect to the ray origin (the receiver's mean)
  __device__ float t_hi() const { return FLT_MAX; }
  __device__ bool stop() const { return T < a.t_min; }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    HitGeom h;
    if (!gauss_hit_geom(a.recs, pos, r, h)) return;
    ++st.hits;
    const float g_alpha = -gVV / (1.0f - h.alpha);
    T *= 1.0f - h.alpha;
    const int gid = a.order[pos];
    atomicAdd(&g.d_opacity[gid], g_alpha * h.G);
    const float g_d2 = g_alpha * (-0.5f * h.alpha);
    // dD^2/dmu_j = -2 A^T a, dD^2/do = 2 A^T a
    float at[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) at[k] = h.A[k] * h.a[0] + h.A[3 + k] * h.a[1] + h.A[6 + k] * h.a[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&g.d_means[3 * gid + k], -2.0f * g_d2 * at[k]);
      go[k] += 2.0f * g_d2 * at[k];
    }
    // A = diag(1/s) R^T: s_k = 1/|A_k.|, R[:,k] = s_k A_k.; dD^2/ds_k = -2 a_k^2 / s_k,
    // dD^2/dR[j][k] = 2 a_k w_j / s_k
    float gR[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float inv_s = sqrtf(h.A[3 * k] * h.A[3 * k] + h.A[3 * k + 1] * h.A[3 * k + 1] +
                                h.A[3 * k + 2] * h.A[3 * k + 2]);  // 1 / s_k
      atomicAdd(&g.d_scales[3 * gid + k], g_d2 * (-2.0f * h.a[k] * h.a[k] * inv_s));
#pragma unroll
      for (int j = 0; j < 3; ++j) gR[j][k] = g_d2 * 2.0f * h.a[k] * h.w[j] * inv_s;
    }
    float gq[4];
    quat_backward(g.quats[4 * gid], g.quats[4 * gid + 1], g.quats[4 * gid + 2], g.quats[4 * gid + 3], gR, gq);
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&g.d_quats[4 * gid + k], gq[k]);
  }
};

__global__ void __launch_bounds__(kTraceThreads, kRoundsMinBlocks) k_trace_bwd(TraceArgs a, GradArgs g) {
  extern __shared__ float smem[];
  float* sdir = smem;                                                               // [S*3]
  unsigned short* slist = reinterpret_cast<unsigned short*>(sdir + 3 * a.S);         // [warps][S]
  __shared__ unsigned int s_next[kTraceWarps];
  for (int i = threadIdx.x; i < 3 * a.S; i += blockDim.x) sdir[i] = a.dirs[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned short* list = slist + warp * a.S;
  const int C = sh_count(a.sh_order);
  const float wq = 4.0f * kPi / (float)a.S;
  const unsigned lt_mask = (1u << lane) - 1u;
  RayStats rs{0u, 0u, 0u, 0u, 0u};
  for (;;) {
    unsigned int wk = 0;
    if (lane == 0) wk = atomicAdd(a.work, 1u);
    wk = __shfl_sync(0xffffffffu, wk, 0);
    if ((int64_t)wk >= a.n) break;
    const int self = (int)wk;
    const float4 q0 = __ldg(a.recs + 4 * self);
    const float4 q3 = __ldg(a.recs + 4 * self + 3);
    const int gid = a.order[self];
    int root = a.roots[find_scene(a.offsets, a.n_scenes, gid)];
    if (root != INT32_MIN && !child_ok(root, a.n, a.status)) root = INT32_MIN;
    float dP[kMaxC];
    bool any = false;
#pragma unroll
    for (int k = 0; k < kMaxC; ++k) {
      dP[k] = (g.dP && k < C) ? g.dP[(int64_t)gid * C + k] : 0.f;
      any |= dP[k] != 0.0f;
    }
    if (g.dP)
      for (int k = kMaxC; k < C; ++k) any |= g.dP[(int64_t)gid * C + k] != 0.0f;  // orders 4-6
    bool any_v = false;
    if (g.dV)
      for (int s = lane; s < a.S; s += 32) any_v |= g.dV[(int64_t)gid * a.S + s] != 0.0f;
    any = any || __any_sync(0xffffffffu, any_v);
    if (!any) continue;  // a receiver with dP_i = 0 (and dV_i = 0) contributes nothing (warp-uniform)
    int cnt = 0;
    for (int base = 0; base < a.S; base += 32) {
      const int s = base + lane;
      const float c = s < a.S ? ray_cos(q3.y, q3.z, q3.w, sdir + 3 * s) : 0.0f;
      const bool up = c > 0.0f;
      const unsigned m = __ballot_sync(0xffffffffu, up);
      if (up) list[cnt + __popc(m & lt_mask)] = (unsigned short)s;
      cnt += __popc(m);
    }
    if (lane == 0) s_next[warp] = 0;
    __syncwarp();
    float gn[3] = {0.f, 0.f, 0.f}, go[3] = {0.f, 0.f, 0.f};
    for (;;) {
      const unsigned t = atomicAdd(&s_next[warp], 1u);
      if ((int)t >= cnt) break;
      const int s = list[t];
      const float* d = sdir + 3 * s;
      const float c = ray_cos(q3.y, q3.z, q3.w, d);
      float gsum = 0.f;  // w * sum_k dP_k Y_k
      if (C <= kMaxC) {
        float Y[kMaxC];
        sh_eval_dyn(a.sh_order, d[0], d[1], d[2], Y);
#pragma unroll
        for (int k = 0; k < kMaxC; ++k)
          if (k < C) gsum = fmaf(dP[k], Y[k], gsum);  // Y holds only the first C values
      } else {  // orders 4-6: the direction set's SH table
        const float* dPi = g.dP + (int64_t)gid * C;
        const float* Ys = a.Ytab + (int64_t)s * C;
        for (int k = 0; k < C; ++k) gsum = fmaf(__ldg(dPi + k), __ldg(Ys + k), gsum);
      }
      gsum *= wq;
      Ray r;
      make_ray(r, q0.x, q0.y, q0.z, d[0], d[1], d[2]);
      float V = 1.0f;
      if (a.flags & PRTGS_SHADOW) {
        ShadowVis sv{a, r, self, rs, 1.0f};
        traverse(a, r, root, 0.0f, sv, rs, rs.nodes);
        V = sv.T;
      }
      // dP/dc = w V Y: the receiver's normal (c = n . w)
      gn[0] += gsum * V * d[0];
      gn[1] += gsum * V * d[1];
      gn[2] += gsum * V * d[2];
      const float gV = gsum * c + (g.dV ? g.dV[(int64_t)gid * a.S + s] : 0.0f);
      if ((a.flags & PRTGS_SHADOW) && gV != 0.0f) {
        BwdVis bv{a, g, r, self, rs, 1.0f, gV * V, {0.f, 0.f, 0.f}};
        traverse(a, r, root, 0.0f, bv, rs, rs.search_nodes);
        go[0] += bv.go[0];
        go[1] += bv.go[1];
        go[2] += bv.go[2];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float vn = warp_sum(gn[k]);
      const float vo = warp_sum(go[k]);
      if (lane == 0) {
        atomicAdd(&g.d_normals[3 * gid + k], vn);
        atomicAdd(&g.d_means[3 * gid + k], vo);
      }
    }
    __syncwarp();
  }
  if (a.stats) {
    unsigned long long c0 = warp_sum_u64(rs.nodes), c1 = warp_sum_u64(rs.search_nodes),
                       c2 = warp_sum_u64(rs.leaves), c3 = warp_sum_u64(rs.hits);
    if (lane == 0) {
      atomicAdd(a.stats + 0, c0);
      atomicAdd(a.stats + 1, c1);
      atomicAdd(a.stats + 2, c2);
      atomicAdd(a.stats + 3, c3);
    }
  }
}

int precompute_transfer_backward(const prtgs_gaussians* gs, const prtgs_bvh* bvh, const prtgs_transfer_params* p,
                                 const float* dP, float* d_means, float* d_scales, float* d_quats, float* d_opacity,
                                 float* d_normals, int32_t* status, void* ws, cudaStream_t stream, const float* dV) {
  const int64_t n = gs->n;
  cudaMemsetAsync(d_means, 0, sizeof(float) * 3 * n, stream);
  cudaMemsetAsync(d_scales, 0, sizeof(float) * 3 * n, stream);
  cudaMemsetAsync(d_quats, 0, sizeof(float) * 4 * n, stream);
  cudaMemsetAsync(d_opacity, 0, sizeof(float) * n, stream);
  cudaMemsetAsync(d_normals, 0, sizeof(float) * 3 * n, stream);
  if (n == 0) return PRTGS_OK;
  Carver c(ws);
  unsigned int* work = c.take<unsigned int>(1);
  const int C = sh_count(p->sh_order);
  float* ytab = C > kMaxC ? c.take<float>((size_t)p->n_dirs * C) : nullptr;
  cudaMemsetAsync(work, 0, sizeof(unsigned int), stream);
  if (ytab) {
    const int rc = sh_table(p->n_dirs, p->sh_order, p->dirs, ytab, stream);
    if (rc != PRTGS_OK) return rc;
  }
  TraceArgs a{};
  a.Ytab = ytab;
  a.nodes = reinterpret_cast<const float4*>(bvh->nodes);
  a.recs = reinterpret_cast<const float4*>(bvh->records);
  a.order = bvh->order;
  a.roots = bvh->roots;
  a.offsets = bvh->scene_offsets;
  a.n_scenes = bvh->n_scenes;
  a.n = n;
  a.dirs = p->dirs;
  a.S = p->n_dirs;
  a.sh_order = p->sh_order;
  a.t_min = p->t_min;
  a.filter_t = p->same_surface_t;
  a.flags = p->flags;
  a.status = status;
  a.work = work;
  a.stats = p->stats;
  a.r0 = 0;
  a.r1 = n;
  GradArgs g{gs->quats, dP, dV, d_means, d_scales, d_quats, d_opacity, d_normals};
  const size_t smem = sizeof(float) * 3 * p->n_dirs + kTraceWarps * (size_t)p->n_dirs * 2;
  int per_sm = 0;
  cudaFuncSetAttribute(k_trace_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_bwd, kTraceThreads, smem);
  k_trace_bwd<<<device_sms() * (per_sm > 0 ? per_sm : 1), kTraceThreads, smem, counted(stream)>>>(a, g);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

size_t transfer_backward_workspace(int64_t, const prtgs_transfer_params* p) {
  const int C = sh_count(p->sh_order);
  return align_up(sizeof(unsigned int)) + (C > kMaxC ? align_up(sizeof(float) * (size_t)p->n_dirs * C) : 0);
}

// ---- self-transfer bounces (Eq. 33; n bounces Eq. 34-35) ----------------------------------------
// One bounce k: T^k_i = sum_s w (n_i.w_s)^+ (rho_j / pi) T^{k-1}_j over the index matrix, per
// channel, with T^0 = P (FROM_P: the same for the three channels). FROM_P writes
// T = P + T^1; later bounces add T^k to T. Tcur (nullable) receives T^k for the next bounce.
// One warp per receiver: lanes 0-15 and 16-31 take alternate rays, lane & 15 the coefficient.
template <bool FROM_P>
__global__ void k_bounce(int64_t n, int C, int S, const float* __restrict__ dirs, const float* __restrict__ normals,
                         const float* __restrict__ albedo, const float* __restrict__ P,
                         const float* __restrict__ Tprev, const int32_t* __restrict__ idx, float* __restrict__ T,
                         float* __restrict__ Tcur, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const int half = lane >> 4;
  const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
  const float wq = 4.0f * kPi / (float)S;
  // coefficients in chunks of 16 (one chunk up to order 3, up to four for order 6)
  for (int kb = 0; kb < C; kb += 16) {
    const int k = kb + (lane & 15);
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
        const float coef = wq * c * (1.0f / kPi);
        if (FROM_P) {
          const float cp = coef * (k < C ? __ldg(P + (int64_t)j * C + k) : 0.f);
          acc0 = fmaf(cp, __ldg(albedo + 3 * j), acc0);
          acc1 = fmaf(cp, __ldg(albedo + 3 * j + 1), acc1);
          acc2 = fmaf(cp, __ldg(albedo + 3 * j + 2), acc2);
        } else if (k < C) {
          const float* tj = Tprev + (int64_t)j * 3 * C + k;
          acc0 = fmaf(coef * __ldg(albedo + 3 * j), __ldg(tj), acc0);
          acc1 = fmaf(coef * __ldg(albedo + 3 * j + 1), __ldg(tj + C), acc1);
          acc2 = fmaf(coef * __ldg(albedo + 3 * j + 2), __ldg(tj + 2 * C), acc2);
        }
      }
    }
    acc0 += __shfl_xor_sync(0xffffffffu, acc0, 16);
    acc1 += __shfl_xor_sync(0xffffffffu, acc1, 16);
    acc2 += __shfl_xor_sync(0xffffffffu, acc2, 16);
    if (half == 0 && k < C) {
      float* t = T + i * 3 * C + k;
      if (FROM_P) {
        const float p = P[i * C + k];
        t[0] = p + acc0;
        t[C] = p + acc1;
        t[2 * C] = p + acc2;
      } else {
        t[0] += acc0;
        t[C] += acc1;
        t[2 * C] += acc2;
      }
      if (Tcur) {
        float* u = Tcur + i * 3 * C + k;
        u[0] = acc0;
        u[C] = acc1;
        u[2 * C] = acc2;
      }
    }
  }
}

// ---- glossy transfer matrices (Eq. 36-41) ---------------------------------------------------
constexpr int kGlossyThreads = 128;


// Ordered compaction of the directions s in [0, S) with pred(s) into list (increasing s), one
// block of kGlossyThreads threads; returns the count (every thread). wt: kGlossyThreads / 32 ints.
template <class Pred>
__device__ __forceinline__ int glossy_compact(int S, Pred pred, int* list, int* wt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kW = kGlossyThreads / 32;
  int count = 0;
  for (int s0 = 0; s0 < S; s0 += kGlossyThreads) {
    const int s = s0 + (int)threadIdx.x;
    const bool p = s < S && pred(s);
    const unsigned b = __ballot_sync(0xffffffffu, p);
    if (lane == 0) wt[warp] = __popc(b);
    __syncthreads();
    int off = count, tot = 0;
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      off += w < warp ? wt[w] : 0;
      tot += wt[w];
    }
    if (p) list[off + __popc(b & ((1u << lane) - 1u))] = s;
    count += tot;
    __syncthreads();
  }
  return count;
}

// C coefficients (orders 1-6); for C > 16 the SH of the direction set come from the table Ytab.
// Per splat the directions with n.w > 0 (the kernel's outgoing side) and, among them, those with
// V > 0 (the incoming side) are first compacted in increasing order, so that every thread of the
// inner loops works on a live term; the sums run over the live terms in the order of the full
// sums, whose other terms are exact zeros.
template <int C>
__global__ void __launch_bounds__(kGlossyThreads) k_glossy(int64_t n_glossy, const int32_t* __restrict__ glossy_ids,
                                                           int S, int order, const float* __restrict__ dirs,
                                                           const float* __restrict__ Ytab,
                                                           const float* __restrict__ normals,
                                                           const float* __restrict__ roughness,
                                                           const float* __restrict__ metallic,
                                                           const float* __restrict__ Vg, float* __restrict__ M) {
  extern __shared__ float smem[];
  float* sdir = smem;              // [S*3]
  float* sY = sdir + 3 * S;        // [S][C]
  float* sU = sY + S * C;          // [live][C]   w^2 (n.w_s)^+ V_s Y(w_s)
  float* sB = sU + S * C;          // [live][C]   sum_o k(s,o) Y(w_o)
  int* sin_list = reinterpret_cast<int*>(sB + S * C);  // [S] incoming live directions
  int* sout_list = sin_list + S;                       // [S] outgoing directions (n.w_o > 0)
  int* wt = sout_list + S;                             // [kGlossyThreads / 32] compaction counts
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) sdir[i] = dirs[i];
  __syncthreads();
  if (C > kMaxC) {
    for (int e = threadIdx.x; e < S * C; e += blockDim.x) sY[e] = Ytab[e];
  } else {
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      float Y[kMaxC];
      sh_eval_dyn(order, sdir[3 * s], sdir[3 * s + 1], sdir[3 * s + 2], Y);
      for (int k = 0; k < C && k < kMaxC; ++k) sY[s * C + k] = Y[k];
    }
  }
  __syncthreads();
  const float wq = 4.0f * kPi / (float)S;
  for (int64_t g = blockIdx.x; g < n_glossy; g += gridDim.x) {
    const int64_t i = glossy_ids[g];
    const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
    const float r = roughness[i];
    const float alpha = r * r, metal = metallic[i];
    auto cosn = [&](int s) {
      const float* w = sdir + 3 * s;
      return fmaf(nx, w[0], fmaf(ny, w[1], nz * w[2]));
    };
    const int n_out = glossy_compact(S, [&](int s) { return cosn(s) > 0.0f; }, sout_list, wt);
    const int n_in =
        glossy_compact(S, [&](int s) { return cosn(s) > 0.0f && Vg[g * S + s] > 0.0f; }, sin_list, wt);
    for (int l = threadIdx.x; l < n_in; l += blockDim.x) {
      const int s = sin_list[l];
      const float* wi = sdir + 3 * s;
      const float ni = cosn(s);
      const float v = Vg[g * S + s];
      const float u = wq * wq * ni * v;
      float Bs[C];
#pragma unroll
      for (int k = 0; k < C; ++k) Bs[k] = 0.f;
      for (int q = 0; q < n_out; ++q) {
        const int o = sout_list[q];
        const float* wo = sdir + 3 * o;
        const float no = cosn(o);
        const float kv = brdf_kernel(nx, ny, nz, wi, wo, ni, no, alpha, metal);
#pragma unroll
        for (int k = 0; k < C; ++k) Bs[k] = fmaf(kv, sY[o * C + k], Bs[k]);
      }
#pragma unroll
      for (int k = 0; k < C; ++k) {
        sB[l * C + k] = Bs[k];
        sU[l * C + k] = u * sY[s * C + k];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
      int ra = e / C, cb = e % C;
      float acc = 0.f;
      for (int l = 0; l < n_in; ++l) acc = fmaf(sU[l * C + ra], sB[l * C + cb], acc);
      M[(g * C + ra) * C + cb] = acc;
    }
    __syncthreads();
  }
}

// Backward of the glossy matrices (Eq. 40). With U_so = Y(w_s)^T dM Y(w_o) and c_s = n.w_s:
//   L = sum_s sum_o w^2 c_s V_s k(s,o) U_so,
//   dL/dV_s = w^2 c_s sum_o k(s,o) U_so,  dL/dr = sum_s w^2 c_s V_s sum_o U_so dk/dr,
//   dL/dm = -sum_s w^2 c_s V_s sum_o U_so,  dL/dn = sum_s w^2 V_s sum_o U_so (k w_s + c_s dk/dn)
// (the cosine takes the raw normal, the kernel n / |n|; the cut-offs n.w > 0 are held fixed).
// One block per glossy splat; Q_o = dM Y(w_o) staged per splat, the threads over s.
template <int C>
__global__ void __launch_bounds__(kGlossyThreads) k_glossy_bwd(int64_t n_glossy, const int32_t* __restrict__ glossy_ids,
                                                               int S, int order, const float* __restrict__ dirs,
                                                               const float* __restrict__ Ytab,
                                                               const float* __restrict__ normals,
                                                               const float* __restrict__ roughness,
                                                               const float* __restrict__ metallic,
                                                               const float* __restrict__ V, const float* __restrict__ dM,
                                                               float* __restrict__ dV, float* __restrict__ d_rough,
                                                               float* __restrict__ d_metal, float* __restrict__ d_normals) {
  extern __shared__ float smem[];
  float* sdir = smem;         // [S*3]
  float* sY = sdir + 3 * S;   // [S][C]
  float* sQ = sY + S * C;     // [S][C]  dM Y(w_o) (rows of the directions with n.w_o > 0)
  float* sdM = sQ + S * C;    // [C*C]
  int* sout_list = reinterpret_cast<int*>(sdM + C * C);  // [S] directions with n.w > 0
  int* sin_list = sout_list + S;                         // [S] the same, those with V != 0 first
  int* wt = sin_list + S;                                // [kGlossyThreads / 32]
  __shared__ float red[5][kGlossyThreads / 32];
  for (int i = threadIdx.x; i < 3 * S; i += blockDim.x) sdir[i] = dirs[i];
  __syncthreads();
  if (C > kMaxC) {
    for (int e = threadIdx.x; e < S * C; e += blockDim.x) sY[e] = Ytab[e];
  } else {
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      float Y[kMaxC];
      sh_eval_dyn(order, sdir[3 * s], sdir[3 * s + 1], sdir[3 * s + 2], Y);
      for (int k = 0; k < C && k < kMaxC; ++k) sY[s * C + k] = Y[k];
    }
  }
  __syncthreads();
  const float wq = 4.0f * kPi / (float)S;
  const float w2 = wq * wq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t g = blockIdx.x; g < n_glossy; g += gridDim.x) {
    const int64_t i = glossy_ids[g];
    const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
    const float r = roughness[i], metal = metallic[i];
    auto cosn = [&](int s) {
      const float* w = sdir + 3 * s;
      return fmaf(nx, w[0], fmaf(ny, w[1], nz * w[2]));
    };
    for (int e = threadIdx.x; e < C * C; e += blockDim.x) sdM[e] = dM[g * C * C + e];
    // the directions with n.w > 0 (increasing); as incoming directions, those with V != 0 (which
    // take every derivative) before those with V = 0 (dV only), so that warps stay converged
    const int n_out = glossy_compact(S, [&](int s) { return cosn(s) > 0.0f; }, sout_list, wt);
    const int n_full =
        glossy_compact(S, [&](int s) { return cosn(s) > 0.0f && V[i * S + s] != 0.0f; }, sin_list, wt);
    const int n_in = n_full + glossy_compact(S, [&](int s) { return cosn(s) > 0.0f && V[i * S + s] == 0.0f; },
                                             sin_list + n_full, wt);
    for (int e = threadIdx.x; e < n_out * C; e += blockDim.x) {
      const int o = sout_list[e / C], a = e % C;
      float q = 0.f;
      for (int b = 0; b < C; ++b) q = fmaf(sdM[a * C + b], sY[o * C + b], q);
      sQ[o * C + a] = q;
    }
    for (int s = threadIdx.x; s < S; s += blockDim.x)
      if (!(cosn(s) > 0.0f)) dV[i * S + s] = 0.f;
    __syncthreads();
    float gr = 0.f, gm = 0.f, gnx = 0.f, gny = 0.f, gnz = 0.f;
    for (int l = threadIdx.x; l < n_in; l += blockDim.x) {
      const int s = sin_list[l];
      const float* wi = sdir + 3 * s;
      const float c = cosn(s);
      const float v = V[i * S + s];
      float Ys[C];
#pragma unroll
      for (int a = 0; a < C; ++a) Ys[a] = sY[s * C + a];
      float kU = 0.f, rU = 0.f, mU = 0.f, nU[3] = {0.f, 0.f, 0.f};
      for (int q = 0; q < n_out; ++q) {
        const int o = sout_list[q];
        const float* wo = sdir + 3 * o;
        const float no = cosn(o);
        float U = 0.f;
#pragma unroll
        for (int a = 0; a < C; ++a) U = fmaf(Ys[a], sQ[o * C + a], U);
        float kv;
        const float dkdr = brdf_kernel_dr(nx, ny, nz, wi, wo, c, no, r, metal, kv);
        kU = fmaf(kv, U, kU);
        if (v != 0.0f) {
          rU = fmaf(U, dkdr, rU);
          mU -= U;
          float dn[3];
          brdf_kernel_dn(nx, ny, nz, wi, wo, r, dn);
          nU[0] = fmaf(U, dn[0], nU[0]);
          nU[1] = fmaf(U, dn[1], nU[1]);
          nU[2] = fmaf(U, dn[2], nU[2]);
        }
      }
      dV[i * S + s] = w2 * c * kU;
      gr = fmaf(w2 * c * v, rU, gr);
      gm = fmaf(w2 * c * v, mU, gm);
      gnx = fmaf(w2 * v, fmaf(kU, wi[0], c * nU[0]), gnx);
      gny = fmaf(w2 * v, fmaf(kU, wi[1], c * nU[1]), gny);
      gnz = fmaf(w2 * v, fmaf(kU, wi[2], c * nU[2]), gnz);
    }
    gr = warp_sum(gr);
    gm = warp_sum(gm);
    gnx = warp_sum(gnx);
    gny = warp_sum(gny);
    gnz = warp_sum(gnz);
    if (lane == 0) {
      red[0][warp] = gr;
      red[1][warp] = gm;
      red[2][warp] = gnx;
      red[3][warp] = gny;
      red[4][warp] = gnz;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      float t = 0.f;
      for (int w = 0; w < kGlossyThreads / 32; ++w) t += red[threadIdx.x][w];
      if (threadIdx.x == 0) d_rough[i] = t;
      else if (threadIdx.x == 1) d_metal[i] = t;
      else d_normals[3 * i + threadIdx.x - 2] = t;
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

__global__ void k_iota_i32(int64_t n, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)i;
}

__global__ void k_mask_u32(int64_t n, const uint8_t* __restrict__ mask, uint32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = mask[i] ? 1u : 0u;
}

static size_t trace_smem(int S) { return sizeof(float) * 3 * S + kTraceWarps * S * (sizeof(float) + 2); }
static size_t glossy_smem(int S, int C) {
  return sizeof(float) * (3 * S + 3 * (size_t)S * C) + sizeof(int) * (2 * (size_t)S + kGlossyThreads / 32);
}

// The glossy matrices' shared memory (directions, three [S][C] tables, two direction lists) must fit one block.
bool glossy_fits(int S, int order) { return glossy_smem(S, sh_count(order)) <= (size_t)227 * 1024; }

template <int C>
static int launch_glossy(int64_t n_glossy, const int32_t* gids, int S, const prtgs_transfer_params* p,
                         const float* ytab, const prtgs_gaussians* g, const float* Vg, float* M, int sms,
                         cudaStream_t stream) {
  const size_t gsm = glossy_smem(S, C);
  if (gsm > (size_t)227 * 1024) return PRTGS_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(k_glossy<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  int gper = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gper, k_glossy<C>, kGlossyThreads, gsm);
  int64_t blocks = (int64_t)sms * (gper > 0 ? gper : 1);
  if (blocks > n_glossy) blocks = n_glossy;
  k_glossy<C><<<(unsigned)blocks, kGlossyThreads, gsm, counted(stream)>>>(n_glossy, gids, S, p->sh_order, p->dirs, ytab,
                                                                          g->normals, g->roughness, g->metallic, Vg, M);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// Receivers per batch: the resolve queue holds at most batch * S rays.
static int64_t trace_batch(int64_t n, int S) {
  int64_t b = (int64_t(1) << 23) / (S > 0 ? S : 1);
  if (b < 1) b = 1;
  return b < n ? b : n;
}

static size_t queue_rec_bytes(int kb) { return 16 + 16 * (size_t)kb; }

static int n_bounces_of(const prtgs_transfer_params* p) { return p->n_bounces > 1 ? p->n_bounces : 1; }

static int index_buffer_of(const prtgs_transfer_params* p) {
  const int kb = p->index_buffer > 0 ? p->index_buffer : kDefaultIndexBuffer;
  return kb <= 1 ? 1 : (kb <= 2 ? 2 : (kb <= 4 ? 4 : 8));
}

// Receivers per packet batch: the visibility scratch holds S * batch floats (at most 2^26).
static int64_t packet_batch(int64_t n, int S) {
  int64_t b = ((int64_t(1) << 26) / (S > 0 ? S : 1)) / 32 * 32;
  if (b < 32) b = 32;
  return b < n ? b : n;
}

static bool use_packets(const prtgs_transfer_params* p) { return p->walk == 0; }

size_t transfer_workspace(int64_t n, int64_t n_glossy, const prtgs_transfer_params* p, bool want_V) {
  size_t b = 2 * align_up(sizeof(unsigned int));
  if (want_V) b += align_up(sizeof(int32_t) * (size_t)n);
  if (use_packets(p)) b += align_up(sizeof(float) * (size_t)packet_batch(n, p->n_dirs) * p->n_dirs);
  if (sh_count(p->sh_order) > kMaxC) b += align_up(sizeof(float) * (size_t)p->n_dirs * sh_count(p->sh_order));
  if (p->flags & PRTGS_BOUNCE) {
    if (!use_packets(p)) {  // the per-ray walk's candidate records and rounds queue
      const size_t rays = (size_t)trace_batch(n, p->n_dirs) * p->n_dirs;
      b += align_up(queue_rec_bytes(index_buffer_of(p)) * rays) + 3 * align_up(sizeof(uint32_t) * rays) +
           scan_workspace((int64_t)rays) + align_up(sizeof(RoundRec) * rays) + align_up(sizeof(unsigned int));
    }
    const size_t tbytes = align_up(sizeof(float) * (size_t)n * 3 * sh_count(p->sh_order));
    if (n_bounces_of(p) > 1) b += tbytes;
    if (n_bounces_of(p) > 2) b += tbytes;
  }
  if (p->flags & PRTGS_GLOSSY) {
    b += 2 * align_up(sizeof(int32_t) * n) + align_up(sizeof(uint32_t) * n) + scan_workspace(n) +
         align_up(sizeof(uint32_t)) + align_up(sizeof(float) * (size_t)n_glossy * p->n_dirs);
  }
  return b;
}

template <bool BOUNCE, int KB>
static int launch_trace(TraceArgs a, size_t smem, int sms, int64_t batch, uint32_t* incl, uint32_t* list,
                        void* scan_ws, RoundRec* more, unsigned int* more_count, cudaStream_t stream) {
  int per_sm = 0, per_sm_b = 0, per_sm_r = 0;
  cudaFuncSetAttribute(k_trace<BOUNCE, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<BOUNCE, KB>, kTraceThreads, smem);
  if (BOUNCE) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_prefix<KB>, 128, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, k_rounds<KB>, 128, 0);
  }
  for (int64_t r0 = 0; r0 < a.n; r0 += batch) {
    a.r0 = r0;
    a.r1 = r0 + batch < a.n ? r0 + batch : a.n;
    cudaMemsetAsync(a.work, 0, sizeof(unsigned int), stream);
    k_trace<BOUNCE, KB><<<sms * (per_sm > 0 ? per_sm : 1), kTraceThreads, smem, counted(stream)>>>(a);
    if (BOUNCE) {
      const int64_t rays = (a.r1 - a.r0) * a.S;
      int rc = scan_u32(a.pending, incl, rays, false, a.queue_count, scan_ws, stream);
      if (rc != PRTGS_OK) return rc;
      k_compact_pending<<<(unsigned)((rays + 255) / 256), 256, 0, counted(stream)>>>(rays, a.pending, incl, list);
      cudaMemsetAsync(more_count, 0, sizeof(unsigned int), stream);
      k_prefix<KB><<<sms * (per_sm_b > 0 ? per_sm_b : 1), 128, 0, counted(stream)>>>(a, list, more, more_count);
      k_rounds<KB><<<sms * (per_sm_r > 0 ? per_sm_r : 1), 128, 0, counted(stream)>>>(a, more, more_count);
    }
  }
  return PRTGS_OK;
}



static int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

int precompute_transfer(const prtgs_gaussians* g, const prtgs_bvh* bvh, const prtgs_transfer_params* p, float* P,
                        float* T, int32_t* idx, float* M, int64_t n_glossy, int32_t* status, void* ws,
                        cudaStream_t stream, float* V_out) {
  const int64_t n = g->n;
  if (n == 0) return PRTGS_OK;
  const int S = p->n_dirs;
  const int C = sh_count(p->sh_order);
  const bool bounce = (p->flags & PRTGS_BOUNCE) != 0;
  const bool glossy = (p->flags & PRTGS_GLOSSY) != 0 && n_glossy > 0;
  Carver c(ws);
  unsigned int* work = c.take<unsigned int>(1);
  unsigned int* qcount = c.take<unsigned int>(1);
  const int kbq = index_buffer_of(p);
  const bool rayq = bounce && !use_packets(p);  // per-ray walk: candidate records and rounds queue
  void* queue = rayq ? c.take<char>(queue_rec_bytes(kbq) * (size_t)trace_batch(n, S) * S) : nullptr;
  const size_t batch_rays = rayq ? (size_t)trace_batch(n, S) * S : 0;
  uint32_t* pending = rayq ? c.take<uint32_t>(batch_rays) : nullptr;
  uint32_t* incl = rayq ? c.take<uint32_t>(batch_rays) : nullptr;
  uint32_t* rlist = rayq ? c.take<uint32_t>(batch_rays) : nullptr;
  void* rscan_ws = rayq ? c.take<char>(scan_workspace((int64_t)batch_rays)) : nullptr;
  RoundRec* more = rayq ? c.take<RoundRec>(batch_rays) : nullptr;
  unsigned int* more_count = rayq ? c.take<unsigned int>(1) : nullptr;
  float* ytab = C > kMaxC ? c.take<float>((size_t)S * C) : nullptr;
  const bool packets = use_packets(p);
  float* vbuf = packets ? c.take<float>((size_t)packet_batch(n, S) * S) : nullptr;
  float* tb[2] = {nullptr, nullptr};  // ping-pong bounce buffers [n,3,C] for n_bounces > 1
  if (bounce && n_bounces_of(p) > 1) tb[0] = c.take<float>((size_t)n * 3 * C);
  if (bounce && n_bounces_of(p) > 2) tb[1] = c.take<float>((size_t)n * 3 * C);
  int32_t* slot = nullptr;
  int32_t* gids = nullptr;
  float* Vg = nullptr;
  if (V_out) {  // every receiver's visibility row: identity slots into V_out (no glossy matrices)
    slot = c.take<int32_t>(n);
    Vg = V_out;
    k_iota_i32<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, slot);
  } else if (p->flags & PRTGS_GLOSSY) {
    slot = c.take<int32_t>(n);
    gids = c.take<int32_t>(n);
    uint32_t* flags = c.take<uint32_t>(n);
    void* sws = c.take<char>(scan_workspace(n));
    uint32_t* total = c.take<uint32_t>(1);
    Vg = c.take<float>((size_t)n_glossy * S);
    k_mask_u32<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, g->glossy_mask, flags);
    int rc = scan_u32(flags, flags, n, false, total, sws, stream);
    if (rc != PRTGS_OK) return rc;
    k_glossy_slots<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, g->glossy_mask, flags, slot, gids);
  }
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
  a.Ytab = ytab;
  if (ytab) {
    k_sh_table<<<(unsigned)((S + 127) / 128), 128, 0, counted(stream)>>>(S, p->sh_order, p->dirs, ytab);
    PRTGS_CHECK_LAUNCH();
  }
  a.t_min = p->t_min;
  a.filter_t = p->same_surface_t;
  a.flags = p->flags;
  a.P = P;
  a.idx = idx;
  a.Vg = (glossy || V_out) ? Vg : nullptr;
  a.glossy_slot = slot;
  a.status = status;
  a.work = work;
  a.stats = p->stats;
  a.r0 = 0;
  a.r1 = n;
  a.queue = queue;
  a.pending = pending;
  a.queue_count = qcount;
  a.packet_dirs = p->packet_dirs;
  size_t smem = trace_smem(S);
  int sms = device_sms();
  const int64_t batch = bounce ? trace_batch(n, S) : n;
  int rct;
  if (packets) {
    rct = PRTGS_OK;
    const int64_t pb = packet_batch(n, S);
    for (int64_t r0 = 0; r0 < n && rct == PRTGS_OK; r0 += pb) {
      a.r0 = r0;
      a.r1 = r0 + pb < n ? r0 + pb : n;
      rct = launch_packet(a, vbuf, bounce, sms, stream);
    }
  } else if (!bounce) {
    rct = launch_trace<false, 1>(a, smem, sms, batch, incl, rlist, rscan_ws, more, more_count, stream);
  } else if (kbq == 1) {
    rct = launch_trace<true, 1>(a, smem, sms, batch, incl, rlist, rscan_ws, more, more_count, stream);
  } else if (kbq == 2) {
    rct = launch_trace<true, 2>(a, smem, sms, batch, incl, rlist, rscan_ws, more, more_count, stream);
  } else if (kbq == 4) {
    rct = launch_trace<true, 4>(a, smem, sms, batch, incl, rlist, rscan_ws, more, more_count, stream);
  } else {
    rct = launch_trace<true, 8>(a, smem, sms, batch, incl, rlist, rscan_ws, more, more_count, stream);
  }
  if (rct != PRTGS_OK) return rct;
  PRTGS_CHECK_LAUNCH();
  if (bounce) {
    const int nb = n_bounces_of(p);
    const unsigned blocks = (unsigned)((n + 7) / 8);
    float* cur = nb > 1 ? tb[0] : nullptr;
    k_bounce<true><<<blocks, 256, 0, counted(stream)>>>(n, C, S, p->dirs, g->normals, g->albedo, P, nullptr, idx, T, cur,
                                               status);
    for (int b = 2; b <= nb; ++b) {  // Eq. 34-35: each bounce gathers the previous one
      float* prev = cur;
      cur = b < nb ? tb[(b - 1) & 1] : nullptr;
      k_bounce<false><<<blocks, 256, 0, counted(stream)>>>(n, C, S, p->dirs, g->normals, g->albedo, P, prev, idx, T, cur,
                                                  status);
    }
    PRTGS_CHECK_LAUNCH();
  }
  if (glossy) {
    int rc = PRTGS_ERR_UNSUPPORTED;
    switch (C) {
      case 4: rc = launch_glossy<4>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      case 9: rc = launch_glossy<9>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      case 16: rc = launch_glossy<16>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      case 25: rc = launch_glossy<25>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      case 36: rc = launch_glossy<36>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      case 49: rc = launch_glossy<49>(n_glossy, gids, S, p, ytab, g, Vg, M, sms, stream); break;
      default: break;
    }
    if (rc != PRTGS_OK) return rc;
  }
  return PRTGS_OK;
}

int bounce_step(int64_t n, int C, int S, const float* dirs, const float* normals, const float* albedo, const float* P,
                const float* Tprev, const int32_t* idx, float* Tscratch, float* Tcur, int32_t* status,
                cudaStream_t stream) {
  if (n == 0) return PRTGS_OK;
  const unsigned blocks = (unsigned)((n + 7) / 8);
  if (!Tprev)
    k_bounce<true><<<blocks, 256, 0, counted(stream)>>>(n, C, S, dirs, normals, albedo, P, nullptr, idx, Tscratch, Tcur,
                                                        status);
  else
    k_bounce<false><<<blocks, 256, 0, counted(stream)>>>(n, C, S, dirs, normals, albedo, P, Tprev, idx, Tscratch, Tcur,
                                                         status);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

size_t glossy_backward_workspace(int64_t n, const prtgs_transfer_params* p) {
  const int C = sh_count(p->sh_order);
  return 2 * align_up(sizeof(int32_t) * n) + align_up(sizeof(uint32_t) * n) + scan_workspace(n) +
         align_up(sizeof(uint32_t)) + (C > kMaxC ? align_up(sizeof(float) * (size_t)p->n_dirs * C) : 0);
}

static size_t glossy_bwd_smem(int S, int C) {
  return sizeof(float) * (3 * S + 2 * (size_t)S * C + (size_t)C * C) + sizeof(int) * (2 * (size_t)S + kGlossyThreads / 32);
}

bool glossy_backward_fits(int S, int order) {
  return glossy_bwd_smem(S, sh_count(order)) <= (size_t)227 * 1024;
}

template <int C>
static int launch_glossy_bwd(int64_t n_glossy, const int32_t* gids, int S, int order, const float* dirs,
                             const float* ytab, const prtgs_gaussians* g, const float* V, const float* dM, float* dV,
                             float* dr, float* dm, float* dn, cudaStream_t stream) {
  const size_t sm = glossy_bwd_smem(S, C);
  if (sm > (size_t)227 * 1024) return PRTGS_ERR_UNSUPPORTED;
  cudaFuncSetAttribute(k_glossy_bwd<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_glossy_bwd<C>, kGlossyThreads, sm);
  int64_t blocks = (int64_t)device_sms() * (per > 0 ? per : 1);
  if (blocks > n_glossy) blocks = n_glossy;
  k_glossy_bwd<C><<<(unsigned)blocks, kGlossyThreads, sm, counted(stream)>>>(n_glossy, gids, S, order, dirs, ytab,
                                                                             g->normals, g->roughness, g->metallic, V,
                                                                             dM, dV, dr, dm, dn);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int glossy_backward(const prtgs_gaussians* g, const prtgs_transfer_params* p, const float* V, const float* dM,
                    int64_t n_glossy, float* dV, float* d_roughness, float* d_metallic, float* d_normals,
                    int32_t* status, void* ws, cudaStream_t stream) {
  const int64_t n = g->n;
  const int S = p->n_dirs;
  const int C = sh_count(p->sh_order);
  cudaMemsetAsync(dV, 0, sizeof(float) * (size_t)n * S, stream);
  cudaMemsetAsync(d_roughness, 0, sizeof(float) * n, stream);
  cudaMemsetAsync(d_metallic, 0, sizeof(float) * n, stream);
  cudaMemsetAsync(d_normals, 0, sizeof(float) * 3 * n, stream);
  if (n == 0 || n_glossy == 0) return PRTGS_OK;
  Carver c(ws);
  int32_t* slot = c.take<int32_t>(n);
  int32_t* gids = c.take<int32_t>(n);
  uint32_t* flags = c.take<uint32_t>(n);
  void* sws = c.take<char>(scan_workspace(n));
  uint32_t* total = c.take<uint32_t>(1);
  float* ytab = C > kMaxC ? c.take<float>((size_t)S * C) : nullptr;
  k_mask_u32<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, g->glossy_mask, flags);
  int rc = scan_u32(flags, flags, n, false, total, sws, stream);
  if (rc != PRTGS_OK) return rc;
  k_glossy_slots<<<(unsigned)((n + 255) / 256), 256, 0, counted(stream)>>>(n, g->glossy_mask, flags, slot, gids);
  if (ytab) {
    rc = sh_table(S, p->sh_order, p->dirs, ytab, stream);
    if (rc != PRTGS_OK) return rc;
  }
  PRTGS_CHECK_LAUNCH();
  switch (C) {
    case 4: return launch_glossy_bwd<4>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    case 9: return launch_glossy_bwd<9>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    case 16: return launch_glossy_bwd<16>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    case 25: return launch_glossy_bwd<25>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    case 36: return launch_glossy_bwd<36>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    case 49: return launch_glossy_bwd<49>(n_glossy, gids, S, p->sh_order, p->dirs, ytab, g, V, dM, dV, d_roughness, d_metallic, d_normals, stream);
    default: return PRTGS_ERR_UNSUPPORTED;
  }
}

int sh_table(int S, int order, const float* dirs, float* Y, cudaStream_t stream) {
  if (S <= 0) return PRTGS_OK;
  k_sh_table<<<(unsigned)((S + 127) / 128), 128, 0, counted(stream)>>>(S, order, dirs, Y);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int transfer_check_dirs(int S) { return (S > 0 && S <= kMaxDirs) ? PRTGS_OK : PRTGS_ERR_UNSUPPORTED; }

}  // namespace prtgs
