// Warp-packet traversal of the transfer rays (Sec. 4.4-4.5).
//
// Every receiver traces the same S world-space directions, so the rays that 32 receivers
// adjacent in Morton order cast along one direction are parallel and start from a small patch
// of the scene. One warp takes such a packet: the lanes walk the LBVH together, testing up to
// 32 nodes per step against the packet's beam (the rectangle the packet's origins span in the
// plane orthogonal to the direction, and the depth range along it that the lanes still need),
// and collect the leaves the beam meets in a shared-memory chunk. Each leaf of a chunk is then
// tested by every lane whose own ray can meet its box, with the same per-ray hit test and the
// same visitors as the per-ray walks in transfer.cu, so every hit decision, product and
// index-matrix rule is that of a single ray; only the traversal is shared.
//
//  k_packet<B>    visibility V_is of every (receiver, direction) of a receiver batch into
//                 V[s][i] (Eq. 4 along a ray, Eq. 27 read as the Gaussian's maximum); with B
//                 (bounce) also the index matrix of Sec. 4.4: the visibility walk finds the
//                 horizon and the nearest front-facing hit, then search rounds walk the hits
//                 from there in key order until the argmax of W_j (Eq. 26) is settled.
//  k_project      P_i = sum_s (4 pi / S) V_is max(0, n_i.w_s) Y(w_s) (Eq. 29 with Eq. 9),
//                 one lane per receiver, compensated sums; also copies V of glossy receivers.
#include "trace.cuh"

namespace prtgs {

constexpr int kPacketWarps = 4;
constexpr int kPacketThreads = 32 * kPacketWarps;
constexpr int kPStack = 384;     // node stack of a warp (ints)
#ifndef PRTGS_PACKET_ROUND_HITS
#define PRTGS_PACKET_ROUND_HITS 14  // 14 keeps the bounce kernel at 4 blocks per SM (16: 3 blocks)
#endif
constexpr int kPacketRoundHits = PRTGS_PACKET_ROUND_HITS;  // hits per index-matrix search round
#ifndef PRTGS_PACKET_LEAVES
#define PRTGS_PACKET_LEAVES 224
#endif
#ifndef PRTGS_PACKET_MIN_BLOCKS
#define PRTGS_PACKET_MIN_BLOCKS 4  // the visibility-only kernel fits 4 blocks per SM without spills
#endif
// leaf chunk of a warp (> 64: a step appends up to 64 leaves; flushed past kPLeaves - 64). Longer
// chunks flush less often: 1M bounce transfer 1.085 s at 96, 0.988 s at 128, 0.970 s at 160,
// 0.962 s at 192, 0.957 s at 224 (4 blocks per SM still fit at S = 256)
constexpr int kPLeaves = PRTGS_PACKET_LEAVES;
#ifndef PRTGS_PACKET_UNROLL
#define PRTGS_PACKET_UNROLL 0
#endif
#ifndef PRTGS_PACKET_BOUNCE_UNROLL
#define PRTGS_PACKET_BOUNCE_UNROLL 8
#endif
constexpr int kPUnrollVis = PRTGS_PACKET_UNROLL;            // leaves tested together (0: one by one): visibility walk
constexpr int kPUnrollBounce = PRTGS_PACKET_BOUNCE_UNROLL;  // ... bounce and index-search walks
// wide pops (32 nodes) only while the stack keeps room for their pushes plus a full one-node-
// at-a-time descent of the deepest possible tree (64 levels)
constexpr int kPHeadroom = 64 + 64 + 4;
// directions per work item by default: one, so that the warps running at a time work on few
// windows and share the BVH nodes around them in L1/L2 (surface-100k visibility 47 ms against 72
// at 16 directions; the 1M tiled transfer 1.69 s against 1.97 s)
constexpr int kPacketDirs = 1;

struct PacketSmem {
  int stack[kPStack];
  int lpos[kPLeaves];      // the chunk's leaves (sorted positions)
  float4 stage[32][4];     // a group of leaves, staged: the exact-test terms of stage_leaf
  // the work item's window of 64 receivers: record row 0 (mean, opacity), scene root, Gaussian
  // index; and, per direction, the window slots of the receivers that face it
  float4 wq0[64];
  int wroot[64], wgid[64];
  int rlist[64];
};
// Bounce mode, per warp after the PacketSmem array: the search round's nearest hits of each lane,
// hits[k][lane] = (t*, position, alpha, m).
using RoundHits = float4[kPacketRoundHits][32];

// Orthonormal frame (e1, e2, w) around a unit direction w (Duff et al. 2017, "Building an
// orthonormal basis, revisited": the branchless form).
struct Frame {
  float e1x, e1y, e1z, e2x, e2y, e2z, wx, wy, wz;
};

__device__ __forceinline__ Frame make_frame(float x, float y, float z) {
  const float sgn = copysignf(1.0f, z);
  const float a = -1.0f / (sgn + z);
  const float b = x * y * a;
  Frame f;
  f.e1x = 1.0f + sgn * x * x * a;
  f.e1y = sgn * b;
  f.e1z = -sgn * x;
  f.e2x = b;
  f.e2y = sgn + y * y * a;
  f.e2z = -y;
  f.wx = x;
  f.wy = y;
  f.wz = z;
  return f;
}

// The packet's beam: the projected origins' rectangle and the depth range along w that the
// lanes still need.
struct Beam {
  float xlo, xhi, ylo, yhi, zlo, zhi;
};

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

__device__ __forceinline__ Beam make_beam(bool need, float xl, float yl, float zlo, float zhi) {
  Beam b;
  b.xlo = warp_min(need ? xl : FLT_MAX);
  b.xhi = warp_max(need ? xl : -FLT_MAX);
  b.ylo = warp_min(need ? yl : FLT_MAX);
  b.yhi = warp_max(need ? yl : -FLT_MAX);
  b.zlo = warp_min(need ? zlo : FLT_MAX);
  b.zhi = warp_max(need ? zhi : -FLT_MAX);
  return b;
}

// The exact ray / Gaussian test of a packet. Every ray of the packet has the direction w, so the
// whitened closest-approach distance depends only on the ray origin's offset from the Gaussian in
// the plane (e1, e2): with u = o - mu = dx e1 + dy e2 + uz w and the rows of A = diag(1/s) R^T,
//   D^2 = |A u x A w|^2 / |A w|^2 = |dx (A e1 x a) + dy (A e2 x a)|^2,  a = A w / |A w|,
//   t*  = -(u^T A^T A w) / |A w|^2 = -uz - dx m1 - dy m2,  m_k = (A e_k . A w) / |A w|^2
// (the component of u along w drops out exactly). The per-Gaussian terms are formed once per
// staged leaf; a lane then needs two additions, six FMAs for the vector and three for its norm.
// Offsets are taken against a reference point R of the packet (one of its ray origins). A leaf's
// R - mu is moved along w to p, the reference ray's point nearest to the Gaussian (D^2 does not
// change along w; the move keeps the frame's own rounding, w.e1 of a few ulp, from mixing the
// distance along w into dx and dy), and p and the lane's o - R are projected on e1, e2 in twice the
// working precision (exact products and sums, hi + lo), so dx = (o - R).e1 + p.e1 carries about one
// rounding of itself: the role that the error-free o - mu and the refinement at the closest point
// play in the per-ray test.
struct Rel {
  float Rx, Ry, Rz;        // reference point (warp-uniform)
  float xr, xr_lo, yr, yr_lo;  // this lane's origin minus R on e1, e2, each as an unevaluated sum hi + lo
  float zr;                // ... and on w
};

// a . b of three terms as an unevaluated sum hi + lo (error-free products by FMA, error-free sums
// by TwoSum, their errors gathered in lo): twice the working precision.
__device__ __forceinline__ void dot3_pair(float ax, float ay, float az, float bx, float by, float bz, float& hi,
                                          float& lo) {
  const float p = ax * bx, ep = fmaf(ax, bx, -p);
  const float q = ay * by, eq = fmaf(ay, by, -q);
  const float r = az * bz, er = fmaf(az, bz, -r);
  float s, t, s2, t2;
  two_sum(p, q, s, t);
  two_sum(s, r, s2, t2);
  hi = s2;
  lo = ((ep + eq) + er) + (t + t2);
}

// The lane's offset o - R from the reference point R on the frame, e1 and e2 parts as hi + lo.
// The frame is orthonormal only to a few ulp: its e1.w and e2.w (taken in twice the working
// precision) times the offset along w are taken off, so that dx e1 + dy e2 is the part of o - R
// across w (up to a multiple of w, which D^2 does not see) and not a few ulp of the packet's depth
// off it, which 1/s_min of a thin Gaussian would magnify.
__device__ __forceinline__ Rel make_rel(const Frame& f, float ox0, float oy0, float oz0, float Rx, float Ry,
                                        float Rz) {
  Rel rel;
  rel.Rx = Rx;
  rel.Ry = Ry;
  rel.Rz = Rz;
  float ox, oy, oz, lox, loy, loz;
  two_sum(ox0, -Rx, ox, lox);
  two_sum(oy0, -Ry, oy, loy);
  two_sum(oz0, -Rz, oz, loz);
  dot3_pair(f.e1x, f.e1y, f.e1z, ox, oy, oz, rel.xr, rel.xr_lo);
  dot3_pair(f.e2x, f.e2y, f.e2z, ox, oy, oz, rel.yr, rel.yr_lo);
  rel.zr = fmaf(f.wx, ox, fmaf(f.wy, oy, f.wz * oz)) + fmaf(f.wx, lox, fmaf(f.wy, loy, f.wz * loz));
  float d1, d1l, d2, d2l;
  dot3_pair(f.e1x, f.e1y, f.e1z, f.wx, f.wy, f.wz, d1, d1l);
  dot3_pair(f.e2x, f.e2y, f.e2z, f.wx, f.wy, f.wz, d2, d2l);
  rel.xr_lo += fmaf(f.e1x, lox, fmaf(f.e1y, loy, f.e1z * loz)) - rel.zr * (d1 + d1l);
  rel.yr_lo += fmaf(f.e2x, lox, fmaf(f.e2y, loy, f.e2z * loz)) - rel.zr * (d2 + d2l);
  return rel;
}

// Stage one leaf for the packet: (p on e1, e2 (high parts), R - mu on w; opacity), (A e1 x a; m1),
// (A e2 x a; m2), (facing term max(-w.n_j, 0); sorted position; p on e1, e2 (low parts)).
__device__ __forceinline__ void stage_leaf(const float4* __restrict__ recs, int pos, const Frame& f, const Rel& rel,
                                           float4* out) {
  const float4 q0 = __ldg(recs + 4 * pos), q1 = __ldg(recs + 4 * pos + 1), q2 = __ldg(recs + 4 * pos + 2),
               q3 = __ldg(recs + 4 * pos + 3);
  // R - mu = h + l exactly; p = R - mu + t_ref w, the offset of mu from the point of the reference
  // ray nearest to it, formed with one rounding per component (the product t_ref w is exact inside
  // the FMA): D^2 does not change along w, so the lanes use p in place of R - mu, and its projections
  // on e1, e2 are small numbers, unaffected by the frame's own rounding (w.e1 of a few ulp times the
  // distance to the Gaussian); uz keeps the distance along w as w.p - t_ref.
  float hx, lx, hy, ly, hz, lz;
  two_sum(rel.Rx, -q0.x, hx, lx);
  two_sum(rel.Ry, -q0.y, hy, ly);
  two_sum(rel.Rz, -q0.z, hz, lz);
  const float t_ref = -fmaf(f.wx, hx, fmaf(f.wy, hy, f.wz * hz));
  // p = h + l + t_ref w per component as hi + lo: the product exactly (FMA), the sum by TwoSum
  float px, pxl, py, pyl, pz, pzl;
  {
    const float ax = t_ref * f.wx, ay = t_ref * f.wy, az = t_ref * f.wz;
    const float eax = fmaf(t_ref, f.wx, -ax), eay = fmaf(t_ref, f.wy, -ay), eaz = fmaf(t_ref, f.wz, -az);
    float e;
    two_sum(hx, ax, px, e);
    pxl = e + eax + lx;
    two_sum(hy, ay, py, e);
    pyl = e + eay + ly;
    two_sum(hz, az, pz, e);
    pzl = e + eaz + lz;
  }
  float cx, cxl, cy, cyl;
  dot3_pair(f.e1x, f.e1y, f.e1z, px, py, pz, cx, cxl);
  dot3_pair(f.e2x, f.e2y, f.e2z, px, py, pz, cy, cyl);
  cxl += fmaf(f.e1x, pxl, fmaf(f.e1y, pyl, f.e1z * pzl));
  cyl += fmaf(f.e2x, pxl, fmaf(f.e2y, pyl, f.e2z * pzl));
  const float cz = fmaf(f.wx, hx, fmaf(f.wy, hy, f.wz * hz)) + fmaf(f.wx, lx, fmaf(f.wy, ly, f.wz * lz));
  // rows of A: (q1.x q1.y q1.z), (q1.w q2.x q2.y), (q2.z q2.w q3.x)
  const float b1x = fmaf(q1.x, f.e1x, fmaf(q1.y, f.e1y, q1.z * f.e1z));
  const float b1y = fmaf(q1.w, f.e1x, fmaf(q2.x, f.e1y, q2.y * f.e1z));
  const float b1z = fmaf(q2.z, f.e1x, fmaf(q2.w, f.e1y, q3.x * f.e1z));
  const float b2x = fmaf(q1.x, f.e2x, fmaf(q1.y, f.e2y, q1.z * f.e2z));
  const float b2y = fmaf(q1.w, f.e2x, fmaf(q2.x, f.e2y, q2.y * f.e2z));
  const float b2z = fmaf(q2.z, f.e2x, fmaf(q2.w, f.e2y, q3.x * f.e2z));
  const float adx = fmaf(q1.x, f.wx, fmaf(q1.y, f.wy, q1.z * f.wz));
  const float ady = fmaf(q1.w, f.wx, fmaf(q2.x, f.wy, q2.y * f.wz));
  const float adz = fmaf(q2.z, f.wx, fmaf(q2.w, f.wy, q3.x * f.wz));
  const float dd = fmaf(adx, adx, fmaf(ady, ady, adz * adz));
  const float id = 1.0f / sqrtf(dd);
  const float ax = adx * id, ay = ady * id, az = adz * id;
  const float idd = 1.0f / dd;
  out[0] = make_float4(cx, cy, cz, q0.w);
  out[1] = make_float4(diff_prod(b1y, az, b1z, ay), diff_prod(b1z, ax, b1x, az), diff_prod(b1x, ay, b1y, ax),
                       fmaf(b1x, adx, fmaf(b1y, ady, b1z * adz)) * idd);
  out[2] = make_float4(diff_prod(b2y, az, b2z, ay), diff_prod(b2z, ax, b2x, az), diff_prod(b2x, ay, b2y, ax),
                       fmaf(b2x, adx, fmaf(b2y, ady, b2z * adz)) * idd);
  out[3] = make_float4(fmaxf(-fmaf(f.wx, q3.y, fmaf(f.wy, q3.z, f.wz * q3.w)), 0.0f), __int_as_float(pos), cxl, cyl);
}

// Projection of a box [lo, hi] on the frame: centre and half-width along e1, e2 and w, widened
// by a margin above the FP32 error of these sums and of a ray's drift off its projected origin
// (|w.e1| of a few ulp times the distance travelled). Any point of the box -- in particular the
// closest approach of a ray that hits a Gaussian inside it -- projects inside these intervals.
__device__ __forceinline__ void project_box(const Frame& f, float lx, float ly, float lz, float hx, float hy,
                                            float hz, float4& A, float2& Z) {
  const float cx = 0.5f * (lx + hx), cy = 0.5f * (ly + hy), cz = 0.5f * (lz + hz);
  const float hxx = 0.5f * (hx - lx), hyy = 0.5f * (hy - ly), hzz = 0.5f * (hz - lz);
  const float px = f.e1x * cx + f.e1y * cy + f.e1z * cz;
  const float py = f.e2x * cx + f.e2y * cy + f.e2z * cz;
  const float pz = f.wx * cx + f.wy * cy + f.wz * cz;
  const float rx = fabsf(f.e1x) * hxx + fabsf(f.e1y) * hyy + fabsf(f.e1z) * hzz;
  const float ry = fabsf(f.e2x) * hxx + fabsf(f.e2y) * hyy + fabsf(f.e2z) * hzz;
  const float rz = fabsf(f.wx) * hxx + fabsf(f.wy) * hyy + fabsf(f.wz) * hzz;
  const float m = 3e-5f * (1.0f + fabsf(cx) + fabsf(cy) + fabsf(cz) + hxx + hyy + hzz);
  A = make_float4(px, py, rx + m, ry + m);
  Z = make_float2(pz - rz - m, pz + rz + m);
}

__device__ __forceinline__ bool beam_meets(const Beam& b, const float4& A, const float2& Z) {
  return A.x + A.z >= b.xlo && A.x - A.z <= b.xhi && A.y + A.w >= b.ylo && A.y - A.w <= b.yhi && Z.y >= b.zlo &&
         Z.x <= b.zhi;
}

// The exact test of one staged leaf for the lane: D^2 and t* (see Rel). The high parts of dx
// cancel without rounding error of their own beyond eps |dx| (exactly where they nearly cancel);
// the low parts carry the roundings of both.
__device__ __forceinline__ void leaf_test(const Rel& rel, const float4* e, float& d2, float& t) {
  const float4 s0 = e[0], s1 = e[1], s2 = e[2], s3 = e[3];
  const float dx = (rel.xr + s0.x) + (rel.xr_lo + s3.z), dy = (rel.yr + s0.y) + (rel.yr_lo + s3.w);
  const float wx = fmaf(dx, s1.x, dy * s2.x), wy = fmaf(dx, s1.y, dy * s2.y), wz = fmaf(dx, s1.z, dy * s2.z);
  d2 = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
  t = -(rel.zr + s0.z) - fmaf(dx, s1.w, dy * s2.w);
}

// Hand one passing leaf test over to the visitor (the receiver's own Gaussian excepted).
template <class Vis>
__device__ __forceinline__ bool hand_over(const float4* e, int self, float d2, float t, Vis& vis, RayStats& st) {
  const float4 s3 = e[3];
  const int pos = __float_as_int(s3.y);
  if (pos == self) return false;
  ++st.hits;
  vis.hit(pos, t, e[0].w * expf(-0.5f * d2), s3.x);
  return true;
}

// One packet walk. Lane state: `active` (this lane's ray takes part), its projected origin
// (xl, yl) and depth zl (for the beam), its offset from the packet's reference point (rel, for the
// exact test), the lower bound t_lo of the hits it wants (0: all hits ahead) and its visitor, whose
// t_hi() bounds the hits it still wants and stop() ends its ray. The leaves of a chunk are staged
// 32 at a time (one record load and the per-Gaussian terms of the exact test per lane), then every
// lane tests its ray against each of them (the test of Rel above) and hands the hits to
// vis.hit(), in chunk order.
template <int UNROLL, class Vis>
__device__ void packet_walk(const TraceArgs& a, const Frame& f, const Ray& r, const Rel& rel, int self, int root,
                            bool active, float xl, float yl, float zl, float t_lo, Vis& vis, PacketSmem& sm,
                            RayStats& st, unsigned& node_count) {
  const int lane = threadIdx.x & 31;
  const float prune_lo = t_lo > 0.f ? t_lo * (1.0f - 1e-5f) - 1e-6f : -FLT_MAX;
  // t > 0 && t >= prune_lo as one strict test against the float below prune_lo (or 0)
  const float tlo = prune_lo > 0.f ? nextafterf(prune_lo, 0.0f) : 0.0f;
  const unsigned above = lane == 31 ? 0u : (0xffffffffu << (lane + 1));  // lanes > lane
  const unsigned below = (1u << lane) - 1u;                                // lanes < lane
  const float zlo_l = t_lo > 0.f ? zl + (t_lo * (1.0f - 1e-5f) - 1e-6f) : zl;
  bool need = active && !vis.stop();
  if (!__any_sync(0xffffffffu, need) || root == INT32_MIN) return;
  if (root < 0) {  // a one-Gaussian scene
    if (need) vis.leaf(~root);
    return;
  }
  float th = vis.t_hi();
  Beam bm = make_beam(need, xl, yl, zlo_l, th == FLT_MAX ? FLT_MAX : zl + th);
  int sp = 1, nl = 0;
  if (lane == 0) sm.stack[0] = root;
  __syncwarp();
  const int64_t max_steps = 4 * a.n + 64;
  for (int64_t step = 0;; ++step) {
    if (step > max_steps) {
      set_status(a.status, PRTGS_STATUS_BAD_INDEX);
      break;
    }
    if (sp > 0) {
      const int npop = sp + kPHeadroom <= kPStack ? min(32, sp) : 1;
      int node = -1;
      if (lane < npop) node = sm.stack[sp - 1 - lane];
      sp -= npop;
      if (lane == 0) node_count += npop;
      bool push0 = false, push1 = false, leaf0 = false, leaf1 = false;
      int c0 = 0, c1 = 0;
      float4 A0, A1;
      float2 Z0, Z1;
      bool near0 = true;
      if (node >= 0) {
        float4 n0, n1, n2;
        load_node(a.nodes, node, n0, n1, n2, c0, c1);
        project_box(f, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, A0, Z0);
        project_box(f, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, A1, Z1);
        const bool h0 = beam_meets(bm, A0, Z0) && child_ok(c0, a.n, a.status);
        const bool h1 = beam_meets(bm, A1, Z1) && child_ok(c1, a.n, a.status);
        push0 = h0 && c0 >= 0;
        push1 = h1 && c1 >= 0;
        leaf0 = h0 && c0 < 0;
        leaf1 = h1 && c1 < 0;
        near0 = Z0.x + Z0.y <= Z1.x + Z1.y;  // nearer box centre along w
      }
      // pushes: far child first, near child on top; lane 0's pushes end on top of the stack
      const int np = (int)push0 + (int)push1;
      const unsigned b1 = __ballot_sync(0xffffffffu, np >= 1), b2 = __ballot_sync(0xffffffffu, np == 2);
      int pos = sp + __popc(b1 & above) + __popc(b2 & above);
      if (pos + np > kPStack) {  // only a malformed tree gets here: report, drop the pushes
        set_status(a.status, PRTGS_STATUS_STACK_OVERFLOW);
      } else if (np == 2) {
        sm.stack[pos] = near0 ? c1 : c0;
        sm.stack[pos + 1] = near0 ? c0 : c1;
      } else if (np == 1) {
        sm.stack[pos] = push0 ? c0 : c1;
      }
      sp = min(sp + __popc(b1) + __popc(b2), kPStack);
      // leaves: appended to the chunk (every lane tests its own ray against them)
      const int nlf = (int)leaf0 + (int)leaf1;
      const unsigned l1 = __ballot_sync(0xffffffffu, nlf >= 1), l2 = __ballot_sync(0xffffffffu, nlf == 2);
      int lp = nl + __popc(l1 & below) + __popc(l2 & below);
      if (leaf0) sm.lpos[lp++] = ~c0;
      if (leaf1) sm.lpos[lp] = ~c1;
      nl += __popc(l1) + __popc(l2);
      __syncwarp();
    }
    if (nl > kPLeaves - 64 || (sp == 0 && nl > 0)) {
      for (int g = 0; g < nl; g += 32) {
        // stage: lane j forms the exact-test terms of leaf g + j
        if (g + lane < nl) stage_leaf(a.recs, sm.lpos[g + lane], f, rel, sm.stage[lane]);
        __syncwarp();
        const int cnt = min(32, nl - g);
        if (lane == 0) st.entries += cnt;
        // per leaf only the test itself; the bookkeeping (the receiver's own Gaussian, the
        // visitor's bound th, whether the lane still wants hits) waits for a passing test, which
        // is rare (a few percent of the leaves); th only falls, and changes only at a hand-over.
        // UNROLL > 0 tests UNROLL leaves at a time (independent chains) and hands the passing
        // ones over in order, each test taken again by the same arithmetic (bit-identical)
        // against the current th: one copy of the visitor's code serves the whole block, which
        // pays where that code is long (the bounce and index-search visitors).
        if (need) st.leaves += cnt;  // leaf tests of the lane (its own Gaussian included)
        float thn = need ? th : -FLT_MAX;  // a lane that wants no hits passes no test
        if constexpr (UNROLL == 0) {
          for (int j = 0; j < cnt; ++j) {
            float d2, t;
            leaf_test(rel, sm.stage[j], d2, t);
            if (d2 <= 9.0f && t > tlo && t <= thn) {
              if (hand_over(sm.stage[j], self, d2, t, vis, st)) {
                need = !vis.stop();
                th = vis.t_hi();
                thn = need ? th : -FLT_MAX;
              }
            }
          }
        } else {
          for (int j0 = 0; j0 < cnt; j0 += UNROLL) {
            unsigned pass = 0u;
#pragma unroll
            for (int k = 0; k < UNROLL; ++k) {
              float d2, t;
              leaf_test(rel, sm.stage[min(j0 + k, 31)], d2, t);  // past cnt: a stale entry, masked below
              if (d2 <= 9.0f && t > tlo && t <= thn) pass |= 1u << k;
            }
            if (cnt - j0 < UNROLL) pass &= (1u << (cnt - j0)) - 1u;
            while (pass) {
              const int j = j0 + __ffs(pass) - 1;
              pass &= pass - 1u;
              float d2, t;
              leaf_test(rel, sm.stage[j], d2, t);
              if (t <= thn && hand_over(sm.stage[j], self, d2, t, vis, st)) {
                need = !vis.stop();
                th = vis.t_hi();
                thn = need ? th : -FLT_MAX;
              }
            }
          }
        }
        __syncwarp();
      }
      nl = 0;
      if (!__any_sync(0xffffffffu, need)) break;
      th = vis.t_hi();
      bm = make_beam(need, xl, yl, zlo_l, th == FLT_MAX ? FLT_MAX : zl + th);
      __syncwarp();
    }
    if (sp == 0 && nl == 0) break;
  }
  __syncwarp();
}

// Visibility walk of the bounce mode. Until T < t_min it multiplies every hit into T (in any
// order, as ShadowVis), records the largest alpha m of the front-facing hits and, at the cut-off,
// the horizon: the largest t* met so far (a hit past it has prefix transmittance below t_min and
// is no index-matrix candidate). It keeps the nearest front-facing hit (by key). After the cut-off
// the walk goes on pruned to the nearer of the horizon and that hit, so that it ends as the
// nearest front-facing hit of the whole ray within the horizon: the first index-matrix candidate.
// It also sums log(1 - alpha) over the hits in front of the current candidate (lpre). That sum
// stays exact while no hit it holds lies behind a nearer candidate found later (checked with the
// largest key summed); when it holds, the index search needs no walk in front of the candidate.
struct BounceVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float T;
  float t_seen;
  float t_hor;
  float tf;  // nearest front-facing hit: t*, position, alpha, facing term
  int pf;
  float af, mf;
  float amax;  // largest alpha m of the front-facing hits multiplied into T
  float lpre;  // sum of log(1 - alpha) of the hits with key below (tf, pf)
  float ts;    // largest key summed into lpre: t*, position
  int ps;
  bool pre_ok;  // lpre is the prefix of (tf, pf)
  __device__ float t_hi() const { return T < a.t_min ? fminf(slack_hi(t_hor), slack_hi(tf)) : FLT_MAX; }
  __device__ bool stop() const { return false; }
  __device__ void hit(int pos, float t, float al, float m) {
    if (!(T < a.t_min)) {
      T *= 1.0f - al;
      t_seen = fmaxf(t_seen, t);
      if (T < a.t_min) t_hor = t_seen;
      if (m > 0.f) amax = fmaxf(amax, al * m);
    } else if (t > t_hor) {
      return;
    }
    if (m > 0.f && key_less(t, pos, tf, pf)) {
      if (ps != INT32_MIN && !key_less(ts, ps, t, pos)) pre_ok = false;  // a summed hit lies behind it
      tf = t;
      pf = pos;
      af = al;
      mf = m;
    } else if (key_less(t, pos, tf, pf)) {
      lpre += log1pf(-al);
      if (ps == INT32_MIN || key_less(ts, ps, t, pos)) {
        ts = t;
        ps = pos;
      }
    }
  }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (!gauss_hit(a.recs, pos, r, t, al, m)) return;
    ++st.hits;
    hit(pos, t, al, m);
  }
};

// One search round of the index matrix: the KR nearest hits of any kind with key past the last
// one processed (and t* within the horizon), kept sorted by key in the lane's column of a shared-
// memory buffer, for processing in key order. In the first round (no hit processed yet) the hits
// in front of the first candidate (key below (tf, pf)) are not kept but summed into lbase = log of
// the prefix transmittance in front of that candidate.
template <int KR>
struct SearchVis {
  const TraceArgs& a;
  const Ray& r;
  int self;
  RayStats& st;
  float t_last;
  int p_last;
  float t_hor;
  float tf;
  int pf;
  float lbase;
  float4 (*buf)[32];  // buf[k][lane]
  int lane;
  int count;
  float t_max;  // key of the last kept hit once the buffer is full
  int p_max;
  __device__ float t_hi() const { return fminf(count == KR ? slack_hi(t_max) : FLT_MAX, slack_hi(t_hor)); }
  __device__ bool stop() const { return false; }
  __device__ void hit(int pos, float t, float al, float m) {
    if (!key_less(t_last, p_last, t, pos)) return;
    if (key_less(t, pos, tf, pf)) {
      lbase += log1pf(-al);
      return;
    }
    if (count == KR && !key_less(t, pos, t_max, p_max)) return;
    // sorted insertion: shift the larger keys up by one (the last falls out when full)
    int k = count < KR ? count : KR - 1;
    while (k > 0) {
      const float4 e = buf[k - 1][lane];
      if (!key_less(t, pos, e.x, __float_as_int(e.y))) break;
      buf[k][lane] = e;
      --k;
    }
    buf[k][lane] = make_float4(t, __int_as_float(pos), al, m);
    if (count < KR) ++count;
    if (count == KR) {
      const float4 e = buf[KR - 1][lane];
      t_max = e.x;
      p_max = __float_as_int(e.y);
    }
  }
  __device__ void leaf(int pos) {
    if (pos == self) return;
    ++st.leaves;
    float t, al, m;
    if (!gauss_hit(a.recs, pos, r, t, al, m)) return;
    ++st.hits;
    hit(pos, t, al, m);
  }
};

// Visibility (and with BOUNCE the index matrix) of the rays of receiver batch [r0, r1):
// V[s * batch + (i - r0)] (0 where n.w <= 0), idx[gid * S + s].
#ifndef PRTGS_PACKET_BOUNCE_MIN_BLOCKS
#define PRTGS_PACKET_BOUNCE_MIN_BLOCKS 4  // 128 registers, no spills; 55.5 KB shared per block at S = 256
#endif
template <bool BOUNCE>
__global__ void __launch_bounds__(kPacketThreads, BOUNCE ? PRTGS_PACKET_BOUNCE_MIN_BLOCKS : PRTGS_PACKET_MIN_BLOCKS)
    k_packet(TraceArgs a, float* __restrict__ V, int dpi) {
  extern __shared__ float4 psmem4[];
  float* sdir = reinterpret_cast<float*>(psmem4);  // [S*3]
  PacketSmem* wsm = reinterpret_cast<PacketSmem*>(sdir + ((3 * a.S + 3) & ~3));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PacketSmem& sm = wsm[warp];
  RoundHits& hbuf = reinterpret_cast<RoundHits*>(wsm + kPacketWarps)[warp];  // bounce mode only
  __shared__ unsigned int s_item[kPacketWarps];
  for (int i = threadIdx.x; i < 3 * a.S; i += blockDim.x) sdir[i] = a.dirs[i];
  __syncthreads();
  const int64_t batch = a.r1 - a.r0;
  const int64_t n_windows = (batch + 63) / 64;
  const int dblocks = (a.S + dpi - 1) / dpi;  // dpi directions per work item
  const unsigned below = (1u << lane) - 1u;
  RayStats rs{0u, 0u, 0u, 0u, 0u, 0u};
  unsigned traced = 0, walks = 0;
  for (;;) {
    if (lane == 0) s_item[warp] = atomicAdd(a.work, 1u);
    __syncwarp();
    const unsigned item = s_item[warp];
    __syncwarp();
    if ((int64_t)item >= n_windows * dblocks) break;
    // a window of 64 receivers adjacent in Morton order; each lane stages two of them
    const int64_t base = a.r0 + 64 * (item / dblocks);
    const int s0 = (int)(item % dblocks) * dpi;
    float4 nq[2];  // record row 3 of the lane's two receivers (its .yzw: the normal)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const bool vj = base + j < a.r1;
      const int sj = vj ? (int)(base + j) : (int)a.r0;
      sm.wq0[j] = __ldg(a.recs + 4 * sj);
      nq[h] = __ldg(a.recs + 4 * sj + 3);
      int rt = INT32_MIN, gj = -1;
      if (vj) {
        gj = a.order[sj];
        rt = a.roots[find_scene(a.offsets, a.n_scenes, gj)];
        if (rt != INT32_MIN && !child_ok(rt, a.n, a.status)) rt = INT32_MIN;
      }
      sm.wroot[j] = rt;
      sm.wgid[j] = gj;
    }
    __syncwarp();
    const int s1 = min(a.S, s0 + dpi);
    for (int s = s0; s < s1; ++s) {
      const float* d = sdir + 3 * s;
      // the receivers of the window that face direction s, compacted into packets of 32 lanes
      // (a window whose receivers all face it gives the two packets of its halves)
      bool upj[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        const bool vj = base + j < a.r1;
        upj[h] = vj && ray_cos(nq[h].y, nq[h].z, nq[h].w, d) > 0.0f;
        if (vj && !upj[h]) {  // untraced ray: no visibility, no index-matrix entry
          V[(int64_t)s * batch + (base + j - a.r0)] = 0.0f;
          if (BOUNCE) a.idx[(int64_t)sm.wgid[j] * a.S + s] = -1;
        }
      }
      const unsigned m0 = __ballot_sync(0xffffffffu, upj[0]), m1 = __ballot_sync(0xffffffffu, upj[1]);
      const int total = __popc(m0) + __popc(m1);
      if (upj[0]) sm.rlist[__popc(m0 & below)] = lane;
      if (upj[1]) sm.rlist[__popc(m0) + __popc(m1 & below)] = lane + 32;
      __syncwarp();
      for (int pass = 0; pass * 32 < total; ++pass) {
      const bool up = pass * 32 + lane < total;
      const int jw = up ? sm.rlist[pass * 32 + lane] : 0;
      const float4 q0 = sm.wq0[jw];
      const int root = up ? sm.wroot[jw] : INT32_MIN;
      const int self = (int)(base + jw);
      float vis = up ? 1.0f : 0.0f;
      int best = -1;  // index-matrix entry (sorted position of the chosen hit)
      if ((a.flags & PRTGS_SHADOW) && __any_sync(0xffffffffu, up)) {
        const Frame f = make_frame(d[0], d[1], d[2]);
        const float xl = f.e1x * q0.x + f.e1y * q0.y + f.e1z * q0.z;
        const float yl = f.e2x * q0.x + f.e2y * q0.y + f.e2z * q0.z;
        const float zl = f.wx * q0.x + f.wy * q0.y + f.wz * q0.z;
        Ray r;
        make_ray(r, q0.x, q0.y, q0.z, d[0], d[1], d[2]);
        traced += up ? 1u : 0u;
        // lanes of different scenes walk their own subtrees, one group at a time
        unsigned todo = __ballot_sync(0xffffffffu, up);
        while (todo) {
          const int leader = __ffs(todo) - 1;
          const int groot = __shfl_sync(0xffffffffu, root, leader);
          const unsigned grp = __ballot_sync(0xffffffffu, up && root == groot) & todo;
          const bool mine = (grp >> lane) & 1u;
          if (lane == 0) ++walks;
          // reference point of the group's exact tests: its leader's ray origin
          const Rel rel = make_rel(f, q0.x, q0.y, q0.z, __shfl_sync(0xffffffffu, q0.x, leader),
                                   __shfl_sync(0xffffffffu, q0.y, leader), __shfl_sync(0xffffffffu, q0.z, leader));
          if (!BOUNCE) {
            ShadowVis sv{a, r, self, rs, 1.0f};
            packet_walk<kPUnrollVis>(a, f, r, rel, self, groot, mine, xl, yl, zl, 0.0f, sv, sm, rs, rs.nodes);
            if (mine) vis = sv.T;
          } else {
            BounceVis bv{a,    r,    self, rs,   1.0f, 0.0f,      FLT_MAX, FLT_MAX,
                         INT32_MAX, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, INT32_MIN, true};
            packet_walk<kPUnrollBounce>(a, f, r, rel, self, groot, mine, xl, yl, zl, 0.0f, bv, sm, rs, rs.nodes);
            if (mine) vis = bv.T;
            // index matrix (Sec. 4.4): argmax of W_j = alpha_j T_j m_j over the hits in key order,
            // T_j the prefix transmittance; candidates need T_j >= t_min and T_j <= filter_t.
            // Every later candidate has W_j <= amax T_j (amax covers every front-facing hit when
            // no cut-off happened, else the trivial bound 1).
            const float lfilter = logf(a.filter_t);
            const float lmin = a.t_min > 0.f ? logf(a.t_min) : -FLT_MAX;
            const float lamax = bv.T < a.t_min ? 0.0f : logf(bv.amax);
            bool searching = mine && bv.tf != FLT_MAX;
            float t_last = -FLT_MAX, lt = 0.0f, lw_best = -FLT_MAX;
            int p_last = INT32_MIN;
            // with an exact prefix of the first candidate, the candidate is taken here, as the
            // rounds would take it (same arithmetic), and the rounds start behind it, if they are
            // still needed: often its weight already settles the argmax
            const bool pre = bv.pre_ok && bv.pf > INT32_MIN;
            if (pre && searching) {
              lt = bv.lpre;
              if (lt < lmin) {
                searching = false;
              } else {
                if (lt <= lfilter) {
                  const float lw = logf(bv.af * bv.mf) + lt;
                  if (lw > lw_best) {
                    lw_best = lw;
                    best = bv.pf;
                  }
                }
                lt += log1pf(-bv.af);
                if (lt < lmin || lt + lamax <= lw_best) searching = false;
                t_last = bv.tf;
                p_last = bv.pf;
              }
            }
            for (int64_t round = 0; __any_sync(0xffffffffu, searching); ++round) {
              if (round > a.n / kPacketRoundHits + 1) {
                if (searching) set_status(a.status, PRTGS_STATUS_BAD_INDEX);
                break;
              }
              SearchVis<kPacketRoundHits> sv{a,     r,      self, rs,      t_last, p_last, bv.t_hor, bv.tf,
                                             bv.pf, 0.0f,   hbuf,   lane, 0,     FLT_MAX, INT32_MAX};
              if (searching) ++rs.rounds;
              packet_walk<kPUnrollBounce>(a, f, r, rel, self, groot, searching, xl, yl, zl, t_last > 0.f ? t_last : 0.0f, sv, sm, rs,
                          rs.search_nodes);
              if (searching) {
                if (round == 0 && !pre) lt = sv.lbase;
                const int nh = sv.count;
                bool decided = false;
                for (int k = 0; k < nh && !decided; ++k) {
                  if (lt < lmin || lt + lamax <= lw_best) {
                    decided = true;
                  } else {
                    const float4 e = hbuf[k][lane];  // t*, position, alpha, m
                    if (e.w > 0.f && lt <= lfilter) {
                      const float lw = logf(e.z * e.w) + lt;
                      if (lw > lw_best) {
                        lw_best = lw;
                        best = __float_as_int(e.y);
                      }
                    }
                    lt += log1pf(-e.z);
                  }
                }
                if (decided || nh < kPacketRoundHits || lt < lmin || lt + lamax <= lw_best) {
                  searching = false;
                } else {
                  t_last = sv.t_max;
                  p_last = sv.p_max;
                }
              }
            }
          }
          todo &= ~grp;
        }
      }
      if (up) {
        V[(int64_t)s * batch + (self - a.r0)] = vis;
        if (BOUNCE) a.idx[(int64_t)sm.wgid[jw] * a.S + s] = best >= 0 ? a.order[best] : -1;
      }
      __syncwarp();
      }  // pass
      __syncwarp();  // the compacted list is rewritten for the next direction
    }
    __syncwarp();  // the window is restaged by the next work item
  }
  if (a.stats) {
    unsigned long long c0 = warp_sum_u64(rs.nodes), c1 = warp_sum_u64(rs.search_nodes),
                       c2 = warp_sum_u64(rs.leaves), c3 = warp_sum_u64(rs.hits), c4 = warp_sum_u64(rs.rounds),
                       c5 = warp_sum_u64(traced), c8 = warp_sum_u64(walks), c9 = warp_sum_u64(rs.entries);
    if (lane == 0) {
      atomicAdd(a.stats + 0, c0);
      atomicAdd(a.stats + 1, c1);
      atomicAdd(a.stats + 4, c4);
      atomicAdd(a.stats + 2, c2);
      atomicAdd(a.stats + 3, c3);
      atomicAdd(a.stats + 5, c5);
      atomicAdd(a.stats + 8, c8);
      atomicAdd(a.stats + 9, c9);
    }
  }
}

// P of the receivers of batch [r0, r1) from V[s][i]: one lane per receiver, a compensated sum
// over the directions per coefficient (orders <= 3 from the Cartesian SH, above from the table).
__global__ void __launch_bounds__(128) k_project(TraceArgs a, const float* __restrict__ V) {
  extern __shared__ float psdir[];  // [S*3]
  for (int i = threadIdx.x; i < 3 * a.S; i += blockDim.x) psdir[i] = a.dirs[i];
  __syncthreads();
  const int64_t batch = a.r1 - a.r0;
  const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= batch) return;
  const int self = (int)(a.r0 + li);
  const float4 q3 = __ldg(a.recs + 4 * self + 3);
  const int gid = a.order[self];
  const int C = sh_count(a.sh_order);
  const float wq = 4.0f * kPi / (float)a.S;
  for (int kb = 0; kb < C; kb += kMaxC) {
    CompSum acc[kMaxC];
    for (int s = 0; s < a.S; ++s) {
      const float* d = psdir + 3 * s;
      const float c = ray_cos(q3.y, q3.z, q3.w, d);
      if (!(c > 0.0f)) continue;
      const float v = V[(int64_t)s * batch + li] * c * wq;
      if (C <= kMaxC) {
        float Y[kMaxC];
        sh_eval_dyn(a.sh_order, d[0], d[1], d[2], Y);
#pragma unroll
        for (int k = 0; k < kMaxC; ++k)
          if (k < C) acc[k].add(v * Y[k]);
      } else {
#pragma unroll
        for (int k = 0; k < kMaxC; ++k)
          if (kb + k < C) acc[k].add(v * __ldg(a.Ytab + (int64_t)s * C + kb + k));
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxC; ++k)
      if (kb + k < C) a.P[(int64_t)gid * C + kb + k] = acc[k].value();
  }
  if (a.Vg) {
    const int slot = a.glossy_slot[gid];
    if (slot >= 0)
      for (int s = 0; s < a.S; ++s) a.Vg[(int64_t)slot * a.S + s] = V[(int64_t)s * batch + li];
  }
}

static size_t packet_smem(int S, bool bounce) {
  return sizeof(float) * ((3 * S + 3) & ~3) + sizeof(PacketSmem) * kPacketWarps +
         (bounce ? sizeof(RoundHits) * kPacketWarps : 0);
}

template <bool BOUNCE>
static int launch_packet_t(const TraceArgs& a, float* V, int sms, cudaStream_t stream) {
  const size_t smem = packet_smem(a.S, BOUNCE);
  cudaFuncSetAttribute(k_packet<BOUNCE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k_packet<BOUNCE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_packet<BOUNCE>, kPacketThreads, smem);
  // work items: (window of 64 receivers, dpi directions); at most 2^26 / 64 of them per batch
  const int dpi = a.packet_dirs > 0 ? a.packet_dirs : kPacketDirs;
  cudaMemsetAsync(a.work, 0, sizeof(unsigned int), stream);
  k_packet<BOUNCE><<<sms * (per_sm > 0 ? per_sm : 1), kPacketThreads, smem, counted(stream)>>>(a, V, dpi);
  PRTGS_CHECK_LAUNCH();
  const int64_t batch = a.r1 - a.r0;
  k_project<<<(unsigned)((batch + 127) / 128), 128, sizeof(float) * 3 * a.S, counted(stream)>>>(a, V);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// Visibility, P (and with bounce the index matrix) of receiver batch [a.r0, a.r1) by packets;
// V is scratch of S * batch floats.
int launch_packet(const TraceArgs& a, float* V, bool bounce, int sms, cudaStream_t stream) {
  return bounce ? launch_packet_t<true>(a, V, sms, stream) : launch_packet_t<false>(a, V, sms, stream);
}

}  // namespace prtgs
