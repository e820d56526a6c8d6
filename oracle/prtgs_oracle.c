/*
 * PRTGS FP64 oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, brute-force CPU restatement of the radiance-transfer precompute of
 * "PRTGS: Precomputed Radiance Transfer of Gaussian Splats" (arxiv 2408.03538). It is
 * used only by the test-suite, by the smoke check and by the timed CPU baseline. It
 * shares no code with the CUDA library: no BVH (every ray is tested against every
 * Gaussian), SH from the associated-Legendre recurrence (the CUDA side uses Cartesian
 * polynomials), the closest-approach distance from the textbook quadratic in FP64.
 *
 * All float inputs are promoted exactly to double. Outputs are double.
 *
 * Functions and the passages they follow:
 *   oracle_sh            real orthonormal SH, Eq. 8-10 (basis), Eq. 13 (orthonormality)
 *   oracle_trace         per receiver and direction: hit set along the ray (Sec. 4.4,
 *                        Eq. 27 read as the Gaussian's maximum along the ray), visibility
 *                        V = prod(1 - alpha_j) (Eq. 4 applied along a ray), the weight
 *                        W_j (Eq. 26), the index matrix (Sec. 4.4, -1 = no hit) and the
 *                        diffuse transfer vector P = sum_s w V (n.w_s)^+ Y(w_s) (Eq. 29
 *                        projected with Eq. 9, f_d factored out, w = 4 pi / S).
 *   oracle_morton_lbvh   Morton codes (FP32 quantisation, the same decision precision as
 *                        the CUDA side) and the binary radix tree over the sorted keys,
 *                        built top-down from its definition (Karras 2012).
 *
 * Parity bookkeeping (not part of the method): rays whose discrete decisions sit within
 * a rounding band of a boundary (D^2 = 9, t* = 0, near-tied weights, near-equal hit
 * distances) are flagged, and a bound on how much the result can change if that
 * decision flips is returned as an allowance.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORACLE_MAX_ORDER 6
#define ORACLE_MAX_C ((ORACLE_MAX_ORDER + 1) * (ORACLE_MAX_ORDER + 1))

/* ---------------------------------------------------------------------------------------
 * Real spherical harmonics (Eq. 8-10). Orthonormal, Condon-Shortley phase carried by
 * P_l^m, flat index k = l*l + l + m.
 * ------------------------------------------------------------------------------------- */
static double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= (double)i;
  return r;
}

/* Associated Legendre P_l^m(x), m >= 0, l <= L, by the standard three-term recurrence. */
static void legendre_all(int L, double x, double P[ORACLE_MAX_ORDER + 1][ORACLE_MAX_ORDER + 1]) {
  double s = sqrt(fmax(0.0, 1.0 - x * x));
  for (int m = 0; m <= L; ++m) {
    /* P_m^m = (-1)^m (2m-1)!! s^m */
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * s;
    P[m][m] = pmm;
    if (m + 1 <= L) P[m + 1][m] = x * (2.0 * m + 1.0) * pmm;
    for (int l = m + 2; l <= L; ++l)
      P[l][m] = ((2.0 * l - 1.0) * x * P[l - 1][m] - (double)(l + m - 1) * P[l - 2][m]) / (double)(l - m);
  }
}

static void sh_eval(int order, const double d_in[3], double* Y) {
  double nrm = sqrt(d_in[0] * d_in[0] + d_in[1] * d_in[1] + d_in[2] * d_in[2]);
  double x = d_in[0] / nrm, y = d_in[1] / nrm, z = d_in[2] / nrm;
  double phi = atan2(y, x);
  double P[ORACLE_MAX_ORDER + 1][ORACLE_MAX_ORDER + 1];
  legendre_all(order, z, P);
  for (int l = 0; l <= order; ++l) {
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
      double v;
      if (m > 0)
        v = sqrt(2.0) * K * cos(m * phi) * P[l][am];
      else if (m < 0)
        v = sqrt(2.0) * K * sin(am * phi) * P[l][am];
      else
        v = K * P[l][0];
      Y[l * l + l + m] = v;
    }
  }
}

int oracle_sh(int order, int64_t n, const double* dirs, double* Y) {
  if (order < 0 || order > ORACLE_MAX_ORDER) return -3;
  int C = (order + 1) * (order + 1);
  for (int64_t i = 0; i < n; ++i) sh_eval(order, dirs + 3 * i, Y + i * C);
  return 0;
}

/* ---------------------------------------------------------------------------------------
 * Gaussian geometry (Eq. 1-2): R from the normalised quaternion (w,x,y,z),
 * Sigma^-1 = R diag(1/s^2) R^T.
 * ------------------------------------------------------------------------------------- */
static void quat_to_rot(const float* qf, double R[3][3]) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

typedef struct {
  double mu[3];
  double sinv[3][3]; /* Sigma^-1 */
  double sigma;      /* opacity */
  double n[3];       /* normal */
  double s_min, s_max;
} OG;

static void make_og(const float* means, const float* scales, const float* quats, const float* opacity,
                    const float* normals, int64_t j, OG* g) {
  double R[3][3];
  quat_to_rot(quats + 4 * j, R);
  double inv2[3];
  g->s_min = 1e300; g->s_max = 0;
  for (int k = 0; k < 3; ++k) {
    double s = scales[3 * j + k];
    inv2[k] = 1.0 / (s * s);
    if (s < g->s_min) g->s_min = s;
    if (s > g->s_max) g->s_max = s;
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += R[a][k] * inv2[k] * R[b][k];
      g->sinv[a][b] = acc;
    }
  for (int k = 0; k < 3; ++k) {
    g->mu[k] = means[3 * j + k];
    g->n[k] = normals[3 * j + k];
  }
  g->sigma = opacity[j];
}

static double quad(const double A[3][3], const double* u, const double* v) {
  double r = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) r += u[a] * A[a][b] * v[b];
  return r;
}

typedef struct {
  double t;      /* closest-approach parameter t* along the ray */
  double d2;     /* squared Mahalanobis distance of the closest approach */
  double alpha;  /* sigma * exp(-d2/2) */
  int64_t j;
  int ambiguous; /* within the rounding band of D^2 = 9 or t* = 0 */
} Hit;

static int hit_cmp(const void* pa, const void* pb) {
  const Hit* a = (const Hit*)pa;
  const Hit* b = (const Hit*)pb;
  if (a->t < b->t) return -1;
  if (a->t > b->t) return 1;
  return (a->j < b->j) ? -1 : (a->j > b->j);
}

/* ray_flags bits */
#define RF_TRACED 1
#define RF_AMBIG_HIT 2     /* an occluder sits within the D^2 / t* rounding band */
#define RF_AMBIG_ARGMAX 4  /* near-tied weights, near-equal t*, or the filter boundary */

/* Rounding bands of the discrete decisions (documented with the parity tests). */
#define BAND_D2_ABS 1e-4
#define BAND_D2_REL_U 2e-8  /* x |u|/s_min */
#define BAND_T_REL 4e-6
#define BAND_W_REL 1e-4
#define BAND_ORDER_REL 4e-6

/*
 * oracle_trace: brute-force tracing for a list of receivers.
 *
 * flags: bit0 = shadow (visibility), bit1 = bounce bookkeeping (weights, index matrix).
 * Index-matrix candidates are the eligible hits whose prefix transmittance (the product in
 * front of them) is at least t_min: hits behind a prefix below the visibility cut-off are
 * not candidates (t_min = 0 gives the unrestricted argmax).
 * Outputs (n_recv rows):
 *   P[n_recv, C]         diffuse transfer vector, raw (no rho, no 1/pi)
 *   V[n_recv, S]         visibility per ray (0 for untraced rays, n.w <= 0)
 *   idx[n_recv, S]       index matrix (argmax W; -1 = no hit / untraced)
 *   cand[n_recv, S, 4]   for bounce: the hits with the 4 largest W (-1 padded)
 *   ray_flags[n_recv, S] RF_* bits
 *   dV[n_recv, S]        bound on |V_gpu - V| from ambiguous occluders (no early exit here)
 *   hits[n_recv]         number of (ray, occluder) intersections over the receiver's traced rays
 *   hits_live[n_recv]    the same, counting each ray's hits in t order only until its
 *                        transmittance first falls below t_min (that hit included): the hits a
 *                        walk with the visibility cut-off must take (nullable)
 */
int oracle_trace(int64_t n, const float* means, const float* scales, const float* quats, const float* opacity,
                 const float* normals, int S, const float* dirs, int order, int flags, double filter_t,
                 double t_min, int64_t n_recv, const int64_t* recv, double* P, double* V, int32_t* idx, int32_t* cand,
                 int32_t* ray_flags, double* dV, double* hits, double* hits_live) {
  if (order < 0 || order > ORACLE_MAX_ORDER) return -3;
  const int C = (order + 1) * (order + 1);
  const double w = 4.0 * M_PI / (double)S;
  OG* g = (OG*)malloc(sizeof(OG) * (size_t)(n > 0 ? n : 1));
  double* Ys = (double*)malloc(sizeof(double) * (size_t)S * C);
  if (!g || !Ys) { free(g); free(Ys); return -5; }
  for (int64_t j = 0; j < n; ++j) make_og(means, scales, quats, opacity, normals, j, &g[j]);
  for (int s = 0; s < S; ++s) {
    double d[3] = {dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2]};
    sh_eval(order, d, Ys + (size_t)s * C);
  }
  int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < n_recv; ++r) {
    int64_t i = recv[r];
    Hit* hl = (Hit*)malloc(sizeof(Hit) * (size_t)(n > 0 ? n : 1));
    if (!hl) { err = -5; continue; }
    double Pacc[ORACLE_MAX_C];
    for (int k = 0; k < C; ++k) Pacc[k] = 0;
    double hit_total = 0, live_total = 0;
    const OG* gi = &g[i];
    for (int s = 0; s < S; ++s) {
      double d[3] = {dirs[3 * s], dirs[3 * s + 1], dirs[3 * s + 2]};
      size_t rs = (size_t)r * S + s;
      double c = gi->n[0] * d[0] + gi->n[1] * d[1] + gi->n[2] * d[2];
      V[rs] = 0; idx[rs] = -1; ray_flags[rs] = 0; dV[rs] = 0;
      if (cand) for (int q = 0; q < 4; ++q) cand[rs * 4 + q] = -1;
      if (c <= 0) continue;
      ray_flags[rs] |= RF_TRACED;
      int nh = 0;
      double vis = 1.0;
      if (flags & 1) {
        for (int64_t j = 0; j < n; ++j) {
          if (j == i) continue;
          const OG* gj = &g[j];
          double u[3] = {gi->mu[0] - gj->mu[0], gi->mu[1] - gj->mu[1], gi->mu[2] - gj->mu[2]};
          double a = quad(gj->sinv, d, d);
          double b = quad(gj->sinv, u, d);
          double cc = quad(gj->sinv, u, u);
          double t = -b / a;
          double d2 = cc - b * b / a;
          if (d2 < 0) d2 = 0;
          double ulen = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
          double band_d2 = BAND_D2_ABS + BAND_D2_REL_U * ulen / gj->s_min;
          double band_t = BAND_T_REL * (ulen + gj->s_max);
          int in_d = d2 <= 9.0, in_t = t > 0.0;
          int near_d = fabs(d2 - 9.0) <= band_d2, near_t = fabs(t) <= band_t;
          int amb = (near_d && (in_t || near_t)) || (near_t && (in_d || near_d));
          if ((in_d && in_t) || amb) {
            Hit h;
            h.t = t; h.d2 = d2; h.j = j; h.ambiguous = amb;
            h.alpha = gj->sigma * exp(-0.5 * d2);
            h.ambiguous = amb;
            if (!(in_d && in_t)) h.ambiguous = 2; /* ambiguous, decided "miss" */
            hl[nh++] = h;
          }
        }
        /* visibility: product over the definite and "hit"-decided occluders */
        for (int q = 0; q < nh; ++q)
          if (hl[q].ambiguous != 2) vis *= (1.0 - hl[q].alpha);
        for (int q = 0; q < nh; ++q) {
          if (hl[q].ambiguous) {
            ray_flags[rs] |= RF_AMBIG_HIT;
            /* flipping this decision changes V by (V excluding j) * alpha_j */
            double vex = hl[q].ambiguous == 2 ? vis : vis / (1.0 - hl[q].alpha);
            dV[rs] += vex * hl[q].alpha;
          }
          if (hl[q].ambiguous != 2) hit_total += 1.0;
        }
      }
      V[rs] = vis;
      for (int k = 0; k < C; ++k) Pacc[k] += w * vis * c * Ys[(size_t)s * C + k];
      if (hits_live && nh > 0) {
        qsort(hl, (size_t)nh, sizeof(Hit), hit_cmp);
        double tl = 1.0;
        for (int q = 0; q < nh; ++q) {
          if (hl[q].ambiguous == 2) continue;
          live_total += 1.0;
          tl *= 1.0 - hl[q].alpha;
          if (tl < t_min) break;
        }
      }

      if ((flags & 2) && nh > 0) {
        qsort(hl, (size_t)nh, sizeof(Hit), hit_cmp);
        /* W_j = alpha_j * prod_{earlier}(1 - alpha) * max(-d.n_j, 0) (Eq. 26), compared in the
         * log domain so that deep prefix products cannot underflow; the argmax is the same. */
        const double lfilter = log(filter_t);
        const double lhorizon = t_min > 0 ? log(t_min) : -INFINITY;
        double lT = 0.0, lwbest = -INFINITY;
        int64_t best = -1;
        int best_pos = -1;
        double top[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        int64_t topj[4] = {-1, -1, -1, -1};
        int amb_arg = 0;
        for (int q = 0; q < nh; ++q) {
          if (hl[q].ambiguous == 2) { amb_arg = amb_arg || (lT > lwbest); continue; }
          const OG* gj = &g[hl[q].j];
          double m = -(d[0] * gj->n[0] + d[1] * gj->n[1] + d[2] * gj->n[2]);
          double lW = (m > 0 && hl[q].alpha > 0) ? log(hl[q].alpha) + lT + log(m) : -INFINITY;
          int eligible = lT <= lfilter && lT >= lhorizon;
          if (filter_t < 1.0 && fabs(lT - lfilter) <= 1e-5) amb_arg = 1;
          if (t_min > 0 && fabs(lT - lhorizon) <= 1e-4 * fabs(lhorizon) + 1e-5) amb_arg = 1;
          if (eligible && lW > -INFINITY) {
            if (lW > lwbest) { lwbest = lW; best = hl[q].j; best_pos = q; }
            /* keep the 4 largest weights as alternative candidates */
            for (int a2 = 0; a2 < 4; ++a2) {
              if (lW > top[a2]) {
                for (int b2 = 3; b2 > a2; --b2) { top[b2] = top[b2 - 1]; topj[b2] = topj[b2 - 1]; }
                top[a2] = lW; topj[a2] = hl[q].j;
                break;
              }
            }
          }
          if (hl[q].ambiguous) amb_arg = amb_arg || (lT > lwbest - BAND_W_REL);
          lT += log1p(-hl[q].alpha);
        }
        idx[rs] = (int32_t)best;
        if (best >= 0) {
          /* near-tied runner-up */
          if (top[1] > -INFINITY && top[1] >= lwbest - BAND_W_REL) amb_arg = 1;
          /* near-equal hit distances up to just past the winner can reorder the prefix products */
          for (int q = 0; q + 1 < nh && q <= best_pos + 1; ++q) {
            double dt = fabs(hl[q + 1].t - hl[q].t);
            if (dt <= BAND_ORDER_REL * (fabs(hl[q].t) + 1e-3)) amb_arg = 1;
          }
          /* further on, a front-facing hit within that band of the hits just in front of it may
           * be ordered before them: its prefix then lacks their factors (1 - alpha), and if it
           * could outweigh the winner that way the argmax is open too */
          double lTq = 0.0;
          for (int q = 0; q < nh; ++q) {
            if (hl[q].ambiguous == 2) continue;
            if (q > best_pos + 1 && hl[q].alpha > 0) {
              const OG* gq = &g[hl[q].j];
              double m = -(d[0] * gq->n[0] + d[1] * gq->n[1] + d[2] * gq->n[2]);
              if (m > 0) {
                double gain = 0.0;
                for (int p = q - 1; p >= 0; --p) {
                  if (hl[p].ambiguous == 2) continue;
                  if (hl[q].t - hl[p].t > BAND_ORDER_REL * (fabs(hl[p].t) + 1e-3)) break;
                  gain -= log1p(-hl[p].alpha);
                }
                if (gain > 0 && log(hl[q].alpha) + lTq + gain + log(m) >= lwbest - BAND_W_REL) amb_arg = 1;
              }
            }
            lTq += log1p(-hl[q].alpha);
          }
        }
        if (amb_arg) ray_flags[rs] |= RF_AMBIG_ARGMAX;
        if (cand)
          for (int q = 0; q < 4; ++q) cand[rs * 4 + q] = (int32_t)topj[q];
      }
    }
    for (int k = 0; k < C; ++k) P[(size_t)r * C + k] = Pacc[k];
    if (hits) hits[r] = hit_total;
    if (hits_live) hits_live[r] = live_total;
    free(hl);
  }
  free(g);
  free(Ys);
  return err;
}

/* ---------------------------------------------------------------------------------------
 * Morton codes and the binary radix tree (LBVH, Karras 2012) used by Sec. 4.4's BVH.
 *
 * The quantisation decides an integer from floats, so it is written in float with the
 * same operation sequence as the CUDA side (this file is compiled with
 * -ffp-contract=off): q = min(floor((c - lo) * (1024 / (hi - lo))), 1023), clamped at 0.
 * Key layout: scene << 57 | code30 << 27 | local index (< 2^27).
 * The tree is derived top-down from its definition: a node covering sorted positions
 * [lo, hi] splits after the last position whose key shares more leading bits with
 * key[lo] than key[hi] does; the child covering [lo, split] is leaf `lo` if it has one
 * element, otherwise internal node `split`; the child covering [split+1, hi] is leaf
 * `split+1` or internal node `split+1`. Internal node 0 is the root of the whole range.
 * ------------------------------------------------------------------------------------- */
static uint32_t spread10(uint32_t v) {
  uint32_t r = 0;
  for (int b = 0; b < 10; ++b) r |= ((v >> b) & 1u) << (3 * b);
  return r;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y);
}

static int clz64(uint64_t x) {
  if (x == 0) return 64;
  int n = 0;
  while (!(x & 0x8000000000000000ull)) { x <<= 1; ++n; }
  return n;
}

typedef struct { int64_t lo, hi, node; } Range;

int oracle_morton_lbvh(int64_t n, const float* means, int n_scenes, const int64_t* offsets, uint32_t* codes,
                       uint64_t* keys_sorted, int32_t* order, int32_t* children, int32_t* roots) {
  if (n <= 0) return 0;
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  if (!keys) return -5;
  for (int b = 0; b < n_scenes; ++b) {
    int64_t s0 = offsets[b], s1 = offsets[b + 1];
    if (s1 <= s0) continue;
    float lo[3], hi[3], sc[3];
    for (int a = 0; a < 3; ++a) { lo[a] = means[3 * s0 + a]; hi[a] = lo[a]; }
    for (int64_t i = s0; i < s1; ++i)
      for (int a = 0; a < 3; ++a) {
        float v = means[3 * i + a];
        if (v < lo[a]) lo[a] = v;
        if (v > hi[a]) hi[a] = v;
      }
    for (int a = 0; a < 3; ++a) {
      float ext = hi[a] - lo[a];
      sc[a] = ext > 0.0f ? 1024.0f / ext : 0.0f;
    }
    for (int64_t i = s0; i < s1; ++i) {
      uint32_t q[3];
      for (int a = 0; a < 3; ++a) {
        float t = means[3 * i + a] - lo[a];
        float m = t * sc[a];
        float f = floorf(m);
        int v = (int)f;
        if (v < 0) v = 0;
        if (v > 1023) v = 1023;
        q[a] = (uint32_t)v;
      }
      uint32_t code = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
      if (codes) codes[i] = code;
      keys[i] = ((uint64_t)b << 57) | ((uint64_t)code << 27) | (uint64_t)(i - s0);
    }
  }
  /* sort (keys are unique) */
  qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
  /* sorted position -> Gaussian id: the scene bits give the offset, the low bits the local index */
  for (int64_t p = 0; p < n; ++p) {
    int b = (int)(keys[p] >> 57);
    order[p] = (int32_t)(offsets[b] + (int64_t)(keys[p] & ((1ull << 27) - 1)));
    if (keys_sorted) keys_sorted[p] = keys[p];
  }
  /* scene roots: the node covering exactly the scene's sorted range */
  for (int b = 0; b < n_scenes; ++b) roots[b] = INT32_MIN;
  if (n == 1) {
    roots[0] = -1 - order[0];
    free(keys);
    return 0;
  }
  Range* st = (Range*)malloc(sizeof(Range) * 256);
  int sp = 0;
  st[sp++] = (Range){0, n - 1, 0};
  /* scene ranges in sorted positions */
  int64_t* sbeg = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_scenes + 1));
  {
    int64_t p = 0;
    for (int b = 0; b < n_scenes; ++b) {
      sbeg[b] = p;
      p += offsets[b + 1] - offsets[b];
    }
    sbeg[n_scenes] = p;
  }
  while (sp > 0) {
    Range r = st[--sp];
    for (int b = 0; b < n_scenes; ++b)
      if (sbeg[b] == r.lo && sbeg[b + 1] - 1 == r.hi) roots[b] = r.node;
    int dnode = clz64(keys[r.lo] ^ keys[r.hi]);
    int64_t split = r.lo;
    for (int64_t p = r.lo; p < r.hi; ++p)
      if (clz64(keys[r.lo] ^ keys[p]) > dnode) split = p;
    int32_t left = (split == r.lo) ? -1 - order[split] : (int32_t)split;
    int32_t right = (split + 1 == r.hi) ? -1 - order[split + 1] : (int32_t)(split + 1);
    children[2 * r.node] = left;
    children[2 * r.node + 1] = right;
    if (split != r.lo) st[sp++] = (Range){r.lo, split, split};
    if (split + 1 != r.hi) st[sp++] = (Range){split + 1, r.hi, split + 1};
  }
  for (int b = 0; b < n_scenes; ++b) {
    if (roots[b] != INT32_MIN) continue;
    /* single-Gaussian scenes are leaves */
    if (sbeg[b + 1] - sbeg[b] == 1) roots[b] = -1 - order[sbeg[b]];
  }
  free(sbeg);
  free(st);
  free(keys);
  return 0;
}
