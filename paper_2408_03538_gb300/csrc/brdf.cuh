// The BRDF kernel of the glossy and training-stage transfers (Eq. 15 times pi):
//   k(w_i, w_o) = (1 - m) + pi f_s,  f_s = D F G / (4 (n.w_i)(n.w_o)),
// GGX D with alpha = r^2, Schlick F with F0 = 0.04 on w_o.h, Smith-Schlick G with k = alpha / 2,
// each for the unit normal n / |n|. Zero unless n.w_i > 0 and n.w_o > 0 (the callers test that).
// Quotients use the fast single-precision divide (__fdividef, 2 ulp): every divisor is a positive
// normal number well inside its range here (den >= min(1, alpha^2), the Smith terms >= alpha/2).
#pragma once
#include "common.cuh"

namespace prtgs {


// k(w_i, w_o) of Eq. 15 times pi for the unit normal n / |n|. ni, no: n . w_i, n . w_o (> 0).
// The GGX denominator (n.h)^2 (a^2 - 1) + 1 is evaluated as (a^2 (n.v)^2 + |n x v|^2) / (|n|^2 |v|^2)
// with v = w_i + w_o kept unnormalised (exactly, as a TwoSum pair) and n x v formed without
// cancellation: near a sharp lobe peak 1 - (n.h)^2 is tiny, and neither the rounding of h nor an
// FP32 normal that is unit only to rounding may leak into it.
__device__ __forceinline__ float brdf_kernel(float nx, float ny, float nz, const float* wi, const float* wo,
                                             float ni, float no, float alpha, float metal) {
  float vx, vy, vz, ex, ey, ez;
  two_sum(wi[0], wo[0], vx, ex);
  two_sum(wi[1], wo[1], vy, ey);
  two_sum(wi[2], wo[2], vz, ez);
  const float cx = diff_prod(ny, vz, nz, vy) + (ny * ez - nz * ey);
  const float cy = diff_prod(nz, vx, nx, vz) + (nz * ex - nx * ez);
  const float cz = diff_prod(nx, vy, ny, vx) + (nx * ey - ny * ex);
  const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
  const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float nv = fmaf(nx, vx, fmaf(ny, vy, nz * vz));
  const float cc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  const float a2 = alpha * alpha;
  const float den = __fdividef(fmaf(a2 * nv, nv, cc), nn * vv);
  const float D = __fdividef(a2, kPi * den * den);
  const float oh = fminf(fmaxf(fmaf(wo[0], vx, fmaf(wo[1], vy, wo[2] * vz)) * rsqrtf(vv), 0.f), 1.f);
  const float x = 1.0f - oh;
  const float x2 = x * x;
  const float F = fmaf(0.96f, x2 * x2 * x, 0.04f);
  const float rn = rsqrtf(nn);
  const float kk = 0.5f * alpha;
  const float gi = __fdividef(1.0f, fmaf(ni * rn, 1.0f - kk, kk));
  const float go = __fdividef(1.0f, fmaf(no * rn, 1.0f - kk, kk));
  return (1.0f - metal) + kPi * 0.25f * D * F * gi * go;
}

// k and dk/dr (r the roughness, alpha = r^2) for the same arguments as brdf_kernel. With
// t = (n.v)^2 / (|n|^2 |v|^2), s = |n x v|^2 / (|n|^2 |v|^2) (v = w_i + w_o), den = a2 t + s,
// a2 = alpha^2 = r^4, D = a2 / (pi den^2) and g = 1 / (x (1 - kk) + kk), kk = r^2 / 2:
//   dD/da2 = (s - a2 t) / (pi den^3),  dg/dkk = -(1 - x) g^2,
//   dk/dr  = pi/4 F [dD/da2 4 r^3 g_i g_o - D r g_i g_o ((1 - x_i) g_i + (1 - x_o) g_o)].
__device__ __forceinline__ float brdf_kernel_dr(float nx, float ny, float nz, const float* wi, const float* wo,
                                                float ni, float no, float r, float metal, float& k) {
  float vx, vy, vz, ex, ey, ez;
  two_sum(wi[0], wo[0], vx, ex);
  two_sum(wi[1], wo[1], vy, ey);
  two_sum(wi[2], wo[2], vz, ez);
  const float cx = diff_prod(ny, vz, nz, vy) + (ny * ez - nz * ey);
  const float cy = diff_prod(nz, vx, nx, vz) + (nz * ex - nx * ez);
  const float cz = diff_prod(nx, vy, ny, vx) + (nx * ey - ny * ex);
  const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
  const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
  const float nv = fmaf(nx, vx, fmaf(ny, vy, nz * vz));
  const float cc = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
  const float alpha = r * r;
  const float a2 = alpha * alpha;
  const float inv = __fdividef(1.0f, nn * vv);
  const float tt = nv * nv * inv, ss = cc * inv;
  const float den = fmaf(a2, tt, ss);
  const float pid2 = __fdividef(1.0f, kPi * den * den);
  const float D = a2 * pid2;
  const float dD = __fdividef((ss - a2 * tt) * pid2, den);
  const float oh = fminf(fmaxf(fmaf(wo[0], vx, fmaf(wo[1], vy, wo[2] * vz)) * rsqrtf(vv), 0.f), 1.f);
  const float x = 1.0f - oh;
  const float x2 = x * x;
  const float F = fmaf(0.96f, x2 * x2 * x, 0.04f);
  const float rn = rsqrtf(nn);
  const float kk = 0.5f * alpha;
  const float xi = ni * rn, xo = no * rn;
  const float gi = __fdividef(1.0f, fmaf(xi, 1.0f - kk, kk));
  const float go = __fdividef(1.0f, fmaf(xo, 1.0f - kk, kk));
  const float q = kPi * 0.25f * F * gi * go;
  k = (1.0f - metal) + q * D;
  return q * (dD * 4.0f * alpha * r - D * r * ((1.0f - xi) * gi + (1.0f - xo) * go));
}

// dk/dn for the raw normal n (the kernel depends on n / |n|; the metallic term does not depend on
// it): with u = n/|n|, h = (w_i + w_o)/|w_i + w_o| and x_h = u.h, x_i = u.w_i, x_o = u.w_o,
//   dk/du = pi/4 F [D'(x_h) g_i g_o h + D g_o g'(x_i) w_i + D g_i g'(x_o) w_o],
//   D'(x) = -4 a2 x (a2 - 1) / (pi den^3), den = x^2 (a2 - 1) + 1,  g'(x) = -(1 - kk) g(x)^2,
// and dk/dn = (dk/du - u (u . dk/du)) / |n|. For gradients; the value of k comes from brdf_kernel.
__device__ __forceinline__ void brdf_kernel_dn(float nx, float ny, float nz, const float* wi, const float* wo, float r,
                                               float* dkdn) {
  const float nn = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
  const float rn = rsqrtf(nn);
  const float ux = nx * rn, uy = ny * rn, uz = nz * rn;
  float hx = wi[0] + wo[0], hy = wi[1] + wo[1], hz = wi[2] + wo[2];
  const float hl = rsqrtf(fmaf(hx, hx, fmaf(hy, hy, hz * hz)));
  hx *= hl;
  hy *= hl;
  hz *= hl;
  const float xh = fmaf(ux, hx, fmaf(uy, hy, uz * hz));
  const float xi = fmaf(ux, wi[0], fmaf(uy, wi[1], uz * wi[2]));
  const float xo = fmaf(ux, wo[0], fmaf(uy, wo[1], uz * wo[2]));
  const float oh = fminf(fmaxf(fmaf(wo[0], hx, fmaf(wo[1], hy, wo[2] * hz)), 0.f), 1.f);
  const float alpha = r * r, a2 = alpha * alpha;
  const float den = fmaf(xh * xh, a2 - 1.0f, 1.0f);
  const float pden = __fdividef(1.0f, kPi * den * den);
  const float D = a2 * pden;
  const float dD = __fdividef(-4.0f * a2 * xh * (a2 - 1.0f) * pden, den);
  const float x = 1.0f - oh, x2 = x * x;
  const float F = fmaf(0.96f, x2 * x2 * x, 0.04f);
  const float kk = 0.5f * alpha;
  const float gi = __fdividef(1.0f, fmaf(xi, 1.0f - kk, kk));
  const float go = __fdividef(1.0f, fmaf(xo, 1.0f - kk, kk));
  const float q = kPi * 0.25f * F;
  const float ch = q * dD * gi * go;
  const float ci = -q * D * go * (1.0f - kk) * gi * gi;
  const float co = -q * D * gi * (1.0f - kk) * go * go;
  const float gx = ch * hx + ci * wi[0] + co * wo[0];
  const float gy = ch * hy + ci * wi[1] + co * wo[1];
  const float gz = ch * hz + ci * wi[2] + co * wo[2];
  const float d = fmaf(ux, gx, fmaf(uy, gy, uz * gz));
  dkdn[0] = (gx - ux * d) * rn;
  dkdn[1] = (gy - uy * d) * rn;
  dkdn[2] = (gz - uz * d) * rn;
}

}  // namespace prtgs
