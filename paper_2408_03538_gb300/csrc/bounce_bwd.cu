// Backward of the self-transfer bounces (Eq. 33-35) with the index matrix held fixed.
//
// Forward, per channel c: T = T^0 + T^1 + ... + T^n, T^0_i = P_i (the same for the three
// channels) and T^k = B T^{k-1}, (B X)_i[c] = sum_s w (n_i.w_s)^+ (rho_j[c]/pi) X_j[c], j = idx[i,s].
// B is linear in X; its adjoint scatters: (B^T L)_j[c] = sum_{(i,s): idx[i,s] = j} w (n_i.w_s)^+
// (rho_j[c]/pi) L_i[c]. With the upstream gradient G = dLoss/dT, the adjoints are
//   A^n = G,  A^{k-1} = G + B^T A^k (k - 1 >= 1),  dLoss/dP_i = sum_c (G + B^T A^1)_i[c],
// and every bounce k adds the partials of B at X = T^{k-1}:
//   dLoss/drho_j[c] += sum_{(i,s): idx = j} w c_is / pi (A^k_i[c] . X_j[c]),
//   dLoss/dn_i      += sum_s w w_s [c_is > 0] sum_c rho_j[c]/pi (A^k_i[c] . X_j[c]).
// The intermediates T^1 .. T^{n-1} are recomputed with the forward's gathers. Scatters use float
// atomics (the last bits vary run to run, like the transfer backward).
#include "common.cuh"
#include "internal.h"

namespace prtgs {

// One warp per receiver i, its lanes over the directions; FROM_P: X = T^0 = P ([n,C]).
template <bool FROM_P>
__global__ void k_bounce_bwd(int64_t n, int C, int S, const float* __restrict__ dirs, const float* __restrict__ normals,
                             const float* __restrict__ albedo, const int32_t* __restrict__ idx,
                             const float* __restrict__ A, const float* __restrict__ X, float* __restrict__ Y,
                             float* __restrict__ d_albedo, float* __restrict__ d_normals, int32_t* status) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const float nx = normals[3 * i], ny = normals[3 * i + 1], nz = normals[3 * i + 2];
  const float wq = 4.0f * kPi / (float)S;
  const float* Ai = A + i * 3 * C;
  float gn0 = 0.f, gn1 = 0.f, gn2 = 0.f;
  for (int s = lane; s < S; s += 32) {
    int j = idx[i * S + s];
    if (j >= n) {
      set_status(status, PRTGS_STATUS_BAD_INDEX);
      j = -1;
    }
    if (j < 0) continue;
    const float* d = dirs + 3 * s;
    const float c = fmaf(nx, d[0], fmaf(ny, d[1], nz * d[2]));
    if (!(c > 0.0f)) continue;
    const float coef = wq * c * (1.0f / kPi);
    float q[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float* xj = FROM_P ? X + (int64_t)j * C : X + ((int64_t)j * 3 + ch) * C;
      const float* ai = Ai + ch * C;
      float acc = 0.f;
      for (int m = 0; m < C; ++m) acc = fmaf(__ldg(ai + m), __ldg(xj + m), acc);
      q[ch] = acc;
    }
    float gc = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float rho = __ldg(albedo + 3 * j + ch);
      atomicAdd(d_albedo + 3 * j + ch, coef * q[ch]);
      gc = fmaf(rho * (1.0f / kPi), q[ch], gc);
      const float cr = coef * rho;
      float* yj = Y + ((int64_t)j * 3 + ch) * C;
      const float* ai = Ai + ch * C;
      for (int m = 0; m < C; ++m) atomicAdd(yj + m, cr * __ldg(ai + m));
    }
    // dc/dn = w_s (c > 0)
    gn0 = fmaf(wq * gc, d[0], gn0);
    gn1 = fmaf(wq * gc, d[1], gn1);
    gn2 = fmaf(wq * gc, d[2], gn2);
  }
  gn0 = warp_sum(gn0);
  gn1 = warp_sum(gn1);
  gn2 = warp_sum(gn2);
  if (lane == 0) {  // the warp owns receiver i: plain accumulation across the bounces
    d_normals[3 * i] += gn0;
    d_normals[3 * i + 1] += gn1;
    d_normals[3 * i + 2] += gn2;
  }
}

// A = G + Y (FINAL: dP_i[m] = sum_c (G + Y)_i[c][m]).
template <bool FINAL>
__global__ void k_bounce_adjoint(int64_t n, int C, const float* __restrict__ G, const float* __restrict__ Y,
                                 float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (FINAL) {
    if (e >= n * C) return;
    const int64_t i = e / C, m = e % C;
    float acc = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) acc += G[(i * 3 + ch) * C + m] + Y[(i * 3 + ch) * C + m];
    out[e] = acc;
  } else {
    if (e >= n * 3 * C) return;
    out[e] = G[e] + Y[e];
  }
}

size_t bounce_backward_workspace(int64_t n, int32_t order, int32_t n_bounces) {
  const int nb = n_bounces > 1 ? n_bounces : 1;
  const size_t buf = align_up(sizeof(float) * (size_t)n * 3 * sh_count(order));
  // T^1 .. T^{n-1}, a scratch T for the forward gathers, the adjoint A and the scatter Y
  return (size_t)(nb - 1) * buf + (nb > 1 ? buf : 0) + 2 * buf;
}

int bounce_backward(int64_t n, int32_t order, int32_t S, const float* dirs, const float* normals,
                    const float* albedo, const float* P, const int32_t* idx, int32_t n_bounces, const float* dT,
                    float* dP, float* d_albedo, float* d_normals, int32_t* status, void* ws, cudaStream_t stream) {
  const int C = sh_count(order);
  const int nb = n_bounces > 1 ? n_bounces : 1;
  cudaMemsetAsync(d_albedo, 0, sizeof(float) * 3 * n, stream);
  cudaMemsetAsync(d_normals, 0, sizeof(float) * 3 * n, stream);
  if (n == 0) return PRTGS_OK;
  Carver cv(ws);
  const size_t per = (size_t)n * 3 * C;
  float* Xk[64];
  for (int k = 1; k < nb; ++k) Xk[k] = cv.take<float>(per);
  float* Tscr = nb > 1 ? cv.take<float>(per) : nullptr;
  float* A = cv.take<float>(per);
  float* Y = cv.take<float>(per);
  // forward intermediates T^1 .. T^{n-1} (the forward's own gathers)
  for (int k = 1; k < nb; ++k) {
    const int rc = bounce_step(n, C, S, dirs, normals, albedo, P, k == 1 ? nullptr : Xk[k - 1], idx, Tscr, Xk[k],
                               status, stream);
    if (rc != PRTGS_OK) return rc;
  }
  const unsigned blocks = (unsigned)((n + 7) / 8);  // 8 warps (receivers) per block
  const float* Acur = dT;
  for (int k = nb; k >= 1; --k) {
    cudaMemsetAsync(Y, 0, sizeof(float) * per, stream);
    if (k == 1)
      k_bounce_bwd<true><<<blocks, 256, 0, counted(stream)>>>(n, C, S, dirs, normals, albedo, idx, Acur, P, Y,
                                                              d_albedo, d_normals, status);
    else
      k_bounce_bwd<false><<<blocks, 256, 0, counted(stream)>>>(n, C, S, dirs, normals, albedo, idx, Acur, Xk[k - 1],
                                                               Y, d_albedo, d_normals, status);
    if (k > 1) {
      k_bounce_adjoint<false><<<(unsigned)((per + 255) / 256), 256, 0, counted(stream)>>>(n, C, dT, Y, A);
      Acur = A;
    } else {
      k_bounce_adjoint<true><<<(unsigned)((n * C + 255) / 256), 256, 0, counted(stream)>>>(n, C, dT, Y, dP);
    }
    PRTGS_CHECK_LAUNCH();
  }
  return PRTGS_OK;
}

}  // namespace prtgs
