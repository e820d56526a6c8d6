// Shared device helpers of libprtgs (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/prtgs.h"

#define PRTGS_CHECK_LAUNCH()                               \
  do {                                                     \
    if (cudaPeekAtLastError() != cudaSuccess) {            \
      (void)cudaGetLastError();                            \
      return PRTGS_ERR_CUDA;                               \
    }                                                      \
  } while (0)

namespace prtgs {

// Kernel launches issued by the library (every launch passes its stream through counted()).
std::atomic<unsigned long long>& launch_counter();
inline cudaStream_t counted(cudaStream_t s) {
  launch_counter().fetch_add(1ull, std::memory_order_relaxed);
  return s;
}

constexpr int kMaxC = 16;           // SH coefficients for order <= 3
constexpr int kStackDepth = 64;     // binary radix tree over 64-bit keys: depth <= 64
constexpr int kSceneShift = 57;     // key: scene << 57 | code << 27 | local index
constexpr int kCodeShift = 27;
constexpr int kMaxScenes = 128;
constexpr int64_t kMaxScenePoints = int64_t(1) << 27;
constexpr float kPi = 3.14159265358979323846f;

__host__ __device__ inline int sh_count(int order) { return (order + 1) * (order + 1); }

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Carve aligned sub-buffers out of a workspace.
struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base(static_cast<char*>(b)), off(0) {}
  template <class T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += align_up(count * sizeof(T));
    return p;
  }
};

__device__ inline void set_status(int32_t* status, int bits) {
  if (status) atomicOr(status, bits);
}

// ---- real spherical harmonics, Cartesian form (l <= 3, Condon-Shortley phase, k = l*l+l+m)
// The constants are sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial factors of
// the associated Legendre functions, evaluated once in double precision.
template <int ORDER>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
  Y[0] = 0.28209479177387814f;
  if (ORDER >= 1) {
    Y[1] = -0.48860251190291992f * y;
    Y[2] = 0.48860251190291992f * z;
    Y[3] = -0.48860251190291992f * x;
  }
  if (ORDER >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.54627421529603959f * (xx - yy);
    if (ORDER >= 3) {
      Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
      Y[10] = 2.8906114426405538f * x * y * z;
      Y[11] = -0.45704579946446572f * y * (5.0f * zz - 1.0f);
      Y[12] = 0.3731763325901154f * z * (5.0f * zz - 3.0f);
      Y[13] = -0.45704579946446572f * x * (5.0f * zz - 1.0f);
      Y[14] = 1.4453057213202769f * z * (xx - yy);
      Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
    }
  }
}

__device__ __forceinline__ void sh_eval_dyn(int order, float x, float y, float z, float* Y) {
  switch (order) {
    case 1: sh_eval<1>(x, y, z, Y); break;
    case 2: sh_eval<2>(x, y, z, Y); break;
    default: sh_eval<3>(x, y, z, Y); break;
  }
}

// ---- real SH of orders 4-6 in FP32 (the same basis and index l*l+l+m): Y_l0 = K_l0 Q_l^0(z),
// Y_l(+-m) = sqrt2 K_lm Q_l^m(z) {Re, Im}(x + i y)^m with Q_l^m = P_l^m / sin^m (Condon-Shortley
// phase): Q_m^m = (-1)^m (2m-1)!!, Q_{m+1}^m = (2m+1) z Q_m^m,
// (l-m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m, K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).
__host__ __device__ constexpr double sh_k2(int l, int m) {
  double r = (2.0 * l + 1.0) / (4.0 * 3.14159265358979323846);
  for (int j = l - m + 1; j <= l + m; ++j) r /= (double)j;
  return r;
}

template <int ORDER>
__device__ __forceinline__ void sh_eval_rec(float x, float y, float z, float* Y) {
  float re = 1.0f, im = 0.0f, qmm = 1.0f;
#pragma unroll
  for (int m = 0; m <= ORDER; ++m) {
    if (m > 0) {
      const float r2 = re * x - im * y, i2 = re * y + im * x;
      re = r2;
      im = i2;
      qmm *= -(2.0f * m - 1.0f);
    }
    float q2 = 0.0f, q1 = qmm;
#pragma unroll
    for (int l = m; l <= ORDER; ++l) {
      float q;
      if (l == m) q = qmm;
      else if (l == m + 1) q = (2.0f * m + 1.0f) * z * qmm;
      else q = ((2.0f * l - 1.0f) * z * q1 - (float)(l + m - 1) * q2) * (1.0f / (float)(l - m));
      if (l > m) {
        q2 = q1;
        q1 = q;
      }
      const float K = (float)sh_k2(l, m);
      if (m == 0) {
        Y[l * l + l] = sqrtf(K) * q;
      } else {
        const float f = sqrtf(2.0f * K) * q;
        Y[l * l + l + m] = f * re;
        Y[l * l + l - m] = f * im;
      }
    }
  }
}

// Orders 1-3 in the Cartesian form above, 4-6 by the recurrence.
template <int ORDER>
__device__ __forceinline__ void sh_eval_any(float x, float y, float z, float* Y) {
  if constexpr (ORDER <= 3) sh_eval<ORDER>(x, y, z, Y);
  else sh_eval_rec<ORDER>(x, y, z, Y);
}

// ---- error-free transformations (Knuth TwoSum) for compensated sums
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a b - c d without cancellation (Kahan's difference of products with an FMA: the rounding
// error of c d is recovered exactly and added back).
__device__ __forceinline__ float diff_prod(float a, float b, float c, float d) {
  const float w = c * d;
  const float e = fmaf(-c, d, w);
  return fmaf(a, b, -w) + e;
}

// Neumaier-style compensated accumulator.
struct CompSum {
  float s, c;
  __device__ __forceinline__ CompSum() : s(0.f), c(0.f) {}
  __device__ __forceinline__ void add(float v) {
    float t, e;
    two_sum(s, v, t, e);
    s = t;
    c = __fadd_rn(c, e);
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// Warp sum of a compensated pair: the error terms are carried along.
__device__ __forceinline__ float warp_comp_sum(float s, float c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float so = __shfl_xor_sync(0xffffffffu, s, off);
    float co = __shfl_xor_sync(0xffffffffu, c, off);
    float t, e;
    two_sum(s, so, t, e);
    s = t;
    c = c + co + e;
  }
  return s + c;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Order-preserving float <-> uint32 map for atomic min/max.
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Index of the scene that contains Gaussian `i` (offsets[0] = 0 <= i < offsets[B]).
__device__ __forceinline__ int find_scene(const int64_t* offsets, int n_scenes, int64_t i) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Gradient of a loss with respect to the (unnormalised) quaternion q = (w,x,y,z) given the
// gradient gR with respect to R(q / |q|), R the rotation matrix of Eq. 2.
__device__ __forceinline__ void quat_backward(float qw0, float qx0, float qy0, float qz0, const float gR[3][3],
                                              float gq[4]) {
  const float qn = sqrtf(qw0 * qw0 + qx0 * qx0 + qy0 * qy0 + qz0 * qz0);
  const float qw = qw0 / qn, qx = qx0 / qn, qy = qy0 / qn, qz = qz0 / qn;
  const float gw = 2.f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] +
                          qx * gR[2][1]);
  const float gx = 2.f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.f * qx * gR[1][1] - qw * gR[1][2] +
                          qz * gR[2][0] + qw * gR[2][1] - 2.f * qx * gR[2][2]);
  const float gy = 2.f * (-2.f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] + qz * gR[1][2] -
                          qw * gR[2][0] + qz * gR[2][1] - 2.f * qy * gR[2][2]);
  const float gz = 2.f * (-2.f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] -
                          2.f * qz * gR[1][1] + qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
  const float dot = qw * gw + qx * gx + qy * gy + qz * gz;
  gq[0] = (gw - qw * dot) / qn;
  gq[1] = (gx - qx * dot) / qn;
  gq[2] = (gy - qy * dot) / qn;
  gq[3] = (gz - qz * dot) / qn;
}

}  // namespace prtgs
