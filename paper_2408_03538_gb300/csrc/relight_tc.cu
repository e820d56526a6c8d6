// Relight contraction on the 5th-generation tensor cores (tcgen05), Eq. 14:
//   scalar T [n,C]:   D[i, 3l+c] = sum_m T[i,m] L[l,c,m]       (one MMA, N = 3k)
//   RGB T [n,3,C]:    D_c[i, l]  = sum_m T[i,c,m] L[l,c,m]     (three MMAs, N = k each)
//   colors[l,i,c] = (rho_i[c] / pi) D
// per tile of 128 Gaussians, N padded to a multiple of 16 (<= 256), accumulated in FP32 in
// tensor memory. K = C is padded to 16 per K block: one block for orders 1-3 (C <= 16), two to
// four for orders 4-6 (C = 25, 36, 49 -> K = 32, 48, 64). The lights of every K block stay in
// shared memory; the A operand is staged one K block at a time, each block's MMAs accumulating
// onto the previous ones after the mbarrier has signalled that they are done reading it.
//
// Precision. PRTGS_PREC_BF16 feeds bf16(T) and bf16(L) (one K = 16 slab). PRTGS_PREC_BF16X3
// splits both operands into three BF16 terms, x = x1 + x2 + x3 (x1 = bf16(x), x2 = bf16(x - x1),
// x3 = bf16(x - x1 - x2)), and accumulates the six products whose order is at most 2^-16
// relative: T1L1 + T1L2 + T2L1 + T1L3 + T2L2 + T3L1, as six K slabs of one MMA chain (the
// split-BF16 scheme of Henry, Tang and Heinecke, "Leveraging the bfloat16 AI datatype for
// higher-precision computations", 2019). The dropped terms are below 2^-24 relative.
//
// Data movement. The operands are transformed on the way in (split into BF16 terms), so they
// are staged with ordinary loads (16-byte loads of the T rows) and stores into shared memory in
// the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices, core matrices
// adjacent in K 128 bytes apart (leading byte offset), 8-row groups 256 bytes apart (stride
// byte offset). One elected thread issues the MMAs; completion is signalled through an
// mbarrier (tcgen05.commit); each warp then reads its 32 accumulator lanes with tcgen05.ld,
// eight lights (24 columns) at a time, and stores each row's three channels directly (staging
// the rows through shared memory for 16-byte stores measured slower: L2 merges them).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace prtgs {

namespace {

constexpr int kTcRows = 128;       // MMA M (one Gaussian per TMEM lane)
#ifndef PRTGS_TC_KSPLIT
#define PRTGS_TC_KSPLIT 2
#endif
constexpr int kKSplit = PRTGS_TC_KSPLIT;  // threads per tile row (each stages 16 / kKSplit of K)
constexpr int kKW = 16 / kKSplit;
constexpr int kTcThreads = 128 * kKSplit;  // warps w, w + 4, ... share TMEM lanes 32(w%4)..+31
constexpr int kSlabBytesA = kTcRows * 16 * 2;  // one K = 16 slab of A: 4 KB
constexpr int kMaxN = 256;
constexpr unsigned kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of a K = 16 slab in the no-swizzle K-major layout.
__device__ __forceinline__ int kmajor_offset(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// tcgen05 shared-memory matrix descriptor: start address, leading / stride byte offsets
// (all >> 4), version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3fffu);
  d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r);
  r = r - __bfloat162float(b);
  c = __float2bfloat16_rn(r);
}

// Two BF16 values as one 32-bit word, the first in the low half (the lower K index).
__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Which split term of T and of L each K slab multiplies (BF16X3).
__device__ __forceinline__ int a_term(int slab) { return slab == 2 || slab == 4 ? 1 : (slab == 5 ? 2 : 0); }
__device__ __forceinline__ int b_term(int slab) { return slab == 1 || slab == 4 ? 1 : (slab == 3 ? 2 : 0); }

// B operand (the split light SH of one scene) into shared memory: for scalar T one group
// whose row o = 3l + c is L[l][c][:]; for RGB T group c whose row l is L[l][c][:].
// Slab (g, kb, slab) of B sits at ((g * KB + kb) * slabs + slab) * n_pad * 32 bytes.
template <int C, int TCH>
__device__ __forceinline__ void load_lights(unsigned char* sB, const float* __restrict__ L, int k, int n_pad,
                                            int slabs) {
  constexpr int KB = (C + 15) / 16;
  const int rows = TCH == 1 ? 3 * k : k;
  const int per_slab = n_pad * 16;
  const int per_group = KB * slabs * per_slab;
  for (int e = threadIdx.x; e < TCH * per_group; e += kTcThreads) {
    const int g = e / per_group, rem0 = e % per_group;
    const int kbs = rem0 / per_slab, rem = rem0 % per_slab;  // kbs = kb * slabs + slab
    const int kb = kbs / slabs, slab = kbs % slabs;
    const int row = rem / 16, kk = rem % 16;
    const int m = 16 * kb + kk;
    float v = 0.f;
    if (row < rows && m < C) v = TCH == 1 ? L[(int64_t)row * C + m] : L[((int64_t)row * 3 + g) * C + m];
    __nv_bfloat16 t1, t2, t3;
    split3(v, t1, t2, t3);
    const int term = slabs == 1 ? 0 : b_term(slab);
    const __nv_bfloat16 sel = term == 0 ? t1 : (term == 1 ? t2 : t3);
    *reinterpret_cast<__nv_bfloat16*>(sB + ((g * KB + kb) * slabs + slab) * n_pad * 32 + kmajor_offset(row, kk)) = sel;
  }
}

// Polls the mbarrier phase at most `polls` times; true once the phase has completed.
__device__ __forceinline__ bool bounded_wait(uint32_t bar, uint32_t phase, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ int64_t ob_of(const int64_t* offsets, int b) { return offsets ? offsets[b] : 0; }
__device__ __forceinline__ int64_t nb_of(const int64_t* offsets, int b, int64_t n) {
  return offsets ? offsets[b + 1] - offsets[b] : n;
}

// NaN for every light's output of this thread's row (a tile whose MMA result is not trusted).
template <bool PIXEL>
__device__ __forceinline__ void write_nan(bool mine, int k, int64_t n, int64_t gi, int64_t ob, int64_t nb,
                                          float* __restrict__ colors) {
  if (!mine || (threadIdx.x >> 7) != 0) return;  // one thread per row
  const float q = __int_as_float(0x7fc00000);
  for (int l = 0; l < k; ++l) {
    if (PIXEL) {
      for (int c = 0; c < 3; ++c) colors[((int64_t)l * 3 + c) * n + gi] = q;
    } else {
      float* out = colors + 3 * (int64_t)k * ob + ((int64_t)l * nb + (gi - ob)) * 3;
      out[0] = q;
      out[1] = q;
      out[2] = q;
    }
  }
}

// offsets == nullptr: one scene with lights L. Otherwise scene b (rows offsets[b] ..
// offsets[b+1]) uses lights L + b * k * 3 * C; a tile that straddles scenes is run once per
// scene with the other rows zeroed. n_pad: N of each MMA; TMEM group g starts at column
// g * n_pad.
// PIXEL: the rows are the n pixels of a transfer image TI[C][3][n] (the composite of the splats'
// (rho/pi) T); colors is the image [k][3][n] and receives D + bg[c] final_T[p] (albedo holds
// final_T); otherwise rows are splats, T is [n][TCH][C] and colors [k][n][3] gets rho/pi D.
template <int C, int TCH, bool PIXEL = false>
__global__ void __launch_bounds__(kTcThreads) k_relight_tc(int64_t n, const float* __restrict__ T,
                                                           const float* __restrict__ albedo,
                                                           const float* __restrict__ L, int k, int n_pad, int slabs,
                                                           int tmem_cols, const int64_t* __restrict__ offsets,
                                                           int n_scenes, float* __restrict__ colors,
                                                           const float* __restrict__ bgv, int32_t* status,
                                                           unsigned wait_polls) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int KB = (C + 15) / 16;  // K blocks of 16
  // layout: [A: groups x slabs of one K block][B: groups x K blocks x slabs]
  unsigned char* sA = smem_raw;
  unsigned char* sB = smem_raw + TCH * slabs * kSlabBytesA;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTcRows - 1), khalf = tid >> 7;  // tile row; K part and light share

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(kTcRows, n_pad);
  const bool t_vec = (reinterpret_cast<uintptr_t>(T) & 15) == 0;  // 16-byte row loads need it
  uint32_t phase = 0;
  const int64_t tiles = (n + kTcRows - 1) / kTcRows;
  int cached = -1;
  bool failed = false;  // a completion wait of this CTA gave up: no further MMAs, NaN outputs
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kTcRows;
    const int64_t row_end = row0 + kTcRows < n ? row0 + kTcRows : n;
    const int b_first = offsets ? find_scene(offsets, n_scenes, row0) : 0;
    const int b_last = offsets ? find_scene(offsets, n_scenes, row_end - 1) : 0;
    const int64_t gi = row0 + row;
    float rho[3] = {0.f, 0.f, 0.f}, add[3] = {0.f, 0.f, 0.f};
    if (gi < n) {
      if (PIXEL) {
        const float ft = __ldg(albedo + gi);  // final transmittance of the pixel
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rho[c] = 1.0f;
          add[c] = bgv ? bgv[c] * ft : 0.f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) rho[c] = __ldg(albedo + 3 * gi + c) * (1.0f / kPi);
      }
    }
    for (int b = b_first; b <= b_last; ++b) {
      const int64_t lo = offsets ? (offsets[b] > row0 ? offsets[b] : row0) : row0;
      const int64_t hi = offsets ? (offsets[b + 1] < row_end ? offsets[b + 1] : row_end) : row_end;
      if (hi <= lo) continue;  // empty scene (uniform over the block)
      const bool mine = gi >= lo && gi < hi;
      if (failed) {  // CTA-uniform: the tensor cores are no longer used by this CTA
        write_nan<PIXEL>(mine, k, n, gi, ob_of(offsets, b), nb_of(offsets, b, n), colors);
        continue;
      }
      if (b != cached) {
        load_lights<C, TCH>(sB, L + (int64_t)b * k * 3 * C, k, n_pad, slabs);
        cached = b;
      }
      // output block of this scene: [k, n_b, 3] at 3 k offsets[b] (the whole [k, n, 3] for one scene)
      const int64_t ob = offsets ? offsets[b] : 0;
      const int64_t nb = offsets ? offsets[b + 1] - ob : n;
      float* cb = colors + 3 * (int64_t)k * ob;
      for (int kb = 0; kb < KB; ++kb) {
        float tv[TCH][kKW];  // this thread's part of the row's K block kb
        if (PIXEL) {
#pragma unroll
          for (int g = 0; g < TCH; ++g)
#pragma unroll
            for (int j = 0; j < kKW; ++j) {
              const int m = 16 * kb + kKW * khalf + j;
              tv[g][j] = (gi < n && m < C) ? __ldg(T + ((int64_t)m * 3 + g) * n + gi) : 0.f;
            }
        } else if (C == 16 && t_vec && gi < n) {
          const float4* src = reinterpret_cast<const float4*>(T + gi * TCH * C + kKW * khalf);
#pragma unroll
          for (int g = 0; g < TCH; ++g)
#pragma unroll
            for (int q = 0; q < kKW / 4; ++q) {
              const float4 v = __ldg(src + 4 * g + q);
              tv[g][4 * q] = v.x;
              tv[g][4 * q + 1] = v.y;
              tv[g][4 * q + 2] = v.z;
              tv[g][4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
          for (int g = 0; g < TCH; ++g)
#pragma unroll
            for (int j = 0; j < kKW; ++j) {
              const int m = 16 * kb + kKW * khalf + j;
              tv[g][j] = (gi < n && m < C) ? __ldg(T + (gi * TCH + g) * C + m) : 0.f;
            }
        }
        // A operand: this thread's part of the row, split into BF16 terms (zero outside the
        // scene). In the K-major layout a row's K = 0..7 and 8..15 are two contiguous 16-byte
        // runs: one 16-byte (or 8-byte) store per slab.
#pragma unroll
        for (int g = 0; g < TCH; ++g) {
          uint32_t pk[3][kKW / 2];  // term x (pairs of K)
#pragma unroll
          for (int j = 0; j < kKW; j += 2) {
            __nv_bfloat16 a1, a2, a3, b1, b2, b3;
            split3(mine ? tv[g][j] : 0.f, a1, a2, a3);
            split3(mine ? tv[g][j + 1] : 0.f, b1, b2, b3);
            pk[0][j / 2] = pack_bf16x2(a1, b1);
            pk[1][j / 2] = pack_bf16x2(a2, b2);
            pk[2][j / 2] = pack_bf16x2(a3, b3);
          }
          for (int slab = 0; slab < slabs; ++slab) {
            const int term = slabs == 1 ? 0 : a_term(slab);
            unsigned char* base = sA + (g * slabs + slab) * kSlabBytesA;
            const uint32_t* q = term == 0 ? pk[0] : (term == 1 ? pk[1] : pk[2]);
            if constexpr (kKW == 8)
              *reinterpret_cast<uint4*>(base + kmajor_offset(row, 8 * khalf)) = make_uint4(q[0], q[1], q[2], q[3]);
            else
              *reinterpret_cast<uint2*>(base + kmajor_offset(row, kKW * khalf)) = make_uint2(q[0], q[1]);
          }
        }
        // make the generic-proxy stores visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          for (int g = 0; g < TCH; ++g)
            for (int slab = 0; slab < slabs; ++slab) {
              const uint64_t da = smem_desc(smem_u32(sA + (g * slabs + slab) * kSlabBytesA), 128, 256);
              const uint64_t db = smem_desc(smem_u32(sB + ((g * KB + kb) * slabs + slab) * n_pad * 32), 128, 256);
              const uint32_t acc = (kb > 0 || slab > 0) ? 1u : 0u;
              asm volatile(
                  "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + (uint32_t)(g * n_pad)),
                  "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar)));
        }
        // bounded wait for this K block's MMA chain (after it, the A operand may be restaged). If
        // any thread gives up, the whole CTA treats the tile as failed: it reports
        // PRTGS_STATUS_TIMEOUT and waits again with the full limit so that the chain has finished
        // reading the operands and writing the accumulator before anything reuses them (or the
        // tensor memory is freed); the tile's outputs become NaN.
        bool done = bounded_wait(smem_u32(&mbar), phase, wait_polls);
        if (__syncthreads_or(!done)) {
          if (tid == 0) set_status(status, PRTGS_STATUS_TIMEOUT);
          bounded_wait(smem_u32(&mbar), phase, kWaitLimit);
          failed = true;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (failed) break;  // CTA-uniform
      }
      if (failed) {
        write_nan<PIXEL>(mine, k, n, gi, ob, nb, colors);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        continue;
      }
      // epilogue: this thread holds accumulator row `row` (TMEM lane row); eight lights at a
      // time, the warps of a lane quarter taking groups of eight in turn
      for (int l0 = 8 * khalf; l0 < k; l0 += 8 * kKSplit) {
        uint32_t r[24];
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          // scalar T: columns 3 l0 + 8 j .. (lights l0..l0+7, channel-minor); RGB T: group j
          const uint32_t col = TCH == 1 ? (uint32_t)(3 * l0 + 8 * j) : (uint32_t)(j * n_pad + l0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
              : "=r"(r[8 * j]), "=r"(r[8 * j + 1]), "=r"(r[8 * j + 2]), "=r"(r[8 * j + 3]), "=r"(r[8 * j + 4]),
                "=r"(r[8 * j + 5]), "=r"(r[8 * j + 6]), "=r"(r[8 * j + 7])
              : "r"(lane_base + col));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int ll = 0; ll < 8; ++ll) {
          const int l = l0 + ll;
          if (l >= k) break;  // uniform
          float v[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const uint32_t bits = TCH == 1 ? r[3 * ll + c] : r[8 * c + ll];
            v[c] = fmaf(__uint_as_float(bits), rho[c], add[c]);
          }
          if (PIXEL) {
            if (mine) {
#pragma unroll
              for (int c = 0; c < 3; ++c) colors[((int64_t)l * 3 + c) * n + gi] = v[c];
            }
          } else if (mine) {
            float* out = cb + ((int64_t)l * nb + (gi - ob)) * 3;
            out[0] = v[0];
            out[1] = v[1];
            out[2] = v[2];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();  // the next pass overwrites the operands and the accumulator
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

}  // namespace

template <int C, int TCH>
static void launch_tc(int grid, size_t smem, cudaStream_t stream, int64_t n, const float* T, const float* albedo,
                      const float* L, int k, int n_pad, int slabs, int tmem_cols, const int64_t* offsets,
                      int n_scenes, float* colors, int32_t* status, unsigned wait_polls) {
  cudaFuncSetAttribute(k_relight_tc<C, TCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_relight_tc<C, TCH><<<grid, kTcThreads, smem, counted(stream)>>>(n, T, albedo, L, k, n_pad, slabs, tmem_cols, offsets,
                                                            n_scenes, colors, nullptr, status, wait_polls);
}

// Dynamic shared memory of one CTA: the A slabs of one K block and the B slabs of every K block.
static size_t tc_smem(int order, int tch, int slabs, int n_pad) {
  const int kb = (sh_count(order) + 15) / 16;
  return (size_t)tch * slabs * kSlabBytesA + (size_t)tch * kb * slabs * n_pad * 32 + 1024;
}

// Whether a tensor-core relight of this shape fits one MMA's N, the TMEM columns and one CTA's
// shared memory.
int relight_tc_fits(int32_t order, int32_t k, int32_t t_channels, int32_t precision) {
  int n_pad = 0, cols = 0;
  if (order < 1 || order > 6 || !relight_tc_shape(k, t_channels, &n_pad, &cols)) return 0;
  const int slabs = precision == PRTGS_PREC_BF16X3 ? 6 : 1;
  return tc_smem(order, t_channels, slabs, n_pad) <= (size_t)227 * 1024 ? 1 : 0;
}

// Tensor-core shape of a relight: N of each MMA and the TMEM columns (a power of two >= 32
// holding every group and the 24 columns the epilogue reads per eight lights), or 0 when the
// shape does not fit one MMA (N <= 256) or the 512 TMEM columns.
int relight_tc_shape(int32_t k, int32_t t_channels, int* n_pad_out, int* tmem_cols_out) {
  if (k <= 0 || (t_channels != 1 && t_channels != 3)) return 0;
  const int k8 = (k + 7) / 8 * 8;
  const int n_pad = t_channels == 1 ? (3 * k + 15) / 16 * 16 : (k + 15) / 16 * 16;
  if (n_pad > kMaxN) return 0;
  int need = t_channels == 1 ? (n_pad > 3 * k8 ? n_pad : 3 * k8) : 3 * n_pad;
  int cols = 32;
  while (cols < need) cols <<= 1;
  if (cols > 512) return 0;
  if (n_pad_out) *n_pad_out = n_pad;
  if (tmem_cols_out) *tmem_cols_out = cols;
  return 1;
}

// Pixel-space relight on the tensor cores: image[l,c,p] = sum_m TI[m,c,p] L[l,c,m] + bg[c] final_T[p].
int relight_tc_pixels(int64_t n_pix, int32_t order, const float* TI, const float* final_T, const float* bg,
                      const float* L, int32_t k, int32_t precision, float* image, int32_t* status,
                      unsigned wait_polls, cudaStream_t stream) {
  if (n_pix == 0 || k == 0) return PRTGS_OK;
  int n_pad = 0, tmem_cols = 0;
  if (!relight_tc_shape(k, 3, &n_pad, &tmem_cols)) return PRTGS_ERR_UNSUPPORTED;
  const int slabs = precision == PRTGS_PREC_BF16X3 ? 6 : 1;
  const size_t smem = tc_smem(order, 3, slabs, n_pad);
  if (smem > 227 * 1024) return PRTGS_ERR_UNSUPPORTED;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n_pix + kTcRows - 1) / kTcRows;
  int per_sm = 512 / tmem_cols;
  const int by_smem = (int)((228 * 1024) / (smem + 1024));
  if (per_sm > by_smem) per_sm = by_smem;
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (int64_t)sms * per_sm;
  const int grid = (int)(tiles < want ? tiles : want);
#define PRTGS_PIX_LAUNCH(CC)                                                                                     \
  cudaFuncSetAttribute(k_relight_tc<CC, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
  k_relight_tc<CC, 3, true><<<grid, kTcThreads, smem, counted(stream)>>>(n_pix, TI, final_T, L, k, n_pad, slabs, tmem_cols, \
                                                                nullptr, 1, image, bg, status, wait_polls)
  switch (order) {
    case 1: PRTGS_PIX_LAUNCH(4); break;
    case 2: PRTGS_PIX_LAUNCH(9); break;
    case 3: PRTGS_PIX_LAUNCH(16); break;
    case 4: PRTGS_PIX_LAUNCH(25); break;
    case 5: PRTGS_PIX_LAUNCH(36); break;
    case 6: PRTGS_PIX_LAUNCH(49); break;
    default: return PRTGS_ERR_UNSUPPORTED;
  }
#undef PRTGS_PIX_LAUNCH
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

int relight_tc(int64_t n, int32_t order, const float* T, int32_t t_channels, const float* albedo, const float* L,
               int32_t k, int32_t precision, const int64_t* offsets, int32_t n_scenes, float* colors,
               int32_t* status, unsigned wait_polls, cudaStream_t stream) {
  if (n == 0 || k == 0) return PRTGS_OK;
  int n_pad = 0, tmem_cols = 0;
  if (!relight_tc_shape(k, t_channels, &n_pad, &tmem_cols)) return PRTGS_ERR_UNSUPPORTED;
  const int slabs = precision == PRTGS_PREC_BF16X3 ? 6 : 1;
  const int tch = t_channels;
  const size_t smem = tc_smem(order, tch, slabs, n_pad);
  if (smem > 227 * 1024) return PRTGS_ERR_UNSUPPORTED;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n + kTcRows - 1) / kTcRows;
  // resident CTAs per SM bounded by the 512 TMEM columns (allocations beyond that would wait
  // for a CTA to finish), by shared memory, and kept at <= 4 so that one CTA's epilogue
  // overlaps another's MMA
  int per_sm = 512 / tmem_cols;
  const int by_smem = (int)((228 * 1024) / (smem + 1024));
  if (per_sm > by_smem) per_sm = by_smem;
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) per_sm = 1;
  const int64_t want = (int64_t)sms * per_sm;
  const int grid = (int)(tiles < want ? tiles : want);
  const bool rgb = tch == 3;
#define PRTGS_TC_LAUNCH(CC)                                                                                       \
  if (rgb) launch_tc<CC, 3>(grid, smem, stream, n, T, albedo, L, k, n_pad, slabs, tmem_cols, offsets, n_scenes,     \
                            colors, status, wait_polls);                                                           \
  else launch_tc<CC, 1>(grid, smem, stream, n, T, albedo, L, k, n_pad, slabs, tmem_cols, offsets, n_scenes, colors, \
                        status, wait_polls)
  switch (order) {
    case 1: PRTGS_TC_LAUNCH(4); break;
    case 2: PRTGS_TC_LAUNCH(9); break;
    case 3: PRTGS_TC_LAUNCH(16); break;
    case 4: PRTGS_TC_LAUNCH(25); break;
    case 5: PRTGS_TC_LAUNCH(36); break;
    case 6: PRTGS_TC_LAUNCH(49); break;
    default: return PRTGS_ERR_UNSUPPORTED;
  }
#undef PRTGS_TC_LAUNCH
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

}  // namespace prtgs
