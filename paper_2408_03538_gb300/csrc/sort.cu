// Prefix sums and a stable LSD radix sort of (uint64 key, int32 value) pairs.
//
// Used by the BVH build (Morton keys, Sec. 4.4) and by the splat rasteriser's
// (tile, depth) ordering (front-to-back order of Eq. 4).
#include "common.cuh"
#include "internal.h"

namespace prtgs {

// ------------------------------------------------------------------------------------------
// Three-phase prefix sum over uint32: per-block totals, a scan of the block totals in one
// block, then per-block scans with their offsets.
// ------------------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* smem_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? smem_warp[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    smem_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  total = smem_warp[(blockDim.x >> 5) - 1];
  uint32_t before = warp > 0 ? smem_warp[warp - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t sw[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  uint32_t total;
  block_exclusive_scan(s, sw, total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_block_sums(uint32_t* __restrict__ sums, int64_t nb, uint32_t* __restrict__ grand_total) {
  __shared__ uint32_t sw[32];
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < nb ? sums[i] : 0u;
    uint32_t total;
    uint32_t ex = block_exclusive_scan(v, sw, total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             const uint32_t* __restrict__ block_offsets, int exclusive) {
  __shared__ uint32_t sw[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, sw, total) + block_offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = exclusive ? run : run + v[k];
    run += v[k];
  }
}

size_t scan_workspace(int64_t n) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  return align_up(sizeof(uint32_t) * (size_t)(nb > 0 ? nb : 1));
}

int scan_u32(const uint32_t* in, uint32_t* out, int64_t n, bool exclusive, uint32_t* total, void* ws,
             cudaStream_t stream) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), stream);
    return PRTGS_OK;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  uint32_t* sums = static_cast<uint32_t*>(ws);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, counted(stream)>>>(in, n, sums);
  k_scan_block_sums<<<1, 1024, 0, counted(stream)>>>(sums, nb, total);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, counted(stream)>>>(in, out, n, sums, exclusive ? 1 : 0);
  PRTGS_CHECK_LAUNCH();
  return PRTGS_OK;
}

// ------------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits. One pass = per-tile digit histograms (digit-major so
// that one exclusive scan gives every (digit, tile) its output offset), the scan, and a
// stable scatter that ranks keys inside a tile round by round: warp-level rank with
// __match_any_sync, then a per-digit prefix over the warps of the block.
// The element count may live on the device (d_count), so the whole sort can be enqueued
// without a host round trip; tiles past the count do no work.
// ------------------------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;

__device__ __forceinline__ int64_t sort_count(const uint32_t* d_count, int64_t capacity) {
  if (!d_count) return capacity;
  int64_t c = (int64_t)*d_count;
  return c < capacity ? c : capacity;
}

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t capacity, const uint32_t* d_count,
                             int shift, int n_tiles, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t n = sort_count(d_count, capacity);
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                                uint64_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t capacity,
                                const uint32_t* d_count, int shift, int n_tiles,
                                const uint32_t* __restrict__ offsets) {
  __shared__ uint32_t base_d[256];
  __shared__ uint32_t cnt[kSortWarps][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base_d[tid] = offsets[(int64_t)tid * n_tiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) cnt[w][tid] = 0;
  __syncthreads();
  int64_t n = sort_count(d_count, capacity);
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= n) return;  // uniform over the block
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + r * kSortThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? keys_in[i] : 0ull;
    int32_t val = valid ? vals_in[i] : 0;
    unsigned digit = valid ? (unsigned)((key >> shift) & 0xffu) : 256u + (unsigned)lane;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0) cnt[warp][digit] = __popc(peers);
    __syncthreads();
    {  // per-digit prefix over the warps, in warp order (keeps the sort stable)
      uint32_t run = base_d[tid];
#pragma unroll
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t c = cnt[w][tid];
        cnt[w][tid] = run;
        run += c;
      }
      base_d[tid] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = cnt[warp][digit] + rank;
      if ((int64_t)pos < n) {  // always true when the histograms are consistent
        keys_out[pos] = key;
        vals_out[pos] = val;
      }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) cnt[w][tid] = 0;
    __syncthreads();
    if (base + (r + 1) * kSortThreads >= n) break;  // uniform
  }
}

size_t radix_sort_workspace(int64_t capacity) {
  int64_t tiles = (capacity + kSortTile - 1) / kSortTile;
  if (tiles < 1) tiles = 1;
  size_t hist = align_up(sizeof(uint32_t) * 256 * (size_t)tiles);
  return hist + scan_workspace(256 * tiles);
}

int radix_sort_pairs(const uint64_t* keys_x, const int32_t* vals_x, uint64_t* keys_f, int32_t* vals_f,
                     uint64_t* keys_y, int32_t* vals_y, int64_t capacity, const uint32_t* d_count, int begin_bit,
                     int end_bit, void* ws, cudaStream_t stream) {
  if (capacity <= 0) return PRTGS_OK;
  int tiles = (int)((capacity + kSortTile - 1) / kSortTile);
  Carver c(ws);
  uint32_t* hist = c.take<uint32_t>(256 * (size_t)tiles);
  void* scan_ws = c.take<char>(scan_workspace(256 * (int64_t)tiles));
  int passes = (end_bit - begin_bit + 7) / 8;
  if (passes < 1) passes = 1;
  const uint64_t* ksrc = keys_x;
  const int32_t* vsrc = vals_x;
  for (int p = 0; p < passes; ++p) {
    // the last pass must land in the final buffers
    bool to_f = ((passes - 1 - p) % 2) == 0;
    uint64_t* kdst = to_f ? keys_f : keys_y;
    int32_t* vdst = to_f ? vals_f : vals_y;
    int shift = begin_bit + 8 * p;
    k_radix_hist<<<tiles, kSortThreads, 0, counted(stream)>>>(ksrc, capacity, d_count, shift, tiles, hist);
    int rc = scan_u32(hist, hist, 256 * (int64_t)tiles, true, nullptr, scan_ws, stream);
    if (rc != PRTGS_OK) return rc;
    k_radix_scatter<<<tiles, kSortThreads, 0, counted(stream)>>>(ksrc, vsrc, kdst, vdst, capacity, d_count, shift, tiles,
                                                         hist);
    PRTGS_CHECK_LAUNCH();
    ksrc = kdst;
    vsrc = vdst;
  }
  return PRTGS_OK;
}

}  // namespace prtgs
