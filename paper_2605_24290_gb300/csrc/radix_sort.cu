// radix_sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs,
// 8-bit digits, used to order every view's instances by (view, tile, depth)
// (Algorithm 1, Stage 1: per-tile depth-sorted lists).  Stability keeps
// equal keys in emission order, which is ascending Gaussian index.
//
// One pass = histogram kernel (per-block digit counts), offset kernel (one
// block per digit: exclusive scan over blocks plus the digit's base), and a
// scatter kernel that ranks each item stably inside its block with warp
// match-any and per-warp digit counters in shared memory.
#include "rxgs_internal.h"

namespace rxgs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;                        // items per lane
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 items per block
constexpr int kDigits = 256;

__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, size_t n, int shift,
                                  uint32_t* __restrict__ hist, uint32_t* __restrict__ totals,
                                  int nblocks, const uint32_t* __restrict__ n_dev) {
  if (n_dev && *n_dev < n) n = *n_dev;
  __shared__ uint32_t h[kDigits];
  h[threadIdx.x] = 0;
  __syncthreads();
  const size_t base = static_cast<size_t>(blockIdx.x) * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const size_t i = base + static_cast<size_t>(r) * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  const uint32_t c = h[threadIdx.x];
  hist[static_cast<size_t>(threadIdx.x) * nblocks + blockIdx.x] = c;
  if (c) atomicAdd(&totals[threadIdx.x], c);
}

// Block d: offsets[d][b] = base(d) + sum_{b' < b} hist[d][b'], base(d) =
// sum_{d' < d} totals[d'].
__global__ void radix_offsets_kernel(uint32_t* __restrict__ hist,
                                     const uint32_t* __restrict__ totals, int nblocks) {
  __shared__ uint32_t sh[kSortThreads];
  __shared__ uint32_t carry_s;
  const int d = blockIdx.x;
  // digit base
  uint32_t t = threadIdx.x < static_cast<unsigned>(d) ? totals[threadIdx.x] : 0;
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = kSortThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < static_cast<unsigned>(o)) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) carry_s = sh[0];
  __syncthreads();
  uint32_t carry = carry_s;
  uint32_t* row = hist + static_cast<size_t>(d) * nblocks;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ uint32_t wsum[kSortWarps];
  for (int base = 0; base < nblocks; base += kSortThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nblocks ? row[i] : 0;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t s = wsum[w];
      if (w < wid) before += s;
      total += s;
    }
    if (i < nblocks) row[i] = carry + before + x - v;
    carry += total;
    __syncthreads();
  }
}

__global__ void radix_scatter_kernel(const uint64_t* __restrict__ keys_in,
                                     const uint32_t* __restrict__ vals_in, size_t n, int shift,
                                     const uint32_t* __restrict__ offsets, int nblocks,
                                     uint64_t* __restrict__ keys_out,
                                     uint32_t* __restrict__ vals_out,
                                     const uint32_t* __restrict__ n_dev) {
  if (n_dev && *n_dev < n) n = *n_dev;
  __shared__ uint32_t wcnt[kSortWarps][kDigits];
  __shared__ uint32_t gbase[kDigits];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kSortWarps * kDigits; d += kSortThreads)
    (&wcnt[0][0])[d] = 0;
  gbase[threadIdx.x] = offsets[static_cast<size_t>(threadIdx.x) * nblocks + blockIdx.x];
  __syncthreads();
  // warp w owns items [base + w*256, base + (w+1)*256), 32 per round in order
  const size_t wbase = static_cast<size_t>(blockIdx.x) * kSortTile +
                       static_cast<size_t>(wid) * (32 * kSortRounds);
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t k[kSortRounds];
  uint32_t val[kSortRounds];
  uint32_t rank[kSortRounds];
  int dig[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const size_t i = wbase + static_cast<size_t>(r) * 32 + lane;
    const bool ok = i < n;
    k[r] = ok ? keys_in[i] : 0;
    val[r] = ok ? vals_in[i] : 0;
    const int d = ok ? static_cast<int>((k[r] >> shift) & 0xff) : kDigits;  // kDigits = none
    dig[r] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned before = __popc(peers & lt_mask);
    const int leader = 31 - __clz(peers);
    uint32_t b = 0;
    if (d < kDigits) b = wcnt[wid][d];
    __syncwarp();
    if (d < kDigits && lane == leader) wcnt[wid][d] = b + __popc(peers);
    __syncwarp();
    rank[r] = b + before;
  }
  __syncthreads();
  // exclusive prefix over warps for each digit
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int d = dig[r];
    if (d < kDigits) {
      const uint32_t pos = gbase[d] + wcnt[wid][d] + rank[r];
      keys_out[pos] = k[r];
      vals_out[pos] = val[r];
    }
  }
}

size_t radix_tmp_words(size_t n) {
  const size_t nb = (n + kSortTile - 1) / kSortTile;
  return nb * kDigits + kDigits;
}

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      size_t n, int bits, uint32_t* tmp, bool* result_in_alt, cudaStream_t s,
                      const uint32_t* n_dev) {
  *result_in_alt = false;
  if (n <= 1 || bits <= 0) return;
  const int nb = static_cast<int>((n + kSortTile - 1) / kSortTile);
  uint32_t* hist = tmp;
  uint32_t* totals = tmp + static_cast<size_t>(nb) * kDigits;
  uint64_t *kin = keys, *kout = keys_alt;
  uint32_t *vin = vals, *vout = vals_alt;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    cudaMemsetAsync(totals, 0, sizeof(uint32_t) * kDigits, s);
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(kin, n, shift, hist, totals, nb, n_dev);
    note_launches(1);
    radix_offsets_kernel<<<kDigits, kSortThreads, 0, s>>>(hist, totals, nb);
    note_launches(1);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(kin, vin, n, shift, hist, nb, kout, vout,
                                                     n_dev);
    note_launches(1);
    uint64_t* tk = kin;
    kin = kout;
    kout = tk;
    uint32_t* tv = vin;
    vin = vout;
    vout = tv;
    alt = !alt;
  }
  *result_in_alt = alt;
}

}  // namespace rxgs
