// radix_sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs,
// used to order every view's instances by (view, tile, depth) (Algorithm 1,
// Stage 1: per-tile depth-sorted lists).  Stability keeps equal keys in
// emission order, which is ascending Gaussian index.
//
// Digits of up to 9 bits (ceil(bits / 9) passes; 44-bit keys take 5).  One
// pass = three kernels over tiles of 2,048 items:
//   sort_count    each tile's digit counts (shared-memory histogram);
//   sort_offsets  one block per digit: where each tile's run of that digit
//                 starts within the digit (exclusive scan over the tiles),
//                 and the digit's total;
//   sort_scatter  adds the digit bases (an exclusive scan of the totals in
//                 each block; no global atomics anywhere in the pass), ranks
//                 the tile's items stably (warp match-any, per-warp digit
//                 counters in shared memory), reorders the tile by digit in
//                 shared memory and writes each digit's run to its place,
//                 consecutive threads on consecutive addresses.
// Every tile's loads are issued before any of its ranks is computed.
#include <algorithm>
#include <utility>

#include "rxgs_internal.h"

namespace rxgs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                   // per thread
constexpr int kTile = kThreads * kItems;    // 2,048 items per tile
constexpr int kMaxWidth = 9;
constexpr int kBins = 1 << kMaxWidth;       // 512
constexpr int kBinsPerThread = kBins / kThreads;
constexpr int kMaxPasses = 8;

struct Plan {
  int passes, width;
};
Plan plan_of(int bits) {
  Plan p;
  p.passes = (bits + kMaxWidth - 1) / kMaxWidth;
  p.width = (bits + p.passes - 1) / p.passes;
  return p;
}

size_t tiles_of(size_t n) { return (n + kTile - 1) / kTile; }

// hist[d * nt + tile] = count of digit d in the tile
__global__ void __launch_bounds__(kThreads) sort_count_kernel(const uint64_t* __restrict__ keys,
                                                              size_t n,
                                                              const uint32_t* __restrict__ n_dev,
                                                              int shift, int width,
                                                              uint32_t* __restrict__ hist, int nt) {
  if (n_dev && *n_dev < n) n = *n_dev;
  __shared__ uint32_t h[kBins];
  for (int d = threadIdx.x; d < kBins; d += kThreads) h[d] = 0;
  const size_t base = static_cast<size_t>(blockIdx.x) * kTile;
  uint64_t k[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(r) * kThreads + threadIdx.x;
    k[r] = i < n ? keys[i] : 0;
  }
  __syncthreads();
  const uint64_t mask = (1ull << width) - 1;
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(r) * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(k[r] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBins; d += kThreads)
    hist[static_cast<size_t>(d) * nt + blockIdx.x] = h[d];
}

// Block d: hist[d][b] <- sum_{b' < b} hist[d][b'] (the run's start within
// the digit) and totals[d] = the digit's count; the digit bases (exclusive
// sums of the totals) are added by the scatter.
__global__ void __launch_bounds__(kThreads) sort_offsets_kernel(uint32_t* __restrict__ hist,
                                                                uint32_t* __restrict__ totals,
                                                                int nt) {
  __shared__ uint32_t wsum[kWarps];
  const int d = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t carry = 0;
  uint32_t* row = hist + static_cast<size_t>(d) * nt;
  for (int base = 0; base < nt; base += kThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nt ? row[i] : 0;
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
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t s = wsum[w];
      if (w < wid) before += s;
      total += s;
    }
    if (i < nt) row[i] = carry + before + x - v;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) totals[d] = carry;
}

struct ScatterSmem {
  uint64_t key[kTile];
  uint32_t val[kTile];
  uint32_t wcnt[kWarps][kBins];  // per-warp digit counts, then their exclusive prefix
  uint32_t toff[kBins];          // the tile's digit runs: start in the reordered tile
  uint32_t gpos[kBins];          // ... and in the output
  uint32_t part[kWarps];
};

__global__ void __launch_bounds__(kThreads) sort_scatter_kernel(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, size_t n, const uint32_t* __restrict__ n_dev, int shift, int width,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ totals, int nt) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatterSmem& S = *reinterpret_cast<ScatterSmem*>(smraw);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (n_dev && *n_dev < n) n = *n_dev;
  const size_t base = static_cast<size_t>(blockIdx.x) * kTile;
  const uint32_t mask = (1u << width) - 1;
  // warp w takes items [base + 256 w, base + 256 (w + 1)), 32 per round;
  // every load in flight before the first rank
  uint64_t k[kItems];
  uint32_t v[kItems], rd[kItems];  // rank in the warp's run << 10 | digit (kBins = none)
  unsigned peers[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(wid) * (32 * kItems) + r * 32 + lane;
    k[r] = i < n ? kin[i] : 0;
    v[r] = i < n ? vin[i] : 0;
  }
  for (int e = t; e < kWarps * kBins; e += kThreads) (&S.wcnt[0][0])[e] = 0;
  {
    // where each digit's run of this tile starts in the output: the digit's
    // base (exclusive sum of the digit totals) plus the tile's offset in it
    uint32_t tv[kBinsPerThread], ts = 0;
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      tv[q] = totals[t * kBinsPerThread + q];
      ts += tv[q];
    }
    uint32_t x = ts;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.part[wid] = x;
    __syncthreads();
    uint32_t b = x - ts;
    for (int w = 0; w < wid; ++w) b += S.part[w];
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      const int d = t * kBinsPerThread + q;
      S.gpos[d] = offsets[static_cast<size_t>(d) * nt + blockIdx.x] + b;
      b += tv[q];
    }
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(wid) * (32 * kItems) + r * 32 + lane;
    const int d = i < n ? static_cast<int>((k[r] >> shift) & mask) : kBins;
    rd[r] = static_cast<uint32_t>(d);
    peers[r] = __match_any_sync(0xffffffffu, d);
  }
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int d = static_cast<int>(rd[r]);
    const unsigned before = __popc(peers[r] & lt_mask);
    const int leader = 31 - __clz(peers[r]);
    uint32_t b = 0;
    if (d < kBins) b = S.wcnt[wid][d];
    __syncwarp();
    if (d < kBins && lane == leader) S.wcnt[wid][d] = b + __popc(peers[r]);
    __syncwarp();
    rd[r] = (b + before) << 10 | static_cast<uint32_t>(d);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, the tile's count, then the
  // tile's runs (exclusive scan over digits)
  uint32_t cnt[kBinsPerThread];
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < kBinsPerThread; ++q) {
    const int d = t * kBinsPerThread + q;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = S.wcnt[w][d];
      S.wcnt[w][d] = run;
      run += c;
    }
    cnt[q] = run;
    s += run;
  }
  {
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.part[wid] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += S.part[w];
    uint32_t off = before + x - s;
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      S.toff[t * kBinsPerThread + q] = off;
      off += cnt[q];
    }
  }
  __syncthreads();
  // the tile reordered by digit in shared memory (every position read before
  // the first store: the compiler cannot tell the arrays apart)
  uint32_t pos[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int d = static_cast<int>(rd[r] & 1023u);
    pos[r] = d < kBins ? S.toff[d] + S.wcnt[wid][d] + (rd[r] >> 10) : kTile;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r)
    if (pos[r] < kTile) {
      S.key[pos[r]] = k[r];
      S.val[pos[r]] = v[r];
    }
  __syncthreads();
  // each digit's run to its place
  const int nin = base < n ? static_cast<int>(min(static_cast<size_t>(kTile), n - base)) : 0;
#pragma unroll 4
  for (int i = t; i < nin; i += kThreads) {
    const uint64_t key = S.key[i];
    const int d = static_cast<int>((key >> shift) & mask);
    const uint32_t p = S.gpos[d] + static_cast<uint32_t>(i) - S.toff[d];
    kout[p] = key;
    vout[p] = S.val[i];
  }
}

}  // namespace

// totals [8][512], then the tile counts [512][tiles] of one pass
size_t radix_tmp_words(size_t n) {
  return static_cast<size_t>(kMaxPasses) * kBins +
         static_cast<size_t>(kBins) * tiles_of(n < 1 ? 1 : n);
}

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      size_t n, int bits, uint32_t* tmp, bool* result_in_alt, cudaStream_t s,
                      const uint32_t* n_dev, unsigned* err) {
  (void)err;  // no kernel of this sort waits on another
  *result_in_alt = false;
  if (n <= 1 || bits <= 0) return;
  const Plan P = plan_of(bits);
  const int nt = static_cast<int>(tiles_of(n));
  uint32_t* totals = tmp;
  uint32_t* hist = tmp + kMaxPasses * kBins;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(sort_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(ScatterSmem)));
    configured = true;
  }
  uint64_t *kin = keys, *kout = keys_alt;
  uint32_t *vin = vals, *vout = vals_alt;
  bool alt = false;
  for (int p = 0; p < P.passes; ++p) {
    const int shift = p * P.width;
    sort_count_kernel<<<nt, kThreads, 0, s>>>(kin, n, n_dev, shift, P.width, hist, nt);
    sort_offsets_kernel<<<kBins, kThreads, 0, s>>>(hist, totals + p * kBins, nt);
    sort_scatter_kernel<<<nt, kThreads, sizeof(ScatterSmem), s>>>(
        kin, vin, kout, vout, n, n_dev, shift, P.width, hist, totals + p * kBins, nt);
    note_launches(3);
    std::swap(kin, kout);
    std::swap(vin, vout);
    alt = !alt;
  }
  *result_in_alt = alt;
}

}  // namespace rxgs
