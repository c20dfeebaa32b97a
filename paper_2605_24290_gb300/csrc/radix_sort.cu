// radix_sort.cu -- stable LSD radix sort of (uint64 or uint32 key, uint32
// value) pairs, used for the per-tile depth-sorted lists (Algorithm 1,
// Stage 1): every view's Gaussians by depth (one segment of K per view, the
// 31-bit depth keys less a bias, 9-bit digits), then the instances emitted
// in that order, in one pass by tile within each view's contiguous run
// (variable segments; the pass also writes each (view, tile) range); with
// more than 512 tiles the instances take the plain sort of (view | tile)
// keys.  Stability keeps equal keys in input order.
//
// Segments: nseg runs of `len` consecutive items (or variable runs), each
// sorted in place on its own (nseg = 1: a plain sort).  Digits of up to 9
// bits (ceil(bits / 9) passes).  One pass = three kernels over tiles of
// 2,048 items, no tile crossing a segment boundary:
//   sort_count    each tile's digit counts (shared-memory histogram);
//   sort_offsets  per (segment, digit): where each tile's run of that digit
//                 starts within the digit (exclusive scan over the
//                 segment's tiles), and the digit's total;
//   sort_scatter  adds the digit bases (an exclusive scan of the segment's
//                 totals in each block; no global atomics anywhere in the
//                 pass), ranks the tile's items stably (warp match-any,
//                 per-warp digit counters in shared memory), reorders the
//                 tile by digit in shared memory and writes each digit's
//                 run to its place, consecutive threads on consecutive
//                 addresses.
// Every tile's loads are issued before any of its ranks is computed.  The
// first pass may read a key array it does not own and no values (each
// item's value is then its index).
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
constexpr int kWarpRowMax = 256;            // tiles per segment scanned by one warp

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

// The segments of one sort: tile b is tile b % tps of segment b / tps.
struct Segs {
  size_t len;  // items per segment
  int nseg;    // segments
  int tps;     // tiles per segment
};

// Items [lo, hi) of tile b (hi <= lo: none); n: the items in all.
struct TileSpan {
  size_t lo, hi;
  int seg, tt;
};
__device__ __forceinline__ TileSpan tile_span(const Segs& S, size_t n) {
  TileSpan t;
  t.seg = static_cast<int>(blockIdx.x / S.tps);
  t.tt = static_cast<int>(blockIdx.x % S.tps);
  const size_t s0 = static_cast<size_t>(t.seg) * S.len;
  t.lo = s0 + static_cast<size_t>(t.tt) * kTile;
  t.hi = min(min(t.lo + kTile, s0 + S.len), n);
  return t;
}

// Variable segments (the instances of each view, one pass by tile):
// segment m holds items [start[m], start[m + 1]) in tiles [tile0[m],
// tile0[m + 1]); tile b belongs to segment tile_seg[b] (nseg: none, no
// items).  Tile counts are laid out [digit][nt]; each segment's first tile
// writes the segment's per-digit [start, end) into ranges[m][T].
struct VarSegs {
  const uint32_t* start;     // [nseg + 1]
  const uint32_t* tile0;     // [nseg + 1]
  const uint32_t* tile_seg;  // [nt]
  int nseg, nt, T;
  uint2* ranges;
};

__device__ __forceinline__ TileSpan var_span(const VarSegs& V) {
  TileSpan t;
  const uint32_t m = V.tile_seg[blockIdx.x];
  t.seg = static_cast<int>(m);
  t.tt = 0;
  t.lo = t.hi = 0;
  if (m < static_cast<uint32_t>(V.nseg)) {
    t.tt = static_cast<int>(blockIdx.x - V.tile0[m]);
    t.lo = V.start[m] + static_cast<size_t>(t.tt) * kTile;
    t.hi = min(t.lo + kTile, static_cast<size_t>(V.start[m + 1]));
  }
  return t;
}

// hist[(seg * kBins + d) * tps + tt] = count of digit d in tile tt of seg
// (kVar: hist[d * nt + tile])
template <typename Key, bool kVar>
__global__ void __launch_bounds__(kThreads) sort_count_kernel(const Key* __restrict__ keys,
                                                              size_t n,
                                                              const uint32_t* __restrict__ n_dev,
                                                              int shift, int width, Key bias,
                                                              uint32_t* __restrict__ hist, Segs S,
                                                              VarSegs V) {
  if (n_dev && *n_dev < n) n = *n_dev;
  __shared__ uint32_t h[kBins];
  for (int d = threadIdx.x; d < kBins; d += kThreads) h[d] = 0;
  TileSpan ts;
  if constexpr (kVar)
    ts = var_span(V);
  else
    ts = tile_span(S, n);
  Key k[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = ts.lo + static_cast<size_t>(r) * kThreads + threadIdx.x;
    k[r] = i < ts.hi ? keys[i] : 0;
  }
  __syncthreads();
  const Key mask = (Key(1) << width) - 1;
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = ts.lo + static_cast<size_t>(r) * kThreads + threadIdx.x;
    if (i < ts.hi) atomicAdd(&h[((k[r] - bias) >> shift) & mask], 1u);
  }
  __syncthreads();
  if constexpr (kVar) {
    for (int d = threadIdx.x; d < kBins; d += kThreads)
      hist[static_cast<size_t>(d) * V.nt + blockIdx.x] = h[d];
  } else {
    uint32_t* row = hist + static_cast<size_t>(ts.seg) * kBins * S.tps + ts.tt;
    for (int d = threadIdx.x; d < kBins; d += kThreads) row[static_cast<size_t>(d) * S.tps] = h[d];
  }
}

// Row r = (seg, digit) of hist (tps entries): each entry <- the exclusive
// sum of the entries before it (the tile's run start within the digit),
// totals[r] = the row's sum; the digit bases (exclusive sums of a segment's
// totals) are added by the scatter.  One block per row ...
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

// ... or one warp per row when rows are short (nt <= kWarpRowMax): lane l
// takes entries [l per, (l + 1) per), all loads in flight at once.
__global__ void __launch_bounds__(kThreads) sort_offsets_warp_kernel(uint32_t* __restrict__ hist,
                                                                     uint32_t* __restrict__ totals,
                                                                     int nt, int rows) {
  constexpr int kPer = kWarpRowMax / 32;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (r >= rows) return;  // whole warps leave together
  uint32_t* row = hist + static_cast<size_t>(r) * nt;
  const int per = (nt + 31) / 32;
  uint32_t v[kPer];
  uint32_t sum = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = lane * per + q;
    v[q] = (q < per && i < nt) ? row[i] : 0u;
    sum += v[q];
  }
  uint32_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  uint32_t run = x - sum;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = lane * per + q;
    if (q < per && i < nt) row[i] = run;
    run += v[q];
  }
  if (lane == 31) totals[r] = x;
}

template <typename Key>
struct ScatterSmem {
  Key key[kTile];
  uint32_t val[kTile];
  uint32_t wcnt[kWarps][kBins];  // per-warp digit counts, then where each warp's
                                 // items of the digit start in the reordered tile
  uint32_t gpos[kBins];          // the digit run's output position, then that
                                 // minus the run's start in the reordered tile
  uint32_t part[kWarps];
};

template <typename Key, bool kVar>
__global__ void __launch_bounds__(kThreads) sort_scatter_kernel(
    const Key* __restrict__ kin, const uint32_t* __restrict__ vin, Key* __restrict__ kout,
    uint32_t* __restrict__ vout, size_t n, const uint32_t* __restrict__ n_dev, int shift, int width,
    Key bias, const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ totals, Segs G,
    const uint32_t* __restrict__ gsrc, uint32_t* __restrict__ gdst, VarSegs V) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ScatterSmem<Key>& S = *reinterpret_cast<ScatterSmem<Key>*>(smraw);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (n_dev && *n_dev < n) n = *n_dev;
  TileSpan ts;
  if constexpr (kVar) {
    ts = var_span(V);
    if (ts.seg >= V.nseg) return;  // a tile past the last segment: no items
  } else {
    ts = tile_span(G, n);
  }
  const size_t base = ts.lo;
  const uint32_t mask = (1u << width) - 1;
  // warp w takes items [base + 256 w, base + 256 (w + 1)), 32 per round;
  // every load in flight before the first rank
  Key k[kItems];
  uint32_t v[kItems], rd[kItems];  // rank in the warp's run << 10 | digit (kBins = none)
  unsigned peers[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(wid) * (32 * kItems) + r * 32 + lane;
    k[r] = i < ts.hi ? kin[i] : 0;
    v[r] = i < ts.hi ? (vin ? vin[i] : static_cast<uint32_t>(i)) : 0;
  }
  for (int e = t; e < kWarps * kBins; e += kThreads) (&S.wcnt[0][0])[e] = 0;
  {
    // where each digit's run of this tile starts in the output: the
    // segment's start, the digit's base in it (exclusive sum of the
    // segment's digit totals) and the tile's offset in the digit
    uint32_t tv[kBinsPerThread], tofs[kBinsPerThread], tsum = 0, seg0;
    if constexpr (kVar) {
      // E(d, x): the exclusive sum of digit d's counts over tiles < x
      auto E = [&](int d, uint32_t x) {
        return x < static_cast<uint32_t>(V.nt) ? offsets[static_cast<size_t>(d) * V.nt + x]
                                               : totals[d];
      };
      const uint32_t p0 = V.tile0[ts.seg], p1 = V.tile0[ts.seg + 1];
#pragma unroll
      for (int q = 0; q < kBinsPerThread; ++q) {
        const int d = t * kBinsPerThread + q;
        const uint32_t a = E(d, p0);
        tv[q] = E(d, p1) - a;
        tofs[q] = E(d, blockIdx.x) - a;
        tsum += tv[q];
      }
      seg0 = V.start[ts.seg];
    } else {
      const uint32_t* segtot = totals + static_cast<size_t>(ts.seg) * kBins;
      const uint32_t* tofsp = offsets + static_cast<size_t>(ts.seg) * kBins * G.tps + ts.tt;
#pragma unroll
      for (int q = 0; q < kBinsPerThread; ++q) {
        const int d = t * kBinsPerThread + q;
        tv[q] = segtot[d];
        tofs[q] = tofsp[static_cast<size_t>(d) * G.tps];
        tsum += tv[q];
      }
      seg0 = static_cast<uint32_t>(static_cast<size_t>(ts.seg) * G.len);
    }
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) S.part[wid] = x;
    __syncthreads();
    uint32_t b = x - tsum + seg0;
    for (int w = 0; w < wid; ++w) b += S.part[w];
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      const int d = t * kBinsPerThread + q;
      S.gpos[d] = tofs[q] + b;
      if constexpr (kVar) {
        // the segment's first tile: each digit's [start, end) in the output
        if (ts.tt == 0 && d < V.T && tv[q] > 0)
          V.ranges[static_cast<size_t>(ts.seg) * V.T + d] = make_uint2(b, b + tv[q]);
      }
      b += tv[q];
    }
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const size_t i = base + static_cast<size_t>(wid) * (32 * kItems) + r * 32 + lane;
    const int d = i < ts.hi ? static_cast<int>(((k[r] - bias) >> shift) & mask) : kBins;
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
    uint32_t off = before + x - s;  // the run's start in the reordered tile
#pragma unroll
    for (int q = 0; q < kBinsPerThread; ++q) {
      const int d = t * kBinsPerThread + q;
      S.gpos[d] -= off;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) S.wcnt[w][d] += off;
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
    pos[r] = d < kBins ? S.wcnt[wid][d] + (rd[r] >> 10) : kTile;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r)
    if (pos[r] < kTile) {
      S.key[pos[r]] = k[r];
      S.val[pos[r]] = v[r];
    }
  __syncthreads();
  // each digit's run to its place
  const int nin = ts.hi > ts.lo ? static_cast<int>(ts.hi - ts.lo) : 0;
#pragma unroll 4
  for (int i = t; i < nin; i += kThreads) {
    const Key key = S.key[i];
    const int d = static_cast<int>(((key - bias) >> shift) & mask);
    const uint32_t p = S.gpos[d] + static_cast<uint32_t>(i);
    const uint32_t val = S.val[i];
    if (kout) kout[p] = key;  // null: the keys are not needed after this pass
    vout[p] = val;
    if (gdst) gdst[p] = gsrc[val];
  }
}


// The view segments of the emitted instances: start[m] = offsets[m K]
// (the emission is view-major) clamped to n (a capacity the emission did not
// write past), tile0 = exclusive scan of the segments' tile counts,
// tile_seg[b] for b < nt.  One block.
__global__ void __launch_bounds__(1024) var_segs_kernel(const uint32_t* __restrict__ offsets, int K,
                                                       int M, int nt, uint32_t n,
                                                       uint32_t* __restrict__ start,
                                                       uint32_t* __restrict__ tile0,
                                                       uint32_t* __restrict__ tile_seg) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 <= M; c0 += 1024) {
    const int m = c0 + t;
    uint32_t cnt = 0;
    if (m <= M) {
      const uint32_t s0 = min(offsets[static_cast<size_t>(m) * K], n);
      start[m] = s0;
      if (m < M) {
        const uint32_t s1 = min(offsets[static_cast<size_t>(m + 1) * K], n);
        cnt = (s1 - s0 + kTile - 1) / kTile;
      }
    }
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    uint32_t before = carry;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    if (m <= M) tile0[m] = before + x - cnt;
    __syncthreads();
    if (t == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < 32; ++w) tot += wsum[w];
      carry += tot;
    }
    __syncthreads();
  }
  // tile b -> the last segment m with tile0[m] <= b (tiles of empty
  // segments are skipped by the search); M past the end
  const uint32_t used = __ldcg(&tile0[M]);  // written by this block (L2)
  for (int b = t; b < nt; b += 1024) {
    uint32_t m = static_cast<uint32_t>(M);
    if (static_cast<uint32_t>(b) < used) {
      int lo = 0, hi = M - 1;  // tile0[lo] <= b < tile0[hi + 1]
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldcg(&tile0[mid]) <= static_cast<uint32_t>(b)) lo = mid;
        else hi = mid - 1;
      }
      m = static_cast<uint32_t>(lo);
    }
    tile_seg[b] = m;
  }
}

size_t tmp_words(const Segs& G) {
  return static_cast<size_t>(G.nseg) * kBins * (1 + static_cast<size_t>(G.tps));
}

// The passes: pass 0 reads (k0, v0) (v0 null: values = indices), pass p
// writes buffer p % 2.  Returns the buffer holding the result, -1 if no
// pass ran.  tmp: the digit totals [nseg][512], then the tile counts
// [nseg][512][tps].
template <typename Key>
int run_passes(const Key* k0, const uint32_t* v0, Key* const (&kb)[2], uint32_t* const (&vb)[2],
               size_t n, const Segs& G, int pfirst, int pend, int width, uint32_t* tmp,
               cudaStream_t s, const uint32_t* n_dev, Key bias = 0,
               const uint32_t* gsrc = nullptr, uint32_t* gdst = nullptr) {
  if (n == 0 || pend <= pfirst) return -1;
  const int nt = G.nseg * G.tps;
  const int rows = G.nseg * kBins;
  uint32_t* totals = tmp;
  uint32_t* hist = tmp + rows;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(sort_scatter_kernel<Key, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(ScatterSmem<Key>)));
    cudaFuncSetAttribute(sort_scatter_kernel<Key, false>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    configured = true;
  }
  const Key* kin = k0;
  const uint32_t* vin = v0;
  int out = 0;
  for (int p = pfirst; p < pend; ++p) {
    out = p & 1;
    const int shift = p * width;
    sort_count_kernel<Key, false><<<nt, kThreads, 0, s>>>(kin, n, n_dev, shift, width, bias,
                                                          hist, G, VarSegs{});
    if (G.tps <= kWarpRowMax)
      sort_offsets_warp_kernel<<<(rows + kWarps - 1) / kWarps, kThreads, 0, s>>>(hist, totals,
                                                                                G.tps, rows);
    else
      sort_offsets_kernel<<<rows, kThreads, 0, s>>>(hist, totals, G.tps);
    const bool last = p + 1 == pend;
    sort_scatter_kernel<Key, false><<<nt, kThreads, sizeof(ScatterSmem<Key>), s>>>(
        kin, vin, last && gdst ? nullptr : kb[out], vb[out], n, n_dev, shift, width, bias, hist,
        totals, G, last ? gsrc : nullptr, last ? gdst : nullptr, VarSegs{});
    note_launches(3);
    kin = kb[out];
    vin = vb[out];
  }
  return out;
}

Segs whole(size_t n) {
  Segs G;
  G.len = n < 1 ? 1 : n;
  G.nseg = 1;
  G.tps = static_cast<int>(tiles_of(G.len));
  return G;
}

Segs segments(size_t len, int nseg) {
  Segs G;
  G.len = len < 1 ? 1 : len;
  G.nseg = nseg < 1 ? 1 : nseg;
  G.tps = static_cast<int>(tiles_of(G.len));
  return G;
}

template <typename Key>
void sort_pairs(Key* keys, uint32_t* vals, Key* keys_alt, uint32_t* vals_alt, size_t n, int bits,
                uint32_t* tmp, bool* result_in_alt, cudaStream_t s, const uint32_t* n_dev) {
  *result_in_alt = false;
  if (n <= 1) return;
  Key* const kb[2] = {keys_alt, keys};
  uint32_t* const vb[2] = {vals_alt, vals};
  if (bits <= 0) return;
  const Plan P = plan_of(bits);
  const int out = run_passes<Key>(keys, vals, kb, vb, n, whole(n), 0, P.passes, P.width, tmp, s,
                                  n_dev);
  *result_in_alt = out == 0;
}

}  // namespace

size_t radix_tmp_words(size_t n) { return tmp_words(whole(n)); }

size_t radix_segments_tmp_words(size_t len, int nseg) { return tmp_words(segments(len, nseg)); }

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                      size_t n, int bits, uint32_t* tmp, bool* result_in_alt, cudaStream_t s,
                      const uint32_t* n_dev, unsigned* err) {
  (void)err;  // no kernel of this sort waits on another
  if (bits > 32) bits = 32;
  sort_pairs<uint32_t>(keys, vals, keys_alt, vals_alt, n, bits, tmp, result_in_alt, s, n_dev);
}

void radix_sort_segments_first(const uint32_t* keys, size_t len, int nseg, uint32_t* keys_a,
                               uint32_t* idx_a, uint32_t* tmp, cudaStream_t s) {
  const Segs G = segments(len, nseg);
  uint32_t* const kb[2] = {keys_a, keys_a};
  uint32_t* const vb[2] = {idx_a, idx_a};
  run_passes<uint32_t>(keys, nullptr, kb, vb, len * static_cast<size_t>(nseg), G, 0, 1, kMaxWidth,
                       tmp, s, nullptr);
}

const uint32_t* radix_sort_segments_rest(size_t len, int nseg, int bits, uint32_t bias,
                                         uint32_t* keys_a, uint32_t* keys_b, uint32_t* idx_a,
                                         uint32_t* idx_b, uint32_t* tmp,
                                         const uint32_t* gather_src, uint32_t* gather_dst,
                                         cudaStream_t s) {
  const size_t n = len * static_cast<size_t>(nseg);
  if (n == 0) return nullptr;
  if (bits > 32) bits = 32;
  const int passes = bits > kMaxWidth ? (bits + kMaxWidth - 1) / kMaxWidth : 1;
  const bool gather = gather_src && gather_dst;
  if (passes == 1) {  // pass 0 was the whole sort
    if (gather) launch_gather_words(gather_src, idx_a, n, gather_dst, s);
    return idx_a;
  }
  const Segs G = segments(len, nseg);
  // pass p writes buffer p % 2: pass 0 wrote keys_a / idx_a, pass 1 reads
  // them and writes keys_b / idx_b, ...
  uint32_t* const kb[2] = {keys_a, keys_b};
  uint32_t* const vb[2] = {idx_a, idx_b};
  const int out = run_passes<uint32_t>(keys_a, idx_a, kb, vb, n, G, 1, passes, kMaxWidth, tmp, s,
                                       nullptr, bias, gather ? gather_src : nullptr,
                                       gather ? gather_dst : nullptr);
  return vb[out];
}

size_t radix_views_tmp_words(size_t n, int M) {
  const size_t nt = tiles_of(n) + static_cast<size_t>(M);
  return static_cast<size_t>(kBins) * (1 + nt) + 2 * (static_cast<size_t>(M) + 1) + nt;
}

void radix_sort_views(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out,
                      uint32_t* vals_out, size_t n, const uint32_t* offsets, int K, int M,
                      int tile_bits, uint2* ranges, int T, uint32_t* tmp, cudaStream_t s) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * static_cast<size_t>(M) * T, s);
  if (n == 0 || M <= 0) return;
  const int nt = static_cast<int>(tiles_of(n) + static_cast<size_t>(M));
  uint32_t* totals = tmp;
  uint32_t* hist = totals + kBins;
  uint32_t* start = hist + static_cast<size_t>(kBins) * nt;
  uint32_t* tile0 = start + (M + 1);
  uint32_t* tile_seg = tile0 + (M + 1);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(sort_scatter_kernel<uint32_t, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(sizeof(ScatterSmem<uint32_t>)));
    cudaFuncSetAttribute(sort_scatter_kernel<uint32_t, true>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    configured = true;
  }
  VarSegs V;
  V.start = start;
  V.tile0 = tile0;
  V.tile_seg = tile_seg;
  V.nseg = M;
  V.nt = nt;
  V.T = T;
  V.ranges = ranges;
  var_segs_kernel<<<1, 1024, 0, s>>>(offsets, K, M, nt, static_cast<uint32_t>(n), start, tile0,
                                     tile_seg);
  const Segs G = whole(n);
  sort_count_kernel<uint32_t, true><<<nt, kThreads, 0, s>>>(keys, n, nullptr, 0, tile_bits, 0u,
                                                            hist, G, V);
  if (nt <= kWarpRowMax)
    sort_offsets_warp_kernel<<<(kBins + kWarps - 1) / kWarps, kThreads, 0, s>>>(hist, totals, nt,
                                                                               kBins);
  else
    sort_offsets_kernel<<<kBins, kThreads, 0, s>>>(hist, totals, nt);
  sort_scatter_kernel<uint32_t, true><<<nt, kThreads, sizeof(ScatterSmem<uint32_t>), s>>>(
      keys, vals, keys_out, vals_out, n, nullptr, 0, tile_bits, 0u, hist, totals, G, nullptr,
      nullptr, V);
  note_launches(4);
}

}  // namespace rxgs
