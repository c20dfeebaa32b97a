// render_tile.cuh -- the compositing of one (view, tile, column block),
// shared by the per-call forward kernel and the persistent batched kernel.
//
// One CTA renders one 256-pixel tile of one view for a block of NB output
// columns (column = receiver j, channel c, real/imag), so every receiver of
// a view shares the tile's sorted list and the per-pixel weights.  The tile
// list is consumed in chunks of 32 Gaussians:
//   phase A  one thread per pixel walks the chunk in depth order and writes
//            A[b][pixel] = T_b w_b (zero when the Gaussian misses the pixel,
//            fails q <= q_max, or the pixel already stopped); the receiver-
//            independent part of the work is done once per tile;
//   phase B  the chunk's contribution to all NB columns is the small dense
//            product  acc[pixel][col] += sum_b A[b][pixel] * s[b][col],
//            register-tiled (NB/8 pixels x 8 columns per thread).
// The radiance rows of the chunk are copied with cp.async while phase A
// runs.  The tile stops as soon as every pixel has T < eps.
//
// With TPP = 2 the CTA has 512 threads, two per pixel (lanes l and l + 16
// of a warp; a warp covers a 16-pixel strip): in phase A the two threads of
// a pixel evaluate the weights of alternate marked Gaussians, exchange them
// by shuffles and both apply the (cheap, sequential) transmittance updates,
// so a wide column block costs one weight evaluation per (pixel, Gaussian).
#pragma once
#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

template <int NB, int TPP = 1>
struct FwdShape {
  static constexpr int kThreads = TPP * kTilePixels;
  static constexpr int SP = 32 / TPP;             // pixels per warp strip
  static constexpr int CG = NB / 8;               // column groups (8 columns each)
  static constexpr int PG = kThreads / CG;        // pixel groups
  static constexpr int PX = kTilePixels / PG;     // pixels per thread
  static constexpr size_t smem = sizeof(float) * (kChunk * kTilePixels + 2 * kChunk * NB) +
                                 sizeof(float4) * 2 * 2 * kChunk;
};

// One (view, tile, column block) of the compositing.  The column block
// covers columns [col0, col0 + NB) of a view whose ncols_v columns start at
// col_base in every radiance row; its receivers are out_rx0, out_rx0 + 1, ...
// in the spectra output, and its per-tile column sums go to partial_row.
struct TileJob {
  int v, tile, col0, col_base, ncols_v, out_rx0;
  float* partial_row;
};

template <int NB, int TPP = 1>
__device__ __forceinline__ void render_tile(const RenderArgs& a, const TileJob& job, float* sA,
                                            float* sR, float4* sRec, float (*sRed)[8]) {
  using S = FwdShape<NB, TPP>;
  const GridConst& g = a.g;
  const int t = threadIdx.x;
  const int lane = t & 31, wp = t >> 5;
  const int h = TPP == 2 ? lane >> 4 : 0;              // which thread of the pixel
  const int px = TPP == 2 ? wp * 16 + (lane & 15) : t;  // this thread's pixel
  const int tile = job.tile, v = job.v;
  const int col0 = job.col0;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + px / g.TW, jj = tc * g.TW + px % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const float* radv = a.rad + job.col_base + static_cast<size_t>(v) * a.rad_view;
  __shared__ unsigned sMask[S::kThreads / 32];  // per warp: chunk entries meeting its strip

  const int pg = t % S::PG, cg = t / S::PG;
  float acc[S::PX][8];
#pragma unroll
  for (int p = 0; p < S::PX; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[p][c] = 0.0f;

  float T = 1.0f;
  bool alive = valid;
  int ncon = 0;
  // Chunks go through a copy pipeline: while chunk n is composited, the
  // records and radiance rows of chunk n + 1 (gathered with indices already
  // in shared memory) and the list indices of chunk n + 2 are in flight
  // (cp.async), so no thread waits on a global load at a chunk boundary.
  __shared__ uint32_t sIdx[3 * kChunk];  // list indices of chunks n, n+1, n+2
  const int nchunks = static_cast<int>((rg.y - rg.x + kChunk - 1) / kChunk);
  auto chunk_len = [&](int n) {
    return min(kChunk, static_cast<int>(rg.y - rg.x - static_cast<uint32_t>(n) * kChunk));
  };
  auto copy_indices = [&](int n) {
    const bool ok = t < chunk_len(n);
    if (t < kChunk)
      cp_async4(&sIdx[(n % 3) * kChunk + t], ok ? &a.vals[rg.x + n * kChunk + t] : a.vals, ok);
  };
  auto gather = [&](int n) {
    const int nbn = chunk_len(n);
    const uint32_t* ks = sIdx + (n % 3) * kChunk;
    float4* rb = sRec + (n & 1) * 2 * kChunk;
    float* rr = sR + (n & 1) * kChunk * NB;
    if (t < kChunk) {
      const bool ok = t < nbn;
      const uint32_t k = ok ? ks[t] : 0u;
      // geometry record (2 x 16 B) and the NB-column radiance slice of row k
      cp_async16(&rb[2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&rb[2 * t + 1], &rec[2 * k + 1], ok);
    }
    constexpr int Q = NB / 4;  // float4 per row slice
    for (int e = t; e < kChunk * Q; e += S::kThreads) {
      const int b = e / Q, q4 = e % Q;
      const bool ok = b < nbn;
      const uint32_t k = ok ? ks[b] : 0u;
      cp_async16(&rr[b * NB + 4 * q4], radv + static_cast<size_t>(k) * a.stride + col0 + 4 * q4,
                 ok);
    }
  };
  if (nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // indices of chunk 0
    __syncthreads();
    gather(0);
    cp_async_commit();
  }
  for (int n = 0; n < nchunks; ++n) {
    const int nb = chunk_len(n);
    cp_async_wait_all();  // chunk n's records and rows, chunk n + 1's indices
    __syncthreads();      // ... visible to all; everyone is done with chunk n - 1
    if (n + 1 < nchunks) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      gather(n + 1);
    }
    cp_async_commit();
    const float4* sRecC = sRec + (n & 1) * 2 * kChunk;
    const float* sRC = sR + (n & 1) * kChunk * NB;
    // ---- phase A: transmittance-weighted alphas, one pixel per thread.
    // Each warp first marks the chunk's Gaussians whose footprint meets its
    // pixel strip (one Gaussian per lane, then a ballot) and walks only
    // those, two at a time: their weights are independent, only the T
    // updates are sequential, in list order.
    if (TPP == 1) {
      const Strip strip = warp_strip(g, tr, tc, wp);
      const bool rel = lane < nb && touches_strip(g, sRecC[2 * lane + 1], strip);
      const unsigned mask = __ballot_sync(0xffffffffu, rel);
      // walk the marked entries while some pixel of the strip is alive; the
      // stored mask keeps only entries that gave some pixel of the strip a
      // non-zero weight (phase B reads nothing else)
      unsigned m = __any_sync(0xffffffffu, alive) ? mask : 0u;
      unsigned used = 0;
      while (m) {
        const int b0 = __ffs(m) - 1;
        m &= m - 1;
        const int b1 = m ? __ffs(m) - 1 : -1;
        if (b1 >= 0) m &= m - 1;
        float w0 = 0.0f, w1 = 0.0f, G;
        bool c0 = false, c1 = false;
        if (alive) {
          c0 = pixel_weight(g, sRecC[2 * b0], sRecC[2 * b0 + 1], i, jj, fi, fj, &w0, &G);
          if (b1 >= 0) c1 = pixel_weight(g, sRecC[2 * b1], sRecC[2 * b1 + 1], i, jj, fi, fj, &w1, &G);
        }
        float Tw0 = 0.0f, Tw1 = 0.0f;
        if (alive && c0) {
          Tw0 = __fmul_rn(T, w0);
          T = __fmul_rn(T, __fsub_rn(1.0f, w0));
          ++ncon;
          if (T < g.eps_T) alive = false;
        }
        if (alive && c1) {
          Tw1 = __fmul_rn(T, w1);
          T = __fmul_rn(T, __fsub_rn(1.0f, w1));
          ++ncon;
          if (T < g.eps_T) alive = false;
        }
        sA[b0 * kTilePixels + t] = Tw0;
        if (b1 >= 0) sA[b1 * kTilePixels + t] = Tw1;
        if (__any_sync(0xffffffffu, Tw0 != 0.0f)) used |= 1u << b0;
        if (b1 >= 0 && __any_sync(0xffffffffu, Tw1 != 0.0f)) used |= 1u << b1;
      }
      if (lane == 0) sMask[wp] = used;
    } else {
      // two threads per pixel: the lower half of the warp evaluates b0, the
      // upper half b1; both apply the updates in list order
      const Strip strip = pixel_strip(g, tr, tc, wp * 16, 16);
      const bool rel = lane < nb && touches_strip(g, sRecC[2 * lane + 1], strip);
      const unsigned mask = __ballot_sync(0xffffffffu, rel);
      unsigned m = __any_sync(0xffffffffu, alive) ? mask : 0u;
      unsigned used = 0;
      const int src0 = lane & 15, src1 = src0 | 16;
      while (m) {
        const int b0 = __ffs(m) - 1;
        m &= m - 1;
        const int b1 = m ? __ffs(m) - 1 : -1;
        if (b1 >= 0) m &= m - 1;
        const int bm = h ? b1 : b0;
        float wm = 0.0f, G;
        bool cm = false;
        if (alive && bm >= 0) cm = pixel_weight(g, sRecC[2 * bm], sRecC[2 * bm + 1], i, jj, fi, fj, &wm, &G);
        const float w0 = __shfl_sync(0xffffffffu, wm, src0);
        const float w1 = __shfl_sync(0xffffffffu, wm, src1);
        const bool c0 = __shfl_sync(0xffffffffu, static_cast<int>(cm), src0) != 0;
        const bool c1 = __shfl_sync(0xffffffffu, static_cast<int>(cm), src1) != 0;
        float Tw0 = 0.0f, Tw1 = 0.0f;
        if (alive && c0) {
          Tw0 = __fmul_rn(T, w0);
          T = __fmul_rn(T, __fsub_rn(1.0f, w0));
          ++ncon;
          if (T < g.eps_T) alive = false;
        }
        if (alive && c1) {
          Tw1 = __fmul_rn(T, w1);
          T = __fmul_rn(T, __fsub_rn(1.0f, w1));
          ++ncon;
          if (T < g.eps_T) alive = false;
        }
        if (h == 0)
          sA[b0 * kTilePixels + px] = Tw0;
        else if (b1 >= 0)
          sA[b1 * kTilePixels + px] = Tw1;
        if (__any_sync(0xffffffffu, Tw0 != 0.0f)) used |= 1u << b0;
        if (b1 >= 0 && __any_sync(0xffffffffu, Tw1 != 0.0f)) used |= 1u << b1;
      }
      if (lane == 0) sMask[wp] = used;
    }
    const int n_alive = __syncthreads_count(alive);
    // ---- phase B: acc[p][c] += A[b][p] * s[b][c] over the (Gaussian, pixel
    // strip) pairs marked in phase A; pixel group p of this thread lies in
    // the strip(s) of warps [p*PG/SP, (p+1)*PG/SP) (SP pixels per strip).
    {
      // pmask: union over the warps of group p (uniform, for skipping);
      // own: the mask of the warp that wrote this thread's pixel of group p
      // (entries outside it were not written this chunk and weigh zero)
      unsigned pmask[S::PX], own[S::PX];
      unsigned any = 0;
#pragma unroll
      for (int p = 0; p < S::PX; ++p) {
        unsigned mm = 0;
        if (S::PG >= S::SP) {
#pragma unroll
          for (int q = 0; q < S::PG / S::SP; ++q) mm |= sMask[p * (S::PG / S::SP) + q];
        } else {
          mm = sMask[(p * S::PG) / S::SP];
        }
        pmask[p] = mm;
        own[p] = sMask[(p * S::PG + pg) / S::SP];
        any |= mm;
      }
      while (any) {
        const int b = __ffs(any) - 1;
        any &= any - 1;
        const float4 b0 = *reinterpret_cast<const float4*>(&sRC[b * NB + cg * 8]);
        const float4 b1 = *reinterpret_cast<const float4*>(&sRC[b * NB + cg * 8 + 4]);
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
        float av[S::PX];
#pragma unroll
        for (int p = 0; p < S::PX; ++p)
          av[p] = (own[p] & (1u << b)) ? sA[b * kTilePixels + p * S::PG + pg] : 0.0f;
#pragma unroll
        for (int p = 0; p < S::PX; ++p)
          if (pmask[p] & (1u << b)) {
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[p][c] = fmaf(av[p], bv[c], acc[p][c]);
          }
      }
    }
    if (n_alive == 0) {
      cp_async_wait_all();  // a prefetch may still be in flight
      break;
    }
  }

  // ---- epilogue
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  if (col0 == 0 && valid && h == 0) {
    const size_t o = static_cast<size_t>(v) * HW + static_cast<size_t>(i) * g.W + jj;
    if (a.ncontrib) a.ncontrib[o] = ncon;
    if (a.tfinal) a.tfinal[o] = T;
  }
  const int twoC = 2 * a.C;
  if (a.spectra) {
#pragma unroll
    for (int p = 0; p < S::PX; ++p) {
      const int pix = p * S::PG + pg;
      const int pi = tr * g.TH + pix / g.TW, pj = tc * g.TW + pix % g.TW;
      if (pi >= g.H || pj >= g.W) continue;
      const size_t po = static_cast<size_t>(pi) * g.W + pj;
#pragma unroll
      for (int c = 0; c < 8; c += 2) {
        const int col = col0 + cg * 8 + c;
        if (col >= job.ncols_v) continue;
        const int j = col / twoC, e = col - j * twoC;
        const size_t off = ((static_cast<size_t>(job.out_rx0) + j) * HW + po) * twoC + e;
        *reinterpret_cast<float2*>(&a.spectra[off]) = make_float2(acc[p][c], acc[p][c + 1]);
      }
    }
  }
  if (job.partial_row) {
    float s[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float x = 0.0f;
#pragma unroll
      for (int p = 0; p < S::PX; ++p) x += acc[p][c];
      s[c] = x;
    }
    constexpr int L = S::PG < 32 ? S::PG : 32;
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
    float* dst = job.partial_row;
    if (S::PG <= 32) {
      if (pg == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int col = col0 + cg * 8 + c;
          if (col < job.ncols_v) dst[col] = s[c];
        }
      }
    } else {
      constexpr int WPG = S::PG / 32;  // warps per column group
      const int w = t >> 5;
      if ((t & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) sRed[w][c] = s[c];
      }
      __syncthreads();
      if (t < S::CG * 8) {
        const int cgi = t / 8, c = t % 8;
        float x = 0.0f;
        for (int q = 0; q < WPG; ++q) x += sRed[cgi * WPG + q][c];
        const int col = col0 + cgi * 8 + c;
        if (col < job.ncols_v) dst[col] = x;
      }
    }
  }
}

}  // namespace rxgs
