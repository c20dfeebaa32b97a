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
#pragma once
#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

template <int NB>
struct FwdShape {
  static constexpr int CG = NB / 8;               // column groups (8 columns each)
  static constexpr int PG = kTilePixels / CG;     // pixel groups
  static constexpr int PX = kTilePixels / PG;     // pixels per thread (= NB/8)
  static constexpr size_t smem = sizeof(float) * (kChunk * kTilePixels + kChunk * NB) +
                                 sizeof(float4) * 2 * kChunk;
};

// One (view, tile, column block) of the compositing.  The column block
// covers columns [col0, col0 + NB) of a view whose ncols_v columns start at
// col_base in every radiance row; its receivers are out_rx0, out_rx0 + 1, ...
// in the spectra output, and its per-tile column sums go to partial_row.
struct TileJob {
  int v, tile, col0, col_base, ncols_v, out_rx0;
  float* partial_row;
};

template <int NB>
__device__ __forceinline__ void render_tile(const RenderArgs& a, const TileJob& job, float* sA,
                                            float* sR, float4* sRec, float (*sRed)[8]) {
  using S = FwdShape<NB>;
  const GridConst& g = a.g;
  const int t = threadIdx.x;
  const int tile = job.tile, v = job.v;
  const int col0 = job.col0;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const float* radv = a.rad + job.col_base;

  const int pg = t % S::PG, cg = t / S::PG;
  float acc[S::PX][8];
#pragma unroll
  for (int p = 0; p < S::PX; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[p][c] = 0.0f;

  float T = 1.0f;
  bool alive = valid;
  int ncon = 0;
  for (uint32_t start = rg.x; start < rg.y; start += kChunk) {
    const int nb = min(kChunk, static_cast<int>(rg.y - start));
    __syncthreads();
    if (t < kChunk) {
      const bool ok = t < nb;
      const uint32_t k = ok ? a.vals[start + t] : 0u;
      // geometry record (2 x 16 B) and the NB-column radiance slice of row k
      cp_async16(&sRec[2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&sRec[2 * t + 1], &rec[2 * k + 1], ok);
    }
    cp_async_commit();
    {
      constexpr int Q = NB / 4;  // float4 per row slice
      for (int e = t; e < kChunk * Q; e += kTilePixels) {
        const int b = e / Q, q4 = e % Q;
        const bool ok = b < nb;
        const uint32_t k = ok ? __ldg(&a.vals[start + b]) : 0u;
        cp_async16(&sR[b * NB + 4 * q4], radv + static_cast<size_t>(k) * a.stride + col0 + 4 * q4,
                   ok);
      }
    }
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // records landed
    __syncthreads();
    // ---- phase A: transmittance-weighted alphas, one pixel per thread
    for (int b = 0; b < nb; ++b) {
      float Tw = 0.0f;
      if (alive) {
        float w, G;
        if (pixel_weight(g, sRec[2 * b], sRec[2 * b + 1], i, jj, fi, fj, &w, &G)) {
          Tw = __fmul_rn(T, w);
          T = __fmul_rn(T, __fsub_rn(1.0f, w));
          ++ncon;
          if (T < g.eps_T) alive = false;
        }
      }
      sA[b * kTilePixels + t] = Tw;
    }
    cp_async_wait_all();
    const int n_alive = __syncthreads_count(alive);
    // ---- phase B: acc[p][c] += A[b][p] * s[b][c], skipping (Gaussian,
    // pixel strip) pairs that are zero for the whole warp: most list entries
    // cover only part of a tile, and stopped pixels contribute nothing.
    for (int b = 0; b < nb; ++b) {
      float av[S::PX];
      unsigned act = 0;  // warp-uniform: strips with a non-zero weight
#pragma unroll
      for (int p = 0; p < S::PX; ++p) {
        av[p] = sA[b * kTilePixels + p * S::PG + pg];
        act |= __any_sync(0xffffffffu, av[p] != 0.0f) ? (1u << p) : 0u;
      }
      if (act == 0) continue;
      const float4 b0 = *reinterpret_cast<const float4*>(&sR[b * NB + cg * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sR[b * NB + cg * 8 + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int p = 0; p < S::PX; ++p)
        if (act & (1u << p)) {
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[p][c] = fmaf(av[p], bv[c], acc[p][c]);
        }
    }
    if (n_alive == 0) break;
  }

  // ---- epilogue
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  if (col0 == 0 && valid) {
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
