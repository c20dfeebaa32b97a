// render_bwd.cu -- backward of the multi-receiver compositing (App. D: the
// backward kernel runs over the same (tile, receiver) grid and accumulates
// Gaussian-level gradients with atomicAdd).
//
// For one pixel with composited sequence k_1..k_n (weights w_m, transmittance
// T_m = prod_{l<m} (1 - w_l)) and cotangent g_c per output column c:
//   dL/ds_{k_m, c}  = T_m w_m g_c
//   dL/dw_m         = T_m (gamma_m - Q_m),   gamma_m = sum_c g_c s_{k_m, c}
//   Q_m             = sum_c g_c S_{m, c},  S_m the normalised colour behind m:
//                     Q_{m-1} = w_m gamma_m + (1 - w_m) Q_m,  Q_n = 0
//   dL/dtau_{k_m}   = exp(-q/2) dL/dw_m
// Q is a convex combination of the gammas, so the error of dL/dw_m scales
// with T_m like the value itself (a forward difference D - E_m would cancel
// catastrophically once T is small).
//
// Nothing is read from the forward: a pre-pass walks each tile's list once
// and recomputes every pixel's final T and stop position with the forward's
// float32 decisions (per-tile recomputation); then each (tile, column block)
// sweeps the list back to front, chunk by chunk, recovering
// T_m = T_{m+1} / (1 - w_m).  Both gradients are linear in
// the columns, so each CTA handles a block of 32 columns and the per-block
// contributions add up.
#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

// Walk 1, once per (view, tile): every pixel's final transmittance and the
// list position one past its last composited Gaussian (its stop), with the
// forward's float32 decisions; tile_stop = the largest stop of the tile.
__global__ void __launch_bounds__(kTilePixels) bwd_prepass_kernel(const RenderArgs a,
                                                                  float* __restrict__ tfin,
                                                                  uint32_t* __restrict__ stops,
                                                                  uint32_t* __restrict__ tile_stop) {
  __shared__ float4 sRec[2][2 * kChunk];
  __shared__ uint32_t sIdx[3 * kChunk];
  __shared__ unsigned sStop;
  const GridConst& g = a.g;
  const int t = threadIdx.x;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  if (t == 0) sStop = rg.x;
  const Strip strip = warp_strip(g, tr, tc, t >> 5);
  float T = 1.0f;
  uint32_t stop = valid ? rg.y : rg.x;
  bool alive = valid;
  // the same copy pipeline as the forward: records of chunk n + 1 and
  // indices of chunk n + 2 in flight while chunk n is walked
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
    if (t < kChunk) {
      const bool ok = t < chunk_len(n);
      const uint32_t k = ok ? sIdx[(n % 3) * kChunk + t] : 0u;
      cp_async16(&sRec[n & 1][2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&sRec[n & 1][2 * t + 1], &rec[2 * k + 1], ok);
    }
  };
  if (nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    gather(0);
    cp_async_commit();
  }
  for (int n = 0; n < nchunks; ++n) {
    const uint32_t start = rg.x + static_cast<uint32_t>(n) * kChunk;
    const int nb = chunk_len(n);
    cp_async_wait_all();
    __syncthreads();
    if (n + 1 < nchunks) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      gather(n + 1);
    }
    cp_async_commit();
    const float4* sR = sRec[n & 1];
    {
      const int lane = t & 31;
      const bool rel = lane < nb && touches_strip(g, sR[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      while (alive && m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        float w, G;
        if (pixel_weight(g, sR[2 * b], sR[2 * b + 1], i, jj, fi, fj, &w, &G)) {
          T = __fmul_rn(T, __fsub_rn(1.0f, w));
          if (T < g.eps_T) {
            alive = false;
            stop = start + b + 1;
          }
        }
      }
    }
    if (__syncthreads_count(alive) == 0) break;
  }
  cp_async_wait_all();  // a prefetch may still be in flight
  atomicMax(&sStop, stop);
  if (valid) {
    const size_t o = static_cast<size_t>(v) * g.H * g.W + static_cast<size_t>(i) * g.W + jj;
    tfin[o] = T;
    stops[o] = stop;
  }
  __syncthreads();
  if (t == 0) tile_stop[static_cast<size_t>(v) * g.T + tile] = sStop;
}

// Walk 2, one CTA of 512 threads per (view, tile, block of NB columns): two
// threads per pixel (lanes l and l + 16 of a warp; a warp covers 16 pixels).
// Per chunk of the list, back to front over the entries that meet the
// warp's 16-pixel strip, two entries b0 > b1 at a time:
//   - the lower half of the warp evaluates the weight of b0 and the upper
//     half that of b1 (exchanged by shuffles), so each (pixel, entry) weight
//     is computed once per NB columns;
//   - each half dots the pixel's cotangent with the radiance over its NB/2
//     columns for both entries; a shuffle adds the halves into gamma;
//   - both halves then run the same recurrence (T recovery, Q suffix);
//   - dL/dtau is summed over the warp's pixels by shuffles.
// Then dL/ds[b][c] = sum_p (T w)[b][p] g[p][c] is register-tiled over all
// 512 threads (4 entries x 8 columns per thread over a slice of the pixels).
template <int NB>
struct BwdShape {
  static constexpr int kThreads = 2 * kTilePixels;
  static constexpr int HC = NB / 2;                 // gamma columns per thread
  static constexpr int GS = NB + 4;                 // padded cotangent row (float4 aligned)
  static constexpr int PE = 2;                      // entries per product block
  static constexpr int PC = 16;                     // columns per product block
  static constexpr int CB = NB / PC;                // column groups in the product
  static constexpr int SL = kThreads / ((kChunk / PE) * CB);  // pixel slices in the product
  static constexpr int kWarps = kThreads / 32;
  // cotangent rows, T w, two radiance / record / index buffers, dtau sums
  static constexpr size_t smem =
      sizeof(float) * (kTilePixels * GS + kChunk * kTilePixels + 2 * kChunk * NB + kWarps * kChunk) +
      sizeof(float4) * 2 * 2 * kChunk + sizeof(uint32_t) * 3 * kChunk;
};

template <int NB>
__global__ void __launch_bounds__(2 * kTilePixels, 1) render_bwd_kernel(const BackwardArgs A) {
  using S = BwdShape<NB>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sG = reinterpret_cast<float*>(smem_raw);          // [256][GS] cotangent rows
  float* sA = sG + kTilePixels * S::GS;                     // [32][256] T w
  float* sR0 = sA + kChunk * kTilePixels;                   // [2][32][NB] radiance slices
  float* sTau = sR0 + 2 * kChunk * NB;                      // [16 warps][32] dL/dtau sums
  float4* sRec0 = reinterpret_cast<float4*>(sTau + S::kWarps * kChunk);  // [2][32][2]
  uint32_t* sK0 = reinterpret_cast<uint32_t*>(sRec0 + 2 * 2 * kChunk);    // [3][32] indices
  __shared__ unsigned sMask[S::kWarps];  // per warp: entries with a non-zero weight

  const RenderArgs& a = A.f;
  const GridConst& g = a.g;
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5, h = lane >> 4;
  const int px = wp * 16 + (lane & 15);
  const int tile = blockIdx.x, v = blockIdx.z;
  const int col0 = blockIdx.y * NB;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + px / g.TW, jj = tc * g.TW + px % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  const int twoC = 2 * a.C;
  const Strip strip = pixel_strip(g, tr, tc, wp * 16, 16);

  // cotangent rows of the tile for the CTA's columns (consecutive threads
  // take consecutive pixels of one column): asynchronous copies when the
  // cotangent is per pixel only, so that all of them are in flight at once
  if (A.g_spec && !A.g_uniform) {
    for (int e = t; e < kTilePixels * NB; e += S::kThreads) {
      const int p = e % kTilePixels, c = e / kTilePixels;
      const int pi = tr * g.TH + p / g.TW, pj = tc * g.TW + p % g.TW;
      const int col = col0 + c;
      const bool ok = pi < g.H && pj < g.W && col < a.ncols;
      const float* src = A.g_spec;
      if (ok) {
        const int j = col / twoC, ec = col - j * twoC;
        const size_t pix = static_cast<size_t>(pi) * g.W + pj;
        src += ((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + ec;
      }
      cp_async4(&sG[p * S::GS + c], src, ok);
    }
    cp_async_commit();
  } else {
#pragma unroll 8
    for (int e = t; e < kTilePixels * NB; e += S::kThreads) {
      const int p = e % kTilePixels, c = e / kTilePixels;
      const int pi = tr * g.TH + p / g.TW, pj = tc * g.TW + p % g.TW;
      const int col = col0 + c;
      float val = 0.0f;
      if (pi < g.H && pj < g.W && col < a.ncols) {
        const int j = col / twoC, ec = col - j * twoC;
        const size_t pix = static_cast<size_t>(pi) * g.W + pj;
        if (A.g_spec) val += A.g_spec[((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + ec];
        if (A.g_uniform) val += A.g_uniform[static_cast<size_t>(v) * a.ncols + col];
      }
      sG[p * S::GS + c] = val;
    }
  }
  // final transmittance and stop position from the per-tile pre-pass
  float T = 1.0f;
  uint32_t stop = rg.x;
  if (valid) {
    const size_t o = static_cast<size_t>(v) * HW + static_cast<size_t>(i) * g.W + jj;
    T = A.tfin[o];
    stop = A.stops[o];
  }
  const uint32_t tile_stop = A.tile_stop[static_cast<size_t>(v) * g.T + tile];

  // product mapping: 16 groups of 2 entries x CB groups of 16 columns, SL
  // pixel slices
  const int slice = t % S::SL, ob = t / S::SL;
  const int bb = (ob / S::CB) * S::PE, cbk = (ob % S::CB) * S::PC;

  float Q = 0.0f;
  const float* gRow = sG + px * S::GS + h * S::HC;
  const int nchunks = static_cast<int>((tile_stop - rg.x + kChunk - 1) / kChunk);
  // Chunks are processed back to front (n-th processed = chunk nchunks-1-n)
  // through a copy pipeline: while chunk n is swept, the records and
  // radiance rows of chunk n + 1 (gathered with the indices already in
  // shared memory) and the indices of chunk n + 2 are in flight (cp.async),
  // so no thread waits on a global load at a chunk boundary.
  auto chunk_start = [&](int n) { return rg.x + static_cast<uint32_t>(nchunks - 1 - n) * kChunk; };
  auto chunk_len = [&](int n) { return min(kChunk, static_cast<int>(tile_stop - chunk_start(n))); };
  auto copy_indices = [&](int n) {
    const uint32_t st0 = chunk_start(n);
    const bool ok = t < chunk_len(n);
    if (t < kChunk) cp_async4(&sK0[(n % 3) * kChunk + t], ok ? &a.vals[st0 + t] : a.vals, ok);
  };
  auto gather = [&](int n) {
    const int nbn = chunk_len(n);
    const uint32_t* ks = sK0 + (n % 3) * kChunk;
    float4* rb = sRec0 + (n & 1) * 2 * kChunk;
    float* rr = sR0 + (n & 1) * kChunk * NB;
    if (t < kChunk) {
      const bool ok = t < nbn;
      const uint32_t k = ok ? ks[t] : 0u;
      cp_async16(&rb[2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&rb[2 * t + 1], &rec[2 * k + 1], ok);
    }
    constexpr int Q4 = NB / 4;  // float4 per radiance row slice
    for (int e = t; e < kChunk * Q4; e += S::kThreads) {
      const int b = e / Q4, q4 = e % Q4;
      const bool ok = b < nbn;
      const uint32_t k = ok ? ks[b] : 0u;
      cp_async16(&rr[b * NB + 4 * q4],
                 a.rad + static_cast<size_t>(v) * a.rad_view + static_cast<size_t>(k) * a.stride +
                     col0 + 4 * q4,
                 ok);
    }
  };
  sTau[t] = 0.0f;  // 512 threads, 16 x 32 entries; the dL/dtau step re-zeroes
  if (nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // cotangent and indices of chunk 0
    __syncthreads();
    gather(0);
    cp_async_commit();
  }
  for (int n = 0; n < nchunks; ++n) {
    const uint32_t start = chunk_start(n);
    const int nb = chunk_len(n);
    cp_async_wait_all();  // chunk n's records and rows, chunk n + 1's indices
    __syncthreads();      // ... visible to all; everyone is done with chunk n - 1
    if (n + 1 < nchunks) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      gather(n + 1);
    }
    cp_async_commit();
    const float4* sRec = sRec0 + (n & 1) * 2 * kChunk;
    const float* sR = sR0 + (n & 1) * kChunk * NB;
    const uint32_t* sK = sK0 + (n % 3) * kChunk;
    {
      const bool rel = lane < nb && touches_strip(g, sRec[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      // no pixel of the strip reaches this chunk: nothing to do here
      if (!__any_sync(0xffffffffu, start < stop)) m = 0;
      unsigned used = 0;
      const int src0 = lane & 15, src1 = src0 | 16;
      while (m) {
        const int b0 = 31 - __clz(m);
        m &= ~(1u << b0);
        const int b1 = m ? 31 - __clz(m) : -1;
        if (b1 >= 0) m &= ~(1u << b1);
        // weights: lower half b0, upper half b1; G = 0 marks "not composited"
        const int bm = h ? b1 : b0;
        float wm = 0.0f, Gm = 0.0f;
        if (bm >= 0 && start + bm < stop) {
          float w, G;
          if (pixel_weight(g, sRec[2 * bm], sRec[2 * bm + 1], i, jj, fi, fj, &w, &G)) {
            wm = w;
            Gm = G;
          }
        }
        const float w0 = __shfl_sync(0xffffffffu, wm, src0);
        const float G0 = __shfl_sync(0xffffffffu, Gm, src0);
        const float w1 = __shfl_sync(0xffffffffu, wm, src1);
        const float G1 = __shfl_sync(0xffffffffu, Gm, src1);
        // gamma over this half's columns, both entries
        float p0 = 0.0f, p1 = 0.0f;
        const bool c0 = G0 != 0.0f, c1 = G1 != 0.0f;
        if (c0 || c1) {
          const float4* r0 = reinterpret_cast<const float4*>(&sR[b0 * NB + h * S::HC]);
          const float4* r1 = reinterpret_cast<const float4*>(&sR[(b1 >= 0 ? b1 : b0) * NB + h * S::HC]);
          const float4* g4 = reinterpret_cast<const float4*>(gRow);
#pragma unroll
          for (int q = 0; q < S::HC / 4; ++q) {
            const float4 gv = g4[q], a0 = r0[q], a1 = r1[q];
            p0 = fmaf(gv.x, a0.x, p0);
            p0 = fmaf(gv.y, a0.y, p0);
            p0 = fmaf(gv.z, a0.z, p0);
            p0 = fmaf(gv.w, a0.w, p0);
            p1 = fmaf(gv.x, a1.x, p1);
            p1 = fmaf(gv.y, a1.y, p1);
            p1 = fmaf(gv.z, a1.z, p1);
            p1 = fmaf(gv.w, a1.w, p1);
          }
        }
        const float gam0 = p0 + __shfl_xor_sync(0xffffffffu, p0, 16);
        const float gam1 = p1 + __shfl_xor_sync(0xffffffffu, p1, 16);
        float Tw0 = 0.0f, Tw1 = 0.0f, dt0 = 0.0f, dt1 = 0.0f;
        if (c0) {
          const float one_m_w = 1.0f - w0;
          T = __fdividef(T, one_m_w);  // transmittance in front of this Gaussian
          Tw0 = T * w0;
          dt0 = T * (gam0 - Q) * G0;
          Q = fmaf(w0, gam0, one_m_w * Q);
        }
        if (c1) {
          const float one_m_w = 1.0f - w1;
          T = __fdividef(T, one_m_w);
          Tw1 = T * w1;
          dt1 = T * (gam1 - Q) * G1;
          Q = fmaf(w1, gam1, one_m_w * Q);
        }
        if (h == 0)
          sA[b0 * kTilePixels + px] = Tw0;
        else if (b1 >= 0)
          sA[b1 * kTilePixels + px] = Tw1;
        if (__any_sync(0xffffffffu, Tw0 != 0.0f)) used |= 1u << b0;
        if (b1 >= 0 && __any_sync(0xffffffffu, Tw1 != 0.0f)) used |= 1u << b1;
        // dL/dtau over the warp's 16 pixels: each half sums its own entry
        float dv = h ? dt1 : dt0;
        if (__any_sync(0xffffffffu, dv != 0.0f)) {
          dv += __shfl_xor_sync(0xffffffffu, dv, 1);
          dv += __shfl_xor_sync(0xffffffffu, dv, 2);
          dv += __shfl_xor_sync(0xffffffffu, dv, 4);
          dv += __shfl_xor_sync(0xffffffffu, dv, 8);
          if (lane == 0) sTau[wp * kChunk + b0] = dv;
          if (lane == 16 && b1 >= 0) sTau[wp * kChunk + b1] = dv;
        }
      }
      if (lane == 0) sMask[wp] = used;
    }
    __syncthreads();
    // dL/ds[b][c] = sum_p A[b][p] g[p][c]: 2 x 16 block per thread over the
    // pixels p = it*SL + slice, then a sum over the SL slices.
    {
      float acc[S::PE][S::PC];
#pragma unroll
      for (int x = 0; x < S::PE; ++x)
#pragma unroll
        for (int c = 0; c < S::PC; ++c) acc[x][c] = 0.0f;
      if (bb < nb) {
        for (int it = 0; it < kTilePixels / S::SL; ++it) {
          // pixels it*SL .. it*SL+SL-1 belong to warp (it*SL)/16, which wrote
          // only the entries of its mask: skip the group when neither of
          // b, b+1 is there
          const unsigned wm = (sMask[(it * S::SL) >> 4] >> bb) & ((1u << S::PE) - 1u);
          if (!wm) continue;
          const int p = it * S::SL + slice;
          float av[S::PE];
#pragma unroll
          for (int x = 0; x < S::PE; ++x)
            av[x] = (wm >> x) & 1u ? sA[(bb + x) * kTilePixels + p] : 0.0f;
          float gv[S::PC];
#pragma unroll
          for (int q = 0; q < S::PC / 4; ++q) {
            const float4 g4 = *reinterpret_cast<const float4*>(&sG[p * S::GS + cbk + 4 * q]);
            gv[4 * q] = g4.x;
            gv[4 * q + 1] = g4.y;
            gv[4 * q + 2] = g4.z;
            gv[4 * q + 3] = g4.w;
          }
#pragma unroll
          for (int x = 0; x < S::PE; ++x)
#pragma unroll
            for (int c = 0; c < S::PC; ++c) acc[x][c] = fmaf(av[x], gv[c], acc[x][c]);
        }
      }
#pragma unroll
      for (int x = 0; x < S::PE; ++x)
#pragma unroll
        for (int c = 0; c < S::PC; ++c) {
          float y = acc[x][c];
#pragma unroll
          for (int o = S::SL / 2; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
          acc[x][c] = y;
        }
      if (slice == 0) {
#pragma unroll
        for (int x = 0; x < S::PE; ++x) {
          const int b = bb + x;
          if (b >= nb) continue;
          float* dst = A.d_rad + static_cast<size_t>(v) * a.rad_view +
                       static_cast<size_t>(sK[b]) * a.stride + col0 + cbk;
#pragma unroll
          for (int c = 0; c < S::PC; ++c)
            if (col0 + cbk + c < a.ncols && acc[x][c] != 0.0f) atomicAdd(&dst[c], acc[x][c]);
        }
      }
    }
    // dL/dtau: the warps' sums in order; each column block adds the part of
    // the gradient its columns carry.  Entry t's sums are re-zeroed by the
    // thread that read them.
    if (t < kChunk) {
      float y = 0.0f;
#pragma unroll
      for (int w = 0; w < S::kWarps; ++w) {
        y += sTau[w * kChunk + t];
        sTau[w * kChunk + t] = 0.0f;
      }
      if (t < nb && y != 0.0f) atomicAdd(&A.d_tau[sK[t]], y);
    }
  }
  cp_async_wait_all();  // the cotangent copies when the tile has no chunk
}

template <int NB>
static void launch_bwd_nb(const BackwardArgs& A, cudaStream_t s) {
  const RenderArgs& a = A.f;
  constexpr size_t smem = BwdShape<NB>::smem;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_bwd_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    configured = true;
  }
  dim3 grid(a.g.T, (a.ncols + NB - 1) / NB, a.M);
  render_bwd_kernel<NB><<<grid, BwdShape<NB>::kThreads, smem, s>>>(A);
  note_launches(1);
}

void launch_bwd_prepass(const BackwardArgs& A, cudaStream_t s) {
  const RenderArgs& a = A.f;
  if (a.M <= 0 || a.ncols <= 0) return;
  bwd_prepass_kernel<<<dim3(a.g.T, 1, a.M), kTilePixels, 0, s>>>(a, A.tfin, A.stops, A.tile_stop);
  note_launches(1);
}

void launch_render_bwd_tc(const BackwardArgs& A, cudaStream_t s);  // render_bwd_tc.cu

void launch_render_bwd(const BackwardArgs& A, cudaStream_t s) {
  const RenderArgs& a = A.f;
  if (a.M <= 0 || a.ncols <= 0) return;
  // radiance rows are padded to a multiple of 128 columns, so every block
  // of 64 or 128 columns lies inside its row; blocks of 128 columns run the
  // tensor-core sweep (render_bwd_tc.cu)
  if (a.ncols <= 64)
    launch_bwd_nb<64>(A, s);
  else
    launch_render_bwd_tc(A, s);
}

}  // namespace rxgs
