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

constexpr int kBNB = 32;      // columns per backward CTA
constexpr int kPad = 257;     // padded per-pixel row (bank spread)
constexpr int kGStride = 36;  // padded cotangent row (float4 aligned)

constexpr size_t bwd_smem_bytes() {
  return sizeof(float) * (kTilePixels * kGStride + 2 * kChunk * kPad + kChunk * kBNB) +
         sizeof(float4) * 2 * kChunk + sizeof(uint32_t) * kChunk;
}

// Walk 1, once per (view, tile): every pixel's final transmittance and the
// list position one past its last composited Gaussian (its stop), with the
// forward's float32 decisions; tile_stop = the largest stop of the tile.
__global__ void __launch_bounds__(kTilePixels) bwd_prepass_kernel(const RenderArgs a,
                                                                  float* __restrict__ tfin,
                                                                  uint32_t* __restrict__ stops,
                                                                  uint32_t* __restrict__ tile_stop) {
  __shared__ float4 sRec[2 * kChunk];
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
  for (uint32_t start = rg.x; start < rg.y; start += kChunk) {
    const int nb = min(kChunk, static_cast<int>(rg.y - start));
    __syncthreads();
    if (t < kChunk) {
      const bool ok = t < nb;
      const uint32_t k = ok ? a.vals[start + t] : 0u;
      cp_async16(&sRec[2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&sRec[2 * t + 1], &rec[2 * k + 1], ok);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    {
      const int lane = t & 31;
      const bool rel = lane < nb && touches_strip(g, sRec[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      while (alive && m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        float w, G;
        if (pixel_weight(g, sRec[2 * b], sRec[2 * b + 1], i, jj, fi, fj, &w, &G)) {
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
  atomicMax(&sStop, stop);
  if (valid) {
    const size_t o = static_cast<size_t>(v) * g.H * g.W + static_cast<size_t>(i) * g.W + jj;
    tfin[o] = T;
    stops[o] = stop;
  }
  __syncthreads();
  if (t == 0) tile_stop[static_cast<size_t>(v) * g.T + tile] = sStop;
}

__global__ void __launch_bounds__(kTilePixels, 2) render_bwd_kernel(const BackwardArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sG = reinterpret_cast<float*>(smem_raw);   // [256][36] cotangent rows
  float* sA = sG + kTilePixels * kGStride;          // [32][257] T w
  float* sT = sA + kChunk * kPad;                   // [32][257] dL/dtau per pixel
  float* sR = sT + kChunk * kPad;                   // [32][32] radiance slice
  float4* sRec = reinterpret_cast<float4*>(sR + kChunk * kBNB);  // [32][2]
  uint32_t* sK = reinterpret_cast<uint32_t*>(sRec + 2 * kChunk);  // [32]
  __shared__ unsigned sMask[kTilePixels / 32];  // per warp: chunk entries meeting its strip

  const RenderArgs& a = A.f;
  const GridConst& g = a.g;
  const int t = threadIdx.x;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int col0 = blockIdx.y * kBNB;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  const size_t pix = static_cast<size_t>(i) * g.W + jj;
  const int twoC = 2 * a.C;
  const Strip strip = warp_strip(g, tr, tc, t >> 5);

  // cotangent of this pixel for the CTA's columns
  float gr[kBNB];
#pragma unroll
  for (int c = 0; c < kBNB; ++c) {
    const int col = col0 + c;
    float val = 0.0f;
    if (valid && col < a.ncols) {
      const int j = col / twoC, e = col - j * twoC;
      if (A.g_spec) val += A.g_spec[((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + e];
      if (A.g_uniform) val += A.g_uniform[static_cast<size_t>(v) * a.ncols + col];
    }
    gr[c] = val;
    sG[t * kGStride + c] = val;
  }
  // final transmittance and stop position from the per-tile pre-pass
  float T = 1.0f;
  uint32_t stop = rg.x;
  if (valid) {
    const size_t o = static_cast<size_t>(v) * HW + pix;
    T = A.tfin[o];
    stop = A.stops[o];
  }
  const uint32_t tile_stop = A.tile_stop[static_cast<size_t>(v) * g.T + tile];

  // dS mapping: 32 output blocks (4 Gaussians x 8 columns) x 8 pixel slices
  const int slice = t & 7, ob = t >> 3;
  const int bb = (ob >> 2) * 4, cbk = (ob & 3) * 8;

  // ---- walk 2: back to front
  float Q = 0.0f;
  const int nchunks = static_cast<int>((tile_stop - rg.x + kChunk - 1) / kChunk);
  for (int ci = nchunks - 1; ci >= 0; --ci) {
    const uint32_t start = rg.x + static_cast<uint32_t>(ci) * kChunk;
    const int nb = min(kChunk, static_cast<int>(tile_stop - start));
    __syncthreads();
    if (t < kChunk) {
      const bool ok = t < nb;
      const uint32_t k = ok ? a.vals[start + t] : 0u;
      sK[t] = k;
      cp_async16(&sRec[2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&sRec[2 * t + 1], &rec[2 * k + 1], ok);
    }
    {
      const int b = t >> 3, q4 = t & 7;  // 32 rows x 32 columns, one float4 each
      const bool ok = b < nb;
      const uint32_t k = ok ? __ldg(&a.vals[start + b]) : 0u;
      cp_async16(&sR[b * kBNB + 4 * q4], a.rad + static_cast<size_t>(k) * a.stride + col0 + 4 * q4,
                 ok);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    {
      // entries meeting this warp's strip, swept from the back
      const int lane = t & 31;
      const bool rel = lane < nb && touches_strip(g, sRec[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      // no pixel of the strip reaches this chunk: nothing to do here
      if (!__any_sync(0xffffffffu, start < stop)) m = 0;
      unsigned used = 0;  // entries with a non-zero weight somewhere in the strip
      while (m) {
        const int b = 31 - __clz(m);
        m &= ~(1u << b);
        float Tw = 0.0f, dtau = 0.0f;
        if (start + b < stop) {
          float w, G;
          if (pixel_weight(g, sRec[2 * b], sRec[2 * b + 1], i, jj, fi, fj, &w, &G)) {
            float gam = 0.0f;
            const float4* r4 = reinterpret_cast<const float4*>(&sR[b * kBNB]);
#pragma unroll
            for (int q = 0; q < kBNB / 4; ++q) {
              const float4 s4 = r4[q];
              gam = fmaf(gr[4 * q + 0], s4.x, gam);
              gam = fmaf(gr[4 * q + 1], s4.y, gam);
              gam = fmaf(gr[4 * q + 2], s4.z, gam);
              gam = fmaf(gr[4 * q + 3], s4.w, gam);
            }
            const float one_m_w = 1.0f - w;
            T = __fdividef(T, one_m_w);  // transmittance in front of this Gaussian
            Tw = T * w;
            dtau = T * (gam - Q) * G;
            Q = fmaf(w, gam, one_m_w * Q);
          }
        }
        sA[b * kPad + t] = Tw;
        sT[b * kPad + t] = dtau;
        if (__any_sync(0xffffffffu, Tw != 0.0f)) used |= 1u << b;
      }
      if (lane == 0) sMask[t >> 5] = used;
    }
    __syncthreads();
    // dL/ds[b][c] = sum_pixels A[b][p] g[p][c]: 4 x 8 block per thread over the
    // pixels p = it*8 + slice, then a sum over the 8 slices.
    {
      float acc[4][8];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[x][c] = 0.0f;
      if (bb < nb) {
        for (int it = 0; it < kTilePixels / 8; ++it) {
          // pixels it*8 .. it*8+7 belong to warp it/4, which wrote only the
          // entries of its mask: skip the group when none of b..b+3 is there
          const unsigned wm = (sMask[it >> 2] >> bb) & 0xfu;
          if (!wm) continue;
          const int p = it * 8 + slice;
          float av[4];
#pragma unroll
          for (int x = 0; x < 4; ++x) av[x] = (wm >> x) & 1u ? sA[(bb + x) * kPad + p] : 0.0f;
          const float4 g0 = *reinterpret_cast<const float4*>(&sG[p * kGStride + cbk]);
          const float4 g1 = *reinterpret_cast<const float4*>(&sG[p * kGStride + cbk + 4]);
          const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[x][c] = fmaf(av[x], gv[c], acc[x][c]);
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float y = acc[x][c];
          y += __shfl_xor_sync(0xffffffffu, y, 4);
          y += __shfl_xor_sync(0xffffffffu, y, 2);
          y += __shfl_xor_sync(0xffffffffu, y, 1);
          acc[x][c] = y;
        }
      if (slice == 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const int b = bb + x;
          if (b >= nb) continue;
          float* dst = A.d_rad + static_cast<size_t>(sK[b]) * a.stride + col0 + cbk;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (col0 + cbk + c < a.ncols && acc[x][c] != 0.0f) atomicAdd(&dst[c], acc[x][c]);
        }
      }
    }
    // dL/dtau: sum over the tile's pixels for each Gaussian of the chunk; each
    // column block adds the part of the gradient its columns carry
    {
      const int b = t >> 3, part = t & 7;
      float y = 0.0f;
      if (b < nb)
        for (int it = 0; it < kTilePixels / 8; ++it)
          if ((sMask[it >> 2] >> b) & 1u) y += sT[b * kPad + it * 8 + part];
      y += __shfl_xor_sync(0xffffffffu, y, 4);
      y += __shfl_xor_sync(0xffffffffu, y, 2);
      y += __shfl_xor_sync(0xffffffffu, y, 1);
      if (part == 0 && b < nb && y != 0.0f) atomicAdd(&A.d_tau[sK[b]], y);
    }
  }
}

void launch_render_bwd(const BackwardArgs& A, int /*cols_per_cta*/, cudaStream_t s) {
  const RenderArgs& a = A.f;
  if (a.M <= 0 || a.ncols <= 0) return;
  constexpr size_t smem = bwd_smem_bytes();
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    configured = true;
  }
  bwd_prepass_kernel<<<dim3(a.g.T, 1, a.M), kTilePixels, 0, s>>>(a, A.tfin, A.stops, A.tile_stop);
  note_launches(1);
  dim3 grid(a.g.T, (a.ncols + kBNB - 1) / kBNB, a.M);
  render_bwd_kernel<<<grid, kTilePixels, smem, s>>>(A);
  note_launches(1);
}

}  // namespace rxgs
