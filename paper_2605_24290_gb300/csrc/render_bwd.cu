// render_bwd.cu -- backward of the multi-receiver compositing (App. D: the
// backward kernel runs over the same (tile, receiver) grid and accumulates
// Gaussian-level gradients with atomicAdd).
//
// For one pixel with composited sequence k_1..k_n (weights w_m, transmittance
// T_m = prod_{l<m} (1 - w_l)) and cotangent g_c per output column c:
//   dL/ds_{k_m, c}  = T_m w_m g_c
//   dL/dw_m         = T_m gamma_m - (D - E_m) / (1 - w_m)
//   with gamma_m    = sum_c g_c s_{k_m, c},  E_m = sum_{l<=m} T_l w_l gamma_l,
//        D          = sum_c g_c C_c (= E_n, the pixel's full sum)
//   dL/dtau_{k_m}   = exp(-q/2) dL/dw_m
// Both gradients are linear in the columns, so each CTA handles a block of 32
// columns and the per-column-block contributions add up.  Nothing per pixel
// is stored by the forward: every tile walks its list again with the same
// float32 decisions (per-tile recomputation).  D comes from the forward
// spectra when they are given; otherwise a first walk accumulates it.
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

template <bool HAVE_D>
__global__ void __launch_bounds__(kTilePixels, 2) render_bwd_kernel(const BackwardArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sG = reinterpret_cast<float*>(smem_raw);   // [256][36] cotangent rows
  float* sA = sG + kTilePixels * kGStride;          // [32][257] T w
  float* sT = sA + kChunk * kPad;                   // [32][257] dL/dtau per pixel
  float* sR = sT + kChunk * kPad;                   // [32][32] radiance slice
  float4* sRec = reinterpret_cast<float4*>(sR + kChunk * kBNB);  // [32][2]
  uint32_t* sK = reinterpret_cast<uint32_t*>(sRec + 2 * kChunk);  // [32]

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

  // cotangent of this pixel for the CTA's columns, and D from the forward
  float gr[kBNB];
  float D = 0.0f;
#pragma unroll
  for (int c = 0; c < kBNB; ++c) {
    const int col = col0 + c;
    float val = 0.0f;
    if (valid && col < a.ncols) {
      const int j = col / twoC, e = col - j * twoC;
      const size_t off = ((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + e;
      if (A.g_spec) val += A.g_spec[off];
      if (A.g_uniform) val += A.g_uniform[static_cast<size_t>(v) * a.ncols + col];
      if (HAVE_D) D = fmaf(val, a.spectra[off], D);
    }
    gr[c] = val;
    sG[t * kGStride + c] = val;
  }

  // dS mapping: 32 output blocks (4 Gaussians x 8 columns) x 8 pixel slices
  const int slice = t & 7, ob = t >> 3;
  const int bb = (ob >> 2) * 4, cbk = (ob & 3) * 8;

  for (int pass = HAVE_D ? 1 : 0; pass < 2; ++pass) {
    float T = 1.0f, E = 0.0f;
    bool alive = valid;
    for (uint32_t start = rg.x; start < rg.y; start += kChunk) {
      const int nb = min(kChunk, static_cast<int>(rg.y - start));
      __syncthreads();
      if (t < kChunk) {
        const bool ok = t < nb;
        const uint32_t k = ok ? a.vals[start + t] : 0u;
        sK[t] = k;
        cp_async16(&sRec[2 * t + 0], &rec[2 * k + 0], ok);
        cp_async16(&sRec[2 * t + 1], &rec[2 * k + 1], ok);
      }
      {
        // 32 rows x 32 columns = 256 float4, one per thread
        const int b = t >> 3, q4 = t & 7;
        const bool ok = b < nb;
        const uint32_t k = ok ? __ldg(&a.vals[start + b]) : 0u;
        cp_async16(&sR[b * kBNB + 4 * q4], a.rad + static_cast<size_t>(k) * a.stride + col0 + 4 * q4,
                   ok);
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      for (int b = 0; b < nb; ++b) {
        float Tw = 0.0f, dtau = 0.0f;
        if (alive) {
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
            Tw = __fmul_rn(T, w);
            E = fmaf(Tw, gam, E);
            if (pass == 1) {
              const float dldw = T * gam - (D - E) / (1.0f - w);
              dtau = dldw * G;
            }
            T = __fmul_rn(T, __fsub_rn(1.0f, w));
            if (T < g.eps_T) alive = false;
          }
        }
        if (pass == 1) {
          sA[b * kPad + t] = Tw;
          sT[b * kPad + t] = dtau;
        }
      }
      const int n_alive = __syncthreads_count(alive);
      if (pass == 1) {
        // dL/ds[b][c] = sum_pixels A[b][p] g[p][c]: 4 x 8 block per thread over
        // the pixels p = it*8 + slice, then a sum over the 8 slices.
        float acc[4][8];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[x][c] = 0.0f;
        if (bb < nb) {
          for (int it = 0; it < kTilePixels / 8; ++it) {
            const int p = it * 8 + slice;
            const float4 g0 = *reinterpret_cast<const float4*>(&sG[p * kGStride + cbk]);
            const float4 g1 = *reinterpret_cast<const float4*>(&sG[p * kGStride + cbk + 4]);
            const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              const float av = sA[(bb + x) * kPad + p];
#pragma unroll
              for (int c = 0; c < 8; ++c) acc[x][c] = fmaf(av, gv[c], acc[x][c]);
            }
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
        // dL/dtau: sum over pixels of each Gaussian of the chunk
        {
          const int b = t >> 3, part = t & 7;
          float y = 0.0f;
          if (b < nb)
            for (int it = 0; it < kTilePixels / 8; ++it) y += sT[b * kPad + it * 8 + part];
          y += __shfl_xor_sync(0xffffffffu, y, 4);
          y += __shfl_xor_sync(0xffffffffu, y, 2);
          y += __shfl_xor_sync(0xffffffffu, y, 1);
          if (part == 0 && b < nb && y != 0.0f) atomicAdd(&A.d_tau[sK[b]], y);
        }
      }
      if (n_alive == 0) break;
    }
    if (pass == 0) D = E;  // the full sum of this pixel's contributions
  }
}

void launch_render_bwd(const BackwardArgs& A, int /*cols_per_cta*/, cudaStream_t s) {
  const RenderArgs& a = A.f;
  if (a.M <= 0 || a.ncols <= 0) return;
  constexpr size_t smem = bwd_smem_bytes();
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    cudaFuncSetAttribute(render_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    configured = true;
  }
  dim3 grid(a.g.T, (a.ncols + kBNB - 1) / kBNB, a.M);
  if (a.spectra)
    render_bwd_kernel<true><<<grid, kTilePixels, smem, s>>>(A);
  else
    render_bwd_kernel<false><<<grid, kTilePixels, smem, s>>>(A);
}

}  // namespace rxgs
