// vis.cu -- CSI / RSSI through visibility weights (Eq. render_reorder):
//   S_j = sum_omega C^(j)(omega) = sum_k W_k s_kj,   W_k = sum_omega T_k(omega) w_k(omega)
// W is receiver-independent, so each view is rasterised once (the same walk
// and float32 decisions as the compositing, but with no receiver columns),
// and the receivers then only need a K-long weighted sum of their radiance:
//   explicit radiance  out[j][v][:] = sum_k rad[j][k][:] W[v][k]: one pass
//                      over each receiver's radiance row for all views (the
//                      [M][K] weights stay in L2), bound by HBM;
//   MLP radiance       out[j][:] = sum_k W[v(j)][k] s(j, k), with s evaluated
//                      on the fly and Gaussians of zero weight skipped, so the
//                      [K][N*2C] radiance is never materialised.
// W is accumulated with float atomics over the tiles a Gaussian meets, so
// its rounding order is not fixed; every other sum runs in a fixed order.
#include <cuda_bf16.h>

#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

// ------------------------------------------------------------- weights W
__global__ void __launch_bounds__(kTilePixels) visibility_kernel(const RenderArgs a,
                                                                 float* __restrict__ Wout) {
  __shared__ float sA[kChunk * kTilePixels];
  __shared__ float4 sRec[2 * kChunk];
  __shared__ uint32_t sK[kChunk];
  const GridConst& g = a.g;
  const int t = threadIdx.x;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  float* W = Wout + static_cast<size_t>(v) * a.K;
  float T = 1.0f;
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
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      float Tw = 0.0f;
      if (alive) {
        float w, G;
        if (pixel_weight(g, sRec[2 * b], sRec[2 * b + 1], i, jj, fi, fj, &w, &G)) {
          Tw = __fmul_rn(T, w);
          T = __fmul_rn(T, __fsub_rn(1.0f, w));
          if (T < g.eps_T) alive = false;
        }
      }
      sA[b * kTilePixels + t] = Tw;
    }
    const int n_alive = __syncthreads_count(alive);
    {
      // sum over the tile's pixels per Gaussian: 8 threads per entry
      const int b = t >> 3, part = t & 7;
      float y = 0.0f;
      if (b < nb)
        for (int q = 0; q < kTilePixels / 8; ++q) y += sA[b * kTilePixels + q * 8 + part];
      y += __shfl_xor_sync(0xffffffffu, y, 4);
      y += __shfl_xor_sync(0xffffffffu, y, 2);
      y += __shfl_xor_sync(0xffffffffu, y, 1);
      if (part == 0 && b < nb && y != 0.0f) atomicAdd(&W[sK[b]], y);
    }
    if (n_alive == 0) break;
  }
}

void launch_visibility(const RenderArgs& a, float* W, cudaStream_t s) {
  if (a.M <= 0) return;
  cudaMemsetAsync(W, 0, sizeof(float) * static_cast<size_t>(a.M) * a.K, s);
  visibility_kernel<<<dim3(a.g.T, 1, a.M), kTilePixels, 0, s>>>(a, W);
  note_launches(1);
}

// ------------------------------------------- explicit radiance: a GEMV pass
// Block (j, chunk of K): out_part[chunk][j][v][e] = sum_{k in chunk}
// rad[j][k][e] W[v][k] for all views v; a second kernel adds the chunks in
// order.  The radiance row is read once for all views.
constexpr int kWsChunk = 4096;   // Gaussians per block
constexpr int kWsMaxViews = 32;  // views handled per pass

__global__ void __launch_bounds__(256) weighted_sum_kernel(const float* __restrict__ rad, int K,
                                                           int C, const float* __restrict__ W,
                                                           int M, int v0, int nv,
                                                           float* __restrict__ part) {
  const int j = blockIdx.y, chunk = blockIdx.x;
  const int twoC = 2 * C;
  const int k0 = chunk * kWsChunk, k1 = min(K, k0 + kWsChunk);
  extern __shared__ float red[];  // [8 warps][nv][twoC]
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // each thread owns (entry e = t % twoC slot) ... simple layout: loop over
  // (k, e) pairs with e fastest; accumulate per (v, e) in registers for e
  // fixed per thread when twoC divides 256
  const int per = 256 / twoC;        // threads per e (twoC <= 256 and divides 256)
  const int e = t % twoC, sub = t / twoC;
  float acc[kWsMaxViews];
#pragma unroll
  for (int q = 0; q < kWsMaxViews; ++q) acc[q] = 0.0f;
  const float* row = rad + static_cast<size_t>(j) * K * twoC;
  if (sub < per) {
    for (int k = k0 + sub; k < k1; k += per) {
      const float x = row[static_cast<size_t>(k) * twoC + e];
#pragma unroll
      for (int q = 0; q < kWsMaxViews; ++q)
        if (q < nv) acc[q] = fmaf(x, W[static_cast<size_t>(v0 + q) * K + k], acc[q]);
    }
  }
  // reduce over the `per` threads sharing e (fixed order through shared memory)
  float* r = red;  // [per][nv][twoC] reused per view group
  for (int q = 0; q < nv; ++q) r[(sub * nv + q) * twoC + e] = acc[q];
  __syncthreads();
  for (int o = t; o < nv * twoC; o += 256) {
    float y = 0.0f;
    for (int s2 = 0; s2 < per; ++s2) y += r[s2 * nv * twoC + o];
    const int q = o / twoC, ee = o % twoC;
    part[((static_cast<size_t>(chunk) * gridDim.y + j) * M + v0 + q) * twoC + ee] = y;
  }
  (void)lane;
  (void)warp;
}

__global__ void weighted_sum_finish_kernel(const float* __restrict__ part, int nchunks, int N,
                                           int M, int C, float* __restrict__ csi,
                                           float* __restrict__ rssi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // (v, j, c)
  if (idx >= M * N * C) return;
  const int c = idx % C, j = (idx / C) % N, v = idx / (C * N);
  const int twoC = 2 * C;
  float re = 0.0f, im = 0.0f;
  for (int ch = 0; ch < nchunks; ++ch) {
    const float* p = part + ((static_cast<size_t>(ch) * N + j) * M + v) * twoC + 2 * c;
    re += p[0];
    im += p[1];
  }
  if (csi) {
    csi[2 * static_cast<size_t>(idx)] = re;
    csi[2 * static_cast<size_t>(idx) + 1] = im;
  }
  if (rssi && C == 1) rssi[idx] = sqrtf(re * re + im * im);
}

size_t weighted_sum_tmp_floats(int M, int K, int N, int C) {
  const size_t nchunks = (K + kWsChunk - 1) / kWsChunk;
  return nchunks * N * M * 2ull * C;
}

bool weighted_sum_supported(int C) { return 256 % (2 * C) == 0; }

void launch_weighted_sum(const float* rad, int N, int K, int C, const float* W, int M, float* tmp,
                         float* csi, float* rssi, cudaStream_t s) {
  const int nchunks = (K + kWsChunk - 1) / kWsChunk;
  const int twoC = 2 * C;
  for (int v0 = 0; v0 < M; v0 += kWsMaxViews) {
    const int nv = min(kWsMaxViews, M - v0);
    const size_t smem = sizeof(float) * (256 / twoC) * nv * twoC;
    weighted_sum_kernel<<<dim3(nchunks, N), 256, smem, s>>>(rad, K, C, W, M, v0, nv, tmp);
    note_launches(1);
  }
  const int n = M * N * C;
  weighted_sum_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(tmp, nchunks, N, M, C, csi, rssi);
  note_launches(1);
}

}  // namespace rxgs

namespace rxgs {

// ------------------------------------ MLP radiance: fused evaluate + reduce
// Block (chunk of Gaussians, receiver j): for the views v of receiver j
// (views v0 .. v0+nv-1 for every receiver, or the single view rx_view[j]),
//   part[chunk][j][v][2C] = sum_{k in chunk} W[v][k] s(j, k)
// with s(j, k) from the conditioning MLP (same formulas and operation order
// as the radiance kernel), evaluated only where some W[v][k] != 0.
constexpr int kMwChunk = 4096;
constexpr int kMwMaxViews = 8;

template <int MAXC2, int MAXV>
__global__ void __launch_bounds__(256) mlp_weighted_kernel(
    const float* __restrict__ P, int C, int bf16, const float* __restrict__ rx,
    const float4* __restrict__ geom, const float* __restrict__ base, int K,
    const float* __restrict__ W, int v0, int nv, const int* __restrict__ rx_view,
    const float* __restrict__ glob, int Mpart, const int* __restrict__ n_dev,
    float* __restrict__ part) {
  extern __shared__ float sw[];  // l_w1 [64*6], l_b1 [64], l_w2 [4C*64], l_b2 [4C]
  __shared__ float red[8][MAXC2];
  const int j = blockIdx.y, chunk = blockIdx.x;
  if (n_dev && j >= *n_dev) return;
  constexpr int H = 64;
  const int n4 = 4 * C, twoC = 2 * C;
  const int off_l = H * 3 + H + n4 * H + n4;  // l_w1 offset in the flat parameters
  const int nw = H * 6 + H + n4 * H + n4;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) {
    float v = P[off_l + e];
    const bool is_w = e < H * 6 || (e >= H * 7 && e < H * 7 + n4 * H);
    sw[e] = (is_w && bf16) ? __bfloat162float(__float2bfloat16_rn(v)) : v;
  }
  __syncthreads();
  const float* W1 = sw;
  const float* B1 = W1 + H * 6;
  const float* W2 = B1 + H;
  const float* B2 = W2 + n4 * H;
  auto rb = [&](float x) { return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x; };
  const int vj = rx_view ? rx_view[j] : v0;
  const int nvj = rx_view ? 1 : nv;
  const float rxj = rx[3 * j], ryj = rx[3 * j + 1], rzj = rx[3 * j + 2];
  const float* gj = glob + static_cast<size_t>(j) * n4;
  const int k0 = chunk * kMwChunk, k1 = min(K, k0 + kMwChunk);
  float acc[MAXV][MAXC2];
#pragma unroll
  for (int q = 0; q < MAXV; ++q)
#pragma unroll
    for (int e = 0; e < MAXC2; ++e) acc[q][e] = 0.0f;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    float wv[MAXV];
    bool any = false;
#pragma unroll
    for (int q = 0; q < MAXV; ++q) {
      wv[q] = q < nvj ? W[static_cast<size_t>(vj + q) * K + k] : 0.0f;
      any |= wv[q] != 0.0f;
    }
    if (!any) continue;
    const float4 p = geom[3 * k];
    const float vx = rxj - p.x, vy = ryj - p.y, vz = rzj - p.z;
    const float d = sqrtf(vx * vx + vy * vy + vz * vz);
    const float inv = 1.0f / d;
    const float x[6] = {rb(vx * inv), rb(vy * inv), rb(vz * inv), rb(d), 1.0f, 0.0f};
    float h[H];
#pragma unroll
    for (int u = 0; u < H; ++u) {
      float a = B1[u];
#pragma unroll
      for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
      h[u] = rb(fmaxf(a, 0.0f));
    }
#pragma unroll
    for (int c = 0; c < MAXC2 / 2; ++c) {
      if (c >= C) break;
      float ol[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float* w = W2 + (4 * c + q) * H;
        float a = B2[4 * c + q];
#pragma unroll
        for (int u = 0; u < H; ++u) a = fmaf(w[u], h[u], a);
        ol[q] = a;
      }
      const float pr = base[(static_cast<size_t>(k) * C + c) * 2 + 0];
      const float pi = base[(static_cast<size_t>(k) * C + c) * 2 + 1];
      const float agr = 1.0f + gj[4 * c + 0], agi = gj[4 * c + 1];
      const float ur = agr * pr - agi * pi + gj[4 * c + 2];
      const float ui = agr * pi + agi * pr + gj[4 * c + 3];
      const float alr = 1.0f + ol[0], ali = ol[1];
      const float sr = alr * ur - ali * ui + ol[2];
      const float si = alr * ui + ali * ur + ol[3];
#pragma unroll
      for (int q = 0; q < MAXV; ++q) {
        acc[q][2 * c] = fmaf(wv[q], sr, acc[q][2 * c]);
        acc[q][2 * c + 1] = fmaf(wv[q], si, acc[q][2 * c + 1]);
      }
    }
  }
  // fixed-order block reduction: warp butterflies, then warps in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < MAXV; ++q) {
    if (q >= nvj) break;
#pragma unroll
    for (int e = 0; e < MAXC2; ++e) {
      float y = acc[q][e];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
      if (lane == 0) red[warp][e] = y;
    }
    __syncthreads();
    if (threadIdx.x < twoC) {
      float y = 0.0f;
      for (int w = 0; w < 8; ++w) y += red[w][threadIdx.x];
      const int vv = rx_view ? 0 : q;  // ragged: one slot per receiver
      part[((static_cast<size_t>(chunk) * gridDim.y + j) * Mpart + (rx_view ? 0 : v0) + vv) * twoC +
           threadIdx.x] = y;
    }
    __syncthreads();
  }
}

size_t mlp_weighted_tmp_floats(int M, int K, int N, int C) {
  const size_t nchunks = (K + kMwChunk - 1) / kMwChunk;
  return nchunks * N * static_cast<size_t>(M) * 2 * C;
}

template <int MAXC2, int MAXV>
static void launch_mw(const MlpParams& m, const float* rx, int N, const float4* geom,
                      const float* base, int K, const float* W, int v0, int nv,
                      const int* rx_view, const float* glob, int Mpart, const int* n_dev,
                      float* part, cudaStream_t s) {
  const int nchunks = (K + kMwChunk - 1) / kMwChunk;
  const size_t smem = sizeof(float) * (64 * 7 + 4 * m.C * 64 + 4 * m.C);
  cudaFuncSetAttribute(mlp_weighted_kernel<MAXC2, MAXV>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  mlp_weighted_kernel<MAXC2, MAXV><<<dim3(nchunks, N), 256, smem, s>>>(
      m.p, m.C, m.bf16, rx, geom, base, K, W, v0, nv, rx_view, glob, Mpart, n_dev, part);
  note_launches(1);
}

// Fused MLP + weighted sum for all (view, receiver) pairs (rx_view == NULL,
// M views) or one view per receiver (rx_view[j]); then the chunk sums are
// added in order into csi[Mpart][N][C][2] / rssi (Mpart = M, or 1 per
// receiver in the ragged case, laid out as [N][C][2]).
void launch_mlp_weighted(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, const float* W, int M, const int* rx_view,
                         const float* glob, float* tmp, float* csi, float* rssi,
                         const int* n_dev, cudaStream_t s) {
  const int Mpart = rx_view ? 1 : M;
  const int C2 = 2 * m.C;
  // views per pass: up to 8 for C <= 4, one at a time for wider channels
  const int vstep = C2 <= 8 ? kMwMaxViews : 1;
  for (int v0 = 0; v0 < (rx_view ? 1 : M); v0 += vstep) {
    const int nv = rx_view ? 1 : min(vstep, M - v0);
    if (C2 <= 2)
      launch_mw<2, kMwMaxViews>(m, rx, N, geom, base, K, W, v0, nv, rx_view, glob, Mpart, n_dev, tmp, s);
    else if (C2 <= 8)
      launch_mw<8, kMwMaxViews>(m, rx, N, geom, base, K, W, v0, nv, rx_view, glob, Mpart, n_dev, tmp, s);
    else
      launch_mw<104, 1>(m, rx, N, geom, base, K, W, v0, nv, rx_view, glob, Mpart, n_dev, tmp, s);
  }
  const int nchunks = (K + kMwChunk - 1) / kMwChunk;
  const int n = Mpart * N * m.C;
  // weighted_sum_finish_kernel reads part[chunk][j][v][2C]; for the ragged
  // case that is [chunk][j][1][2C] and the output [1][N][C][2] = [N][C][2]
  weighted_sum_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(tmp, nchunks, N, Mpart, m.C, csi,
                                                             rssi);
  note_launches(1);
}

}  // namespace rxgs
