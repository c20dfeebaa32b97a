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
constexpr int kWsChunk = 1024;   // Gaussians per block
constexpr int kWsSub = 256;      // Gaussians per shared-memory stage
constexpr int kWsMaxViews = 16;  // views handled per pass

// Block (chunk of 1024 Gaussians, 32 complex columns q = (j, c)), eight
// threads per column: sub-lane u takes the column's Gaussians
// k0 + 4u + 32i, four at a time, so one warp load covers four rows x 256
// contiguous bytes (few pages per instruction: the rows of a 1M-Gaussian
// radiance are 8 MB apart).  The chunk's visibility weights are staged 256
// Gaussians at a time in shared memory as [view][k] (16-byte reads, eight
// distinct per quarter warp); all eight loads of a stage are issued before
// its products, and the eight sub-lanes' sums are added by shuffles at the
// end (fixed order).  With C = 1 (K even) four Gaussians are 32 contiguous
// bytes (two 16-byte loads).
constexpr int kWsCols = 32;      // complex columns per block
constexpr int kWsPer = kWsSub / 32;  // four-Gaussian groups per sub-lane and stage

template <bool kVec>
__device__ __forceinline__ void ws_load4(const float2* col, int k, int kk, int kn, int C,
                                         bool act, float2 (&sv)[4]) {
  if (kVec && act && kk + 4 <= kn) {
    const float4 a4 = *reinterpret_cast<const float4*>(col + k);
    const float4 b4 = *reinterpret_cast<const float4*>(col + k + 2);
    sv[0] = make_float2(a4.x, a4.y);
    sv[1] = make_float2(a4.z, a4.w);
    sv[2] = make_float2(b4.x, b4.y);
    sv[3] = make_float2(b4.z, b4.w);
  } else {
#pragma unroll
    for (int x = 0; x < 4; ++x)
      sv[x] = (act && kk + x < kn) ? col[static_cast<size_t>(k + x) * C] : make_float2(0.f, 0.f);
  }
}

template <bool kVec>
__global__ void __launch_bounds__(256, 2) weighted_sum_kernel(const float* __restrict__ rad, int N,
                                                           int K, int C,
                                                           const float* __restrict__ W, int M,
                                                           int v0, int nv,
                                                           float* __restrict__ part) {
  __shared__ __align__(16) float sW[kWsMaxViews][kWsSub];
  const int chunk = blockIdx.x, t = threadIdx.x, u = t & 7;
  const int ncq = N * C;
  const int qcol = blockIdx.y * kWsCols + (t >> 3);
  const bool act = qcol < ncq;
  const int jq = act ? qcol / C : 0, cq = act ? qcol - jq * C : 0;
  const float2* col = reinterpret_cast<const float2*>(rad) + static_cast<size_t>(jq) * K * C + cq;
  const int k0 = chunk * kWsChunk, k1 = min(K, k0 + kWsChunk);
  float acc[kWsMaxViews][2];
#pragma unroll
  for (int v = 0; v < kWsMaxViews; ++v) acc[v][0] = acc[v][1] = 0.0f;
  for (int ks = k0; ks < k1; ks += kWsSub) {
    const int kn = min(kWsSub, k1 - ks);
    // this stage's radiance first (in flight while the weights are staged)
    float2 sv[kWsPer][4];
#pragma unroll
    for (int i = 0; i < kWsPer; ++i) {
      const int kk = 32 * i + 4 * u;
      ws_load4<kVec>(col, ks + kk, kk, kn, C, act, sv[i]);
    }
    __syncthreads();  // the previous stage is consumed
#pragma unroll
    for (int v = 0; v < kWsMaxViews; ++v)
      sW[v][t] = (v < nv && t < kn) ? W[static_cast<size_t>(v0 + v) * K + ks + t] : 0.0f;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kWsPer; ++i) {
      const int kk = 32 * i + 4 * u;
#pragma unroll
      for (int v = 0; v < kWsMaxViews; ++v) {
        const float4 w4 = *reinterpret_cast<const float4*>(&sW[v][kk]);
        float re = acc[v][0], im = acc[v][1];
        re = fmaf(w4.x, sv[i][0].x, re);
        im = fmaf(w4.x, sv[i][0].y, im);
        re = fmaf(w4.y, sv[i][1].x, re);
        im = fmaf(w4.y, sv[i][1].y, im);
        re = fmaf(w4.z, sv[i][2].x, re);
        im = fmaf(w4.z, sv[i][2].y, im);
        re = fmaf(w4.w, sv[i][3].x, re);
        im = fmaf(w4.w, sv[i][3].y, im);
        acc[v][0] = re;
        acc[v][1] = im;
      }
    }
  }
  // the eight sub-lanes of a column (lanes 8a .. 8a + 7 of the warp)
#pragma unroll
  for (int v = 0; v < kWsMaxViews; ++v)
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) acc[v][e] += __shfl_xor_sync(0xffffffffu, acc[v][e], o);
  if (!act || u != 0) return;
  const int twoC = 2 * C;
#pragma unroll
  for (int v = 0; v < kWsMaxViews; ++v) {
    if (v >= nv) break;
    float* dst = part + ((static_cast<size_t>(chunk) * N + jq) * M + v0 + v) * twoC + 2 * cq;
    dst[0] = acc[v][0];
    dst[1] = acc[v][1];
  }
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

bool weighted_sum_supported(int C) { return C >= 1; }

void launch_weighted_sum(const float* rad, int N, int K, int C, const float* W, int M, float* tmp,
                         float* csi, float* rssi, cudaStream_t s) {
  const int nchunks = (K + kWsChunk - 1) / kWsChunk;
  const unsigned colblocks = static_cast<unsigned>((N * C + kWsCols - 1) / kWsCols);
  // 16-byte loads need each receiver row of a single channel to start on 16 B
  const bool vec = C == 1 && K % 2 == 0 && (reinterpret_cast<uintptr_t>(rad) & 15) == 0;
  for (int v0 = 0; v0 < M; v0 += kWsMaxViews) {
    const int nv = min(kWsMaxViews, M - v0);
    if (vec)
      weighted_sum_kernel<true><<<dim3(nchunks, colblocks), 256, 0, s>>>(rad, N, K, C, W, M, v0,
                                                                          nv, tmp);
    else
      weighted_sum_kernel<false><<<dim3(nchunks, colblocks), 256, 0, s>>>(rad, N, K, C, W, M, v0,
                                                                           nv, tmp);
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
    // channels unrolled for the narrow spectra only (wide float32 spectra
    // would unroll 52 x 256 FMAs)
#pragma unroll(MAXC2 <= 8 ? MAXC2 / 2 : 1)
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

size_t mlp_weighted_tc_extra_floats(int C);

size_t mlp_weighted_tmp_floats(int M, int K, int N, int C) {
  const size_t nchunks = (K + kMwChunk - 1) / kMwChunk;
  // chunk partials, plus room for packed tensor-core weight fragments
  return nchunks * N * static_cast<size_t>(M) * 2 * C + mlp_weighted_tc_extra_floats(C);
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
bool launch_mlp_weighted_tc(const MlpParams& m, const float* rx, int N, const float4* geom,
                            const float* base, int K, const float* W, int M, const int* rx_view,
                            const float* glob, float* tmp, float* csi, float* rssi,
                            const int* n_dev, cudaStream_t s);

void launch_mlp_weighted(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, const float* W, int M, const int* rx_view,
                         const float* glob, float* tmp, float* csi, float* rssi,
                         const int* n_dev, cudaStream_t s) {
  // bf16 MLPs: output layer on tensor cores
  if (launch_mlp_weighted_tc(m, rx, N, geom, base, K, W, M, rx_view, glob, tmp, csi, rssi, n_dev, s))
    return;
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

namespace rxgs {

// --------------------------- bf16 MLP on tensor cores, fused with the sum
// Same result as mlp_weighted in bf16 mode (inputs, weights and hidden
// activations rounded to bf16, float32 accumulation), with the output layer
// [16 Gaussians x 64] x [64 x 4C] on warp-level tensor-core MMAs
// (mma.sync m16n8k16 bf16 -> f32).  A pack kernel lays W2^T out once per
// call as the MMA's B fragments (bf16 pairs); every block copies them to
// shared memory.  Block (chunk of 4096 Gaussians, receiver j), each warp a
// 512-Gaussian segment of the chunk:
//   1. the warp compacts its segment's Gaussians with W[v][k] != 0 (ballots
//      over coalesced reads, ascending k);
//   2. 16 listed Gaussians at a time: lanes compute the hidden layer (bf16)
//      into shared memory, the MMAs produce the local (alpha, beta) of every
//      channel, and lanes holding alpha combine them with beta (from the
//      neighbour lane), phi_base and the global branch into s, accumulating
//      W s per channel;
//   3. lanes, then warps, are summed in a fixed order into part[chunk][j].
constexpr int kTcMaxNT = 26;  // 8-wide output tiles: 4C <= 208, C <= 52
constexpr int kTcHStride = 72;
constexpr int kTcSeg = kMwChunk / 8;  // Gaussians per warp segment

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

static int tc_tiles(int C) { return (4 * C + 7) / 8; }
static size_t tc_pack_words(int C) { return static_cast<size_t>(tc_tiles(C)) * 4 * 32 * 2; }

// B fragments of W2^T (element (k, n) = W2[n][k]), [NT][4 k-steps][32 lanes][2]
__global__ void mlp_pack_w2_kernel(const float* __restrict__ P, int C, uint32_t* __restrict__ out) {
  constexpr int H = 64;
  const int n4 = 4 * C, NT = (n4 + 7) / 8;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NT * 4 * 32) return;
  const float* W2 = P + (H * 3 + H + n4 * H + n4) + H * 7;
  const int nt = e / 128, ks = (e / 32) % 4, l = e % 32;
  const int n = nt * 8 + (l >> 2), k0 = ks * 16 + (l & 3) * 2;
  float w[4] = {0.f, 0.f, 0.f, 0.f};
  if (n < n4) {
    w[0] = W2[n * H + k0];
    w[1] = W2[n * H + k0 + 1];
    w[2] = W2[n * H + k0 + 8];
    w[3] = W2[n * H + k0 + 9];
  }
  out[2 * e + 0] = pack_bf16(w[0], w[1]);
  out[2 * e + 1] = pack_bf16(w[2], w[3]);
}

__global__ void __launch_bounds__(256, 2) mlp_weighted_tc_kernel(
    const float* __restrict__ P, int C, const uint32_t* __restrict__ packed,
    const float* __restrict__ rx, const float4* __restrict__ geom,
    const float* __restrict__ base, int K, const float* __restrict__ W, int v0,
    const int* __restrict__ rx_view, const float* __restrict__ glob, int Mpart,
    const int* __restrict__ n_dev, float* __restrict__ part) {
  constexpr int H = 64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n4 = 4 * C, NT = (n4 + 7) / 8;
  uint32_t* sBf = reinterpret_cast<uint32_t*>(smem_raw);               // [NT][4][32][2]
  float* sW1 = reinterpret_cast<float*>(sBf + NT * 4 * 32 * 2);         // [64][6] bf16-rounded
  float* sB1 = sW1 + H * 6;                                             // [64]
  float* sB2 = sB1 + H;                                                 // [NT*8]
  float* sG = sB2 + NT * 8;                                             // [4C] global branch
  __nv_bfloat16* sH = reinterpret_cast<__nv_bfloat16*>(sG + n4);         // [8 warps][16][72]
  int* sList = reinterpret_cast<int*>(sH + 8 * 16 * kTcHStride);         // [8 warps][512]
  __shared__ float sRed[8][2 * 52];
  const int j = blockIdx.y, chunk = blockIdx.x;
  if (n_dev && j >= *n_dev) return;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int off_l = H * 3 + H + n4 * H + n4;  // l_w1 in the flat parameters
  {
    const int n16 = NT * 4 * 32 * 2 / 4;  // 16-byte pieces of the packed fragments
    for (int e = t; e < n16; e += 256) cp_async16(&sBf[4 * e], &packed[4 * e], true);
    cp_async_commit();
  }
  for (int e = t; e < H * 6; e += 256) sW1[e] = __bfloat162float(__float2bfloat16_rn(P[off_l + e]));
  for (int e = t; e < H; e += 256) sB1[e] = P[off_l + H * 6 + e];
  for (int e = t; e < NT * 8; e += 256) sB2[e] = e < n4 ? P[off_l + H * 7 + n4 * H + e] : 0.0f;
  for (int e = t; e < n4; e += 256) sG[e] = glob[static_cast<size_t>(j) * n4 + e];
  const int vj = rx_view ? rx_view[j] : v0;
  const float* Wv = W + static_cast<size_t>(vj) * K;
  // ---- per-warp compaction of the segment's non-zero weights (ascending k)
  int* wl = sList + warp * kTcSeg;
  const int s0 = chunk * kMwChunk + warp * kTcSeg;
  int nact = 0;
#pragma unroll 4
  for (int r = 0; r < kTcSeg / 32; ++r) {
    const int k = s0 + r * 32 + lane;
    const bool nz = k < K && Wv[k] != 0.0f;
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (nz) wl[nact + __popc(bal & ((1u << lane) - 1u))] = k;
    nact += __popc(bal);
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- 16-Gaussian tiles of the warp's list
  const float rxj = rx[3 * j], ryj = rx[3 * j + 1], rzj = rx[3 * j + 2];
  const int g = lane >> 2, tig = lane & 3;
  float acc[kTcMaxNT][2];
#pragma unroll
  for (int nt = 0; nt < kTcMaxNT; ++nt) acc[nt][0] = acc[nt][1] = 0.0f;
  __nv_bfloat16* hW = sH + warp * 16 * kTcHStride;
  for (int tile = 0; tile * 16 < nact; ++tile) {
    // hidden layer: lane computes units [32*half, 32*half + 32) of row r
    {
      const int r = lane & 15, half = lane >> 4;
      const int li = tile * 16 + r;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      const bool ok = li < nact;
      if (ok) {
        const float4 p = geom[3 * wl[li]];
        const float vx = rxj - p.x, vy = ryj - p.y, vz = rzj - p.z;
        const float d = sqrtf(vx * vx + vy * vy + vz * vz);
        const float inv = 1.0f / d;
        x[0] = __bfloat162float(__float2bfloat16_rn(vx * inv));
        x[1] = __bfloat162float(__float2bfloat16_rn(vy * inv));
        x[2] = __bfloat162float(__float2bfloat16_rn(vz * inv));
        x[3] = __bfloat162float(__float2bfloat16_rn(d));
      }
#pragma unroll 8
      for (int uu = 0; uu < 32; ++uu) {
        const int u = half * 32 + uu;
        float a = sB1[u];
#pragma unroll
        for (int i = 0; i < 4; ++i) a = fmaf(sW1[u * 6 + i], x[i], a);
        a += sW1[u * 6 + 4];  // inputs 4 and 5 are the constants 1 and 0
        hW[r * kTcHStride + u] = __float2bfloat16_rn(ok ? fmaxf(a, 0.0f) : 0.0f);
      }
    }
    __syncwarp();
    // A fragments of the 16 x 64 hidden tile
    uint32_t af[4][4];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int c0 = ks * 16 + tig * 2;
      af[ks][0] = *reinterpret_cast<const uint32_t*>(&hW[g * kTcHStride + c0]);
      af[ks][1] = *reinterpret_cast<const uint32_t*>(&hW[(g + 8) * kTcHStride + c0]);
      af[ks][2] = *reinterpret_cast<const uint32_t*>(&hW[g * kTcHStride + c0 + 8]);
      af[ks][3] = *reinterpret_cast<const uint32_t*>(&hW[(g + 8) * kTcHStride + c0 + 8]);
    }
    __syncwarp();  // hW is rewritten by the next tile
    const int la = tile * 16 + g, lb = la + 8;
    const int ka = la < nact ? wl[la] : -1, kb = lb < nact ? wl[lb] : -1;
    const float wa = ka >= 0 ? Wv[ka] : 0.0f, wb = kb >= 0 ? Wv[kb] : 0.0f;
#pragma unroll
    for (int nt = 0; nt < kTcMaxNT; ++nt) {
      if (nt >= NT) break;
      float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint2 bp = *reinterpret_cast<const uint2*>(&sBf[((nt * 4 + ks) * 32 + lane) * 2]);
        mma_bf16_16816(d, af[ks], bp.x, bp.y);
      }
      const int col = nt * 8 + tig * 2;
      d[0] += sB2[col];
      d[1] += sB2[col + 1];
      d[2] += sB2[col];
      d[3] += sB2[col + 1];
      // beta of the same channel sits in the neighbouring lane (tig + 1)
      const float b0 = __shfl_xor_sync(0xffffffffu, d[0], 1);
      const float b1 = __shfl_xor_sync(0xffffffffu, d[1], 1);
      const float b2 = __shfl_xor_sync(0xffffffffu, d[2], 1);
      const float b3 = __shfl_xor_sync(0xffffffffu, d[3], 1);
      const int ch = 2 * nt + (tig >> 1);
      if ((tig & 1) == 0 && ch < C) {
        const float agr = 1.0f + sG[4 * ch + 0], agi = sG[4 * ch + 1];
        const float bgr = sG[4 * ch + 2], bgi = sG[4 * ch + 3];
        if (ka >= 0) {
          const float2 ph = *reinterpret_cast<const float2*>(&base[(static_cast<size_t>(ka) * C + ch) * 2]);
          const float ur = agr * ph.x - agi * ph.y + bgr, ui = agr * ph.y + agi * ph.x + bgi;
          const float alr = 1.0f + d[0], ali = d[1];
          acc[nt][0] = fmaf(wa, alr * ur - ali * ui + b0, acc[nt][0]);
          acc[nt][1] = fmaf(wa, alr * ui + ali * ur + b1, acc[nt][1]);
        }
        if (kb >= 0) {
          const float2 ph = *reinterpret_cast<const float2*>(&base[(static_cast<size_t>(kb) * C + ch) * 2]);
          const float ur = agr * ph.x - agi * ph.y + bgr, ui = agr * ph.y + agi * ph.x + bgi;
          const float alr = 1.0f + d[2], ali = d[3];
          acc[nt][0] = fmaf(wb, alr * ur - ali * ui + b2, acc[nt][0]);
          acc[nt][1] = fmaf(wb, alr * ui + ali * ur + b3, acc[nt][1]);
        }
      }
    }
  }
  // ---- lanes with the same tig (rows g = 0..7), then warps, in fixed order
#pragma unroll
  for (int nt = 0; nt < kTcMaxNT; ++nt) {
    if (nt >= NT) break;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float y = acc[nt][e];
      y += __shfl_xor_sync(0xffffffffu, y, 4);
      y += __shfl_xor_sync(0xffffffffu, y, 8);
      y += __shfl_xor_sync(0xffffffffu, y, 16);
      acc[nt][e] = y;
    }
    const int ch = 2 * nt + (tig >> 1);
    if (g == 0 && (tig & 1) == 0 && ch < C) {
      sRed[warp][2 * ch] = acc[nt][0];
      sRed[warp][2 * ch + 1] = acc[nt][1];
    }
  }
  __syncthreads();
  if (t < 2 * C) {
    float y = 0.0f;
    for (int w = 0; w < 8; ++w) y += sRed[w][t];
    part[((static_cast<size_t>(chunk) * gridDim.y + j) * Mpart + (rx_view ? 0 : v0)) * 2 * C + t] = y;
  }
}

size_t mlp_weighted_tc_smem(int C) {
  const int n4 = 4 * C, NT = (n4 + 7) / 8;
  return sizeof(uint32_t) * NT * 4 * 32 * 2 + sizeof(float) * (64 * 6 + 64 + NT * 8 + n4) +
         sizeof(__nv_bfloat16) * 8 * 16 * kTcHStride + sizeof(int) * kMwChunk;
}

// Wide spectra through tensor cores (bf16 MLPs with 4 < C <= 52).  The
// packed W2^T fragments sit at the start of tmp, the chunk partials after.
bool mlp_weighted_uses_tc(const MlpParams& m) { return m.bf16 && m.C > 4 && m.C <= 52; }

bool launch_mlp_weighted_tc(const MlpParams& m, const float* rx, int N, const float4* geom,
                            const float* base, int K, const float* W, int M, const int* rx_view,
                            const float* glob, float* tmp, float* csi, float* rssi,
                            const int* n_dev, cudaStream_t s) {
  if (!mlp_weighted_uses_tc(m)) return false;
  uint32_t* packed = reinterpret_cast<uint32_t*>(tmp);
  float* part = tmp + tc_pack_words(m.C);
  const int nfrag = tc_tiles(m.C) * 4 * 32;
  mlp_pack_w2_kernel<<<(nfrag + 255) / 256, 256, 0, s>>>(m.p, m.C, packed);
  note_launches(1);
  const int Mpart = rx_view ? 1 : M;
  const int nchunks = (K + kMwChunk - 1) / kMwChunk;
  const size_t smem = mlp_weighted_tc_smem(m.C);
  cudaFuncSetAttribute(mlp_weighted_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  for (int v0 = 0; v0 < (rx_view ? 1 : M); ++v0) {
    mlp_weighted_tc_kernel<<<dim3(nchunks, N), 256, smem, s>>>(
        m.p, m.C, packed, rx, geom, base, K, W, v0, rx_view, glob, Mpart, n_dev, part);
    note_launches(1);
  }
  const int n = Mpart * N * m.C;
  weighted_sum_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(part, nchunks, N, Mpart, m.C, csi,
                                                             rssi);
  note_launches(1);
  return true;
}

size_t mlp_weighted_tc_extra_floats(int C) { return tc_pack_words(C); }

}  // namespace rxgs
