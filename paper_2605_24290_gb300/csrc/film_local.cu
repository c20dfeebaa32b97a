// film_local.cu -- the local branch of the receiver conditioning (Eq. local)
// composed with the global FiLM branch over the FLE components (Eq.
// combined_local, Sec. 3.3.2):
//   phi_jkl = (1 + alpha_jk) [(1 + a_jl) phi_base,kl + b_jl] + beta_jk
// (alpha_jk, beta_jk) = MLP_loc([v_hat, d, T, rho_bar]) per (receiver j,
// Gaussian k): Linear(6, 64) -> ReLU -> Linear(64, 4), the scene's
// conditioning MLP's local branch with one channel, outputs (alpha.re,
// alpha.im, beta.re, beta.im); v_hat and d from the Gaussian to the receiver,
// (T, rho_bar) the occlusion probes (or (1, 0) for a clear scene).
//
// Forward: local_factors (one thread per pair, weights in shared memory);
// the FiLM coefficient kernel applies them (fle_tc.cu).  Backward, from the
// composed coefficients' gradient G'[j][k][.][l]:
//   dL/dalpha_jk = sum_l conj(c_jkl) G'_jkl,  dL/dbeta_jk = sum_l G'_jkl
//   G_jkl = conj(1 + alpha_jk) G'_jkl   (in place: the FiLM fold's input)
// with c the FiLM-modulated coefficient (film_local_grad: one warp per pair,
// lanes over components), then the local MLP's weight gradients summed over
// all pairs (local_mlp_backward: lanes = hidden units, a block's warps
// reduced in shared memory, one float atomic per weight and block).
#include "rxgs_internal.h"

namespace rxgs {

namespace {

constexpr int kH = 64;                       // hidden units of the local branch
constexpr int kLocW = kH * 6 + kH + 4 * kH + 4;  // l_w1, l_b1, l_w2, l_b2
constexpr int kPairsPerBlock = 4096;

// offset of the local branch in the flat parameters (one channel):
// g_w1 [64][3], g_b1 [64], g_w2 [4][64], g_b2 [4], then l_w1 ...
constexpr int kLocOff = kH * 3 + kH + 4 * kH + 4;

__device__ __forceinline__ void local_inputs(const float* rx, const float4* geom, const float2* feat,
                                             int K, int j, int k, float (&x)[6]) {
  const float4 p = geom[3 * k];
  const float vx = rx[3 * j + 0] - p.x, vy = rx[3 * j + 1] - p.y, vz = rx[3 * j + 2] - p.z;
  const float d = sqrtf(vx * vx + vy * vy + vz * vz);
  const float inv = 1.0f / d;
  const float2 oc = feat ? feat[static_cast<size_t>(j) * K + k] : make_float2(1.0f, 0.0f);
  x[0] = vx * inv;
  x[1] = vy * inv;
  x[2] = vz * inv;
  x[3] = d;
  x[4] = oc.x;
  x[5] = oc.y;
}

__global__ void __launch_bounds__(256) local_factors_kernel(const float* __restrict__ P,
                                                            const float* __restrict__ rx, int N,
                                                            const float4* __restrict__ geom, int K,
                                                            const float2* __restrict__ feat,
                                                            float4* __restrict__ loc) {
  __shared__ float sw[kLocW];
  for (int e = threadIdx.x; e < kLocW; e += blockDim.x) sw[e] = P[kLocOff + e];
  __syncthreads();
  const float* W1 = sw;
  const float* B1 = W1 + kH * 6;
  const float* W2 = B1 + kH;
  const float* B2 = W2 + 4 * kH;
  const size_t pair = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;  // (j, k)
  if (pair >= static_cast<size_t>(N) * K) return;
  const int j = static_cast<int>(pair / K), k = static_cast<int>(pair % K);
  float x[6];
  local_inputs(rx, geom, feat, K, j, k, x);
  float o[4] = {B2[0], B2[1], B2[2], B2[3]};
#pragma unroll 8
  for (int u = 0; u < kH; ++u) {
    float a = B1[u];
#pragma unroll
    for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
    const float h = fmaxf(a, 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = fmaf(W2[q * kH + u], h, o[q]);
  }
  loc[pair] = make_float4(o[0], o[1], o[2], o[3]);
}

// one warp per pair (j, k): lanes over the components
__global__ void __launch_bounds__(256) film_local_grad_kernel(float* __restrict__ G,
                                                              const float* __restrict__ base,
                                                              const float4* __restrict__ ab,
                                                              const float4* __restrict__ loc,
                                                              int N, int K, int L,
                                                              float4* __restrict__ d_loc) {
  const size_t pair = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pair >= static_cast<size_t>(N) * K) return;
  const int j = static_cast<int>(pair / K), k = static_cast<int>(pair % K);
  const float4 lf = loc[pair];
  const float alr = 1.0f + lf.x, ali = lf.y;
  float* g = G + pair * 2 * L;
  float dar = 0.0f, dai = 0.0f, dbr = 0.0f, dbi = 0.0f;
  for (int l = lane; l < L; l += 32) {
    const float4 q = ab[static_cast<size_t>(j) * L + l];
    const float pr = base[static_cast<size_t>(k) * 2 * L + l];
    const float pi = base[static_cast<size_t>(k) * 2 * L + L + l];
    const float ar = 1.0f + q.x;
    const float cr = fmaf(ar, pr, fmaf(-q.y, pi, q.z));  // c = (1 + a) base + b
    const float ci = fmaf(ar, pi, fmaf(q.y, pr, q.w));
    const float gr = g[l], gi = g[L + l];
    dar = fmaf(cr, gr, fmaf(ci, gi, dar));  // conj(c) G'
    dai = fmaf(cr, gi, fmaf(-ci, gr, dai));
    dbr += gr;
    dbi += gi;
    g[l] = fmaf(alr, gr, ali * gi);        // conj(1 + alpha) G'
    g[L + l] = fmaf(alr, gi, -ali * gr);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    dar += __shfl_xor_sync(0xffffffffu, dar, o);
    dai += __shfl_xor_sync(0xffffffffu, dai, o);
    dbr += __shfl_xor_sync(0xffffffffu, dbr, o);
    dbi += __shfl_xor_sync(0xffffffffu, dbi, o);
  }
  if (lane == 0) d_loc[pair] = make_float4(dar, dai, dbr, dbi);
}

// lanes = hidden units (two per lane), a block takes kPairsPerBlock pairs
__global__ void __launch_bounds__(256) local_mlp_backward_kernel(
    const float* __restrict__ P, const float* __restrict__ rx, int N,
    const float4* __restrict__ geom, int K, const float2* __restrict__ feat,
    const float4* __restrict__ d_loc, float* __restrict__ grad) {
  __shared__ float sw[kLocW];
  __shared__ float red[8][kLocW];
  for (int e = threadIdx.x; e < kLocW; e += blockDim.x) sw[e] = P[kLocOff + e];
  __syncthreads();
  const float* W1 = sw;
  const float* B1 = W1 + kH * 6;
  const float* W2 = B1 + kH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t npairs = static_cast<size_t>(N) * K;
  const size_t p0 = static_cast<size_t>(blockIdx.x) * kPairsPerBlock;
  const size_t p1 = p0 + kPairsPerBlock < npairs ? p0 + kPairsPerBlock : npairs;
  float dw1[2][6], db1[2], dw2[4][2], db2[4];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    db1[s] = 0.0f;
#pragma unroll
    for (int i = 0; i < 6; ++i) dw1[s][i] = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) dw2[q][s] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) db2[q] = 0.0f;
  for (size_t pair = p0 + warp; pair < p1; pair += 8) {
    const int j = static_cast<int>(pair / K), k = static_cast<int>(pair % K);
    float x[6];
    local_inputs(rx, geom, feat, K, j, k, x);  // the same address in every lane
    const float4 dl = d_loc[pair];
    const float dol[4] = {dl.x, dl.y, dl.z, dl.w};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int u = lane + 32 * s;
      float a = B1[u];
#pragma unroll
      for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
      const float h = fmaxf(a, 0.0f);
      float dh = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        dw2[q][s] = fmaf(dol[q], h, dw2[q][s]);
        dh = fmaf(dol[q], W2[q * kH + u], dh);
      }
      dh = a > 0.0f ? dh : 0.0f;
      db1[s] += dh;
#pragma unroll
      for (int i = 0; i < 6; ++i) dw1[s][i] = fmaf(dh, x[i], dw1[s][i]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) db2[q] += dol[q];
  }
  // warps' sums in shared memory, then the block's sum in warp order
  float* r = red[warp];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int u = lane + 32 * s;
#pragma unroll
    for (int i = 0; i < 6; ++i) r[u * 6 + i] = dw1[s][i];
    r[kH * 6 + u] = db1[s];
#pragma unroll
    for (int q = 0; q < 4; ++q) r[kH * 7 + q * kH + u] = dw2[q][s];
  }
  if (lane < 4) r[kH * 7 + 4 * kH + lane] = db2[lane];
  __syncthreads();
  for (int e = threadIdx.x; e < kLocW; e += blockDim.x) {
    float y = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) y += red[w][e];
    if (y != 0.0f) atomicAdd(&grad[kLocOff + e], y);
  }
}

}  // namespace

bool local_branch_supported(int hidden, int C) { return hidden == kH && C == 1; }

void launch_local_factors(const float* mlp, const float* rx, int N, const float4* geom, int K,
                          const float2* feat, float4* loc, cudaStream_t s) {
  const size_t n = static_cast<size_t>(N) * K;
  if (n == 0) return;
  local_factors_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(mlp, rx, N, geom, K,
                                                                             feat, loc);
  note_launches(1);
}

void launch_film_local_backward(float* G, const float* base, const float4* ab, const float4* loc,
                                const float* mlp, const float* rx, int N, const float4* geom,
                                int K, int lmax, const float2* feat, float4* d_loc,
                                float* grad_mlp, cudaStream_t s) {
  const size_t n = static_cast<size_t>(N) * K;
  if (n == 0) return;
  const int L = (lmax + 1) * (lmax + 1);
  film_local_grad_kernel<<<static_cast<unsigned>((n * 32 + 255) / 256), 256, 0, s>>>(
      G, base, ab, loc, N, K, L, d_loc);
  note_launches(1);
  if (grad_mlp) {
    local_mlp_backward_kernel<<<static_cast<unsigned>((n + kPairsPerBlock - 1) / kPairsPerBlock),
                                256, 0, s>>>(mlp, rx, N, geom, K, feat, d_loc, grad_mlp);
    note_launches(1);
  }
}

}  // namespace rxgs
