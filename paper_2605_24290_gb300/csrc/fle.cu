// fle.cu -- Fourier-Legendre directional radiance (App. E.2) and its
// gradient, the per-receiver directional signal of Algorithm 1.
//
// For view v (transmitter t_v) and Gaussian k, with u = p_k - t_v, polar
// angle theta (cos theta = u_z / |u|) and azimuth phi (atan2(u_y, u_x)):
//   Y_lm = N_l|m| P_l^|m|(cos theta) e^{i m phi},   component l*l + l + m,
//   s[v][k][j] = sum_lm (a_jk,lm + i b_jk,lm) Y_lm          (forward)
//   dL/d(a + i b)_jk,lm = sum_v g[v][k][j] conj(Y_lm)     (backward)
// with P_l^m by the three-term recurrence (no Condon-Shortley phase) and
// e^{i m phi} by repeated complex multiplication.  The basis depends on the
// transmitter only; for one Gaussian both directions are small dense
// products, [views x L] x [L x receivers] and [receivers x views] x
// [views x L], so a block takes one Gaussian and stages its basis for 32
// views and its coefficients (or gradients) for 64 receivers in shared
// memory; the coefficient tensor is read once for all views.  With the global
// FiLM branch (Eq. film_apply) the coefficients are formed from the base
// coefficients and the per-(receiver, component) modulation while staged,
// and the backward folds the coefficient gradient into the base and
// modulation gradients without storing it.
#include <algorithm>
#include <cmath>

#include "rxgs_internal.h"

namespace rxgs {

constexpr int kFleMaxL = 100;  // lmax <= 9
constexpr int kFleViews = 32;  // views per pass
constexpr int kFleRx = 64;     // receivers per pass
constexpr int kFleStride = kFleMaxL + 1;  // padded row (bank spread)

struct FleNorm {
  float n[kFleMaxL];  // N_l|m| by component index l*l + l + m
};

static FleNorm fle_norm_table(int lmax) {
  FleNorm t{};
  for (int l = 0; l <= lmax; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = m < 0 ? -m : m;
      double ratio = 1.0;  // (l - |m|)! / (l + |m|)!
      for (int q = l - am + 1; q <= l + am; ++q) ratio /= q;
      t.n[l * l + l + m] = static_cast<float>(std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio));
    }
  return t;
}

// The basis of direction u for components 0 .. (lmax+1)^2 - 1 into Y (re, im).
__device__ void fle_basis_dir(float ux, float uy, float uz, int lmax, const FleNorm& nrm,
                              float2* Y) {
  const float rho = sqrtf(ux * ux + uy * uy + uz * uz);
  const float hh = sqrtf(ux * ux + uy * uy);
  // a centre on the transmitter itself (culled by the projection anyway)
  // takes the +z direction
  const float ct = rho > 0.0f ? uz / rho : 1.0f, st = rho > 0.0f ? hh / rho : 0.0f;
  float cp = 1.0f, sp = 0.0f;
  if (hh > 0.0f) {
    cp = ux / hh;
    sp = uy / hh;
  }
  float pmm = 1.0f, er = 1.0f, ei = 0.0f;  // P_m^m and e^{i m phi}
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) {
      pmm *= static_cast<float>(2 * m - 1) * st;
      const float r = er * cp - ei * sp;
      ei = er * sp + ei * cp;
      er = r;
    }
    auto put = [&](int l, float p) {
      const float val = nrm.n[l * l + l + m] * p;
      Y[l * l + l + m] = make_float2(val * er, val * ei);
      if (m > 0) Y[l * l + l - m] = make_float2(val * er, -val * ei);
    };
    put(m, pmm);
    if (m + 1 <= lmax) {
      float p0 = pmm, p1 = static_cast<float>(2 * m + 1) * ct * pmm;
      put(m + 1, p1);
      for (int l = m + 2; l <= lmax; ++l) {
        const float p2 = (static_cast<float>(2 * l - 1) * ct * p1 -
                          static_cast<float>(l + m - 1) * p0) / static_cast<float>(l - m);
        put(l, p2);
        p0 = p1;
        p1 = p2;
      }
    }
  }
}

// kFilm: the coefficients are (1 + a_jl) base_kl + b_jl (Eq. film_apply),
// formed while they are staged; otherwise they are read from coeffs.
template <bool kFilm>
__global__ void __launch_bounds__(256) fle_radiance_kernel(
    const float* __restrict__ coeffs, int N, int K, int lmax, const float4* __restrict__ geom,
    const float* __restrict__ tx, int M, int stride, size_t rad_view, FleNorm nrm,
    float* __restrict__ rad, const float* __restrict__ base, const float4* __restrict__ ab) {
  extern __shared__ __align__(16) unsigned char fle_smem[];
  auto sY = reinterpret_cast<float2(*)[kFleStride]>(fle_smem);                 // [32][101]
  auto sC = reinterpret_cast<float2(*)[kFleStride]>(fle_smem + sizeof(float2) * kFleViews * kFleStride);  // [64][101]
  const int k = blockIdx.x, t = threadIdx.x;
  const int L = (lmax + 1) * (lmax + 1);
  const float4 p = geom[3 * k];
  const int vv = t / 16, jj = t % 16;
  for (int v0 = 0; v0 < M; v0 += kFleViews) {
    const int nv = min(kFleViews, M - v0);
    __syncthreads();
    if (t < nv)
      fle_basis_dir(p.x - tx[3 * (v0 + t)], p.y - tx[3 * (v0 + t) + 1], p.z - tx[3 * (v0 + t) + 2],
                    lmax, nrm, sY[t]);
    for (int j0 = 0; j0 < N; j0 += kFleRx) {
      const int nr = min(kFleRx, N - j0);
      __syncthreads();  // sY is complete; the previous receivers are done with sC
      for (int e = t; e < nr * L; e += 256) {
        const int j = e / L, l = e % L;
        if (kFilm) {
          const float4 q = ab[static_cast<size_t>(j0 + j) * L + l];
          const float pr = base[static_cast<size_t>(k) * 2 * L + l];
          const float pi = base[static_cast<size_t>(k) * 2 * L + L + l];
          const float ar = 1.0f + q.x;
          sC[j][l] = make_float2(fmaf(ar, pr, fmaf(-q.y, pi, q.z)), fmaf(ar, pi, fmaf(q.y, pr, q.w)));
        } else {
          const float* c = coeffs + (static_cast<size_t>(j0 + j) * K + k) * 2 * L;
          sC[j][l] = make_float2(c[l], c[L + l]);
        }
      }
      __syncthreads();
      float ar[2][4], ai[2][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int q = 0; q < 4; ++q) ar[a][q] = ai[a][q] = 0.0f;
      for (int l = 0; l < L; ++l) {
        const float2 y0 = sY[vv][l], y1 = sY[vv + 16][l];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 c = sC[jj + 16 * q][l];
          ar[0][q] = fmaf(c.x, y0.x, fmaf(-c.y, y0.y, ar[0][q]));
          ai[0][q] = fmaf(c.x, y0.y, fmaf(c.y, y0.x, ai[0][q]));
          ar[1][q] = fmaf(c.x, y1.x, fmaf(-c.y, y1.y, ar[1][q]));
          ai[1][q] = fmaf(c.x, y1.y, fmaf(c.y, y1.x, ai[1][q]));
        }
      }
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int v = vv + 16 * a;
        if (v >= nv) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = jj + 16 * q;
          if (j >= nr) continue;
          float* dst = rad + static_cast<size_t>(v0 + v) * rad_view + static_cast<size_t>(k) * stride +
                       2 * (j0 + j);
          *reinterpret_cast<float2*>(dst) = make_float2(ar[a][q], ai[a][q]);
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256) fle_backward_kernel(
    const float* __restrict__ d_rad, int N, int K, int lmax, const float4* __restrict__ geom,
    const float* __restrict__ tx, int M, int stride, size_t rad_view, FleNorm nrm,
    float* __restrict__ grad) {
  __shared__ float2 sY[kFleViews][kFleStride];
  __shared__ float2 sG[kFleViews][kFleRx + 1];
  const int k = blockIdx.x, t = threadIdx.x;
  const int L = (lmax + 1) * (lmax + 1);
  const float4 p = geom[3 * k];
  // receivers jj + 16 q, components ll + 16 r: consecutive lanes take
  // consecutive components of one receiver, so the gradient rows are
  // updated in contiguous segments
  const int ll = t % 16, jj = t / 16;
  constexpr int kR = (kFleMaxL + 15) / 16;
  for (int j0 = 0; j0 < N; j0 += kFleRx) {
    const int nr = min(kFleRx, N - j0);
    float gr[4][kR], gi[4][kR];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < kR; ++r) gr[q][r] = gi[q][r] = 0.0f;
    for (int v0 = 0; v0 < M; v0 += kFleViews) {
      const int nv = min(kFleViews, M - v0);
      __syncthreads();  // the previous pass is done with sY and sG
      if (t < nv)
        fle_basis_dir(p.x - tx[3 * (v0 + t)], p.y - tx[3 * (v0 + t) + 1],
                      p.z - tx[3 * (v0 + t) + 2], lmax, nrm, sY[t]);
      for (int e = t; e < nv * nr; e += 256) {
        const int v = e / nr, j = e % nr;
        const float* g = d_rad + static_cast<size_t>(v0 + v) * rad_view +
                         static_cast<size_t>(k) * stride + 2 * (j0 + j);
        sG[v][j] = make_float2(g[0], g[1]);
      }
      __syncthreads();
      for (int v = 0; v < nv; ++v) {
        float2 gq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) gq[q] = sG[v][min(jj + 16 * q, kFleRx - 1)];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const int l = ll + 16 * r;
          const float2 y = sY[v][l < kFleMaxL ? l : 0];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            // g conj(y): (gr yr + gi yi, gi yr - gr yi)
            gr[q][r] = fmaf(gq[q].x, y.x, fmaf(gq[q].y, y.y, gr[q][r]));
            gi[q][r] = fmaf(gq[q].y, y.x, fmaf(-gq[q].x, y.y, gi[q][r]));
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = jj + 16 * q;
      if (j >= nr) continue;
      float* dst = grad + (static_cast<size_t>(j0 + j) * K + k) * 2 * L;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int l = ll + 16 * r;
        if (l >= L) continue;
        dst[l] += gr[q][r];
        dst[L + l] += gi[q][r];
      }
    }
  }
}

// The FiLM backward (Eq. film_apply): blocks stay resident and take Gaussians
// k = blockIdx.x, + gridDim.x, ... for each pass of 32 receivers.  As in
// fle_backward_kernel, thread (jj, ll) forms G_jkl = sum_v g conj(Y) for
// receivers jj, jj + 16 and components ll + 16 r.  Then
//   dL/dbase_kl = sum_j conj(1 + a_jl) G_jkl   (a warp shuffle and a fixed-order
//                                               sum over the eight warps)
//   dL/da_jl += conj(base_kl) G_jkl, dL/db_jl += G_jkl   (kept in registers
//                                               over the block's Gaussians,
//                                               added to d_ab once per pass)
constexpr int kFbRx = 32;  // receivers per pass

__global__ void __launch_bounds__(256) film_fle_backward_kernel(
    const float* __restrict__ d_rad, int N, int K, int lmax, const float4* __restrict__ geom,
    const float* __restrict__ tx, int M, int stride, size_t rad_view, FleNorm nrm,
    const float* __restrict__ base, const float4* __restrict__ ab, float* __restrict__ grad_base,
    float* __restrict__ d_ab) {
  __shared__ float2 sY[kFleViews][kFleStride];
  __shared__ float2 sG[kFleViews][kFbRx + 1];
  __shared__ float2 sP[8][kFleMaxL];
  const int t = threadIdx.x, ll = t % 16, jj = t / 16, warp = t / 32;
  const int L = (lmax + 1) * (lmax + 1);
  constexpr int kR = (kFleMaxL + 15) / 16;
  for (int j0 = 0; j0 < N; j0 += kFbRx) {
    const int nr = min(kFbRx, N - j0);
    float4 acc[2][kR];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < kR; ++r) acc[q][r] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = blockIdx.x; k < K; k += gridDim.x) {
      const float4 p = geom[3 * k];
      float gr[2][kR], gi[2][kR];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < kR; ++r) gr[q][r] = gi[q][r] = 0.0f;
      for (int v0 = 0; v0 < M; v0 += kFleViews) {
        const int nv = min(kFleViews, M - v0);
        __syncthreads();  // the previous pass is done with sY, sG and sP
        if (t < nv)
          fle_basis_dir(p.x - tx[3 * (v0 + t)], p.y - tx[3 * (v0 + t) + 1],
                        p.z - tx[3 * (v0 + t) + 2], lmax, nrm, sY[t]);
        for (int e = t; e < nv * nr; e += 256) {
          const int v = e / nr, j = e % nr;
          const float* g = d_rad + static_cast<size_t>(v0 + v) * rad_view +
                           static_cast<size_t>(k) * stride + 2 * (j0 + j);
          sG[v][j] = make_float2(g[0], g[1]);
        }
        __syncthreads();
        for (int v = 0; v < nv; ++v) {
          float2 gq[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) gq[q] = sG[v][jj + 16 * q];
#pragma unroll
          for (int r = 0; r < kR; ++r) {
            const int l = ll + 16 * r;
            const float2 y = sY[v][l < kFleMaxL ? l : 0];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              gr[q][r] = fmaf(gq[q].x, y.x, fmaf(gq[q].y, y.y, gr[q][r]));
              gi[q][r] = fmaf(gq[q].y, y.x, fmaf(-gq[q].x, y.y, gi[q][r]));
            }
          }
        }
      }
      // receivers of this pass that do not exist carry unset staging values:
      // they take no part below
      float2 dp[kR];
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        dp[r] = make_float2(0.0f, 0.0f);
        const int l = ll + 16 * r;
        if (l >= L) continue;
        const float pr = base[static_cast<size_t>(k) * 2 * L + l];
        const float pi = base[static_cast<size_t>(k) * 2 * L + L + l];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = jj + 16 * q;
          if (j >= nr) continue;
          const float4 a = ab[static_cast<size_t>(j0 + j) * L + l];
          const float ar = 1.0f + a.x, ai = a.y;
          const float xr = gr[q][r], xi = gi[q][r];
          dp[r].x = fmaf(ar, xr, fmaf(ai, xi, dp[r].x));
          dp[r].y = fmaf(ar, xi, fmaf(-ai, xr, dp[r].y));
          acc[q][r].x = fmaf(pr, xr, fmaf(pi, xi, acc[q][r].x));
          acc[q][r].y = fmaf(pr, xi, fmaf(-pi, xr, acc[q][r].y));
          acc[q][r].z += xr;
          acc[q][r].w += xi;
        }
      }
      if (grad_base) {
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          dp[r].x += __shfl_xor_sync(0xffffffffu, dp[r].x, 16);
          dp[r].y += __shfl_xor_sync(0xffffffffu, dp[r].y, 16);
          const int l = ll + 16 * r;
          if ((t & 16) == 0 && l < L) sP[warp][l] = dp[r];
        }
        __syncthreads();
        if (t < L) {
          float sr = 0.0f, si = 0.0f;
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            sr += sP[w][t].x;
            si += sP[w][t].y;
          }
          grad_base[static_cast<size_t>(k) * 2 * L + t] += sr;
          grad_base[static_cast<size_t>(k) * 2 * L + L + t] += si;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int j = jj + 16 * q;
      if (j >= nr) continue;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const int l = ll + 16 * r;
        if (l >= L) continue;
        float* dst = d_ab + (static_cast<size_t>(j0 + j) * L + l) * 4;
        atomicAdd(dst + 0, acc[q][r].x);
        atomicAdd(dst + 1, acc[q][r].y);
        atomicAdd(dst + 2, acc[q][r].z);
        atomicAdd(dst + 3, acc[q][r].w);
      }
    }
  }
}

void launch_fle_radiance(const float* coeffs, int N, int K, int lmax, const float4* geom,
                         const float* tx, int M, int stride, size_t rad_view, float* rad,
                         cudaStream_t s, const float* base, const float4* ab) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  constexpr size_t smem = sizeof(float2) * (kFleViews + kFleRx) * kFleStride;
  auto kern = base ? fle_radiance_kernel<true> : fle_radiance_kernel<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  kern<<<K, 256, smem, s>>>(coeffs, N, K, lmax, geom, tx, M, stride, rad_view,
                            fle_norm_table(lmax), rad, base, ab);
  note_launches(1);
}

void launch_film_fle_backward(const float* d_rad, int N, int K, int lmax, const float4* geom,
                              const float* tx, int M, int stride, size_t rad_view,
                              const float* base, const float4* ab, float* grad_base,
                              float* d_ab, cudaStream_t s) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, film_fle_backward_kernel, 256, 0);
  const int grid = std::max(1, std::min(K, std::max(1, nsm) * std::max(1, per_sm)));
  film_fle_backward_kernel<<<grid, 256, 0, s>>>(d_rad, N, K, lmax, geom, tx, M, stride, rad_view,
                                                fle_norm_table(lmax), base, ab, grad_base, d_ab);
  note_launches(1);
}

void launch_fle_backward(const float* d_rad, int N, int K, int lmax, const float4* geom,
                         const float* tx, int M, int stride, size_t rad_view, float* grad,
                         cudaStream_t s) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  fle_backward_kernel<<<K, 256, 0, s>>>(d_rad, N, K, lmax, geom, tx, M, stride, rad_view,
                                        fle_norm_table(lmax), grad);
  note_launches(1);
}

}  // namespace rxgs
