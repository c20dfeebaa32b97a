// vis_bwd.cu -- backward of CSI / RSSI through visibility weights, for
// explicit radiance (App. D backward; Eq. render_reorder).
//
// When the cotangent is on CSI or RSSI only, the per-pixel cotangent of view
// v is the same at every pixel: g[v][q] for the complex column q = (j, c).
// The gradients of the compositing then factor:
//   dL/ds[j][k][c]  = sum_v W[v][k] g[v][j][c]       W[v][k] = sum_pixels T_k w_k
//   dL/dtau_k       = sum_v sum_pixels G_k T_k (gamma[v][k] - Q)
// with gamma[v][k] = sum_q <g[v][q], s[j][k][c]> (one real number per view
// and Gaussian) and Q the same suffix recurrence as the per-pixel backward,
// now over scalars: Q <- w gamma + (1 - w) Q.  Three kernels:
//   gamma_kernel      gamma[M][K], streaming the receiver-major radiance once
//                     per 16 views;
//   bwd_uniform       per (view, tile): the back-to-front sweep of the
//                     per-pixel backward with the scalar gamma, summing
//                     T w and dL/dtau per Gaussian (warp sums + atomics);
//   outer_kernel      grad_radiance[j][k][c] += sum_v W[v][k] g[v][j][c].
// No [K][N*2C] radiance copy or radiance-gradient buffer is made.
#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

constexpr int kVbViews = 16;   // views per pass of the column kernels
constexpr int kGamCols = 128;  // complex columns staged per step in gamma_kernel

// gamma[v][k] for v in [v0, v0 + nv): thread = 4 consecutive Gaussians
// (1,024 per block), 16 views x 4 Gaussians in registers, walking all
// complex columns q = (j, c); the cotangents of 128 columns for the pass's
// views are staged in shared memory as [q][view] (re, im) and read as
// 16-byte broadcasts.  With C = 1 (K even) the four Gaussians of a column
// are 32 contiguous bytes (two 16-byte loads).
template <bool kVec>
__global__ void __launch_bounds__(256) gamma_kernel(const float* __restrict__ rad, int N, int K,
                                                    int C, const float* __restrict__ gu, int M,
                                                    int v0, int nv, float* __restrict__ gamma) {
  __shared__ __align__(16) float sg[kGamCols][kVbViews][2];
  const int t = threadIdx.x;
  const int k0 = (blockIdx.x * 256 + t) * 4;
  const int ncq = N * C;
  float acc[kVbViews][4];
#pragma unroll
  for (int v = 0; v < kVbViews; ++v)
#pragma unroll
    for (int x = 0; x < 4; ++x) acc[v][x] = 0.0f;
  const float2* r2 = reinterpret_cast<const float2*>(rad);
  const bool full = k0 + 4 <= K;
  for (int q0 = 0; q0 < ncq; q0 += kGamCols) {
    const int nq = min(kGamCols, ncq - q0);
    __syncthreads();
    for (int e = t; e < kGamCols * kVbViews; e += 256) {
      const int qq = e / kVbViews, v = e % kVbViews;
      float2 x = make_float2(0.0f, 0.0f);
      if (qq < nq && v < nv)
        x = reinterpret_cast<const float2*>(gu)[static_cast<size_t>(v0 + v) * ncq + q0 + qq];
      sg[qq][v][0] = x.x;
      sg[qq][v][1] = x.y;
    }
    __syncthreads();
    if (k0 < K) {
      // the column's four Gaussians; a ring of four register buffers keeps
      // three columns' loads in flight (unrolled by four: no buffer copy,
      // which would wait for its load)
      auto load = [&](int qq, float2 (&sv)[4]) {
        const int q = q0 + qq, j = q / C, c = q - j * C;
        const float2* cp = r2 + (static_cast<size_t>(j) * K + k0) * C + c;
        if (kVec && full) {
          const float4 a4 = *reinterpret_cast<const float4*>(cp);
          const float4 b4 = *reinterpret_cast<const float4*>(cp + 2);
          sv[0] = make_float2(a4.x, a4.y);
          sv[1] = make_float2(a4.z, a4.w);
          sv[2] = make_float2(b4.x, b4.y);
          sv[3] = make_float2(b4.z, b4.w);
        } else {
#pragma unroll
          for (int x = 0; x < 4; ++x)
            sv[x] = k0 + x < K ? cp[static_cast<size_t>(x) * C] : make_float2(0.f, 0.f);
        }
      };
      auto step = [&](int qq, const float2 (&sv)[4]) {
#pragma unroll
        for (int v2 = 0; v2 < kVbViews / 2; ++v2) {
          const float4 g4 = *reinterpret_cast<const float4*>(&sg[qq][2 * v2][0]);
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            acc[2 * v2][x] = fmaf(g4.x, sv[x].x, fmaf(g4.y, sv[x].y, acc[2 * v2][x]));
            acc[2 * v2 + 1][x] = fmaf(g4.z, sv[x].x, fmaf(g4.w, sv[x].y, acc[2 * v2 + 1][x]));
          }
        }
      };
      float2 rb[4][4];
#pragma unroll
      for (int b = 0; b < 3; ++b)
        if (b < nq) load(b, rb[b]);
      for (int qb = 0; qb < nq; qb += 4) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int qq = qb + b;
          if (qq >= nq) break;
          if (qq + 3 < nq) load(qq + 3, rb[(b + 3) & 3]);
          step(qq, rb[b]);
        }
      }
    }
  }
  if (k0 >= K) return;
#pragma unroll
  for (int v = 0; v < kVbViews; ++v) {
    if (v >= nv) break;
#pragma unroll
    for (int x = 0; x < 4; ++x)
      if (k0 + x < K) gamma[static_cast<size_t>(v0 + v) * K + k0 + x] = acc[v][x];
  }
}

// Back-to-front sweep of one (view, tile) with the scalar gamma: one thread
// per pixel, the copy pipeline of the forward (indices two chunks ahead,
// records and gamma values one chunk ahead), the per-pixel final T and stop
// from the pre-pass.
__global__ void __launch_bounds__(kTilePixels) bwd_uniform_kernel(
    const RenderArgs a, const float* __restrict__ gamma, const float* __restrict__ tfin,
    const uint32_t* __restrict__ stops, const uint32_t* __restrict__ tile_stop,
    float* __restrict__ W, float* __restrict__ d_tau) {
  __shared__ float4 sRec[2][2 * kChunk];
  __shared__ float sGam[2][kChunk];
  __shared__ uint32_t sIdx[3 * kChunk];
  __shared__ float sWs[kTilePixels / 32][kChunk], sTs[kTilePixels / 32][kChunk];
  const GridConst& g = a.g;
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const float* gv = gamma + static_cast<size_t>(v) * a.K;
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  float T = 1.0f;
  uint32_t stop = rg.x;
  if (valid) {
    const size_t o = static_cast<size_t>(v) * HW + static_cast<size_t>(i) * g.W + jj;
    T = tfin[o];
    stop = stops[o];
  }
  const uint32_t tstop = tile_stop[static_cast<size_t>(v) * g.T + tile];
  const Strip strip = warp_strip(g, tr, tc, wp);
  const int nchunks = static_cast<int>((tstop - rg.x + kChunk - 1) / kChunk);
  auto chunk_start = [&](int n) { return rg.x + static_cast<uint32_t>(nchunks - 1 - n) * kChunk; };
  auto chunk_len = [&](int n) { return min(kChunk, static_cast<int>(tstop - chunk_start(n))); };
  auto copy_indices = [&](int n) {
    const bool ok = t < chunk_len(n);
    if (t < kChunk)
      cp_async4(&sIdx[(n % 3) * kChunk + t], ok ? &a.vals[chunk_start(n) + t] : a.vals, ok);
  };
  auto gather = [&](int n) {
    if (t < kChunk) {
      const bool ok = t < chunk_len(n);
      const uint32_t k = ok ? sIdx[(n % 3) * kChunk + t] : 0u;
      cp_async16(&sRec[n & 1][2 * t + 0], &rec[2 * k + 0], ok);
      cp_async16(&sRec[n & 1][2 * t + 1], &rec[2 * k + 1], ok);
      cp_async4(&sGam[n & 1][t], &gv[k], ok);
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
  float Q = 0.0f;
  for (int n = 0; n < nchunks; ++n) {
    const uint32_t start = chunk_start(n);
    const int nb = chunk_len(n);
    cp_async_wait_all();
    __syncthreads();
    if (n + 1 < nchunks) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      gather(n + 1);
    }
    cp_async_commit();
    const float4* sR = sRec[n & 1];
    const float* sG = sGam[n & 1];
    const uint32_t* sK = sIdx + (n % 3) * kChunk;
    sWs[wp][lane] = 0.0f;
    sTs[wp][lane] = 0.0f;
    __syncwarp();
    {
      const bool rel = lane < nb && touches_strip(g, sR[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      if (!__any_sync(0xffffffffu, start < stop)) m = 0;
      while (m) {
        const int b = 31 - __clz(m);
        m &= ~(1u << b);
        float Tw = 0.0f, dt = 0.0f;
        if (start + b < stop) {
          float w, G;
          if (pixel_weight(g, sR[2 * b], sR[2 * b + 1], i, jj, fi, fj, &w, &G)) {
            const float gam = sG[b];
            const float one_m_w = 1.0f - w;
            T = __fdividef(T, one_m_w);  // transmittance in front of this Gaussian
            Tw = T * w;
            dt = T * (gam - Q) * G;
            Q = fmaf(w, gam, one_m_w * Q);
          }
        }
        if (__any_sync(0xffffffffu, Tw != 0.0f || dt != 0.0f)) {
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1) {
            Tw += __shfl_xor_sync(0xffffffffu, Tw, o);
            dt += __shfl_xor_sync(0xffffffffu, dt, o);
          }
          if (lane == 0) {
            sWs[wp][b] = Tw;
            sTs[wp][b] = dt;
          }
        }
      }
    }
    __syncthreads();
    if (t < nb) {
      float ws = 0.0f, ts = 0.0f;
#pragma unroll
      for (int w8 = 0; w8 < kTilePixels / 32; ++w8) {
        ws += sWs[w8][t];
        ts += sTs[w8][t];
      }
      const uint32_t k = sK[t];
      if (W && ws != 0.0f) atomicAdd(&W[static_cast<size_t>(v) * a.K + k], ws);
      if (ts != 0.0f) atomicAdd(&d_tau[k], ts);
    }
  }
  cp_async_wait_all();
}

// grad[j][k][c] += sum_v W[v][k] g[v][j][c]: thread = 4 consecutive
// Gaussians (their W for the pass's views in registers), looping over the
// complex columns of its block; the cotangents of those columns are staged
// in shared memory.
constexpr int kOutCols = 64;

template <bool kVec>
__global__ void __launch_bounds__(256) outer_kernel(const float* __restrict__ W, int K,
                                                    const float* __restrict__ gu, int N, int C,
                                                    int v0, int nv, float* __restrict__ grad) {
  __shared__ __align__(16) float sg[kOutCols][kVbViews][2];
  const int t = threadIdx.x;
  const int k0 = (blockIdx.x * 256 + t) * 4;
  const int ncq = N * C;
  const int q0 = blockIdx.y * kOutCols, nq = min(kOutCols, ncq - q0);
  for (int e = t; e < kOutCols * kVbViews; e += 256) {
    const int qq = e / kVbViews, v = e % kVbViews;
    float2 x = make_float2(0.0f, 0.0f);
    if (qq < nq && v < nv)
      x = reinterpret_cast<const float2*>(gu)[static_cast<size_t>(v0 + v) * ncq + q0 + qq];
    sg[qq][v][0] = x.x;
    sg[qq][v][1] = x.y;
  }
  __syncthreads();
  if (k0 >= K) return;
  float w[kVbViews][4];
#pragma unroll
  for (int v = 0; v < kVbViews; ++v)
#pragma unroll
    for (int x = 0; x < 4; ++x)
      w[v][x] = (v < nv && k0 + x < K) ? W[static_cast<size_t>(v0 + v) * K + k0 + x] : 0.0f;
  // per column: the four gradient entries read, the update added, written
  // back; a ring of four register buffers keeps three columns' reads in
  // flight (unrolled by four: no buffer copy)
  const bool vec = kVec && k0 + 4 <= K;
  auto dst_of = [&](int qq) {
    const int q = q0 + qq, j = q / C, c = q - j * C;
    return reinterpret_cast<float2*>(grad) + (static_cast<size_t>(j) * K + k0) * C + c;
  };
  auto load = [&](int qq, float2 (&o)[4]) {
    const float2* d = dst_of(qq);
    if (vec) {
      const float4 a4 = reinterpret_cast<const float4*>(d)[0];
      const float4 b4 = reinterpret_cast<const float4*>(d)[1];
      o[0] = make_float2(a4.x, a4.y);
      o[1] = make_float2(a4.z, a4.w);
      o[2] = make_float2(b4.x, b4.y);
      o[3] = make_float2(b4.z, b4.w);
    } else {
#pragma unroll
      for (int x = 0; x < 4; ++x)
        o[x] = k0 + x < K ? d[static_cast<size_t>(x) * C] : make_float2(0.f, 0.f);
    }
  };
  auto step = [&](int qq, float2 (&o)[4]) {
#pragma unroll
    for (int v2 = 0; v2 < kVbViews / 2; ++v2) {
      const float4 g4 = *reinterpret_cast<const float4*>(&sg[qq][2 * v2][0]);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        o[x].x = fmaf(w[2 * v2][x], g4.x, fmaf(w[2 * v2 + 1][x], g4.z, o[x].x));
        o[x].y = fmaf(w[2 * v2][x], g4.y, fmaf(w[2 * v2 + 1][x], g4.w, o[x].y));
      }
    }
    float2* d = dst_of(qq);
    if (vec) {
      reinterpret_cast<float4*>(d)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
      reinterpret_cast<float4*>(d)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    } else {
#pragma unroll
      for (int x = 0; x < 4; ++x)
        if (k0 + x < K) d[static_cast<size_t>(x) * C] = o[x];
    }
  };
  float2 rb[4][4];
#pragma unroll
  for (int b = 0; b < 3; ++b)
    if (b < nq) load(b, rb[b]);
  for (int qb = 0; qb < nq; qb += 4) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int qq = qb + b;
      if (qq >= nq) break;
      if (qq + 3 < nq) load(qq + 3, rb[(b + 3) & 3]);
      step(qq, rb[b]);
    }
  }
}

void launch_vis_backward(const BackwardArgs& A, const float* rad_rm, const float* gu,
                         float* gamma, float* W, float* grad_radiance, cudaStream_t s) {
  const RenderArgs& a = A.f;
  const int M = a.M, K = a.K, N = a.N, C = a.C;
  if (M <= 0 || K <= 0) return;
  // 16-byte access to a single channel's rows needs K even and 16-byte bases
  const bool vec_r = C == 1 && K % 2 == 0 && (reinterpret_cast<uintptr_t>(rad_rm) & 15) == 0;
  const unsigned kb = static_cast<unsigned>((K + 1023) / 1024);
  for (int v0 = 0; v0 < M; v0 += kVbViews) {
    const int nv = min(kVbViews, M - v0);
    if (vec_r)
      gamma_kernel<true><<<kb, 256, 0, s>>>(rad_rm, N, K, C, gu, M, v0, nv, gamma);
    else
      gamma_kernel<false><<<kb, 256, 0, s>>>(rad_rm, N, K, C, gu, M, v0, nv, gamma);
    note_launches(1);
  }
  bwd_uniform_kernel<<<dim3(a.g.T, 1, M), kTilePixels, 0, s>>>(a, gamma, A.tfin, A.stops,
                                                               A.tile_stop, grad_radiance ? W : nullptr,
                                                               A.d_tau);
  note_launches(1);
  if (!grad_radiance) return;
  const bool vec_g = C == 1 && K % 2 == 0 && (reinterpret_cast<uintptr_t>(grad_radiance) & 15) == 0;
  const unsigned qb = static_cast<unsigned>((N * C + kOutCols - 1) / kOutCols);
  for (int v0 = 0; v0 < M; v0 += kVbViews) {
    const int nv = min(kVbViews, M - v0);
    if (vec_g)
      outer_kernel<true><<<dim3(kb, qb), 256, 0, s>>>(W, K, gu, N, C, v0, nv, grad_radiance);
    else
      outer_kernel<false><<<dim3(kb, qb), 256, 0, s>>>(W, K, gu, N, C, v0, nv, grad_radiance);
    note_launches(1);
  }
}

}  // namespace rxgs
