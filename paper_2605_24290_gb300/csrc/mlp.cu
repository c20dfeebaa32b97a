// mlp.cu -- receiver-conditioned radiance (Sec. 3.3.2; Algorithm 1, Stage 2):
//   global branch  (a_g, b_g) = MLP_g(r_j)                      (Eq. film)
//   local branch   (a_l, b_l) = MLP_l([v_hat, d, T=1, rho=0])   (Eq. local)
//   combination    s = (1 + a_l) * ((1 + a_g) * phi_base + b_g) + b_l,
//                  complex products per channel         (Eq. combined_local)
// Each branch is Linear -> ReLU -> Linear with outputs (a.re, a.im, b.re,
// b.im) per channel.  v_hat = (r - p)/|r - p| points from the Gaussian to
// the receiver.  The occlusion inputs are held at a clear path (T = 1,
// rho_bar = 0).  bf16 mode rounds the matmul operands (inputs, weights and
// hidden activations) to bf16 and accumulates in float32.
#include <cuda_bf16.h>

#include "rxgs_internal.h"

namespace rxgs {

constexpr int kHidden = 64;

struct MlpOffsets {
  int g_w1, g_b1, g_w2, g_b2, l_w1, l_b1, l_w2, l_b2, total;
};

__host__ __device__ inline MlpOffsets mlp_offsets(int h, int C) {
  MlpOffsets o;
  o.g_w1 = 0;
  o.g_b1 = o.g_w1 + h * 3;
  o.g_w2 = o.g_b1 + h;
  o.g_b2 = o.g_w2 + 4 * C * h;
  o.l_w1 = o.g_b2 + 4 * C;
  o.l_b1 = o.l_w1 + h * 6;
  o.l_w2 = o.l_b1 + h;
  o.l_b2 = o.l_w2 + 4 * C * h;
  o.total = o.l_b2 + 4 * C;
  return o;
}

__device__ __forceinline__ float rb(float x, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// glob[j][4C] = MLP_g(r_j); one block per receiver.
__global__ void mlp_global_kernel(const float* __restrict__ P, int C, int bf16,
                                  const float* __restrict__ rx, float* __restrict__ glob) {
  __shared__ float h[kHidden];
  const MlpOffsets o = mlp_offsets(kHidden, C);
  const int j = blockIdx.x;
  const float x0 = rb(rx[3 * j + 0], bf16), x1 = rb(rx[3 * j + 1], bf16),
              x2 = rb(rx[3 * j + 2], bf16);
  for (int u = threadIdx.x; u < kHidden; u += blockDim.x) {
    const float* w = P + o.g_w1 + u * 3;
    float a = P[o.g_b1 + u];
    a = fmaf(rb(w[0], bf16), x0, a);
    a = fmaf(rb(w[1], bf16), x1, a);
    a = fmaf(rb(w[2], bf16), x2, a);
    h[u] = rb(fmaxf(a, 0.0f), bf16);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 4 * C; q += blockDim.x) {
    const float* w = P + o.g_w2 + q * kHidden;
    float a = P[o.g_b2 + q];
    for (int u = 0; u < kHidden; ++u) a = fmaf(rb(w[u], bf16), h[u], a);
    glob[static_cast<size_t>(j) * 4 * C + q] = a;
  }
}

// One thread per (Gaussian k, receiver j), j fastest.  Writes the
// Gaussian-major radiance row k, columns j*2C .. j*2C + 2C - 1.
__global__ void __launch_bounds__(256) mlp_local_kernel(const float* __restrict__ P, int C,
                                                        int bf16, const float* __restrict__ rx,
                                                        int N, const float4* __restrict__ geom,
                                                        const float* __restrict__ base, int K,
                                                        int stride,
                                                        const float* __restrict__ glob,
                                                        float* __restrict__ out) {
  extern __shared__ float sw[];  // l_w1 [64*6], l_b1 [64], l_w2 [4C*64], l_b2 [4C]
  const MlpOffsets o = mlp_offsets(kHidden, C);
  const int nw = kHidden * 6 + kHidden + 4 * C * kHidden + 4 * C;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) {
    float v = P[o.l_w1 + e];
    // weights (not biases) are matmul operands
    const bool is_w = e < kHidden * 6 || (e >= kHidden * 7 && e < kHidden * 7 + 4 * C * kHidden);
    sw[e] = is_w ? rb(v, bf16) : v;
  }
  __syncthreads();
  const float* W1 = sw;
  const float* B1 = W1 + kHidden * 6;
  const float* W2 = B1 + kHidden;
  const float* B2 = W2 + 4 * C * kHidden;
  const size_t pair = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (pair >= static_cast<size_t>(N) * K) return;
  const int j = static_cast<int>(pair % N);
  const int k = static_cast<int>(pair / N);
  const float4 p = geom[3 * k];
  const float vx = rx[3 * j + 0] - p.x, vy = rx[3 * j + 1] - p.y, vz = rx[3 * j + 2] - p.z;
  const float d = sqrtf(vx * vx + vy * vy + vz * vz);
  const float inv = 1.0f / d;
  const float x[6] = {rb(vx * inv, bf16), rb(vy * inv, bf16), rb(vz * inv, bf16), rb(d, bf16),
                      1.0f, 0.0f};
  float h[kHidden];
#pragma unroll
  for (int u = 0; u < kHidden; ++u) {
    float a = B1[u];
#pragma unroll
    for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
    h[u] = rb(fmaxf(a, 0.0f), bf16);
  }
  const float* gj = glob + static_cast<size_t>(j) * 4 * C;
  float* dst = out + static_cast<size_t>(k) * stride + static_cast<size_t>(j) * 2 * C;
  for (int c = 0; c < C; ++c) {
    float ol[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float* w = W2 + (4 * c + q) * kHidden;
      float a = B2[4 * c + q];
#pragma unroll
      for (int u = 0; u < kHidden; ++u) a = fmaf(w[u], h[u], a);
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
    *reinterpret_cast<float2*>(&dst[2 * c]) = make_float2(sr, si);
  }
}

void launch_mlp_radiance(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, float* out, float* glob,
                         cudaStream_t s) {
  if (N <= 0 || K <= 0) return;
  // pad columns of every row stay zero
  cudaMemsetAsync(out, 0, sizeof(float) * static_cast<size_t>(K) * stride, s);
  mlp_global_kernel<<<N, 128, 0, s>>>(m.p, m.C, m.bf16, rx, glob);
  note_launches(1);
  const size_t pairs = static_cast<size_t>(N) * K;
  const size_t smem = sizeof(float) * (kHidden * 7 + 4 * m.C * kHidden + 4 * m.C);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(mlp_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  mlp_local_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, smem, s>>>(
      m.p, m.C, m.bf16, rx, N, geom, base, K, stride, glob, out);
  note_launches(1);
}



// ------------------------------------------------------------------ backward
// Gradients of L through the combination and both MLPs, given
// dS[k][j*2C + 2c + {0,1}] = dL/ds_kj (Gaussian-major).  With complex
// products z = a b:  dL/da = g conj(b), dL/db = g conj(a).
//   u = (1 + a_g) phi + b_g,  s = (1 + a_l) u + b_l
//   dL/da_l = g conj(u), dL/db_l = g, dL/du = g conj(1 + a_l)
//   dL/da_g = sum_k dL/du conj(phi), dL/db_g = sum_k dL/du,
//   dL/dphi = sum_j dL/du conj(1 + a_g)
// The local-branch weight gradients are sums over all (j, k) pairs: each
// persistent block accumulates its pairs in registers (one parameter per
// thread), writes one partial, and a second kernel adds the partials in a
// fixed order.
constexpr int kBwdPairs = 256;  // pairs per tile (one per thread)
constexpr int kMaxBwdC = 4;     // MLP backward supports C <= 4

static int mlp_bwd_blocks() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  return sms;  // one resident block per SM (the tile buffers take ~150 KB)
}

size_t mlp_backward_tmp_floats(const MlpParams& m, int N, int /*K*/) {
  const int nloc = kHidden * 6 + kHidden + 4 * m.C * kHidden + 4 * m.C;
  const int blocks = mlp_bwd_blocks();
  return static_cast<size_t>(blocks) * (nloc + static_cast<size_t>(N) * 4 * m.C) +
         static_cast<size_t>(N) * 4 * m.C;
}

__global__ void __launch_bounds__(kBwdPairs) mlp_local_bwd_kernel(
    const float* __restrict__ P, int C, const float* __restrict__ rx, int N,
    const float4* __restrict__ geom, const float* __restrict__ base, int K, int stride,
    const float* __restrict__ dS, const float* __restrict__ glob, float* __restrict__ grad_base,
    float* __restrict__ part) {
  extern __shared__ float sm[];
  const MlpOffsets o = mlp_offsets(kHidden, C);
  const int n4 = 4 * C;
  float* W1 = sm;                          // [64][6]
  float* B1 = W1 + kHidden * 6;            // [64]
  float* W2 = B1 + kHidden;                // [4C][64]
  float* sX = W2 + n4 * kHidden;           // [256][6]
  float* sH = sX + kBwdPairs * 6;          // [256][65]  post-ReLU hidden (padded)
  float* sDol = sH + kBwdPairs * 65;       // [256][4C]
  float* sDh = sDol + kBwdPairs * n4;      // [256][65]
  float* sDB = sDh + kBwdPairs * 65;       // [256][2C]  dL/dphi contributions
  float* sOG = sDB + kBwdPairs * 2 * C;    // [256][4C]  dL/d(a_g, b_g) contributions
  float* accOG = sOG + kBwdPairs * n4;     // [N][4C]    block accumulator
  const int t = threadIdx.x;
  for (int e = t; e < kHidden * 6; e += kBwdPairs) W1[e] = P[o.l_w1 + e];
  for (int e = t; e < kHidden; e += kBwdPairs) B1[e] = P[o.l_b1 + e];
  for (int e = t; e < n4 * kHidden; e += kBwdPairs) W2[e] = P[o.l_w2 + e];
  for (int e = t; e < N * n4; e += kBwdPairs) accOG[e] = 0.0f;
  // owned parameter accumulators
  float aW2 = 0.0f, aW1a = 0.0f, aW1b = 0.0f, aB1 = 0.0f, aB2 = 0.0f;
  const size_t pairs = static_cast<size_t>(N) * K;
  const size_t ntiles = (pairs + kBwdPairs - 1) / kBwdPairs;
  __syncthreads();
  for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const size_t p0 = tile * kBwdPairs;
    const size_t pair = p0 + t;
    const bool ok = pair < pairs;
    // ---- phase 1: forward recompute and the complex-affine backward
    {
      float x[6] = {0, 0, 0, 0, 0, 0};
      float dol[4 * kMaxBwdC], db[2 * kMaxBwdC], dog[4 * kMaxBwdC];
#pragma unroll
      for (int q = 0; q < 4 * kMaxBwdC; ++q) dol[q] = dog[q] = 0.0f;
#pragma unroll
      for (int q = 0; q < 2 * kMaxBwdC; ++q) db[q] = 0.0f;
      if (ok) {
        const int j = static_cast<int>(pair % N), k = static_cast<int>(pair / N);
        const float4 p = geom[3 * k];
        const float vx = rx[3 * j + 0] - p.x, vy = rx[3 * j + 1] - p.y, vz = rx[3 * j + 2] - p.z;
        const float d = sqrtf(vx * vx + vy * vy + vz * vz);
        const float inv = 1.0f / d;
        x[0] = vx * inv; x[1] = vy * inv; x[2] = vz * inv; x[3] = d; x[4] = 1.0f; x[5] = 0.0f;
        float h[kHidden];
#pragma unroll
        for (int u = 0; u < kHidden; ++u) {
          float a = B1[u];
#pragma unroll
          for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
          h[u] = fmaxf(a, 0.0f);
          sH[t * 65 + u] = h[u];
        }
        const float* gj = glob + static_cast<size_t>(j) * n4;
        const float* gs = dS + static_cast<size_t>(k) * stride + static_cast<size_t>(j) * 2 * C;
        for (int c = 0; c < C; ++c) {
          float ol[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float* w = W2 + (4 * c + q) * kHidden;
            float a = P[o.l_b2 + 4 * c + q];
#pragma unroll
            for (int u = 0; u < kHidden; ++u) a = fmaf(w[u], h[u], a);
            ol[q] = a;
          }
          const float pr = base[(static_cast<size_t>(k) * C + c) * 2 + 0];
          const float pi = base[(static_cast<size_t>(k) * C + c) * 2 + 1];
          const float agr = 1.0f + gj[4 * c + 0], agi = gj[4 * c + 1];
          const float ur = agr * pr - agi * pi + gj[4 * c + 2];
          const float ui = agr * pi + agi * pr + gj[4 * c + 3];
          const float alr = 1.0f + ol[0], ali = ol[1];
          const float gr = gs[2 * c], gi = gs[2 * c + 1];
          // dL/da_l = g conj(u); dL/db_l = g
          dol[4 * c + 0] = gr * ur + gi * ui;
          dol[4 * c + 1] = gi * ur - gr * ui;
          dol[4 * c + 2] = gr;
          dol[4 * c + 3] = gi;
          // dL/du = g conj(1 + a_l)
          const float dur = gr * alr + gi * ali, dui = gi * alr - gr * ali;
          // dL/da_g = du conj(phi); dL/db_g = du; dL/dphi = du conj(1 + a_g)
          dog[4 * c + 0] = dur * pr + dui * pi;
          dog[4 * c + 1] = dui * pr - dur * pi;
          dog[4 * c + 2] = dur;
          dog[4 * c + 3] = dui;
          db[2 * c + 0] = dur * agr + dui * agi;
          db[2 * c + 1] = dui * agr - dur * agi;
        }
      } else {
        for (int u = 0; u < kHidden; ++u) sH[t * 65 + u] = 0.0f;
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) sX[t * 6 + i] = x[i];
      for (int q = 0; q < n4; ++q) {
        sDol[t * n4 + q] = dol[q];
        sOG[t * n4 + q] = dog[q];
      }
      for (int q = 0; q < 2 * C; ++q) sDB[t * 2 * C + q] = db[q];
    }
    __syncthreads();
    // ---- phase 2: dL/dh = W2^T dol masked by ReLU
    for (int u = 0; u < kHidden; ++u) {
      float a = 0.0f;
      for (int q = 0; q < n4; ++q) a = fmaf(W2[q * kHidden + u], sDol[t * n4 + q], a);
      sDh[t * 65 + u] = sH[t * 65 + u] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    // ---- phase 3: owned parameter sums over the tile's pairs
    if (t < n4 * kHidden) {
      const int q = t / kHidden, u = t % kHidden;
      float a = 0.0f;
      for (int pp = 0; pp < kBwdPairs; ++pp) a = fmaf(sDol[pp * n4 + q], sH[pp * 65 + u], a);
      aW2 += a;
    }
    {
      const int e0 = t, e1 = t + kBwdPairs;  // dW1 entries u*6 + i
      float a0 = 0.0f, a1 = 0.0f;
      for (int pp = 0; pp < kBwdPairs; ++pp) {
        a0 = fmaf(sDh[pp * 65 + e0 / 6], sX[pp * 6 + e0 % 6], a0);
        if (e1 < kHidden * 6) a1 = fmaf(sDh[pp * 65 + e1 / 6], sX[pp * 6 + e1 % 6], a1);
      }
      aW1a += a0;
      aW1b += a1;
    }
    if (t < kHidden) {
      float a = 0.0f;
      for (int pp = 0; pp < kBwdPairs; ++pp) a += sDh[pp * 65 + t];
      aB1 += a;
    }
    if (t < n4) {
      float a = 0.0f;
      for (int pp = 0; pp < kBwdPairs; ++pp) a += sDol[pp * n4 + t];
      aB2 += a;
    }
    // ---- phase 4: dL/dphi per Gaussian (atomics: a Gaussian's pairs may span
    // tiles), dL/d(a_g, b_g) per receiver into the block accumulator
    {
      const size_t kfirst = p0 / N;
      const size_t plast = min(p0 + kBwdPairs, pairs) - 1;
      const size_t klast = plast / N;
      const size_t nk = klast - kfirst + 1;
      for (size_t kk = t; kk < nk; kk += kBwdPairs) {
        const size_t k = kfirst + kk;
        const size_t a0 = max(k * N, p0) - p0, a1 = min((k + 1) * N, plast + 1) - p0;
        for (int q = 0; q < 2 * C; ++q) {
          float s = 0.0f;
          for (size_t pp = a0; pp < a1; ++pp) s += sDB[pp * 2 * C + q];
          atomicAdd(&grad_base[k * 2 * C + q], s);
        }
      }
      for (int j = t; j < N; j += kBwdPairs) {
        for (size_t pp = (j + N - p0 % N) % N; pp < kBwdPairs && p0 + pp < pairs; pp += N)
          for (int q = 0; q < n4; ++q) accOG[j * n4 + q] += sOG[pp * n4 + q];
      }
    }
    __syncthreads();
  }
  // ---- block partial: [local params (flat order l_w1 l_b1 l_w2 l_b2)] [N][4C]
  const int nloc = kHidden * 6 + kHidden + n4 * kHidden + n4;
  float* dst = part + static_cast<size_t>(blockIdx.x) * (nloc + static_cast<size_t>(N) * n4);
  dst[t] = aW1a;
  if (t + kBwdPairs < kHidden * 6) dst[t + kBwdPairs] = aW1b;
  if (t < kHidden) dst[kHidden * 6 + t] = aB1;
  if (t < n4 * kHidden) dst[kHidden * 7 + t] = aW2;
  if (t < n4) dst[kHidden * 7 + n4 * kHidden + t] = aB2;
  for (int e = t; e < N * n4; e += kBwdPairs) dst[nloc + e] = accOG[e];
}

// Sums the block partials in block order: local parameters go into
// grad_mlp, the per-receiver (a_g, b_g) gradients into dog[N][4C].
__global__ void mlp_partial_reduce_kernel(const float* __restrict__ part, int blocks, int nloc,
                                          int nog, int l_off, float* __restrict__ grad_mlp,
                                          float* __restrict__ dog) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nloc + nog) return;
  float s = 0.0f;
  for (int b = 0; b < blocks; ++b) s += part[static_cast<size_t>(b) * (nloc + nog) + e];
  if (e < nloc)
    grad_mlp[l_off + e] += s;
  else
    dog[e - nloc] = s;
}

// Global branch backward for all receivers in one block (N is small).
__global__ void mlp_global_bwd_kernel(const float* __restrict__ P, int C,
                                      const float* __restrict__ rx, int N,
                                      const float* __restrict__ dog,
                                      float* __restrict__ grad_mlp) {
  __shared__ float h[kHidden], dh[kHidden];
  const MlpOffsets o = mlp_offsets(kHidden, C);
  const int n4 = 4 * C;
  const int t = threadIdx.x;
  // owned accumulators: W1 (192), B1 (64), W2 (4C*64), B2 (4C)
  for (int j = 0; j < N; ++j) {
    const float x0 = rx[3 * j], x1 = rx[3 * j + 1], x2 = rx[3 * j + 2];
    for (int u = t; u < kHidden; u += blockDim.x) {
      const float* w = P + o.g_w1 + u * 3;
      float a = P[o.g_b1 + u];
      a = fmaf(w[0], x0, a);
      a = fmaf(w[1], x1, a);
      a = fmaf(w[2], x2, a);
      h[u] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    const float* dj = dog + static_cast<size_t>(j) * n4;
    for (int u = t; u < kHidden; u += blockDim.x) {
      float a = 0.0f;
      for (int q = 0; q < n4; ++q) a = fmaf(P[o.g_w2 + q * kHidden + u], dj[q], a);
      dh[u] = h[u] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    for (int e = t; e < n4 * kHidden; e += blockDim.x)
      grad_mlp[o.g_w2 + e] += dj[e / kHidden] * h[e % kHidden];
    for (int e = t; e < n4; e += blockDim.x) grad_mlp[o.g_b2 + e] += dj[e];
    for (int e = t; e < kHidden * 3; e += blockDim.x) {
      const float xv = e % 3 == 0 ? x0 : (e % 3 == 1 ? x1 : x2);
      grad_mlp[o.g_w1 + e] += dh[e / 3] * xv;
    }
    for (int e = t; e < kHidden; e += blockDim.x) grad_mlp[o.g_b1 + e] += dh[e];
    __syncthreads();
  }
}

void launch_mlp_backward(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, const float* dS,
                         const float* glob, float* grad_base, float* grad_mlp, float* tmp,
                         cudaStream_t s) {
  const int C = m.C, n4 = 4 * C;
  const int nloc = kHidden * 6 + kHidden + n4 * kHidden + n4;
  const int blocks = mlp_bwd_blocks();
  const size_t smem = sizeof(float) * (kHidden * 7 + n4 * kHidden + kBwdPairs * 6 +
                                       kBwdPairs * 65 * 2 + kBwdPairs * n4 * 2 +
                                       kBwdPairs * 2 * C + static_cast<size_t>(N) * n4);
  cudaFuncSetAttribute(mlp_local_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  float* part = tmp;
  float* dog = tmp + static_cast<size_t>(blocks) * (nloc + static_cast<size_t>(N) * n4);
  mlp_local_bwd_kernel<<<blocks, kBwdPairs, smem, s>>>(m.p, C, rx, N, geom, base, K, stride, dS,
                                                       glob, grad_base, part);
  note_launches(1);
  const int tot = nloc + N * n4;
  const MlpOffsets o = mlp_offsets(kHidden, C);
  mlp_partial_reduce_kernel<<<(tot + 255) / 256, 256, 0, s>>>(part, blocks, nloc, N * n4, o.l_w1,
                                                              grad_mlp, dog);
  note_launches(1);
  mlp_global_bwd_kernel<<<1, 256, 0, s>>>(m.p, C, rx, N, dog, grad_mlp);
  note_launches(1);
}

}  // namespace rxgs
