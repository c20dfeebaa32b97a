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
  const size_t pairs = static_cast<size_t>(N) * K;
  const size_t smem = sizeof(float) * (kHidden * 7 + 4 * m.C * kHidden + 4 * m.C);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(mlp_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  mlp_local_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, smem, s>>>(
      m.p, m.C, m.bf16, rx, N, geom, base, K, stride, glob, out);
}

}  // namespace rxgs
