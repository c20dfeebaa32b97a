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
                                  const float* __restrict__ rx, float* __restrict__ glob,
                                  const int* __restrict__ n_dev) {
  __shared__ float h[kHidden];
  const MlpOffsets o = mlp_offsets(kHidden, C);
  const int j = blockIdx.x;
  if (n_dev && j >= *n_dev) return;
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
                                                        float* __restrict__ out,
                                                        const int* __restrict__ n_dev,
                                                        const int* __restrict__ col_of,
                                                        const float2* __restrict__ feat) {
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
  if (n_dev && j >= *n_dev) return;
  const float4 p = geom[3 * k];
  const float vx = rx[3 * j + 0] - p.x, vy = rx[3 * j + 1] - p.y, vz = rx[3 * j + 2] - p.z;
  const float d = sqrtf(vx * vx + vy * vy + vz * vz);
  const float inv = 1.0f / d;
  float2 oc = make_float2(1.0f, 0.0f);  // occlusion inputs (T, rho_bar)
  if (feat) oc = feat[static_cast<size_t>(j) * K + k];
  const float x[6] = {rb(vx * inv, bf16), rb(vy * inv, bf16), rb(vz * inv, bf16), rb(d, bf16),
                      rb(oc.x, bf16), rb(oc.y, bf16)};
  float h[kHidden];
#pragma unroll
  for (int u = 0; u < kHidden; ++u) {
    float a = B1[u];
#pragma unroll
    for (int i = 0; i < 6; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
    h[u] = rb(fmaxf(a, 0.0f), bf16);
  }
  const float* gj = glob + static_cast<size_t>(j) * 4 * C;
  float* dst = out + static_cast<size_t>(k) * stride +
               (col_of ? static_cast<size_t>(col_of[j]) : static_cast<size_t>(j) * 2 * C);
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

// Narrow spectra (C <= 4): the same arithmetic with the hidden units
// streamed into the 4C output accumulators (bias first, then units in
// ascending order, as above), so no 64-entry hidden vector is kept.  Each
// thread evaluates PP pairs (block-strided, so every slice of a block stays
// coalesced) and reuses each weight it reads from shared memory PP times.
template <int CC, int PP, bool OCC>
__global__ void __launch_bounds__(256) mlp_local_narrow_kernel(
    const float* __restrict__ P, int bf16, const float* __restrict__ rx, int N,
    const float4* __restrict__ geom, const float* __restrict__ base, int K, int stride,
    const float* __restrict__ glob, float* __restrict__ out, const int* __restrict__ n_dev,
    const int* __restrict__ col_of, const float2* __restrict__ feat) {
  constexpr int n4 = 4 * CC;
  // per hidden unit u, as 16-byte broadcasts: (w1[0..3]), (w1[4], w1[5], b1, 0)
  // and the unit's output weights (W2[4c..4c+3][u]) per channel c
  __shared__ float4 W1a[kHidden], W1b[kHidden], W2t[kHidden * CC];
  __shared__ float B2[n4];
  const MlpOffsets o = mlp_offsets(kHidden, CC);
  for (int u = threadIdx.x; u < kHidden; u += blockDim.x) {
    const float* w = P + o.l_w1 + u * 6;
    W1a[u] = make_float4(rb(w[0], bf16), rb(w[1], bf16), rb(w[2], bf16), rb(w[3], bf16));
    W1b[u] = make_float4(rb(w[4], bf16), rb(w[5], bf16), P[o.l_b1 + u], 0.0f);
#pragma unroll
    for (int c = 0; c < CC; ++c)
      W2t[u * CC + c] = make_float4(rb(P[o.l_w2 + (4 * c + 0) * kHidden + u], bf16),
                                    rb(P[o.l_w2 + (4 * c + 1) * kHidden + u], bf16),
                                    rb(P[o.l_w2 + (4 * c + 2) * kHidden + u], bf16),
                                    rb(P[o.l_w2 + (4 * c + 3) * kHidden + u], bf16));
  }
  for (int e = threadIdx.x; e < n4; e += blockDim.x) B2[e] = P[o.l_b2 + e];
  __syncthreads();
  const size_t npairs = static_cast<size_t>(N) * K;
  const int nlim = n_dev ? *n_dev : N;
  float x[PP][4], xo[PP][2];  // direction, distance; occlusion (T, rho_bar)
  bool ok[PP];
  int jv[PP], kv[PP];
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    const size_t pair = (static_cast<size_t>(blockIdx.x) * PP + r) * blockDim.x + threadIdx.x;
    ok[r] = pair < npairs;
    const int j = ok[r] ? static_cast<int>(pair % N) : 0;
    const int k = ok[r] ? static_cast<int>(pair / N) : 0;
    ok[r] = ok[r] && j < nlim;
    jv[r] = j;
    kv[r] = k;
    x[r][0] = x[r][1] = x[r][2] = x[r][3] = 0.0f;
    xo[r][0] = 1.0f;
    xo[r][1] = 0.0f;
    if (OCC && ok[r]) {
      const float2 f = feat[static_cast<size_t>(j) * K + k];
      xo[r][0] = rb(f.x, bf16);
      xo[r][1] = rb(f.y, bf16);
    }
    if (ok[r]) {
      const float4 p = geom[3 * k];
      const float vx = rx[3 * j + 0] - p.x, vy = rx[3 * j + 1] - p.y, vz = rx[3 * j + 2] - p.z;
      const float d = sqrtf(vx * vx + vy * vy + vz * vz);
      const float inv = 1.0f / d;
      x[r][0] = rb(vx * inv, bf16);
      x[r][1] = rb(vy * inv, bf16);
      x[r][2] = rb(vz * inv, bf16);
      x[r][3] = rb(d, bf16);
    }
  }
  float ol[PP][n4];
#pragma unroll
  for (int r = 0; r < PP; ++r)
#pragma unroll
    for (int q = 0; q < n4; ++q) ol[r][q] = B2[q];
#pragma unroll 4
  for (int u = 0; u < kHidden; ++u) {
    float w1[6], w2[n4];
    const float4 a4 = W1a[u], b4 = W1b[u];
    w1[0] = a4.x; w1[1] = a4.y; w1[2] = a4.z; w1[3] = a4.w;
    w1[4] = b4.x; w1[5] = b4.y;
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      const float4 t4 = W2t[u * CC + c];
      w2[4 * c] = t4.x; w2[4 * c + 1] = t4.y; w2[4 * c + 2] = t4.z; w2[4 * c + 3] = t4.w;
    }
    const float b1 = b4.z;
#pragma unroll
    for (int r = 0; r < PP; ++r) {
      // inputs 4 and 5 are the constants 1 and 0: the same fmaf chain as the
      // general kernel (fmaf(w, 1, a) = a + w and fmaf(w, 0, a) = a)
      float a = b1;
#pragma unroll
      for (int i = 0; i < 4; ++i) a = fmaf(w1[i], x[r][i], a);
      if (OCC) {
        a = fmaf(w1[4], xo[r][0], a);
        a = fmaf(w1[5], xo[r][1], a);
      } else {
        a = a + w1[4];
      }
      const float hu = rb(fmaxf(a, 0.0f), bf16);
#pragma unroll
      for (int q = 0; q < n4; ++q) ol[r][q] = fmaf(w2[q], hu, ol[r][q]);
    }
  }
#pragma unroll
  for (int r = 0; r < PP; ++r) {
    if (!ok[r]) continue;
    const int j = jv[r], k = kv[r];
    const float* gj = glob + static_cast<size_t>(j) * n4;
    float* dst = out + static_cast<size_t>(k) * stride +
                 (col_of ? static_cast<size_t>(col_of[j]) : static_cast<size_t>(j) * 2 * CC);
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      const float pr = base[(static_cast<size_t>(k) * CC + c) * 2 + 0];
      const float pi = base[(static_cast<size_t>(k) * CC + c) * 2 + 1];
      const float agr = 1.0f + gj[4 * c + 0], agi = gj[4 * c + 1];
      const float ur = agr * pr - agi * pi + gj[4 * c + 2];
      const float ui = agr * pi + agi * pr + gj[4 * c + 3];
      const float alr = 1.0f + ol[r][4 * c], ali = ol[r][4 * c + 1];
      const float sr = alr * ur - ali * ui + ol[r][4 * c + 2];
      const float si = alr * ui + ali * ur + ol[r][4 * c + 3];
      *reinterpret_cast<float2*>(&dst[2 * c]) = make_float2(sr, si);
    }
  }
}

void launch_mlp_global(const MlpParams& m, const float* rx, int N, float* glob, cudaStream_t s,
                       const int* n_dev) {
  if (N <= 0) return;
  mlp_global_kernel<<<N, 128, 0, s>>>(m.p, m.C, m.bf16, rx, glob, n_dev);
  note_launches(1);
}

void launch_mlp_radiance(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, float* out, float* glob,
                         cudaStream_t s, const int* n_dev, const int* col_of, bool clear) {
  if (N <= 0 || K <= 0) return;
  // pad columns of every row stay zero
  if (clear) cudaMemsetAsync(out, 0, sizeof(float) * static_cast<size_t>(K) * stride, s);
  mlp_global_kernel<<<N, 128, 0, s>>>(m.p, m.C, m.bf16, rx, glob, n_dev);
  note_launches(1);
  const size_t pairs = static_cast<size_t>(N) * K;
  switch (m.C) {
#define RXGS_NARROW(CCV, PPV)                                                                  \
  case CCV: {                                                                                 \
    const unsigned nblk = static_cast<unsigned>((pairs + 256 * PPV - 1) / (256 * PPV));       \
    if (m.feat)                                                                               \
      mlp_local_narrow_kernel<CCV, PPV, true><<<nblk, 256, 0, s>>>(                           \
          m.p, m.bf16, rx, N, geom, base, K, stride, glob, out, n_dev, col_of, m.feat);       \
    else                                                                                      \
      mlp_local_narrow_kernel<CCV, PPV, false><<<nblk, 256, 0, s>>>(                          \
          m.p, m.bf16, rx, N, geom, base, K, stride, glob, out, n_dev, col_of, nullptr);      \
    note_launches(1);                                                                         \
    return;                                                                                   \
  }
    RXGS_NARROW(1, 4)
    RXGS_NARROW(2, 4)
    RXGS_NARROW(3, 2)
    RXGS_NARROW(4, 2)
#undef RXGS_NARROW
    default:
      break;
  }
  const size_t smem = sizeof(float) * (kHidden * 7 + 4 * m.C * kHidden + 4 * m.C);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(mlp_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
  mlp_local_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, smem, s>>>(
      m.p, m.C, m.bf16, rx, N, geom, base, K, stride, glob, out, n_dev, col_of, m.feat);
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
// One thread per (j, k) pair, grid-stride with a stride that is a multiple
// of N so each thread keeps one receiver j (phase 1: features, hidden
// layer, outputs, the combination's gradients).  The local-branch weight
// gradients are sums over pairs of outer products (dol x h, dh x x); they
// are accumulated with the warp transposed (phase 2): lane l owns hidden
// units l and l + 32, walks the warp's 32 pairs (features and dol staged in
// shared memory), recomputes h for its units and accumulates in registers.
// At the end warps and blocks are combined in a fixed order.
constexpr int kBwdThreads = 256;

static int mlp_bwd_blocks(int N) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 152;
  }
  int gcd = kBwdThreads, b = N;
  while (b) {
    const int t = gcd % b;
    gcd = b;
    b = t;
  }
  const int m = N / gcd;  // blocks * 256 must be a multiple of N
  int blocks = 2 * sms;
  blocks = blocks < m ? m : (blocks / m) * m;
  return blocks;
}

size_t mlp_backward_tmp_floats(const MlpParams& m, int N, int /*K*/) {
  const int nloc = kHidden * 6 + kHidden + 4 * m.C * kHidden + 4 * m.C;
  const int blocks = mlp_bwd_blocks(N);
  return static_cast<size_t>(blocks) * (nloc + static_cast<size_t>(N) * 4 * m.C) +
         static_cast<size_t>(N) * 4 * m.C;
}

template <int CC, bool OCC>
__global__ void __launch_bounds__(kBwdThreads) mlp_local_bwd_kernel(
    const float* __restrict__ P, const float* __restrict__ rx, int N,
    const float4* __restrict__ geom, const float* __restrict__ base, int K, int stride,
    const float* __restrict__ dS, const float* __restrict__ glob, float* __restrict__ grad_base,
    float* __restrict__ part, const float2* __restrict__ feat, int c0, int Ct) {
  // channels c0 .. c0 + CC - 1 of Ct (one group of a wide spectrum)
  constexpr int n4 = 4 * CC;
  constexpr int nloc = kHidden * 6 + kHidden + n4 * kHidden + n4;
  constexpr int kWarps = kBwdThreads / 32;
  __shared__ float W1[kHidden * 6], B1[kHidden], W2[n4 * kHidden], B2[n4];
  __shared__ float B1x[kHidden];                // B1 + W1[., 4]: the start of a without occlusion
  __shared__ float4 sX[kBwdThreads];            // features of each thread's pair
  __shared__ float2 sO[kBwdThreads];            // its occlusion inputs (T, rho_bar)
  __shared__ float4 sD[kBwdThreads * CC];       // dol of each thread's pair
  extern __shared__ float sdyn[];  // [kWarps][nloc] warp partials, then [256][4C]
  const MlpOffsets o = mlp_offsets(kHidden, Ct);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int e = t; e < kHidden * 6; e += kBwdThreads) W1[e] = P[o.l_w1 + e];
  for (int e = t; e < kHidden; e += kBwdThreads) B1[e] = P[o.l_b1 + e];
  for (int e = t; e < n4 * kHidden; e += kBwdThreads) W2[e] = P[o.l_w2 + 4 * c0 * kHidden + e];
  for (int e = t; e < n4; e += kBwdThreads) B2[e] = P[o.l_b2 + 4 * c0 + e];
  for (int e = t; e < kHidden; e += kBwdThreads) B1x[e] = P[o.l_b1 + e] + P[o.l_w1 + e * 6 + 4];
  __syncthreads();

  // phase-2 operands of this lane's hidden units u = lane, lane + 32
  float w1u[2][6], w2u[2][n4];
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int u = hf * 32 + lane;
#pragma unroll
    for (int i = 0; i < 6; ++i) w1u[hf][i] = W1[u * 6 + i];
#pragma unroll
    for (int q = 0; q < n4; ++q) w2u[hf][q] = W2[q * kHidden + u];
  }
  float b1u[2] = {B1[lane], B1[32 + lane]};
  const float b1x[2] = {B1x[lane], B1x[32 + lane]};

  constexpr int NI = OCC ? 6 : 4;  // inputs with a weight gradient of their own
  float aw2[n4][2], aw1[NI][2], ab1[2], ab2[n4], aog[n4];
#pragma unroll
  for (int q = 0; q < n4; ++q) aw2[q][0] = aw2[q][1] = ab2[q] = aog[q] = 0.0f;
#pragma unroll
  for (int i = 0; i < NI; ++i) aw1[i][0] = aw1[i][1] = 0.0f;
  ab1[0] = ab1[1] = 0.0f;

  const size_t pairs = static_cast<size_t>(N) * K;
  const size_t gstride = static_cast<size_t>(gridDim.x) * kBwdThreads;
  const size_t first = static_cast<size_t>(blockIdx.x) * kBwdThreads + t;
  const int j = static_cast<int>(first % N);  // fixed: gstride is a multiple of N
  const float rxj = rx[3 * j + 0], ryj = rx[3 * j + 1], rzj = rx[3 * j + 2];
  float gj[n4];
#pragma unroll
  for (int q = 0; q < n4; ++q) gj[q] = glob[static_cast<size_t>(j) * 4 * Ct + 4 * c0 + q];

  const size_t rounds = (pairs + gstride - 1) / gstride;
  for (size_t r = 0; r < rounds; ++r) {
    const size_t pair = first + r * gstride;
    const bool ok = pair < pairs;
    const int k = ok ? static_cast<int>(pair / N) : 0;
    float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float2 oc = make_float2(1.0f, 0.0f);  // occlusion inputs (T, rho_bar)
    float dol[n4], db[2 * CC];
#pragma unroll
    for (int q = 0; q < n4; ++q) dol[q] = 0.0f;
#pragma unroll
    for (int q = 0; q < 2 * CC; ++q) db[q] = 0.0f;
    if (ok) {
      const float4 p = geom[3 * k];
      const float vx = rxj - p.x, vy = ryj - p.y, vz = rzj - p.z;
      const float d = sqrtf(vx * vx + vy * vy + vz * vz);
      const float inv = 1.0f / d;
      x[0] = vx * inv;
      x[1] = vy * inv;
      x[2] = vz * inv;
      x[3] = d;
      if (OCC) oc = feat[static_cast<size_t>(j) * K + k];
      // hidden units streamed into the outputs (same summation order as
      // the forward: bias first, then units in ascending order)
      float oall[n4];
#pragma unroll
      for (int q = 0; q < n4; ++q) oall[q] = B2[q];
#pragma unroll 8
      for (int u = 0; u < kHidden; ++u) {
        float a;
        if (OCC) {  // the forward's order: inputs 0..5
          a = B1[u];
#pragma unroll
          for (int i = 0; i < 4; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
          a = fmaf(W1[u * 6 + 4], oc.x, a);
          a = fmaf(W1[u * 6 + 5], oc.y, a);
        } else {
          a = B1x[u];  // input 4 is T = 1, input 5 is rho = 0
#pragma unroll
          for (int i = 0; i < 4; ++i) a = fmaf(W1[u * 6 + i], x[i], a);
        }
        const float hu = fmaxf(a, 0.0f);
#pragma unroll
        for (int q = 0; q < n4; ++q) oall[q] = fmaf(W2[q * kHidden + u], hu, oall[q]);
      }
      const float* gs = dS + static_cast<size_t>(k) * stride + static_cast<size_t>(j) * 2 * Ct + 2 * c0;
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const float ol[4] = {oall[4 * c], oall[4 * c + 1], oall[4 * c + 2], oall[4 * c + 3]};
        const float pr = base[(static_cast<size_t>(k) * Ct + c0 + c) * 2 + 0];
        const float pi = base[(static_cast<size_t>(k) * Ct + c0 + c) * 2 + 1];
        const float agr = 1.0f + gj[4 * c + 0], agi = gj[4 * c + 1];
        const float ur = agr * pr - agi * pi + gj[4 * c + 2];
        const float ui = agr * pi + agi * pr + gj[4 * c + 3];
        const float alr = 1.0f + ol[0], ali = ol[1];
        const float gr = gs[2 * c], gi = gs[2 * c + 1];
        dol[4 * c + 0] = gr * ur + gi * ui;  // dL/da_l = g conj(u)
        dol[4 * c + 1] = gi * ur - gr * ui;
        dol[4 * c + 2] = gr;                 // dL/db_l = g
        dol[4 * c + 3] = gi;
        const float dur = gr * alr + gi * ali, dui = gi * alr - gr * ali;  // g conj(1 + a_l)
        aog[4 * c + 0] += dur * pr + dui * pi;  // dL/da_g = du conj(phi)
        aog[4 * c + 1] += dui * pr - dur * pi;
        aog[4 * c + 2] += dur;                  // dL/db_g = du
        aog[4 * c + 3] += dui;
        db[2 * c + 0] = dur * agr + dui * agi;  // dL/dphi = du conj(1 + a_g)
        db[2 * c + 1] = dui * agr - dur * agi;
      }
    }
    // dL/dphi: one atomic per warp when the warp's pairs share k
    {
      const int k0 = __shfl_sync(0xffffffffu, k, 0);
      const bool same = __all_sync(0xffffffffu, !ok || k == k0) &&
                        __shfl_sync(0xffffffffu, static_cast<int>(ok), 0);
      if (same) {
#pragma unroll
        for (int q = 0; q < 2 * CC; ++q) {
          float y = db[q];
#pragma unroll
          for (int off = 16; off >= 1; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
          if (lane == 0) atomicAdd(&grad_base[(static_cast<size_t>(k0) * Ct + c0) * 2 + q], y);
        }
      } else if (ok) {
#pragma unroll
        for (int q = 0; q < 2 * CC; ++q)
          atomicAdd(&grad_base[(static_cast<size_t>(k) * Ct + c0) * 2 + q], db[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < n4; ++q) ab2[q] += dol[q];
    // ---- phase 2: the warp's 32 pairs, lane = hidden units lane, lane + 32
    sX[t] = make_float4(x[0], x[1], x[2], x[3]);
    if (OCC) sO[t] = oc;
#pragma unroll
    for (int c = 0; c < CC; ++c)
      sD[t * CC + c] = make_float4(dol[4 * c], dol[4 * c + 1], dol[4 * c + 2], dol[4 * c + 3]);
    __syncwarp();
#pragma unroll 4
    for (int pp = 0; pp < 32; ++pp) {
      const int p = warp * 32 + pp;
      const float4 xp = sX[p];
      const float2 op = OCC ? sO[p] : make_float2(1.0f, 0.0f);
      float dv[n4];
#pragma unroll
      for (int c = 0; c < CC; ++c) {
        const float4 d4 = sD[p * CC + c];
        dv[4 * c + 0] = d4.x;
        dv[4 * c + 1] = d4.y;
        dv[4 * c + 2] = d4.z;
        dv[4 * c + 3] = d4.w;
      }
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        float a;
        if (OCC) {
          a = b1u[hf];
          a = fmaf(w1u[hf][0], xp.x, a);
          a = fmaf(w1u[hf][1], xp.y, a);
          a = fmaf(w1u[hf][2], xp.z, a);
          a = fmaf(w1u[hf][3], xp.w, a);
          a = fmaf(w1u[hf][4], op.x, a);
          a = fmaf(w1u[hf][5], op.y, a);
        } else {
          a = b1x[hf];
          a = fmaf(w1u[hf][0], xp.x, a);
          a = fmaf(w1u[hf][1], xp.y, a);
          a = fmaf(w1u[hf][2], xp.z, a);
          a = fmaf(w1u[hf][3], xp.w, a);
        }
        const float hv = fmaxf(a, 0.0f);
        float g = 0.0f;
#pragma unroll
        for (int q = 0; q < n4; ++q) g = fmaf(w2u[hf][q], dv[q], g);
        const float dh = hv > 0.0f ? g : 0.0f;  // dL/dh = W2^T dol on active units
        ab1[hf] += dh;
        aw1[0][hf] = fmaf(dh, xp.x, aw1[0][hf]);
        aw1[1][hf] = fmaf(dh, xp.y, aw1[1][hf]);
        aw1[2][hf] = fmaf(dh, xp.z, aw1[2][hf]);
        aw1[3][hf] = fmaf(dh, xp.w, aw1[3][hf]);
        if (OCC) {
          aw1[NI - 2][hf] = fmaf(dh, op.x, aw1[NI - 2][hf]);
          aw1[NI - 1][hf] = fmaf(dh, op.y, aw1[NI - 1][hf]);
        }
#pragma unroll
        for (int q = 0; q < n4; ++q) aw2[q][hf] = fmaf(dv[q], hv, aw2[q][hf]);
      }
    }
    __syncwarp();  // sX / sD are rewritten in the next round
  }

  // ---- warp partials -> shared, then a fixed-order sum over warps
  float* wp = sdyn + warp * nloc;
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int u = hf * 32 + lane;
#pragma unroll
    for (int i = 0; i < 4; ++i) wp[u * 6 + i] = aw1[i][hf];
    // inputs 4 and 5: the occlusion features, or the constants 1 and 0
    // (the gradient of input 4 then equals the bias gradient)
    wp[u * 6 + 4] = OCC ? aw1[NI - 2][hf] : ab1[hf];
    wp[u * 6 + 5] = OCC ? aw1[NI - 1][hf] : 0.0f;
    wp[kHidden * 6 + u] = ab1[hf];
#pragma unroll
    for (int q = 0; q < n4; ++q) wp[kHidden * 7 + q * kHidden + u] = aw2[q][hf];
  }
#pragma unroll
  for (int q = 0; q < n4; ++q) {
    float y = ab2[q];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) y += __shfl_xor_sync(0xffffffffu, y, off);
    if (lane == 0) wp[kHidden * 7 + n4 * kHidden + q] = y;
  }
  float* og = sdyn + kWarps * nloc;  // [256][4C]
#pragma unroll
  for (int q = 0; q < n4; ++q) og[t * n4 + q] = aog[q];
  __syncthreads();
  float* dst = part + static_cast<size_t>(blockIdx.x) * (nloc + static_cast<size_t>(N) * n4);
  for (int e = t; e < nloc; e += kBwdThreads) {
    float y = 0.0f;
    for (int w = 0; w < kWarps; ++w) y += sdyn[w * nloc + e];
    dst[e] = y;
  }
  const int shift = static_cast<int>((static_cast<size_t>(blockIdx.x) * kBwdThreads) % N);
  for (int e = t; e < N * n4; e += kBwdThreads) {
    const int jj = e / n4, q = e % n4;
    float y = 0.0f;
    for (int tt = (jj - shift + N) % N; tt < kBwdThreads; tt += N) y += og[tt * n4 + q];
    dst[nloc + e] = y;
  }
}

// Sums the block partials in block order: local parameters go into
// grad_mlp, the per-receiver (a_g, b_g) gradients into dog[N][4C].
// Sums the block partials of one channel group (channels c0 .. c0 + cc - 1
// of Ct) in block order: W1 and B1 add into grad_mlp (every group
// contributes), the group's W2 rows and B2 entries go to their places, and
// the per-receiver (a_g, b_g) gradients to dog[N][4 Ct].
__global__ void mlp_partial_reduce_kernel(const float* __restrict__ part, int blocks, int nloc,
                                          int nog, MlpOffsets o, int c0, int cc, int Ct,
                                          float* __restrict__ grad_mlp, float* __restrict__ dog) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nloc + nog) return;
  float s = 0.0f;
  for (int b = 0; b < blocks; ++b) s += part[static_cast<size_t>(b) * (nloc + nog) + e];
  const int n4 = 4 * cc;
  const int w1b1 = kHidden * 7, w2 = n4 * kHidden;
  if (e < w1b1) {
    grad_mlp[o.l_w1 + e] += s;
  } else if (e < w1b1 + w2) {
    grad_mlp[o.l_w2 + 4 * c0 * kHidden + (e - w1b1)] += s;
  } else if (e < nloc) {
    grad_mlp[o.l_b2 + 4 * c0 + (e - w1b1 - w2)] += s;
  } else {
    const int jq = e - nloc, jj = jq / n4, q = jq % n4;
    dog[static_cast<size_t>(jj) * 4 * Ct + 4 * c0 + q] = s;
  }
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

template <int CC>
static void launch_mlp_local_bwd(int blocks, const MlpParams& m, const float* rx, int N,
                                 const float4* geom, const float* base, int K, int stride,
                                 const float* dS, const float* glob, float* grad_base, float* part,
                                 int c0, cudaStream_t s) {
  constexpr int n4 = 4 * CC;
  constexpr int nloc = kHidden * 6 + kHidden + n4 * kHidden + n4;
  const size_t smem = sizeof(float) * ((kBwdThreads / 32) * nloc + kBwdThreads * n4);
  if (m.feat) {
    cudaFuncSetAttribute(mlp_local_bwd_kernel<CC, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    mlp_local_bwd_kernel<CC, true><<<blocks, kBwdThreads, smem, s>>>(
        m.p, rx, N, geom, base, K, stride, dS, glob, grad_base, part, m.feat, c0, m.C);
  } else {
    cudaFuncSetAttribute(mlp_local_bwd_kernel<CC, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    mlp_local_bwd_kernel<CC, false><<<blocks, kBwdThreads, smem, s>>>(
        m.p, rx, N, geom, base, K, stride, dS, glob, grad_base, part, nullptr, c0, m.C);
  }
  note_launches(1);
}

void launch_mlp_backward(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, const float* dS,
                         const float* glob, float* grad_base, float* grad_mlp, float* tmp,
                         cudaStream_t s) {
  const int C = m.C, n4 = 4 * C;
  const int nloc = kHidden * 6 + kHidden + n4 * kHidden + n4;
  const int blocks = mlp_bwd_blocks(N);
  float* part = tmp;  // one channel group's block partials at a time
  float* dog = tmp + static_cast<size_t>(blocks) * (nloc + static_cast<size_t>(N) * n4);
  const MlpOffsets o = mlp_offsets(kHidden, C);
  // channels in groups of up to 4: the hidden-layer gradient is a sum over
  // output channels, so the groups' contributions to W1 and B1 add up
  for (int c0 = 0; c0 < C; c0 += 4) {
    const int cc = C - c0 < 4 ? C - c0 : 4;
    switch (cc) {
      case 1: launch_mlp_local_bwd<1>(blocks, m, rx, N, geom, base, K, stride, dS, glob, grad_base, part, c0, s); break;
      case 2: launch_mlp_local_bwd<2>(blocks, m, rx, N, geom, base, K, stride, dS, glob, grad_base, part, c0, s); break;
      case 3: launch_mlp_local_bwd<3>(blocks, m, rx, N, geom, base, K, stride, dS, glob, grad_base, part, c0, s); break;
      default: launch_mlp_local_bwd<4>(blocks, m, rx, N, geom, base, K, stride, dS, glob, grad_base, part, c0, s); break;
    }
    const int gl = kHidden * 7 + 4 * cc * kHidden + 4 * cc, gog = N * 4 * cc;
    mlp_partial_reduce_kernel<<<(gl + gog + 255) / 256, 256, 0, s>>>(part, blocks, gl, gog, o, c0,
                                                                     cc, C, grad_mlp, dog);
    note_launches(1);
  }
  mlp_global_bwd_kernel<<<1, 256, 0, s>>>(m.p, C, rx, N, dog, grad_mlp);
  note_launches(1);
}

}  // namespace rxgs
