// loss.cu -- the L1 term of the Stage II loss (App. E.3) and its cotangent in
// one pass: on the amplitude |R| = sqrt(Re^2 + Im^2 + 1e-8) (App. E.2) of
// rendered spectra, or on RSSI values.
//   L = (1/n) sum_i | a_i - y_i |
//   spectra: dL/dR_i = sign(a_i - y_i) / n * R_i / a_i      (a_i = |R_i|)
//   RSSI:    dL/drssi_i = sign(rssi_i - y_i) / n
// The sum is taken per block (grid-stride, then a fixed-order block
// reduction) and the block partial sums are added in block order by one more
// block, so the loss is the same from run to run.
#include "rxgs_internal.h"

namespace rxgs {

constexpr int kLossThreads = 256;

template <bool kSpectra>
__global__ void __launch_bounds__(kLossThreads) l1_loss_kernel(const float* __restrict__ values,
                                                               const float* __restrict__ target,
                                                               size_t n, float inv_n,
                                                               float* __restrict__ grad,
                                                               float* __restrict__ part) {
  __shared__ float red[kLossThreads / 32];
  float acc = 0.0f;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (kSpectra) {
      const float2 r = reinterpret_cast<const float2*>(values)[i];
      const float a = sqrtf(r.x * r.x + r.y * r.y + 1e-8f);
      const float d = a - target[i];
      acc += fabsf(d);
      const float s = d > 0.0f ? inv_n : (d < 0.0f ? -inv_n : 0.0f);
      reinterpret_cast<float2*>(grad)[i] = make_float2(s * r.x / a, s * r.y / a);
    } else {
      const float d = values[i] - target[i];
      acc += fabsf(d);
      grad[i] = d > 0.0f ? inv_n : (d < 0.0f ? -inv_n : 0.0f);
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
#pragma unroll
    for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void l1_loss_finish_kernel(const float* __restrict__ part, int nparts, float inv_n,
                                      float* __restrict__ loss) {
  __shared__ float red[kLossThreads];
  float s = 0.0f;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[b];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float y = 0.0f;
    for (int t = 0; t < static_cast<int>(blockDim.x); ++t) y += red[t];
    loss[0] = y * inv_n;
  }
}

int l1_loss_blocks() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return 4 * (nsm > 0 ? nsm : 1);
}

void launch_l1_loss(bool spectra, const float* values, const float* target, size_t n, float* loss,
                    float* grad, float* part, int nparts, cudaStream_t s) {
  const float inv_n = n > 0 ? static_cast<float>(1.0 / static_cast<double>(n)) : 0.0f;
  if (spectra)
    l1_loss_kernel<true><<<nparts, kLossThreads, 0, s>>>(values, target, n, inv_n, grad, part);
  else
    l1_loss_kernel<false><<<nparts, kLossThreads, 0, s>>>(values, target, n, inv_n, grad, part);
  l1_loss_finish_kernel<<<1, kLossThreads, 0, s>>>(part, nparts, inv_n, loss);
  note_launches(2);
}

}  // namespace rxgs
