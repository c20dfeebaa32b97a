// fle_bwd_tc.cu -- the coefficient gradient of the FLE radiance (App. E.2;
// the backward of Algorithm 1 eval_fle) as a tcgen05 contraction per
// Gaussian:
//   dL/d(a + i b)_jk,l = G_jkl = sum_v g[v][k][j] conj(Y_vkl)
// with g the gradient of the per-view radiance.  Real-ified with the
// cotangent rows interleaved (row 2j = Re g_j, row 2j + 1 = Im g_j) as the A
// operand (M = 128 rows of 64 receivers, K = 32 views) and the basis of the
// views as two B operands (N = 112 components: Re Y, Im Y):
//   Q1 = g Yr,  Q2 = g Yi   (float32 in TMEM, accumulated over view groups)
//   Re G_j = Q1[2j] + Q2[2j+1],  Im G_j = Q1[2j+1] - Q2[2j]
// (lanes 2j and 2j + 1 exchange one value).  Operands split into two bf16
// terms (three MMAs per product, tc_common.cuh).  The finished tile goes
// through shared memory so that the gradient rows are read, added to and
// written back coalesced (or only written, when the caller asks for the
// gradient itself rather than an accumulation).
//
// One CTA per SM (512 threads) walks jobs (Gaussian, receiver group, view
// group); a group (Gaussian, receiver group) accumulates over its view
// groups in one of two TMEM sets (224 columns each), and its tile is written
// out while the next group's MMAs run.  Operand buffers are double-buffered
// by job with one mbarrier each; every wait is bounded (kErrTimeout).
#include <cuda_bf16.h>

#include <algorithm>

#include "fle_basis.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {
namespace {

constexpr int kThreads = 512;
constexpr int kRx = 64;
constexpr int kViews = 32;
constexpr int kLp = 112;
constexpr int kOct = kLp / 8;
// A[row][v] read MN-major: core (v/8, row/8) at (v/8) * kAK + (row/8) * kAM,
// 8 consecutive rows per 16-byte core row (one view)
constexpr uint32_t kAM = 144, kAK = 16 * kAM;
constexpr uint32_t kABytes = 4 * kAK;
// B[v][l] read MN-major: core (v/8, l/8) at (v/8) * kBK + (l/8) * 128
constexpr uint32_t kBN = 128, kBK = kOct * 128;
constexpr uint32_t kBBytes = 4 * kBK;
constexpr uint32_t kSetBytes = 2 * kABytes + 4 * kBBytes;  // A hi, lo; Yr hi, lo; Yi hi, lo
constexpr int kYPitch = kLp + 1;                           // float2 per basis row
constexpr uint32_t kOffY = 2 * kSetBytes;                  // float2 Y[32][kYPitch]
constexpr uint32_t kOutPitch = kLp + 1;                    // floats per staged row
constexpr uint32_t kOffOut = kOffY + kViews * kYPitch * 8; // float [128][kOutPitch]
constexpr uint32_t kOffNorm = kOffOut + 128 * kOutPitch * 4;  // float N_l|m|[100]
constexpr uint32_t kOffBar = kOffNorm + 100 * 4;
constexpr uint32_t kOffMisc = kOffBar + 16;
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
constexpr uint32_t kTmemCols = 512;  // 2 sets x (Q1: 112, Q2: 112) at 0 and 256
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kIdesc = tc::idesc_bf16(128, kLp, 1, 1);

struct Job {
  int k, j0, v0, nr, nv, grp, last;
};

__device__ __forceinline__ Job job_of(int n, int N, int M) {
  const int njg = (N + kRx - 1) / kRx, nvg = (M + kViews - 1) / kViews;
  const int per_k = njg * nvg;
  const int i = n / per_k, r = n % per_k;
  Job J;
  J.k = blockIdx.x + i * gridDim.x;
  J.j0 = (r / nvg) * kRx;
  J.v0 = (r % nvg) * kViews;
  J.nr = min(kRx, N - J.j0);
  J.nv = min(kViews, M - J.v0);
  J.grp = n / nvg;
  J.last = (r % nvg) == nvg - 1;
  return J;
}

__global__ void __launch_bounds__(kThreads, 1)
    fle_backward_tc_kernel(const float* __restrict__ d_rad, int N, int K, int lmax,
                           const float4* __restrict__ geom, const float* __restrict__ tx, int M,
                           int stride, size_t rad_view, FleNorm nrm, float* __restrict__ grad,
                           int accumulate, unsigned* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  float2* sY = reinterpret_cast<float2*>(sm + kOffY);
  float* sOut = reinterpret_cast<float*>(sm + kOffOut);
  float* sNorm = reinterpret_cast<float*>(sm + kOffNorm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int L = (lmax + 1) * (lmax + 1);
  const uint32_t sbase = tc::smem_u32(sm);
  const int njg = (N + kRx - 1) / kRx, nvg = (M + kViews - 1) / kViews;
  const int nk = blockIdx.x < K ? (K - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int njobs = nk * njg * nvg;
  auto set_off = [](int n) { return (n & 1) ? kSetBytes : 0u; };

  auto stage = [&](int n) {
    const Job J = job_of(n, N, M);
    const uint32_t so = set_off(n);
    fle_basis_group(geom[3 * J.k], tx, J.v0, J.nv, lmax, sNorm, sY, kYPitch, t, kThreads);
    // cotangent rows: thread (view v, row octet ro) loads 8 consecutive
    // columns of the view's radiance row
    {
      const int v = t >> 4, ro = t & 15;
      float x[8];
      const bool ok = v < J.nv && 8 * ro < 2 * J.nr;
      if (ok) {
        const float4* src = reinterpret_cast<const float4*>(
            d_rad + static_cast<size_t>(J.v0 + v) * rad_view + static_cast<size_t>(J.k) * stride +
            2 * J.j0 + 8 * ro);
        const float4 a0 = src[0], a1 = src[1];
        x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
        x[4] = a1.x; x[5] = a1.y; x[6] = a1.z; x[7] = a1.w;
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (8 * ro + e >= 2 * J.nr) x[e] = 0.0f;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0.0f;
      }
      uint4 hi, lo;
      tc::split8(x, hi, lo);
      const uint32_t off = (v >> 3) * kAK + ro * kAM + (v & 7) * 16;
      *reinterpret_cast<uint4*>(sm + so + off) = hi;
      *reinterpret_cast<uint4*>(sm + so + kABytes + off) = lo;
    }
    __syncthreads();  // sY complete
    for (int e = t; e < kViews * kOct; e += kThreads) {
      const int v = e / kOct, o = e % kOct;
      float yr[8], yi[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float2 y = sY[v * kYPitch + 8 * o + q];
        yr[q] = y.x;
        yi[q] = y.y;
      }
      const uint32_t off = (v >> 3) * kBK + o * kBN + (v & 7) * 16;
      uint4 hi, lo;
      tc::split8(yr, hi, lo);
      *reinterpret_cast<uint4*>(sm + so + 2 * kABytes + off) = hi;
      *reinterpret_cast<uint4*>(sm + so + 2 * kABytes + kBBytes + off) = lo;
      tc::split8(yi, hi, lo);
      *reinterpret_cast<uint4*>(sm + so + 2 * kABytes + 2 * kBBytes + off) = hi;
      *reinterpret_cast<uint4*>(sm + so + 2 * kABytes + 3 * kBBytes + off) = lo;
    }
  };
  auto issue = [&](uint32_t tmem, int n) {
    const Job J = job_of(n, N, M);
    const uint32_t so = sbase + set_off(n);
    const uint64_t dA[2] = {tc::smem_desc(so, kAK, kAM), tc::smem_desc(so + kABytes, kAK, kAM)};
    const uint32_t first = J.v0 == 0;
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {  // Q1 (Re Y), Q2 (Im Y)
      const uint32_t yb = so + 2 * kABytes + 2 * pr * kBBytes;
      const uint64_t dB[2] = {tc::smem_desc(yb, kBK, kBN), tc::smem_desc(yb + kBBytes, kBK, kBN)};
      const uint32_t d = tmem + 256 * (J.grp & 1) + kLp * pr;
#pragma unroll
      for (int k = 0; k < kViews / 16; ++k)
#pragma unroll
        for (int term = 0; term < 3; ++term)
          tc::mma_bf16(d, dA[term == 2] + ((2 * k * kAK) >> 4), dB[term == 1] + ((2 * k * kBK) >> 4),
                       kIdesc, !(first && k == 0 && term == 0));
    }
    tc::mma_commit(&bar[n & 1]);
  };
  // the finished tile of job n's group: TMEM -> shared (warps 0-3), then the
  // gradient rows += (all threads)
  auto write_out = [&](uint32_t tmem, int n) {
    const Job J = job_of(n, N, M);
    if (warp < 4) {
      const uint32_t base = tmem + (static_cast<uint32_t>(32 * warp) << 16) + 256 * (J.grp & 1);
      const int row = 32 * warp + lane;
      const bool odd = lane & 1;
#pragma unroll 1
      for (int c0 = 0; c0 < kLp; c0 += 16) {
        float q1a[8], q1b[8], q2a[8], q2b[8];
        tc::tmem_ld8(base + c0, q1a);
        tc::tmem_ld8(base + c0 + 8, q1b);
        tc::tmem_ld8(base + kLp + c0, q2a);
        tc::tmem_ld8(base + kLp + c0 + 8, q2b);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float oa = __shfl_xor_sync(0xffffffffu, q2a[e], 1);
          const float ob = __shfl_xor_sync(0xffffffffu, q2b[e], 1);
          sOut[row * kOutPitch + c0 + e] = odd ? q1a[e] - oa : q1a[e] + oa;
          sOut[row * kOutPitch + c0 + 8 + e] = odd ? q1b[e] - ob : q1b[e] + ob;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // row r = 2j + part -> grad[j0 + j][k][part][l]; 128 threads per row pass
    for (int e = t; e < 2 * J.nr * 128; e += kThreads) {
      const int row = e >> 7, l = e & 127;
      if (l < L) {
        float* dst = grad + (static_cast<size_t>(J.j0 + (row >> 1)) * K + J.k) * 2 * L +
                     (row & 1) * L + l;
        *dst = accumulate ? *dst + sOut[row * kOutPitch + l] : sOut[row * kOutPitch + l];
      }
    }
  };

  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (t == 32) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
    sMisc[1] = 0;
  }
  for (int l = t; l < 100; l += kThreads) sNorm[l] = nrm.n[l];
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sMisc[0];
  auto fail = [&]() {
    atomicOr(&sMisc[1], 1u);
    if (err) atomicOr(err, kErrTimeout);
  };
  for (int n = 0; n < min(2, njobs); ++n) {
    stage(n);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      issue(tmem, n);
    }
  }
  for (int n = 1; n <= njobs; ++n) {
    const int pn = n - 1;
    if (!tc::mbar_wait(&bar[pn & 1], (pn >> 1) & 1, kWaitLimit)) fail();
    tc::fence_after_sync();
    __syncthreads();
    if (sMisc[1]) break;
    if (job_of(pn, N, M).last) write_out(tmem, pn);
    const bool more = n + 1 < njobs;
    if (more) stage(n + 1);  // into operand set (n + 1) & 1 = pn & 1 (job pn is done)
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (more && t == 0) {
      tc::fence_after_sync();
      issue(tmem, n + 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

void launch_fle_backward_tc(const float* d_rad, int N, int K, int lmax, const float4* geom,
                            const float* tx, int M, int stride, size_t rad_view, float* grad,
                            bool accumulate, cudaStream_t s, unsigned* err) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(fle_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmem));
    configured = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(K, nsm));
  fle_backward_tc_kernel<<<grid, kThreads, kSmem, s>>>(d_rad, N, K, lmax, geom, tx, M, stride,
                                                       rad_view, fle_norm_table(lmax), grad,
                                                       accumulate ? 1 : 0, err);
  note_launches(1);
}

}  // namespace rxgs
