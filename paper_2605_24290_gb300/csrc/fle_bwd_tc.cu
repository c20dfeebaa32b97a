// fle_bwd_tc.cu -- the coefficient gradient of the FLE radiance (App. E.2;
// the backward of Algorithm 1 eval_fle) as a tcgen05 contraction per
// Gaussian, over the folded components (fle_tc.cuh).  With g the gradient
// of the per-view radiance s = sum_P Yr c+ + i sum_Q Yi c-:
//   D+[2j] = sum_v Re g_vj Yr_v,  D+[2j+1] = sum_v Im g_vj Yr_v   (dL/dRe c+, dL/dIm c+)
//   D-[2j] = sum_v Im g_vj Yi_v,  D-[2j+1] = -sum_v Re g_vj Yi_v  (dL/dRe c-, dL/dIm c-)
//   dL/dc_{l,+m} = D+ + D-,  dL/dc_{l,-m} = D+ - D-,  dL/dc_{l,0} = D+
// The A operands (M = 128 rows 2j, 2j + 1, K = 32 views) are the cotangent
// rows and their swapped copy (row 2j = Im g_j, row 2j + 1 = -Re g_j), split
// into bf16 terms and stored in tensor memory; the B operand is the step's
// basis read MN-major (N = components, K = views); D+ and D- accumulate over
// a job's view groups in tensor memory.
//
// Warp-specialised like the forward (fle_tc.cu), on the same basis image:
//   warp 0      one bulk copy of the step's basis block per step;
//   warps 4-7   load the cotangent of a step (lane = row; the loads of the
//               next step are in flight while this one is split and stored);
//   warp 1      one thread issues the MMAs;
//   warps 8-11  read a job's D+ and D- (tcgen05.ld), unfold them into the
//               (lmax + 1)^2 components of the lane's half-row, stage the
//               job's rows in shared memory as one tensor-map box and add it
//               to (or store it into) the gradient with one TMA reduction.
// Every wait is bounded (kErrTimeout).  A degree whose half-rows are not
// whole 16-byte units or an unaligned gradient array is written directly.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "fle_tc.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {
namespace {

using namespace fle;

constexpr int kThreads = 384;
// the gradient rows of a job as one box [64 receivers][2L floats] (the TMA
// layout; at degree 9 the 8 lanes of a quarter warp write 8 bank groups),
// two boxes
constexpr uint32_t kBox = kRx * 200 * 4;
constexpr uint32_t kOffOut = 0;
constexpr uint32_t kOffB = 2 * kBox;
constexpr uint32_t kOffBar = kOffB + 2 * kBStage;
constexpr int kNumBars = 11;
constexpr uint32_t kOffMisc = kOffBar + 8 * kNumBars;
constexpr uint32_t kSmem = kOffMisc + 48;  // TMEM base, abort, write-out flags [2][4]
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffBar % 8 == 0 && kBox % 1024 == 0, "alignment");
constexpr uint32_t kTmemCols = 512;
// tensor memory: D at 128 * (job & 1) (D+: 64 columns, D-: 48 at +64);
// A operands at 256 + 64 * (step & 1): G+ hi, G+ lo, G- hi, G- lo (16 each)
constexpr uint32_t kColA = 256;

template <bool kBulk>
__global__ void __launch_bounds__(kThreads, 1)
    fle_backward_tc_kernel(const float* __restrict__ d_rad, int N, int K, int lmax,
                           const unsigned char* __restrict__ image, int M, int stride,
                           size_t rad_view, float* __restrict__ grad,
                           int accumulate, unsigned* __restrict__ err,
                           const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint64_t* afull = bar;        // [2] A operands of a step in TMEM
  uint64_t* bfull = bar + 2;    // [2] B operand of a step staged
  uint64_t* sdone = bar + 4;    // [2] MMAs of a step complete
  uint64_t* dfull = bar + 6;    // [2] MMAs of a job complete
  uint64_t* dempty = bar + 8;   // [2] a job's D read
  uint64_t* fin = bar + 10;
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);
  volatile uint32_t* abort_flag = &sMisc[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = (lmax + 1) * (lmax + 1);
  const int njobs = jobs_of_cta(K, N), nvg = (M + kViews - 1) / kViews;
  const int nsteps = njobs * nvg;

  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (threadIdx.x == 32) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&afull[i], 4);
      tc::mbar_init(&bfull[i], 1);
      tc::mbar_init(&sdone[i], 1);
      tc::mbar_init(&dfull[i], 1);
      tc::mbar_init(&dempty[i], 4);
    }
    tc::mbar_init(fin, 1);
    tc::mbar_fence_init();
    sMisc[1] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sMisc[0];
  auto fail = [&]() {
    atomicOr(&sMisc[1], 1u);
    if (err) atomicOr(err, kErrTimeout);
  };
  auto wait_warp = [&](uint64_t* b, uint32_t parity) -> bool {
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(b, parity, kWaitLimit));
    if (!ok && lane == 0) fail();
    return ok;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // per step the view group's basis block into one of two B stages
    if (lane == 0) {
      int s = 0, issued = 0;
      bool stop = false;
      JobIter it(K);
      for (int n = 0; n < njobs && !stop; ++n, it.next()) {
        for (int vg = 0; vg < nvg; ++vg, ++s) {
          if (*abort_flag) { stop = true; break; }
          if (s >= 2 && !tc::mbar_wait(&sdone[s & 1], ((s >> 1) - 1) & 1, kWaitLimit)) {
            fail();
            stop = true;
            break;
          }
          tc::mbar_arrive_expect_tx(&bfull[s & 1], kBStage);
          tc::bulk_g2s(sm + kOffB + (s & 1) * kBStage,
                       image + (static_cast<size_t>(it.k) * nvg + vg) * kBStage, kBStage,
                       &bfull[s & 1]);
          issued = s + 1;
        }
      }
      // copies of a walk cut short land before the CTA exits
      for (int q = max(0, issued - 2); q < issued; ++q)
        tc::mbar_wait(&bfull[q & 1], (q >> 1) & 1, kWaitLimit);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const int kp = kp_of(lmax), kq = kq_of(lmax);
      const uint32_t idp = tc::idesc_bf16(128, kp, 0, 1);
      const uint32_t idq = kq > 0 ? tc::idesc_bf16(128, kq, 0, 1) : 0u;
      const uint32_t sb = tc::smem_u32(sm) + kOffB;
      int s = 0;
      bool stop = false;
      for (int n = 0; n < njobs && !stop; ++n) {
        for (int vg = 0; vg < nvg; ++vg, ++s) {
          if (*abort_flag) { stop = true; break; }
          if (!tc::mbar_wait(&afull[s & 1], (s >> 1) & 1, kWaitLimit)) { fail(); stop = true; break; }
          if (!tc::mbar_wait(&bfull[s & 1], (s >> 1) & 1, kWaitLimit)) { fail(); stop = true; break; }
          if (vg == 0 && n >= 2 &&
              !tc::mbar_wait(&dempty[n & 1], ((n >> 1) - 1) & 1, kWaitLimit)) {
            fail(); stop = true; break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + 128 * (n & 1);
          const uint32_t a = tmem + kColA + 64 * (s & 1);
          const uint32_t b = sb + (s & 1) * kBStage;
#pragma unroll
          for (int ks = 0; ks < kViews / 16; ++ks) {
            // B read MN-major: LBO = distance of core matrices 8 views apart,
            // SBO = distance of those 8 components apart
            const uint32_t more = vg == 0 && ks == 0 ? 0u : 1u;
            const uint64_t ph = tc::smem_desc(b + kYrHi + ks * 2 * kSboP, kSboP, 128);
            const uint64_t pl = tc::smem_desc(b + kYrLo + ks * 2 * kSboP, kSboP, 128);
            tc::mma_bf16_ts(d, a + ks * 8, ph, idp, more);
            tc::mma_bf16_ts(d, a + ks * 8, pl, idp, 1);
            tc::mma_bf16_ts(d, a + 16 + ks * 8, ph, idp, 1);
            if (kq > 0) {
              const uint64_t qh = tc::smem_desc(b + kYiHi + ks * 2 * kSboQ, kSboQ, 128);
              const uint64_t ql = tc::smem_desc(b + kYiLo + ks * 2 * kSboQ, kSboQ, 128);
              tc::mma_bf16_ts(d + 64, a + 32 + ks * 8, qh, idq, more);
              tc::mma_bf16_ts(d + 64, a + 32 + ks * 8, ql, idq, 1);
              tc::mma_bf16_ts(d + 64, a + 48 + ks * 8, qh, idq, 1);
            }
          }
          tc::mma_commit(&sdone[s & 1]);
          if (vg == nvg - 1) tc::mma_commit(&dfull[n & 1]);
        }
      }
      tc::mma_commit(fin);
      if (!tc::mbar_wait(fin, 0, kWaitLimit)) fail();
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------------- A operands
    const int q = warp - 4, row = 32 * q + lane;
    const bool odd = lane & 1;
    // (job, view group) of the step being loaded
    JobIter lit(K);
    int lvg = 0;
    auto load = [&](float (&g)[kViews]) {
      const int v0 = lvg * kViews;
      const int nv = min(kViews, M - v0);
      const bool ok = row < 2 * (N - lit.jg * kRx);
      const float* src = d_rad + static_cast<size_t>(lit.k) * stride + 2 * lit.jg * kRx + row +
                         static_cast<size_t>(v0) * rad_view;
#pragma unroll
      for (int v = 0; v < kViews; ++v)
        g[v] = (ok && v < nv) ? src[static_cast<size_t>(v) * rad_view] : 0.0f;
      if (++lvg == nvg) {
        lvg = 0;
        lit.next();
      }
    };
    auto put = [&](int s, const float (&g)[kViews]) -> bool {
      if (*abort_flag) return false;
      if (s >= 2 && !wait_warp(&sdone[s & 1], ((s >> 1) - 1) & 1)) return false;
      tc::fence_after_sync();
      const uint32_t a = tmem + (static_cast<uint32_t>(32 * q) << 16) + kColA + 64 * (s & 1);
      uint32_t h[16], lo[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) tc::split2(g[2 * e], g[2 * e + 1], h[e], lo[e]);
      tc::tmem_st16(a, h);
      tc::tmem_st16(a + 16, lo);
      float x[kViews];  // row 2j: Im g_j, row 2j + 1: -Re g_j
#pragma unroll
      for (int v = 0; v < kViews; ++v) {
        const float o = __shfl_xor_sync(0xffffffffu, g[v], 1);
        x[v] = odd ? -o : o;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) tc::split2(x[2 * e], x[2 * e + 1], h[e], lo[e]);
      tc::tmem_st16(a + 32, h);
      tc::tmem_st16(a + 48, lo);
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&afull[s & 1]);
      return true;
    };
    // two register sets: the loads of step s + 1 are in flight while step s is stored
    float ga[kViews], gb[kViews];
    if (nsteps > 0) load(ga);
    for (int s = 0; s < nsteps; s += 2) {
      if (s + 1 < nsteps) load(gb);
      if (!put(s, ga) || s + 1 >= nsteps) break;
      if (s + 2 < nsteps) load(ga);
      if (!put(s + 1, gb)) break;
    }
  } else if (warp >= 8) {
    // ---------------------------------------------------------------- write-out
    const int q = warp - 8, row = 32 * q + lane, jl = row >> 1, p = row & 1;
    const bool has_q = kq_of(lmax) > 0;
    JobIter it(K);
    // the four warps agree on going on (they meet at named barriers below,
    // so none may leave the walk alone): flags [n & 1][warp], read after
    // the barrier of job n and next written for job n + 2
    volatile uint32_t* go = sMisc + 4;
    for (int n = 0; n < njobs; ++n, it.next()) {
      const bool ok = !*abort_flag && wait_warp(&dfull[n & 1], (n >> 1) & 1);
      if (lane == 0) go[(n & 1) * 4 + q] = ok ? 1u : 0u;
      tc::named_barrier(1, 128);
      if (!(go[(n & 1) * 4] & go[(n & 1) * 4 + 1] & go[(n & 1) * 4 + 2] & go[(n & 1) * 4 + 3]))
        break;
      tc::fence_after_sync();
      uint32_t dp[64], dq[48];
      const uint32_t d = tmem + (static_cast<uint32_t>(32 * q) << 16) + 128 * (n & 1);
      {
        uint32_t r[32];
        tc::tmem_ld32_async(d, r);
#pragma unroll
        for (int e = 0; e < 32; ++e) dp[e] = r[e];
      }
      {
        uint32_t r[32];
        tc::tmem_ld32_async(d + 32, r);
#pragma unroll
        for (int e = 0; e < 32; ++e) dp[32 + e] = r[e];
      }
      {
        uint32_t r[32];
        tc::tmem_ld32_async(d + 64, r);
#pragma unroll
        for (int e = 0; e < 32; ++e) dq[e] = r[e];
      }
      {
        uint32_t r[16];
        tc::tmem_ld16_async(d + 96, r);
#pragma unroll
        for (int e = 0; e < 16; ++e) dq[32 + e] = r[e];
      }
      tc::tmem_wait_ld();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&dempty[n & 1]);
      // the lane's half-row in component order l*l + l + m
      float o[100];
#pragma unroll
      for (int l = 0; l < 10; ++l)
#pragma unroll
        for (int m = -l; m <= l; ++m) {
          const int am = m < 0 ? -m : m;
          const float vp = __uint_as_float(dp[kappa_p(l, am)]);
          const float vq = (am > 0 && has_q) ? __uint_as_float(dq[kappa_q(l, am)]) : 0.0f;
          o[l * l + l + m] = m == 0 ? vp : (m > 0 ? vp + vq : vp - vq);
        }
      const bool on = jl < N - it.jg * kRx;
      if (kBulk) {
        // box n & 1 is free once the copy issued from it two jobs ago has
        // read it; the four warps fill it, then one thread adds (or stores)
        // it to the gradient rows (rows past N are not written)
        if (row == 0) tc::bulk_wait_read<1>();
        tc::named_barrier(1, 128);
        unsigned char* box = sm + kOffOut + (n & 1) * kBox;
        if (on) {
          float4* srow = reinterpret_cast<float4*>(box + (jl * 2 * L + p * L) * 4);
#pragma unroll
          for (int t = 0; t < 25; ++t)
            if (4 * t < L) srow[t] = make_float4(o[4 * t], o[4 * t + 1], o[4 * t + 2], o[4 * t + 3]);
        }
        tc::fence_smem_to_async();
        tc::named_barrier(1, 128);
        if (row == 0) {
          if (accumulate)
            tc::tma_reduce_add_3d(&tmap, 0, it.k, it.jg * kRx, box);
          else
            tc::tma_store_3d(&tmap, 0, it.k, it.jg * kRx, box);
          tc::bulk_commit();
        }
      } else if (on) {
        float* dst = grad + (static_cast<size_t>(it.jg * kRx + jl) * K + it.k) * 2 * L + p * L;
#pragma unroll
        for (int i = 0; i < 100; ++i)
          if (i < L) dst[i] = accumulate ? dst[i] + o[i] : o[i];
      }
    }
    if (kBulk && row == 0) tc::bulk_wait_all();
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool kBulk>
void launch_backward(const float* d_rad, int N, int K, int lmax, const unsigned char* image,
                     int M, int stride, size_t rad_view, float* grad, bool accumulate, int grid,
                     cudaStream_t s, unsigned* err, const CUtensorMap& tmap) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(fle_backward_tc_kernel<kBulk>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmem));
    configured = true;
  }
  fle_backward_tc_kernel<kBulk><<<grid, kThreads, kSmem, s>>>(
      d_rad, N, K, lmax, image, M, stride, rad_view, grad, accumulate ? 1 : 0, err, tmap);
}

}  // namespace

void launch_fle_backward_tc(const float* d_rad, int N, int K, int lmax,
                            const unsigned char* image, int M, int stride, size_t rad_view,
                            float* grad, bool accumulate, cudaStream_t s, unsigned* err) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long jobs = static_cast<long long>(K) * ((N + kRx - 1) / kRx);
  const int grid = static_cast<int>(std::max(1LL, std::min<long long>(jobs, nsm)));
  const int L = (lmax + 1) * (lmax + 1);
  CUtensorMap tmap{};
  if (encode_fle_rows(&tmap, grad, N, K, L))
    launch_backward<true>(d_rad, N, K, lmax, image, M, stride, rad_view, grad, accumulate, grid, s,
                          err, tmap);
  else
    launch_backward<false>(d_rad, N, K, lmax, image, M, stride, rad_view, grad, accumulate, grid,
                           s, err, tmap);
  note_launches(1);
}

}  // namespace rxgs
