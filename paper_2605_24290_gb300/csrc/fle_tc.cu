// fle_tc.cu -- the FLE directional radiance (App. E.2; Algorithm 1 eval_fle)
// as a tcgen05 contraction per Gaussian.
//
// For Gaussian k, receivers j (a group of 64) and views v (a group of 32):
//   s[v][k][j] = sum_l Y_vl (c_jl),   Y_vl = N_l|m| P_l^|m|(cos theta_v) e^{i m phi_v}
// with c_jl the coefficients (a + i b)_jk,l (given, or formed from the base
// coefficients by the global FiLM branch, film_coeffs below).  Real-ified, with the
// coefficient rows interleaved (row 2j = Re c_j, row 2j + 1 = Im c_j) as the
// A operand (M = 128, K = components padded to a multiple of 16) and the
// basis of the 32 views as two B operands (N = 32: Re Y and Im Y):
//   P1 = A Yr^T,  P2 = A Yi^T   (float32 in TMEM)
//   Re s_j = P1[2j] - P2[2j+1],  Im s_j = P1[2j+1] + P2[2j]
// so lanes 2j and 2j + 1 of a warp exchange one value (shuffle) and row r of
// the accumulator is column r of the radiance row the views write.  Operands
// are split into two bf16 terms (three MMAs per product, tc_common.cuh).
//
// One CTA per SM (512 threads) walks jobs (Gaussian, receiver group, view
// group) with two operand buffers and two TMEM accumulator sets: while the
// MMAs of job n run, the threads write out job n - 1 (warps 0-3 read its
// accumulators) and stage job n + 1 (basis evaluated in float32 per (view,
// order m) and split; coefficients split from registers that were loaded a
// whole iteration earlier, so their memory latency is hidden).  Each buffer
// set has its own mbarrier, so no wait is ever more than one phase behind;
// every wait is bounded (kErrTimeout).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fle_basis.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {

// N_l|m| = sqrt((2l + 1) / (4 pi) (l - |m|)! / (l + |m|)!) by component index
// l*l + l + m (the orthonormal basis of App. E.2).
FleNorm fle_norm_table(int lmax) {
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

namespace {

constexpr int kThreads = 512;
constexpr int kRx = 64;      // receivers per job (128 accumulator rows)
constexpr int kViews = 32;   // views per job (N of the MMA)
constexpr int kLp = 112;     // components, padded: (lmax + 1)^2 <= 100
constexpr int kOct = kLp / 8;
// A[row][l]: core (row/8, l/8) at (row/8) * kSboA + (l/8) * 128 (K-major)
// B[v][l]  : core (v/8, l/8)   at (v/8) * kSboB + (l/8) * 128 (K-major)
constexpr uint32_t kLbo = 128;
constexpr uint32_t kSboA = kOct * 128, kSboB = kOct * 128;
constexpr uint32_t kABytes = 16 * kSboA;  // 128 rows
constexpr uint32_t kBBytes = 4 * kSboB;   // 32 views
// per buffer set: A hi, A lo, Yr hi, Yr lo, Yi hi, Yi lo
constexpr uint32_t kSetBytes = 2 * kABytes + 4 * kBBytes;
constexpr uint32_t kOffSet0 = 0, kOffSet1 = kSetBytes;
constexpr int kYPitch = kLp + 1;                           // float2 per basis row (bank spread)
constexpr uint32_t kOffY = 2 * kSetBytes;                  // float2 Y[32][kYPitch] (float32 basis)
constexpr uint32_t kOffNorm = kOffY + kViews * kYPitch * 8; // float N_l|m|[100]
constexpr uint32_t kOffBar = kOffNorm + 100 * 4;            // u64 [2]
constexpr uint32_t kOffMisc = kOffBar + 16;                 // TMEM base, abort
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "shared memory");
constexpr uint32_t kTmemCols = 128;  // 2 sets x (P1: 32, P2: 32)
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kIdesc = tc::idesc_bf16(128, kViews, 0, 0);

struct Job {
  int k, j0, v0, nr, nv;
};

__device__ __forceinline__ Job job_of(int n, int K, int N, int M) {
  const int njg = (N + kRx - 1) / kRx, nvg = (M + kViews - 1) / kViews;
  const int per_k = njg * nvg;
  const int i = n / per_k, r = n % per_k;
  Job J;
  J.k = blockIdx.x + i * gridDim.x;
  J.j0 = (r / nvg) * kRx;
  J.v0 = (r % nvg) * kViews;
  J.nr = min(kRx, N - J.j0);
  J.nv = min(kViews, M - J.v0);
  (void)K;
  return J;
}

__device__ __forceinline__ void put16(unsigned char* base, uint32_t off, const uint4& x) {
  *reinterpret_cast<uint4*>(base + off) = x;
}

}  // namespace

namespace {

// Coefficient tasks of one job: (receiver j, component octet o), thread t
// takes tasks t and t + 512; the 16 values of a task (8 real, 8 imaginary
// parts) are loaded one iteration ahead of their conversion.
constexpr int kTasks = kRx * kOct;
constexpr int kTasksPerThread = (kTasks + kThreads - 1) / kThreads;
struct ARegs {
  float4 v[kTasksPerThread][4];
};

__global__ void __launch_bounds__(kThreads, 1)
    fle_radiance_tc_kernel(const float* __restrict__ coeffs, int N, int K, int lmax,
                           const float4* __restrict__ geom, const float* __restrict__ tx, int M,
                           int stride, size_t rad_view, FleNorm nrm, float* __restrict__ rad,
                           unsigned* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  float2* sY = reinterpret_cast<float2*>(sm + kOffY);
  float* sNorm = reinterpret_cast<float*>(sm + kOffNorm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int L = (lmax + 1) * (lmax + 1);
  const uint32_t sbase = tc::smem_u32(sm);
  const int njg = (N + kRx - 1) / kRx, nvg = (M + kViews - 1) / kViews;
  const int nk = static_cast<int>(blockIdx.x) < K ? (K - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
  const int njobs = nk * njg * nvg;
  auto set_off = [](int n) { return (n & 1) ? kOffSet1 : kOffSet0; };

  // coefficient rows of job n into registers
  auto load_A = [&](int n, ARegs& R) {
    const Job J = job_of(n, K, N, M);
#pragma unroll
    for (int u = 0; u < kTasksPerThread; ++u) {
      const int e = t + u * kThreads;
      const int j = e / kOct, o = e % kOct;
#pragma unroll
      for (int q = 0; q < 4; ++q) R.v[u][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e >= kTasks || j >= J.nr || 8 * o >= L) continue;
      const float* c = coeffs + (static_cast<size_t>(J.j0 + j) * K + J.k) * 2 * L;
      if (8 * o + 8 <= L && (L & 3) == 0) {
        const float4* c4 = reinterpret_cast<const float4*>(c + 8 * o);
        const float4* d4 = reinterpret_cast<const float4*>(c + L + 8 * o);
        R.v[u][0] = c4[0];
        R.v[u][1] = c4[1];
        R.v[u][2] = d4[0];
        R.v[u][3] = d4[1];
      } else {
        float re[8], im[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int l = 8 * o + q;
          re[q] = l < L ? c[l] : 0.0f;
          im[q] = l < L ? c[L + l] : 0.0f;
        }
        R.v[u][0] = make_float4(re[0], re[1], re[2], re[3]);
        R.v[u][1] = make_float4(re[4], re[5], re[6], re[7]);
        R.v[u][2] = make_float4(im[0], im[1], im[2], im[3]);
        R.v[u][3] = make_float4(im[4], im[5], im[6], im[7]);
      }
    }
  };
  // ... split into bf16 terms, rows 2j (real) and 2j + 1 (imaginary)
  auto store_A = [&](int n, const ARegs& R) {
    const uint32_t so = set_off(n);
#pragma unroll
    for (int u = 0; u < kTasksPerThread; ++u) {
      const int e = t + u * kThreads;
      if (e >= kTasks) continue;
      const int j = e / kOct, o = e % kOct;
      const float re[8] = {R.v[u][0].x, R.v[u][0].y, R.v[u][0].z, R.v[u][0].w,
                           R.v[u][1].x, R.v[u][1].y, R.v[u][1].z, R.v[u][1].w};
      const float im[8] = {R.v[u][2].x, R.v[u][2].y, R.v[u][2].z, R.v[u][2].w,
                           R.v[u][3].x, R.v[u][3].y, R.v[u][3].z, R.v[u][3].w};
      uint4 hi, lo;
      const int r0 = 2 * j;
      const uint32_t off0 = (r0 >> 3) * kSboA + o * kLbo + (r0 & 7) * 16;
      tc::split8(re, hi, lo);
      put16(sm, so + off0, hi);
      put16(sm, so + kABytes + off0, lo);
      tc::split8(im, hi, lo);
      put16(sm, so + off0 + 16, hi);  // row 2j + 1 (same core matrix)
      put16(sm, so + kABytes + off0 + 16, lo);
    }
  };
  // basis of job n's views, split into Re / Im bf16 terms
  auto stage_B = [&](int n) {
    const Job J = job_of(n, K, N, M);
    const uint32_t so = set_off(n);
    fle_basis_group(geom[3 * J.k], tx, J.v0, J.nv, lmax, sNorm, sY, kYPitch, t, kThreads);
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
      const uint32_t off = (v >> 3) * kSboB + o * kLbo + (v & 7) * 16;
      uint4 hi, lo;
      tc::split8(yr, hi, lo);
      put16(sm, so + 2 * kABytes + off, hi);
      put16(sm, so + 2 * kABytes + kBBytes + off, lo);
      tc::split8(yi, hi, lo);
      put16(sm, so + 2 * kABytes + 2 * kBBytes + off, hi);
      put16(sm, so + 2 * kABytes + 3 * kBBytes + off, lo);
    }
  };
  // ---- MMAs of job n (thread 0)
  auto issue = [&](uint32_t tmem, int n) {
    const uint32_t so = sbase + set_off(n);
    const uint64_t dA[2] = {tc::smem_desc(so, kLbo, kSboA), tc::smem_desc(so + kABytes, kLbo, kSboA)};
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {  // P1 (Re Y), P2 (Im Y)
      const uint32_t yb = so + 2 * kABytes + 2 * pr * kBBytes;
      const uint64_t dB[2] = {tc::smem_desc(yb, kLbo, kSboB), tc::smem_desc(yb + kBBytes, kLbo, kSboB)};
      const uint32_t d = tmem + 64 * (n & 1) + 32 * pr;
#pragma unroll
      for (int k = 0; k < kOct / 2; ++k)
#pragma unroll
        for (int term = 0; term < 3; ++term)
          tc::mma_bf16(d, dA[term == 2] + ((2 * k * kLbo) >> 4), dB[term == 1] + ((2 * k * kLbo) >> 4),
                       kIdesc, (k | term) != 0);
    }
    tc::mma_commit(&bar[n & 1]);
  };
  // ---- write-out of job n (warps 0-3: accumulator rows = radiance columns)
  auto write_out = [&](uint32_t tmem, int n) {
    const Job J = job_of(n, K, N, M);
    const uint32_t lanes = static_cast<uint32_t>(32 * warp) << 16;
    float p1[32], p2[32];
    tc::tmem_ld32(tmem + lanes + 64 * (n & 1), p1);
    tc::tmem_ld32(tmem + lanes + 64 * (n & 1) + 32, p2);
    const int row = 32 * warp + lane;  // 2j + part
    const bool odd = lane & 1;
    const bool ok = row < 2 * J.nr;
    float* dst = rad + static_cast<size_t>(J.k) * stride + 2 * J.j0 + row;
#pragma unroll
    for (int v = 0; v < kViews; ++v) {
      const float other = __shfl_xor_sync(0xffffffffu, p2[v], 1);
      const float val = odd ? p1[v] + other : p1[v] - other;
      if (ok && v < J.nv) dst[static_cast<size_t>(J.v0 + v) * rad_view] = val;
    }
  };

  // ---- set-up
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
  ARegs R;
  // prologue: jobs 0 and 1 staged and issued, job 2's coefficients in flight
  for (int n = 0; n < min(2, njobs); ++n) {
    load_A(n, R);
    stage_B(n);
    store_A(n, R);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0) {
      tc::fence_after_sync();
      issue(tmem, n);
    }
  }
  if (njobs > 2) load_A(2, R);
  // steady state: job n - 1 written out and job n + 1 staged while job n runs
  for (int n = 1; n <= njobs; ++n) {
    const int pn = n - 1;  // the job to finish
    if (!tc::mbar_wait(&bar[pn & 1], (pn >> 1) & 1, kWaitLimit)) fail();
    tc::fence_after_sync();
    __syncthreads();
    if (sMisc[1]) break;
    if (warp < 4) write_out(tmem, pn);
    const bool more = n + 1 < njobs;
    if (more) {
      stage_B(n + 1);  // into set (n + 1) & 1 = pn & 1, free since job pn is done
      store_A(n + 1, R);
      if (n + 2 < njobs) load_A(n + 2, R);  // arrives during the next iteration
    }
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

void launch_fle_radiance_tc(const float* coeffs, int N, int K, int lmax, const float4* geom,
                            const float* tx, int M, int stride, size_t rad_view, float* rad,
                            cudaStream_t s, unsigned* err) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(fle_radiance_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmem));
    configured = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(K, nsm));
  fle_radiance_tc_kernel<<<grid, kThreads, kSmem, s>>>(coeffs, N, K, lmax, geom, tx, M, stride,
                                                       rad_view, fle_norm_table(lmax), rad, err);
  note_launches(1);
}

}  // namespace rxgs

namespace rxgs {

// ---- the global FiLM branch over the FLE coefficients (Eq. film_apply)
// c[j][k][.][l] = (1 + a_jl) base[k][.][l] + b_jl (complex), ab[j][l] =
// (a.re, a.im, b.re, b.im): the coefficients that the tensor-core contraction
// above then reduces against the basis.  With the local branch (loc[j][k] =
// (alpha.re, alpha.im, beta.re, beta.im), Eq. combined_local) they become
// (1 + alpha_jk) c_jkl + beta_jk.
__global__ void film_coeffs_kernel(const float* __restrict__ base, const float4* __restrict__ ab,
                                   const float4* __restrict__ loc, int N, int K, int L,
                                   float* __restrict__ out) {
  const size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;  // (j, k, l)
  const size_t total = static_cast<size_t>(N) * K * L;
  if (idx >= total) return;
  const int l = static_cast<int>(idx % L);
  const size_t jk = idx / L;
  const int k = static_cast<int>(jk % K), j = static_cast<int>(jk / K);
  const float4 q = ab[static_cast<size_t>(j) * L + l];
  const float pr = base[static_cast<size_t>(k) * 2 * L + l];
  const float pi = base[static_cast<size_t>(k) * 2 * L + L + l];
  const float ar = 1.0f + q.x;
  float cr = fmaf(ar, pr, fmaf(-q.y, pi, q.z));
  float ci = fmaf(ar, pi, fmaf(q.y, pr, q.w));
  if (loc) {
    const float4 lf = loc[jk];
    const float alr = 1.0f + lf.x;
    const float r = fmaf(alr, cr, fmaf(-lf.y, ci, lf.z));
    ci = fmaf(alr, ci, fmaf(lf.y, cr, lf.w));
    cr = r;
  }
  float* o = out + jk * 2 * L;
  o[l] = cr;
  o[L + l] = ci;
}

void launch_film_coeffs(const float* base, const float4* ab, const float4* loc, int N, int K,
                        int lmax, float* out, cudaStream_t s) {
  const int L = (lmax + 1) * (lmax + 1);
  const size_t total = static_cast<size_t>(N) * K * L;
  if (total == 0) return;
  film_coeffs_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(base, ab, loc, N,
                                                                               K, L, out);
  note_launches(1);
}

// ---- its backward, from the coefficient gradient G[j][k][.][l]:
//   dL/dbase_kl = sum_j conj(1 + a_jl) G_jkl      (film_fold_base: a block holds
//                 the modulation of all receivers in shared memory and takes
//                 a range of Gaussians, one thread per component)
//   dL/da_jl    = sum_k conj(base_kl) G_jkl,  dL/db_jl = sum_k G_jkl
//                 (film_fold_ab: a block per (receiver, range of Gaussians),
//                 one thread per component, one float atomic per entry)
constexpr int kFoldBaseK = 64;   // Gaussians per block
constexpr int kFoldAbK = 1024;   // Gaussians per block

__global__ void film_fold_base_kernel(const float* __restrict__ G, const float4* __restrict__ ab,
                                      int N, int K, int L, float* __restrict__ grad_base) {
  extern __shared__ float4 sAb[];  // [N][L]
  for (int e = threadIdx.x; e < N * L; e += blockDim.x) sAb[e] = ab[e];
  __syncthreads();
  const int l = threadIdx.x;
  if (l >= L) return;
  const int k0 = blockIdx.x * kFoldBaseK, k1 = min(K, k0 + kFoldBaseK);
  for (int k = k0; k < k1; ++k) {
    float sr = 0.0f, si = 0.0f;
    for (int j = 0; j < N; ++j) {
      const float* g = G + (static_cast<size_t>(j) * K + k) * 2 * L;
      const float gr = g[l], gi = g[L + l];
      const float4 q = sAb[j * L + l];
      const float ar = 1.0f + q.x, ai = q.y;  // conj(1 + a) G
      sr = fmaf(ar, gr, fmaf(ai, gi, sr));
      si = fmaf(ar, gi, fmaf(-ai, gr, si));
    }
    grad_base[static_cast<size_t>(k) * 2 * L + l] += sr;
    grad_base[static_cast<size_t>(k) * 2 * L + L + l] += si;
  }
}

__global__ void film_fold_ab_kernel(const float* __restrict__ G, const float* __restrict__ base,
                                    int K, int L, float* __restrict__ d_ab) {
  const int l = threadIdx.x, j = blockIdx.y;
  if (l >= L) return;
  const int k0 = blockIdx.x * kFoldAbK, k1 = min(K, k0 + kFoldAbK);
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int k = k0; k < k1; ++k) {
    const float* g = G + (static_cast<size_t>(j) * K + k) * 2 * L;
    const float gr = g[l], gi = g[L + l];
    const float pr = base[static_cast<size_t>(k) * 2 * L + l];
    const float pi = base[static_cast<size_t>(k) * 2 * L + L + l];
    acc.x = fmaf(pr, gr, fmaf(pi, gi, acc.x));  // conj(base) G
    acc.y = fmaf(pr, gi, fmaf(-pi, gr, acc.y));
    acc.z += gr;
    acc.w += gi;
  }
  float* dst = d_ab + (static_cast<size_t>(j) * L + l) * 4;
  atomicAdd(dst + 0, acc.x);
  atomicAdd(dst + 1, acc.y);
  atomicAdd(dst + 2, acc.z);
  atomicAdd(dst + 3, acc.w);
}

void launch_film_fold(const float* G, int N, int K, int lmax, const float* base,
                      const float4* ab, float* grad_base, float* d_ab, cudaStream_t s) {
  const int L = (lmax + 1) * (lmax + 1);
  if (N <= 0 || K <= 0) return;
  if (grad_base) {
    const size_t smem = sizeof(float4) * static_cast<size_t>(N) * L;
    cudaFuncSetAttribute(film_fold_base_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    film_fold_base_kernel<<<(K + kFoldBaseK - 1) / kFoldBaseK, 128, smem, s>>>(G, ab, N, K, L,
                                                                              grad_base);
    note_launches(1);
  }
  if (d_ab) {
    film_fold_ab_kernel<<<dim3((K + kFoldAbK - 1) / kFoldAbK, N), 128, 0, s>>>(G, base, K, L, d_ab);
    note_launches(1);
  }
}

}  // namespace rxgs
