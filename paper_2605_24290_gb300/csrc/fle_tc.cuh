// fle_tc.cuh -- pieces shared by the tensor-core FLE kernels (fle_tc.cu,
// fle_bwd_tc.cu): the folded component order, the job/step walk and the
// basis operand of one group of views.
//
// Folding +m and -m (App. E.2).  With Y_{l,m} = N_l|m| P_l^|m|(cos theta)
// e^{i m phi} the basis of -m is the conjugate of that of +m, so writing
// Yr = N P cos(m phi), Yi = N P sin(m phi) (m >= 0):
//   sum_{m=-l..l} Y_{l,m} c_{l,m} = sum_{m>=0} Yr c+_{l,m} + i sum_{m>0} Yi c-_{l,m}
//   c+_{l,m} = c_{l,m} + c_{l,-m} (m > 0),  c+_{l,0} = c_{l,0},  c-_{l,m} = c_{l,m} - c_{l,-m}
// which halves the contraction: (lmax+1)(lmax+2)/2 "P" components (l, m >= 0)
// against Yr and lmax(lmax+1)/2 "Q" components (l, m > 0) against Yi,
// instead of (lmax+1)^2 against each of Re Y and Im Y.  The components are
// ordered l-major: kappa_p(l, m) = l(l+1)/2 + m, kappa_q(l, m) = l(l-1)/2 + m - 1.
// The gradient unfolds the same way: dL/dc_{l,+-m} = dL/dc+ +- dL/dc-.
//
// Operand layouts (fixed at the lmax = 9 extents, a smaller degree runs
// fewer K steps): the basis of one step (32 views, lane = view) as K-major
// core matrices of 8 views x 8 components, Yr over kP = 64 and Yi over
// kQ = 48 components, each as hi and lo bf16 terms (14,336 bytes).
#pragma once
#include <cuda.h>

#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {
namespace fle {

constexpr int kRx = 64;      // receivers per job (128 accumulator rows: 2j, 2j + 1)
constexpr int kViews = 32;   // views per step
constexpr int kP = 64;       // P components, padded (55 at lmax = 9)
constexpr int kQ = 48;       // Q components, padded (45 at lmax = 9)
constexpr uint32_t kSboP = (kP / 8) * 128;  // distance of core matrices 8 views apart
constexpr uint32_t kSboQ = (kQ / 8) * 128;
constexpr uint32_t kYrHi = 0, kYrLo = 4 * kSboP, kYiHi = 8 * kSboP, kYiLo = 8 * kSboP + 4 * kSboQ;
constexpr uint32_t kBStage = 8 * kSboP + 8 * kSboQ;  // 14,336 bytes
constexpr uint32_t kWaitLimit = 1u << 20;

// The coefficient (or gradient) array [N][K][2L] float32 as a rank-3 tensor
// (2L, K, N) whose box of 2L x 1 x min(64, N) elements is the half-row pairs
// of one job (Gaussian k, receivers j0 ..): one TMA copy per job.  False when
// the encoder is unavailable or refuses the layout (the kernels then read or
// write the rows directly).
bool encode_fle_rows(CUtensorMap* map, const float* base, int N, int K, int L);

__host__ __device__ constexpr int kappa_p(int l, int m) { return l * (l + 1) / 2 + m; }
__host__ __device__ constexpr int kappa_q(int l, int m) { return l * (l - 1) / 2 + m - 1; }
// K extents (multiples of 16) of a degree
__host__ __device__ inline int kp_of(int lmax) { return ((lmax + 1) * (lmax + 2) / 2 + 15) & ~15; }
__host__ __device__ inline int kq_of(int lmax) { return (lmax * (lmax + 1) / 2 + 15) & ~15; }

// The CTA's jobs are (Gaussian k, receiver group jg) for global index
// g = blockIdx.x + n * gridDim.x (n = 0, 1, ...), k = g % K, jg = g / K; each
// job has one step per group of 32 views.  The iterator advances (k, jg)
// without divisions.
__device__ __forceinline__ int jobs_of_cta(int K, int N) {
  const long long total = static_cast<long long>(K) * ((N + kRx - 1) / kRx);
  const long long b = blockIdx.x;
  return b < total ? static_cast<int>((total - 1 - b) / gridDim.x + 1) : 0;
}
struct JobIter {
  int K, k, jg;
  __device__ explicit JobIter(int K_) : K(K_), k(static_cast<int>(blockIdx.x)), jg(0) {
    while (k >= K) {
      k -= K;
      ++jg;
    }
  }
  __device__ void next() {
    k += static_cast<int>(gridDim.x);
    while (k >= K) {
      k -= K;
      ++jg;
    }
  }
};

// Eight values of one view's row -> hi and lo 16-byte core rows.
__device__ __forceinline__ void put_octet(unsigned char* hi, unsigned char* lo, uint32_t off,
                                          const float (&x)[8]) {
  uint4 h, l;
  tc::split2(x[0], x[1], h.x, l.x);
  tc::split2(x[2], x[3], h.y, l.y);
  tc::split2(x[4], x[5], h.z, l.z);
  tc::split2(x[6], x[7], h.w, l.w);
  *reinterpret_cast<uint4*>(hi + off) = h;
  *reinterpret_cast<uint4*>(lo + off) = l;
}

// Scratch row pitch of the float32 basis (odd: the lanes' rows fall in
// different banks).
constexpr int kBPitch = kP + kQ + 1;
constexpr uint32_t kBScratch = 32 * kBPitch * 4;  // bytes per basis warp

// The basis operands of one step: lane = view v0 + lane (zero rows past nv),
// direction u = p - t_v (polar angle from +z, azimuth atan2(u_y, u_x)),
// y_lm = N_lm P_l^m(cos theta) by the recurrence in l of `rec` (shared, see
// FleRec; no Condon-Shortley phase), e^{i m phi} by repeated complex
// products.  Each degree l updates the ten orders at once (independent
// chains), m from high to low so that the diagonal reads y_{l-1,l-1} before
// it is replaced.  The values go to the lane's float32 scratch row (P
// components, then Q), then 8 at a time into hi and lo core rows.  Ends with
// the proxy fence that makes the rows visible to the tensor core.
__device__ __forceinline__ void basis_rows(unsigned char* stage, float* scratch, const float4 p,
                                           const float* __restrict__ tx, int v0, int nv, int lmax,
                                           const float2* rec, int lane) {
  const bool on = lane < nv;
  float ct = 1.0f, st = 0.0f, cp = 1.0f, sp = 0.0f;
  if (on) {
    const float ux = p.x - tx[3 * (v0 + lane)], uy = p.y - tx[3 * (v0 + lane) + 1],
                uz = p.z - tx[3 * (v0 + lane) + 2];
    const float hh2 = ux * ux + uy * uy;
    const float rho2 = hh2 + uz * uz;
    // a centre on the transmitter itself (culled by the projection anyway)
    // takes the +z direction
    const float irho = rho2 > 0.0f ? rsqrtf(rho2) : 0.0f;
    const float ihh = hh2 > 0.0f ? rsqrtf(hh2) : 0.0f;
    ct = rho2 > 0.0f ? uz * irho : 1.0f;
    st = hh2 * ihh * irho;
    cp = hh2 > 0.0f ? ux * ihh : 1.0f;
    sp = uy * ihh;
  }
  const float zero = on ? 1.0f : 0.0f;  // rows past nv are zero
  float cm[10], sn[10];
  cm[0] = zero;
  sn[0] = 0.0f;
#pragma unroll
  for (int m = 1; m < 10; ++m) {
    cm[m] = cm[m - 1] * cp - sn[m - 1] * sp;
    sn[m] = cm[m - 1] * sp + sn[m - 1] * cp;
  }
  float* row = scratch + lane * kBPitch;
  const int np = (lmax + 1) * (lmax + 2) / 2, nq = lmax * (lmax + 1) / 2;
  for (int e = np; e < kP; ++e) row[e] = 0.0f;
  for (int e = nq; e < kQ; ++e) row[kP + e] = 0.0f;
  float p1[10], p2[10];  // y_{l-1,m}, y_{l-2,m}
#pragma unroll
  for (int m = 0; m < 10; ++m) p1[m] = p2[m] = 0.0f;
#pragma unroll 1
  for (int l = 0; l <= lmax; ++l) {
    const float2* rl = rec + 10 * l;
    float* rp = row + l * (l + 1) / 2;
    float* rq = row + kP + l * (l - 1) / 2 - 1;
    // the degree's table row first (no scratch store may come between: the
    // compiler cannot tell the scratch and the table apart), then the ten
    // orders branch-free (orders past l computed and dropped)
    float2 cr[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) cr[m] = rl[m];
#pragma unroll
    for (int m = 9; m >= 0; --m) {
      const float2 c = cr[m];
      const float off = c.x * ct * p1[m] - c.y * p2[m];
      const float diag = m == 0 ? c.x : c.x * st * p1[m > 0 ? m - 1 : 0];
      const bool live = m <= l;
      const float y = m == l ? diag : off;
      if (live) {
        rp[m] = y * cm[m];
        if (m > 0) rq[m] = y * sn[m];
      }
      p2[m] = live ? p1[m] : p2[m];
      p1[m] = live ? y : p1[m];
    }
  }
  __syncwarp();
  const uint32_t sub = (lane & 7) * 16;  // the view's row within a core matrix
  const uint32_t offP = (lane >> 3) * kSboP + sub, offQ = (lane >> 3) * kSboQ + sub;
  // all of a row's reads before its stores (same aliasing reason), P then Q
  {
    float x[kP];
#pragma unroll
    for (int e = 0; e < kP; ++e) x[e] = row[e];
#pragma unroll
    for (int o = 0; o < kP / 8; ++o)
      put_octet(stage + kYrHi, stage + kYrLo, offP + o * 128,
                *reinterpret_cast<const float(*)[8]>(&x[8 * o]));
  }
  {
    float x[kQ];
#pragma unroll
    for (int e = 0; e < kQ; ++e) x[e] = row[kP + e];
#pragma unroll
    for (int o = 0; o < kQ / 8; ++o)
      put_octet(stage + kYiHi, stage + kYiLo, offQ + o * 128,
                *reinterpret_cast<const float(*)[8]>(&x[8 * o]));
  }
  tc::fence_smem_to_async();
}

}  // namespace fle
}  // namespace rxgs
