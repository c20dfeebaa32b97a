// fle_tc.cuh -- pieces shared by the tensor-core FLE kernels (fle_tc.cu,
// fle_bwd_tc.cu): the folded component order, the layout of the basis
// operand of one group of views, the job walk and the coefficient tensor map.
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
// fewer K steps): the basis of one step (32 views) as K-major core matrices
// of 8 views x 8 components, Yr over kP = 64 and Yi over kQ = 48 components,
// each as hi and lo bf16 terms (14,336 bytes).  The basis image holds one
// such block per (Gaussian, view group) in HBM; the kernels copy it whole.
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
// without divisions.  With G > 0 (the FiLM-conditioned contraction, whose
// CTAs keep one receiver group's modulation in shared memory) the grid is
// G x P CTAs: CTA b keeps group jg = b % G and takes k = b / G, b / G + P, ...
__device__ __forceinline__ int jobs_of_cta(int K, int N, int G = 0) {
  if (G > 0) {
    const int kb = static_cast<int>(blockIdx.x) / G, P = static_cast<int>(gridDim.x) / G;
    return kb < K ? (K - 1 - kb) / P + 1 : 0;
  }
  const long long total = static_cast<long long>(K) * ((N + kRx - 1) / kRx);
  const long long b = blockIdx.x;
  return b < total ? static_cast<int>((total - 1 - b) / gridDim.x + 1) : 0;
}
struct JobIter {
  int K, k, jg, step;
  bool fixed;
  __device__ explicit JobIter(int K_, int G = 0) : K(K_), k(0), jg(0), step(0), fixed(G > 0) {
    if (fixed) {
      jg = static_cast<int>(blockIdx.x) % G;
      k = static_cast<int>(blockIdx.x) / G;
      step = static_cast<int>(gridDim.x) / G;
      return;
    }
    k = static_cast<int>(blockIdx.x);
    while (k >= K) {
      k -= K;
      ++jg;
    }
  }
  __device__ void next() {
    if (fixed) {
      k += step;
      return;
    }
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

}  // namespace fle
}  // namespace rxgs
