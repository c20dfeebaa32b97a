// fle_tc.cu -- the FLE directional radiance (App. E.2; Algorithm 1 eval_fle)
// as a tcgen05 contraction per Gaussian.
//
// For Gaussian k, receivers j (a group of 64) and views v (a group of 32):
//   s[v][k][j] = sum_l Y_vl c_jl = sum_P Yr c+_j + i sum_Q Yi c-_j
// with the +m / -m components folded (fle_tc.cuh) and c_jl the coefficients
// (a + i b)_jk,l (given, or formed from the base coefficients by the global
// FiLM branch inside the converters, kFilm).  Real-ified, with the coefficient rows
// interleaved (row 2j = Re, row 2j + 1 = Im) as the A operand (M = 128) and
// the folded basis of the 32 views as the B operand (N = 32):
//   P1 = A+ Yr^T (K = P components),  P2 = A- Yi^T (K = Q components)
//   Re s_j = P1[2j] - P2[2j+1],  Im s_j = P1[2j+1] + P2[2j]
// (lanes 2j and 2j + 1 exchange one value).  Operands are split into two
// bf16 terms (three MMAs per product, tc_common.cuh).
//
// The basis operand of every (Gaussian, group of 32 views) is computed
// first (fle_basis_image: fully parallel, one thread per view, written in
// the staged layout).  Then one CTA per SM walks jobs (Gaussian, receiver
// group), each with one step per group of 32 views, through warp-specialised
// stages on mbarriers:
//   warp 0       per job one TMA copy (a tensor-map box of the job's 64
//                coefficient rows) into one of three shared-memory stages;
//   warp 2       per step one bulk copy of the basis block into one of two
//                B stages (a producer of its own, so that neither copy
//                stream waits behind the other);
//   warps 4-7,   fold and split the coefficients (lane = accumulator row)
//   12-15        and store the A operand into tensor memory (tcgen05.st),
//                double-buffered; the two groups take even and odd jobs;
//   warp 1       one thread issues the MMAs (A from tensor memory, B from
//                shared memory) into one of two accumulators;
//   warps 8-11   read the accumulators (tcgen05.ld), combine and store.
// Every wait is bounded: on a timeout the CTA records kErrTimeout, stops
// walking, lets its copies and MMAs in flight complete and frees its tensor
// memory.  A degree whose half-rows are not whole 16-byte units
// ((lmax + 1)^2 odd) or an unaligned coefficient array takes the same kernel
// with the converters reading the coefficients directly.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "fle_tc.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {

// N_lm = sqrt((2l + 1) / (4 pi) (l - m)! / (l + m)!) (the orthonormal basis of
// App. E.2, m >= 0) and the three-term recurrence of P_l^m in l, both folded
// into the coefficients of the recurrence of y_lm = N_lm P_l^m (double, then
// rounded once).
FleRec fle_rec_table() {
  auto norm = [](int l, int m) {
    double ratio = 1.0;  // (l - m)! / (l + m)!
    for (int q = l - m + 1; q <= l + m; ++q) ratio /= q;
    return std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
  };
  FleRec t{};
  t.r[0][0][0] = static_cast<float>(norm(0, 0));
  for (int l = 1; l < 10; ++l) {
    // P_l^l = (2l - 1) st P_{l-1}^{l-1},  P_l^{l-1} = (2l - 1) ct P_{l-1}^{l-1}
    t.r[l][l][0] = static_cast<float>((2.0 * l - 1.0) * norm(l, l) / norm(l - 1, l - 1));
    t.r[l][l - 1][0] = static_cast<float>((2.0 * l - 1.0) * norm(l, l - 1) / norm(l - 1, l - 1));
    // (l - m) P_l^m = (2l - 1) ct P_{l-1}^m - (l + m - 1) P_{l-2}^m
    for (int m = 0; m + 2 <= l; ++m) {
      t.r[l][m][0] = static_cast<float>((2.0 * l - 1.0) / (l - m) * norm(l, m) / norm(l - 1, m));
      t.r[l][m][1] = static_cast<float>((l + m - 1.0) / (l - m) * norm(l, m) / norm(l - 2, m));
    }
  }
  return t;
}

namespace tc {

bool encode_f32_tiled(CUtensorMap* map, const float* base, int rank, const uint64_t* dims,
                      const uint64_t* strides, const uint32_t* box) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<Encode>(fn);
  }
  if (!encode || rank < 1 || rank > 5 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return false;
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], unit[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    unit[i] = 1;
    if (box[i] < 1 || box[i] > 256) return false;
    if (i + 1 < rank) {
      st[i] = strides[i];
      if ((strides[i] & 15) != 0) return false;
    }
  }
  if ((box[0] * 4u) % 16u != 0) return false;
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, static_cast<cuuint32_t>(rank),
                const_cast<float*>(base), d, st, bx, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

namespace fle {

bool encode_fle_rows(CUtensorMap* map, const float* base, int N, int K, int L) {
  if ((L & 3) != 0 || 2 * L > 256) return false;
  const uint64_t dims[3] = {static_cast<uint64_t>(2 * L), static_cast<uint64_t>(K),
                            static_cast<uint64_t>(N)};
  const uint64_t strides[2] = {static_cast<uint64_t>(2 * L) * 4,
                               static_cast<uint64_t>(K) * 2 * L * 4};
  const uint32_t box[3] = {static_cast<uint32_t>(2 * L), 1,
                           static_cast<uint32_t>(N < kRx ? N : kRx)};
  return tc::encode_f32_tiled(map, base, 3, dims, strides, box);
}

}  // namespace fle

namespace {

using namespace fle;

constexpr int kThreads = 512;
constexpr int kStages = 3;                      // coefficient stages
// one stage: the job's box [64 receivers][2L floats] as the TMA lays it out
// (at degree 9 a receiver's Re and Im half-rows are 25 16-byte units apart
// and receivers 50, so the 8 lanes of a quarter warp read 8 bank groups)
constexpr uint32_t kCStage = kRx * 200 * 4;
constexpr uint32_t kOffB = kStages * kCStage;
constexpr uint32_t kOffBar = kOffB + 2 * kBStage;
constexpr int kNumBars = 2 * kStages + 11;
constexpr uint32_t kOffMisc = kOffBar + 8 * kNumBars;
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffBar % 8 == 0 && kOffB % 1024 == 0, "alignment");
constexpr uint32_t kTmemCols = 512;
// tensor memory: accumulators (P1: 32 columns, P2: 32) at 64 * (step & 1);
// A operands at 128 + 128 * (job & 1): A+ hi, A+ lo (32 columns each), A- hi,
// A- lo (24 each)
constexpr uint32_t kColA = 128, kAPlo = 32, kAQhi = 64, kAQlo = 88;

// The basis image: thread = (Gaussian, view), warp = (Gaussian, view
// group).  Fully unrolled (degree and order known at compile time, the
// recurrence table in the constant bank, components past lmax zero): each
// component is written as soon as its core-matrix row of 8 is complete.
constexpr int kImgThreads = 128;

__global__ void __launch_bounds__(kImgThreads) fle_basis_image_kernel(
    const float4* __restrict__ geom, const float* __restrict__ tx, int K, int M, int lmax,
    FleRec rec, unsigned char* __restrict__ image) {
  const int nvg = (M + kViews - 1) / kViews, lane = threadIdx.x & 31;
  const long long g = static_cast<long long>(blockIdx.x) * (kImgThreads / 32) + (threadIdx.x >> 5);
  if (g >= static_cast<long long>(K) * nvg) return;
  const int k = static_cast<int>(g / nvg), v0 = static_cast<int>(g % nvg) * kViews;
  const bool on = lane < M - v0;
  const float4 p = geom[3 * k];
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
  float cm[10], sn[10];
  cm[0] = on ? 1.0f : 0.0f;  // rows past the views are zero
  sn[0] = 0.0f;
#pragma unroll
  for (int m = 1; m < 10; ++m) {
    cm[m] = cm[m - 1] * cp - sn[m - 1] * sp;
    sn[m] = cm[m - 1] * sp + sn[m - 1] * cp;
  }
  unsigned char* blk = image + g * kBStage;
  const uint32_t sub = (lane & 7) * 16;
  const uint32_t offP = (lane >> 3) * kSboP + sub, offQ = (lane >> 3) * kSboQ + sub;
  float bp[8], bq[8];
  float p1[10], p2[10];  // y_{l-1,m}, y_{l-2,m}
#pragma unroll
  for (int l = 0; l < 10; ++l) {
    const float keep = l <= lmax ? 1.0f : 0.0f;
    float y[10];
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      const float a = rec.r[l][m][0], b = rec.r[l][m][1];
      if (m == l)
        y[m] = l == 0 ? a : a * st * p1[m - 1 >= 0 ? m - 1 : 0];
      else if (m == l - 1)
        y[m] = a * ct * p1[m];
      else
        y[m] = a * ct * p1[m] - b * p2[m];
      const int kp = kappa_p(l, m);
      bp[kp & 7] = keep * y[m] * cm[m];
      if ((kp & 7) == 7) put_octet(blk + kYrHi, blk + kYrLo, offP + (kp >> 3) * 128, bp);
      if (m > 0) {
        const int kq = kappa_q(l, m);
        bq[kq & 7] = keep * y[m] * sn[m];
        if ((kq & 7) == 7) put_octet(blk + kYiHi, blk + kYiLo, offQ + (kq >> 3) * 128, bq);
      }
    }
#pragma unroll
    for (int m = 0; m <= l; ++m) {
      p2[m] = p1[m];
      p1[m] = y[m];
    }
  }
  // tails: P components 55..63 and Q components 45..47 are zero
  bp[7] = 0.0f;
  put_octet(blk + kYrHi, blk + kYrLo, offP + 6 * 128, bp);
#pragma unroll
  for (int e = 0; e < 8; ++e) bp[e] = 0.0f;
  put_octet(blk + kYrHi, blk + kYrLo, offP + 7 * 128, bp);
  bq[5] = bq[6] = bq[7] = 0.0f;
  put_octet(blk + kYiHi, blk + kYiLo, offQ + 5 * 128, bq);
}

// The coefficients of one job -> the A operand in tensor memory: lane = row
// 2j + p of the warp's quarter, c its half-row (row past N: zeros).
// A+ = c_{l,m} + c_{l,-m} (m > 0), c_{l,0}; A- = c_{l,m} - c_{l,-m}; 16
// components at a time split into hi and lo terms (8 columns each).
__device__ __forceinline__ void store_a(uint32_t a, const float (&c)[100]) {
  {
    float v[16];
#pragma unroll
    for (int l = 0; l < 10; ++l)
#pragma unroll
      for (int m = 0; m <= l; ++m) {
        const int kp = kappa_p(l, m);
        v[kp & 15] = m == 0 ? c[l * l + l] : c[l * l + l + m] + c[l * l + l - m];
        if ((kp & 15) == 15 || kp == kappa_p(9, 9)) {
          if (kp == kappa_p(9, 9))
#pragma unroll
            for (int e = (kappa_p(9, 9) & 15) + 1; e < 16; ++e) v[e] = 0.0f;
          uint32_t h[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) tc::split2(v[2 * e], v[2 * e + 1], h[e], lo[e]);
          tc::tmem_st8(a + (kp >> 4) * 8, h);
          tc::tmem_st8(a + kAPlo + (kp >> 4) * 8, lo);
        }
      }
  }
  {
    float v[16];
#pragma unroll
    for (int l = 1; l < 10; ++l)
#pragma unroll
      for (int m = 1; m <= l; ++m) {
        const int kq = kappa_q(l, m);
        v[kq & 15] = c[l * l + l + m] - c[l * l + l - m];
        if ((kq & 15) == 15 || kq == kappa_q(9, 9)) {
          if (kq == kappa_q(9, 9))
#pragma unroll
            for (int e = (kappa_q(9, 9) & 15) + 1; e < 16; ++e) v[e] = 0.0f;
          uint32_t h[8], lo[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) tc::split2(v[2 * e], v[2 * e + 1], h[e], lo[e]);
          tc::tmem_st8(a + kAQhi + (kq >> 4) * 8, h);
          tc::tmem_st8(a + kAQlo + (kq >> 4) * 8, lo);
        }
      }
  }
}

// kFilm: the coefficients are formed in the converters from the base
// coefficients and the modulations (Eq. film_apply; with loc, Eq.
// combined_local), never written to memory: the CTA keeps its receiver
// group's (a, b) table [component][receiver] in shared memory (loaded once)
// and warp 0 stages each job's base coefficients phi_k (2L floats).
template <bool kBulk, bool kFilm>
__global__ void __launch_bounds__(kThreads, 1)
    fle_radiance_tc_kernel(const float* __restrict__ coeffs, int N, int K, int lmax,
                           const unsigned char* __restrict__ image, int M, int stride,
                           size_t rad_view, float* __restrict__ rad, unsigned* __restrict__ err,
                           const __grid_constant__ CUtensorMap tmap, const float* __restrict__ base,
                           const float4* __restrict__ ab, const float4* __restrict__ loc) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint64_t* cfull = bar;                 // [kStages] coefficients landed
  uint64_t* cempty = bar + kStages;      // [kStages] converters done with them
  uint64_t* afull = bar + 2 * kStages;   // [2] A operand of a job in TMEM
  uint64_t* adone = afull + 2;           // [2] MMAs of a job complete
  uint64_t* bfull = afull + 4;           // [2] B operand of a step landed
  uint64_t* sdone = afull + 6;           // [2] MMAs of a step complete
  uint64_t* aempty = afull + 8;          // [2] accumulators of a step read
  uint64_t* fin = afull + 10;            // every MMA complete
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);
  volatile uint32_t* abort_flag = &sMisc[1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int L = (lmax + 1) * (lmax + 1);
  const int G = kFilm ? (N + kRx - 1) / kRx : 0;
  const int njobs = jobs_of_cta(K, N, G), nvg = (M + kViews - 1) / kViews;
  // kFilm: the (a, b) table float4 [L][kRx] and kStages stages of phi (2L floats)
  float4* sTab = reinterpret_cast<float4*>(sm);
  float* sPhi = reinterpret_cast<float*>(sm + kRx * 100 * 16);
  if constexpr (kFilm) {
    const int jg = static_cast<int>(blockIdx.x) % G, j0 = jg * kRx;
    for (int e = threadIdx.x; e < kRx * L; e += kThreads) {
      const int l = e / kRx, jl = e - l * kRx;
      sTab[e] = j0 + jl < N ? ab[static_cast<size_t>(j0 + jl) * L + l]
                            : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (threadIdx.x == 32) {
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&cfull[i], kFilm ? 32 : 1);
      tc::mbar_init(&cempty[i], 4);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&afull[i], 4);
      tc::mbar_init(&adone[i], 1);
      tc::mbar_init(&bfull[i], 1);
      tc::mbar_init(&sdone[i], 1);
      tc::mbar_init(&aempty[i], 4);
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
  // a whole warp waits; any lane that gave up stops the warp
  auto wait_warp = [&](uint64_t* b, uint32_t parity) -> bool {
    const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(b, parity, kWaitLimit));
    if (!ok && lane == 0) fail();
    return ok;
  };

  if (warp == 0 && kFilm) {
    // ------------------------------------------------- base coefficients
    // per job phi_k (2L floats) into one of kStages stages, all lanes
    JobIter it(K, G);
    for (int n = 0; n < njobs; ++n, it.next()) {
      if (*abort_flag) break;
      const int st = n % kStages;
      if (n >= kStages && !wait_warp(&cempty[st], ((n / kStages) - 1) & 1)) break;
      const float* src = base + static_cast<size_t>(it.k) * 2 * L;
      float* dst = sPhi + st * 200;
      for (int e = lane; e < 2 * L; e += 32) dst[e] = __ldg(src + e);
      tc::mbar_arrive(&cfull[st]);  // release: each lane's stores before its arrival
    }
  } else if (warp == 0) {
    // ------------------------------------------------- coefficient producer
    // per job one box of the coefficient rows (rows j0 .. j0 + 63 of Gaussian
    // k; rows past N read as zero)
    if (kBulk && lane == 0) {
      const uint32_t box_bytes = static_cast<uint32_t>(min(kRx, N)) * 8u * L;
      int issued = 0;
      JobIter it(K, G);
      for (int n = 0; n < njobs; ++n, it.next()) {
        if (*abort_flag) break;
        const int st = n % kStages;
        if (n >= kStages && !tc::mbar_wait(&cempty[st], ((n / kStages) - 1) & 1, kWaitLimit)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(&cfull[st], box_bytes);
        tc::tma_load_3d(sm + st * kCStage, &tmap, 0, it.k, it.jg * kRx, &cfull[st]);
        issued = n + 1;
      }
      // copies of a walk cut short land before the CTA exits
      for (int n = max(0, issued - kStages); n < issued; ++n)
        tc::mbar_wait(&cfull[n % kStages], (n / kStages) & 1, kWaitLimit);
    }
    __syncwarp();
  } else if (warp == 2) {
    // ------------------------------------------------------- basis producer
    // per step the view group's basis block into one of two B stages
    if (lane == 0) {
      int s = 0, issued = 0;
      bool stop = false;
      JobIter it(K, G);
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
      for (int q = max(0, issued - 2); q < issued; ++q)
        tc::mbar_wait(&bfull[q & 1], (q >> 1) & 1, kWaitLimit);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      const int kp16 = kp_of(lmax) / 16, kq16 = kq_of(lmax) / 16;
      constexpr uint32_t idesc = tc::idesc_bf16(128, kViews, 0, 0);
      const uint32_t sb = tc::smem_u32(sm) + kOffB;
      int s = 0;
      bool stop = false;
      for (int n = 0; n < njobs && !stop; ++n) {
        for (int vg = 0; vg < nvg; ++vg, ++s) {
          if (*abort_flag) { stop = true; break; }
          if (vg == 0 && !tc::mbar_wait(&afull[n & 1], (n >> 1) & 1, kWaitLimit)) {
            fail(); stop = true; break;
          }
          if (!tc::mbar_wait(&bfull[s & 1], (s >> 1) & 1, kWaitLimit)) { fail(); stop = true; break; }
          if (s >= 2 && !tc::mbar_wait(&aempty[s & 1], ((s >> 1) - 1) & 1, kWaitLimit)) {
            fail(); stop = true; break;
          }
          tc::fence_after_sync();
          const uint32_t acc = tmem + 64 * (s & 1);
          const uint32_t a = tmem + kColA + 128 * (n & 1);
          const uint32_t b = sb + (s & 1) * kBStage;
          for (int ks = 0; ks < kp16; ++ks) {  // P1 = A+ Yr^T
            const uint64_t bh = tc::smem_desc(b + kYrHi + ks * 256, 128, kSboP);
            const uint64_t bl = tc::smem_desc(b + kYrLo + ks * 256, 128, kSboP);
            tc::mma_bf16_ts(acc, a + ks * 8, bh, idesc, ks > 0);
            tc::mma_bf16_ts(acc, a + ks * 8, bl, idesc, 1);
            tc::mma_bf16_ts(acc, a + kAPlo + ks * 8, bh, idesc, 1);
          }
          for (int ks = 0; ks < kq16; ++ks) {  // P2 = A- Yi^T
            const uint64_t bh = tc::smem_desc(b + kYiHi + ks * 256, 128, kSboQ);
            const uint64_t bl = tc::smem_desc(b + kYiLo + ks * 256, 128, kSboQ);
            tc::mma_bf16_ts(acc + 32, a + kAQhi + ks * 8, bh, idesc, ks > 0);
            tc::mma_bf16_ts(acc + 32, a + kAQhi + ks * 8, bl, idesc, 1);
            tc::mma_bf16_ts(acc + 32, a + kAQlo + ks * 8, bh, idesc, 1);
          }
          tc::mma_commit(&sdone[s & 1]);
          if (vg == nvg - 1) tc::mma_commit(&adone[n & 1]);
        }
      }
      tc::mma_commit(fin);
      if (!tc::mbar_wait(fin, 0, kWaitLimit)) fail();
    }
    __syncwarp();
  } else if ((warp >= 4 && warp < 8) || warp >= 12) {
    // ---------------------------------------------------------------- A operand
    // two groups of four warps take the even and the odd jobs
    const int grp = warp >= 12, q = warp & 3, row = 32 * q + lane, jl = row >> 1, p = row & 1;
    JobIter it(K, G);
    if (grp) it.next();
    for (int n = grp; n < njobs; n += 2, it.next(), it.next()) {
      if (*abort_flag) break;
      const int st = n % kStages;
      if ((kBulk || kFilm) && !wait_warp(&cfull[st], (n / kStages) & 1)) break;
      if (n >= 2 && !wait_warp(&adone[n & 1], ((n >> 1) - 1) & 1)) break;
      tc::fence_after_sync();
      const bool on = jl < N - it.jg * kRx;
      float c[100];
      if (kFilm) {
        // c = (1 + a) phi + b (complex, per component), then (1 + alpha) c +
        // beta with the local factors; this lane keeps the Re (p = 0) or Im
        // (p = 1) part
        // Re: (1 + a.re) phi.re - a.im phi.im + b.re; Im: (1 + a.re) phi.im +
        // a.im phi.re + b.im -- with x, y = this part's and the other part of
        // phi and sg = -1 / +1, both are fma(1 + a.re, x, fma(sg a.im, y, b))
        const float* ph = sPhi + st * 200;
        const float* px = ph + p * L;
        const float* py = ph + (1 - p) * L;
        const float sg = p ? 1.0f : -1.0f;
        const float4 lf = (loc && on) ? loc[static_cast<size_t>(it.jg * kRx + jl) * K + it.k]
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
        const float alr = 1.0f + lf.x, sal = sg * lf.y, bl = p ? lf.w : lf.z;
#pragma unroll
        for (int l = 0; l < 100; ++l) {
          float v = 0.0f;
          if (l < L) {
            const float4 q4 = sTab[l * kRx + jl];
            v = fmaf(1.0f + q4.x, px[l], fmaf(sg * q4.y, py[l], p ? q4.w : q4.z));
          }
          c[l] = v;
        }
        if (loc) {
          // (1 + alpha) c + beta: the other part from the partner lane
#pragma unroll
          for (int l = 0; l < 100; ++l) {
            const float o = __shfl_xor_sync(0xffffffffu, c[l], 1);
            if (l < L) c[l] = fmaf(alr, c[l], fmaf(sal, o, bl));
          }
        }
        if (!on)
#pragma unroll
          for (int l = 0; l < 100; ++l) c[l] = 0.0f;
      } else if (kBulk) {
        const float4* r4 =
            reinterpret_cast<const float4*>(sm + st * kCStage + (jl * 2 * L + p * L) * 4);
#pragma unroll
        for (int t = 0; t < 25; ++t) {
          const float4 v = (on && 4 * t < L) ? r4[t] : make_float4(0.f, 0.f, 0.f, 0.f);
          c[4 * t] = v.x;
          c[4 * t + 1] = v.y;
          c[4 * t + 2] = v.z;
          c[4 * t + 3] = v.w;
        }
      } else {
        const float* g =
            coeffs + (static_cast<size_t>(it.jg * kRx + jl) * K + it.k) * 2 * L + p * L;
#pragma unroll
        for (int i = 0; i < 100; ++i) c[i] = (on && i < L) ? __ldg(g + i) : 0.0f;
      }
      store_a(tmem + (static_cast<uint32_t>(32 * q) << 16) + kColA + 128 * (n & 1), c);
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&afull[n & 1]);
        if (kBulk || kFilm) tc::mbar_arrive(&cempty[st]);
      }
    }
  } else if (warp >= 8 && warp < 12) {
    // ---------------------------------------------------------------- write-out
    const int q = warp - 8, row = 32 * q + lane;
    const bool odd = lane & 1, has_q = kq_of(lmax) > 0;
    JobIter it(K, G);
    int s = 0;
    bool stop = false;
    for (int n = 0; n < njobs && !stop; ++n, it.next()) {
      const bool ok = row < 2 * (N - it.jg * kRx);
      float* dst = rad + static_cast<size_t>(it.k) * stride + 2 * it.jg * kRx + row;
      for (int vg = 0; vg < nvg; ++vg, ++s) {
        if (*abort_flag || !wait_warp(&sdone[s & 1], (s >> 1) & 1)) { stop = true; break; }
        tc::fence_after_sync();
        uint32_t r1[32], r2[32];
        const uint32_t acc = tmem + (static_cast<uint32_t>(32 * q) << 16) + 64 * (s & 1);
        tc::tmem_ld32_async(acc, r1);
        tc::tmem_ld32_async(acc + 32, r2);
        tc::tmem_wait_ld();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&aempty[s & 1]);
        const int v0 = vg * kViews, nv = min(kViews, M - v0);
        float* d = dst + static_cast<size_t>(v0) * rad_view;
#pragma unroll
        for (int v = 0; v < kViews; ++v) {
          const float other =
              __shfl_xor_sync(0xffffffffu, has_q ? __uint_as_float(r2[v]) : 0.0f, 1);
          const float p1 = __uint_as_float(r1[v]);
          if (ok && v < nv) d[static_cast<size_t>(v) * rad_view] = odd ? p1 + other : p1 - other;
        }
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <bool kBulk, bool kFilm>
void launch_radiance(const float* coeffs, int N, int K, int lmax, const unsigned char* image,
                     int M, int stride, size_t rad_view, float* rad, int grid, cudaStream_t s,
                     unsigned* err, const CUtensorMap& tmap, const float* base = nullptr,
                     const float4* ab = nullptr, const float4* loc = nullptr) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(fle_radiance_tc_kernel<kBulk, kFilm>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmem));
    configured = true;
  }
  fle_radiance_tc_kernel<kBulk, kFilm><<<grid, kThreads, kSmem, s>>>(
      coeffs, N, K, lmax, image, M, stride, rad_view, rad, err, tmap, base, ab, loc);
}

}  // namespace

size_t fle_basis_image_bytes(int K, int M) {
  return static_cast<size_t>(K) * ((M + kViews - 1) / kViews) * kBStage;
}

void launch_fle_basis_image(const float4* geom, const float* tx, int K, int M, int lmax,
                            unsigned char* image, cudaStream_t s) {
  if (K <= 0 || M <= 0) return;
  const long long blocks = (static_cast<long long>(K) * ((M + kViews - 1) / kViews) +
                            kImgThreads / 32 - 1) / (kImgThreads / 32);
  fle_basis_image_kernel<<<static_cast<unsigned>(blocks), kImgThreads, 0, s>>>(
      geom, tx, K, M, lmax, fle_rec_table(), image);
  note_launches(1);
}

void launch_fle_radiance_tc(const float* coeffs, int N, int K, int lmax,
                            const unsigned char* image, int M, int stride, size_t rad_view,
                            float* rad, cudaStream_t s, unsigned* err) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long jobs = static_cast<long long>(K) * ((N + kRx - 1) / kRx);
  const int grid = static_cast<int>(std::max(1LL, std::min<long long>(jobs, nsm)));
  const int L = (lmax + 1) * (lmax + 1);
  CUtensorMap tmap{};
  if (encode_fle_rows(&tmap, coeffs, N, K, L))
    launch_radiance<true, false>(coeffs, N, K, lmax, image, M, stride, rad_view, rad, grid, s,
                                 err, tmap);
  else
    launch_radiance<false, false>(coeffs, N, K, lmax, image, M, stride, rad_view, rad, grid, s,
                                  err, tmap);
  note_launches(1);
}

void launch_fle_radiance_film_tc(const float* base, const float4* ab, const float4* loc, int N,
                                 int K, int lmax, const unsigned char* image, int M, int stride,
                                 size_t rad_view, float* rad, cudaStream_t s, unsigned* err) {
  if (K <= 0 || N <= 0 || M <= 0) return;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // G receiver groups, P CTAs per group (each keeps its group's modulation)
  const int G = (N + kRx - 1) / kRx;
  const int P = std::max(1, std::min(K, nsm / G));
  CUtensorMap tmap{};
  launch_radiance<false, true>(nullptr, N, K, lmax, image, M, stride, rad_view, rad, G * P, s,
                               err, tmap, base, ab, loc);
  note_launches(1);
}

}  // namespace rxgs

namespace rxgs {


// ---- its backward, from the coefficient gradient G[j][k][.][l]:
//   dL/dbase_kl = sum_j conj(1 + a_jl) G_jkl      (film_fold_base: one thread
//                 per (Gaussian, component), the receivers summed in order,
//                 the modulation read through the cache)
//   dL/da_jl    = sum_k conj(base_kl) G_jkl,  dL/db_jl = sum_k G_jkl
//                 (film_fold_ab: a block per (receiver, range of Gaussians),
//                 one thread per component, one float atomic per entry)
constexpr int kFoldAbK = 1024;   // Gaussians per block

__global__ void __launch_bounds__(256) film_fold_base_kernel(const float* __restrict__ G,
                                                             const float4* __restrict__ ab, int N,
                                                             int K, int L,
                                                             float* __restrict__ grad_base) {
  const size_t idx = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;  // (k, l)
  if (idx >= static_cast<size_t>(K) * L) return;
  const int k = static_cast<int>(idx / L), l = static_cast<int>(idx % L);
  const size_t jstride = static_cast<size_t>(K) * 2 * L;
  const float* g = G + static_cast<size_t>(k) * 2 * L + l;
  float sr = 0.0f, si = 0.0f;
#pragma unroll 8
  for (int j = 0; j < N; ++j) {
    const float gr = g[j * jstride], gi = g[j * jstride + L];
    const float4 q = __ldg(&ab[static_cast<size_t>(j) * L + l]);
    const float ar = 1.0f + q.x, ai = q.y;  // conj(1 + a) G
    sr = fmaf(ar, gr, fmaf(ai, gi, sr));
    si = fmaf(ar, gi, fmaf(-ai, gr, si));
  }
  grad_base[static_cast<size_t>(k) * 2 * L + l] += sr;
  grad_base[static_cast<size_t>(k) * 2 * L + L + l] += si;
}

__global__ void film_fold_ab_kernel(const float* __restrict__ G, const float* __restrict__ base,
                                    int K, int L, float* __restrict__ d_ab) {
  const int l = threadIdx.x, j = blockIdx.y;
  if (l >= L) return;
  const int k0 = blockIdx.x * kFoldAbK, k1 = min(K, k0 + kFoldAbK);
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 4
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
    const size_t n = static_cast<size_t>(K) * L;
    film_fold_base_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(G, ab, N, K, L,
                                                                                grad_base);
    note_launches(1);
  }
  if (d_ab) {
    film_fold_ab_kernel<<<dim3((K + kFoldAbK - 1) / kFoldAbK, N), 128, 0, s>>>(G, base, K, L, d_ab);
    note_launches(1);
  }
}

}  // namespace rxgs
