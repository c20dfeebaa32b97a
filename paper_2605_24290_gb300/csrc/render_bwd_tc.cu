// render_bwd_tc.cu -- the back-to-front sweep of the compositing backward
// (App. D) for blocks of 128 output columns, with its two per-chunk
// contractions on the tcgen05 tensor cores and their accumulators in tensor
// memory.
//
// For one (view, tile, 128-column block) and one chunk of 32 list entries
// b (back to front), with g[p][c] the cotangent of pixel p and column c and
// s[b][c] the radiance of entry b:
//   gamma[p][b] = sum_c g[p][c] s[b][c]             (M = 256 pixels, N = 32, K = 128)
//   dL/ds[b][c] = sum_p (T w)[b][p] g[p][c]          (M = 128 columns, N = 32, K = 256)
// Between the two, each pixel runs the scalar recurrence of the backward
// (T recovery T_m = T_{m+1} / (1 - w_m), the suffix Q_{m-1} = w_m gamma_m +
// (1 - w_m) Q_m, dL/dtau_m = T_m (gamma_m - Q_m) G_m) over the chunk's entries
// that meet its warp's strip, writing (T w)[b][p] for the second product.
// Both products take their float32 operands split into two bf16 terms
// (tc_common.cuh): three MMAs per product, about 1.2e-5 relative error per
// term, float32 accumulation.  The cotangent tile g is loaded and split once
// per CTA and serves both products: K-major as the A operand of gamma,
// MN-major as the A operand of dL/ds.
//
// 512 threads.  Warps 0-7 own one pixel each (thread = pixel = TMEM lane of
// its gamma row); warps 8-15 stage the next chunk's radiance, drain the
// previous chunk's dL/ds accumulator (TMEM lanes = columns) into the
// gradient with float atomics, sum the dL/dtau of the previous chunk, and
// thread 256 issues the MMAs.  Per chunk n:
//   1. all 512 threads evaluate the weights G[b][p] of chunk n (the entries
//      that meet each warp's 32-pixel strip, shared between the two warps of
//      a strip);
//   2. warps 0-7 wait for gamma(n), run the recurrence, write T w (bf16 x 2);
//      warps 8-15 wait for gamma(n), stage radiance(n+1) (bf16 x 2), drain
//      dL/ds(n-1) and dL/dtau(n-1);
//   3. one barrier, then dL/ds(n) and gamma(n+1) are issued.
// Every mbarrier wait is bounded: a wait that gives up sets kErrTimeout in the
// device error word and the CTA leaves the loop, frees its tensor memory and
// returns.
#include <cuda_bf16.h>

#include "render_common.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {
namespace {

constexpr int kP = kTilePixels;  // 256 pixels per tile
constexpr int kNB = 128;         // columns per CTA
constexpr int kCH = kChunk;      // 32 list entries per chunk
constexpr int kThreads = 512;

// Operand buffers, 8x8 bf16 core matrices (128 bytes each):
//   g[p][c]: core (p/8, c/8) at (p/8 * 16 + c/8) * 128
//   s[b][c]: core (b/8, c/8) at (b/8) * kSboS + (c/8) * kLboS
//   a[b][p]: core (b/8, p/8) at (b/8) * kSboA + (p/8) * kLboA
// (s and a are written every chunk; their 144-byte core pitch along K spreads
// a warp's stores over all banks).
constexpr uint32_t kLboG = 128, kSboG = 16 * 128;
constexpr uint32_t kLboS = 144, kSboS = 16 * kLboS;
constexpr uint32_t kLboA = 144, kSboA = 32 * kLboA;
constexpr uint32_t kGBytes = kP * kNB * 2;
constexpr uint32_t kSBytes = 4 * kSboS;
constexpr uint32_t kABytes = 4 * kSboA;
constexpr uint32_t kOffG1 = 0, kOffG2 = kGBytes;
constexpr uint32_t kOffS1 = 2 * kGBytes, kOffS2 = kOffS1 + kSBytes;
constexpr uint32_t kOffA1 = kOffS2 + kSBytes, kOffA2 = kOffA1 + kABytes;
constexpr uint32_t kOffW = kOffA2 + kABytes;              // float G[32][256]
constexpr uint32_t kOffRec = kOffW + kCH * kP * 4;        // float4 [2][32][2]
constexpr uint32_t kOffIdx = kOffRec + 2 * kCH * 2 * 16;  // u32 [4][32] list indices
constexpr uint32_t kOffTau = kOffIdx + 4 * kCH * 4;       // float [2][32][8] dL/dtau per warp
constexpr uint32_t kOffMask = kOffTau + 2 * kCH * 8 * 4;  // u32 [8] strip masks
constexpr uint32_t kOffBar = kOffMask + 64;               // u64 [2] mbarriers
constexpr uint32_t kOffMisc = kOffBar + 16;               // u32 TMEM base, abort, #gamma, #dlds
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");

constexpr uint32_t kTmemCols = 128;  // gamma: columns 0-63 (two M tiles), dL/ds: 64-95
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kIdescGamma = tc::idesc_bf16(128, 32, 0, 0);
constexpr uint32_t kIdescDlds = tc::idesc_bf16(128, 32, 1, 0);

__device__ __forceinline__ uint32_t g_off(int p, int c) {
  return ((p >> 3) * 16 + (c >> 3)) * 128 + (p & 7) * 16 + (c & 7) * 2;
}

__global__ void __launch_bounds__(kThreads, 1) render_bwd_tc_kernel(const BackwardArgs A) {
  extern __shared__ __align__(128) unsigned char sm[];
  float* sW = reinterpret_cast<float*>(sm + kOffW);
  float4* sRec0 = reinterpret_cast<float4*>(sm + kOffRec);
  uint32_t* sIdx = reinterpret_cast<uint32_t*>(sm + kOffIdx);
  float* sTau = reinterpret_cast<float*>(sm + kOffTau);
  uint32_t* sMask = reinterpret_cast<uint32_t*>(sm + kOffMask);
  uint64_t* barG = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint64_t* barD = barG + 1;
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);

  const RenderArgs& a = A.f;
  const GridConst& g = a.g;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int col0 = blockIdx.y * kNB;
  const int tr = tile / g.tiles_w, tcol = tile % g.tiles_w;
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const float* radv = a.rad + static_cast<size_t>(v) * a.rad_view;
  float* drad = A.d_rad + static_cast<size_t>(v) * a.rad_view;
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  const int twoC = 2 * a.C;
  const uint32_t tile_stop = A.tile_stop[static_cast<size_t>(v) * g.T + tile];
  const int nchunks = static_cast<int>((tile_stop - rg.x + kCH - 1) / kCH);
  const uint32_t sbase = tc::smem_u32(sm);

  // this thread's pixel (warps 8-15 mirror warps 0-7 in the weight phase)
  const int p = t & (kP - 1);
  const int i = tr * g.TH + p / g.TW, jj = tcol * g.TW + p % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  float T = 1.0f, Q = 0.0f;
  uint32_t stop = rg.x;
  if (valid) {
    const size_t o = static_cast<size_t>(v) * HW + static_cast<size_t>(i) * g.W + jj;
    T = A.tfin[o];
    stop = A.stops[o];
  }
  const int wp = warp & 7, half = warp >> 3;
  const Strip strip = pixel_strip(g, tr, tcol, 32 * wp, 32);

  // chunk n of the sweep covers list positions [chunk_start(n), +chunk_len(n))
  auto chunk_start = [&](int n) { return rg.x + static_cast<uint32_t>(nchunks - 1 - n) * kCH; };
  auto chunk_len = [&](int n) { return min(kCH, static_cast<int>(tile_stop - chunk_start(n))); };
  auto fail = [&]() {
    atomicOr(&sMisc[1], 1u);
    if (A.err) atomicOr(A.err, kErrTimeout);
  };
  // warp 8: list indices of chunk n (ring of 4) and records (two buffers)
  auto copy_indices = [&](int n) {
    const int l = t - 256;
    const bool ok = l < chunk_len(n);
    cp_async4(&sIdx[(n & 3) * kCH + l], ok ? &a.vals[chunk_start(n) + l] : a.vals, ok);
  };
  auto gather_rec = [&](int n) {
    const int l = t - 256;
    const bool ok = l < chunk_len(n);
    const uint32_t k = ok ? sIdx[(n & 3) * kCH + l] : 0u;
    float4* rb = sRec0 + (n & 1) * 2 * kCH;
    cp_async16(&rb[2 * l + 0], &rec[2 * k + 0], ok);
    cp_async16(&rb[2 * l + 1], &rec[2 * k + 1], ok);
  };
  // warps 8-15: radiance rows of chunk n, 16 columns per thread
  auto load_rad = [&](int n, float (&x)[16]) {
    const int h = t - 256, b = h >> 3, cg = h & 7;
    const bool ok = b < chunk_len(n);
    const uint32_t k = ok ? sIdx[(n & 3) * kCH + b] : 0u;
    const float4* src =
        reinterpret_cast<const float4*>(radv + static_cast<size_t>(k) * a.stride + col0 + cg * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 r = ok ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[4 * q + 0] = r.x;
      x[4 * q + 1] = r.y;
      x[4 * q + 2] = r.z;
      x[4 * q + 3] = r.w;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e)
      if (col0 + cg * 16 + e >= a.ncols) x[e] = 0.0f;
  };
  auto store_rad = [&](const float (&x)[16]) {
    const int h = t - 256, b = h >> 3, cg = h & 7;
    float x0[8], x1[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      x0[e] = x[e];
      x1[e] = x[8 + e];
    }
    uint4 hi, lo;
    const uint32_t row = (b >> 3) * kSboS + (b & 7) * 16;
    tc::split8(x0, hi, lo);
    *reinterpret_cast<uint4*>(sm + kOffS1 + row + (2 * cg) * kLboS) = hi;
    *reinterpret_cast<uint4*>(sm + kOffS2 + row + (2 * cg) * kLboS) = lo;
    tc::split8(x1, hi, lo);
    *reinterpret_cast<uint4*>(sm + kOffS1 + row + (2 * cg + 1) * kLboS) = hi;
    *reinterpret_cast<uint4*>(sm + kOffS2 + row + (2 * cg + 1) * kLboS) = lo;
  };
  // warps 8-11: dL/ds of chunk n from TMEM (lane = column) into the gradient
  auto drain_dlds = [&](int n) {
    float d[32];
    tc::tmem_ld32(sMisc[0] + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 64, d);
    const int col = col0 + 32 * (warp & 3) + lane;
    const int nb = chunk_len(n);
    const uint32_t* ks = sIdx + (n & 3) * kCH;
    if (col < a.ncols) {
#pragma unroll
      for (int b = 0; b < kCH; ++b)
        if (b < nb && d[b] != 0.0f)
          atomicAdd(&drad[static_cast<size_t>(ks[b]) * a.stride + col], d[b]);
    }
  };
  // warp 12: dL/dtau of chunk n, the eight pixel warps' sums in order
  auto drain_tau = [&](int n) {
    const int b = lane;
    if (b < chunk_len(n)) {
      const float* src = sTau + (n & 1) * kCH * 8 + b * 8;
      float y = 0.0f;
#pragma unroll
      for (int w = 0; w < 8; ++w) y += src[w];
      if (y != 0.0f) atomicAdd(&A.d_tau[sIdx[(n & 3) * kCH + b]], y);
    }
  };
  // thread 256: the MMAs of gamma(n) (g x s) and dL/ds(n) (g^T x a)
  auto issue_gamma = [&](uint32_t tmem) {
#pragma unroll 1
    for (int m = 0; m < 2; ++m)
#pragma unroll 1
      for (int k = 0; k < kNB / 16; ++k)
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t ga = sbase + (term == 2 ? kOffG2 : kOffG1) + ((16 * m) * 16 + 2 * k) * 128;
          const uint32_t sb = sbase + (term == 1 ? kOffS2 : kOffS1) + 2 * k * kLboS;
          tc::mma_bf16(tmem + 32 * m, tc::smem_desc(ga, kLboG, kSboG),
                       tc::smem_desc(sb, kLboS, kSboS), kIdescGamma, (k | term) != 0);
        }
  };
  auto issue_dlds = [&](uint32_t tmem) {
#pragma unroll 1
    for (int k = 0; k < kP / 16; ++k)
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        // g read MN-major: M = columns (core pitch 128 B), K = pixels (core pitch 2048 B)
        const uint32_t ga = sbase + (term == 2 ? kOffG2 : kOffG1) + k * 2 * kSboG;
        const uint32_t ab = sbase + (term == 1 ? kOffA2 : kOffA1) + 2 * k * kLboA;
        tc::mma_bf16(tmem + 64, tc::smem_desc(ga, kSboG, kLboG), tc::smem_desc(ab, kLboA, kSboA),
                     kIdescDlds, (k | term) != 0);
      }
  };

  // ---- set-up: tensor memory, mbarriers, first indices
  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (t == 256) {
    tc::mbar_init(barG, 1);
    tc::mbar_init(barD, 1);
    tc::mbar_fence_init();
    sMisc[1] = 0;
    sMisc[2] = 0;
    sMisc[3] = 0;
  }
  if (warp == 8 && nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
  }
  // cotangent tile -> g (bf16 x 2), 8 columns per store
#pragma unroll 1
  for (int r = 0; r < 8; ++r) {
    const int oc = (t >> 8) + 2 * r;
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = col0 + oc * 8 + e;
      float val = 0.0f;
      if (valid && col < a.ncols) {
        const int j = col / twoC, ec = col - j * twoC;
        const size_t pix = static_cast<size_t>(i) * g.W + jj;
        if (A.g_spec) val += A.g_spec[((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + ec];
        if (A.g_uniform) val += A.g_uniform[static_cast<size_t>(v) * a.ncols + col];
      }
      x[e] = val;
    }
    uint4 hi, lo;
    tc::split8(x, hi, lo);
    const uint32_t off = g_off(p, oc * 8);
    *reinterpret_cast<uint4*>(sm + kOffG1 + off) = hi;
    *reinterpret_cast<uint4*>(sm + kOffG2 + off) = lo;
  }
  if (warp == 8 && nchunks > 0) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  __syncthreads();  // indices of chunk 0, mbarriers, TMEM address
  if (warp == 8 && nchunks > 0) {
    gather_rec(0);
    cp_async_commit();
  }
  if (warp >= 8 && nchunks > 0) {
    float x[16];
    load_rad(0, x);
    store_rad(x);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sMisc[0];
  if (t == 256 && nchunks > 0) {
    issue_gamma(tmem);
    tc::mma_commit(barG);
    sMisc[2] = 1;
  }

  // ---- the sweep, back to front
  for (int n = 0; n < nchunks; ++n) {
    cp_async_wait_all();  // records of chunk n, indices of chunk n + 1
    __syncthreads();
    if (sMisc[1]) break;
    const uint32_t start = chunk_start(n);
    const int nb = chunk_len(n);
    if (warp == 8) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      if (n + 1 < nchunks) gather_rec(n + 1);
      cp_async_commit();
    }
    const float4* sR = sRec0 + (n & 1) * 2 * kCH;
    // 1. weights G[b][p] of the entries meeting this warp's strip, the two
    //    warps of a strip taking alternate entries
    {
      const bool rel = lane < nb && touches_strip(g, sR[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      if (!__any_sync(0xffffffffu, start < stop)) m = 0;  // no pixel reaches this chunk
      if (half == 0 && lane == 0) sMask[wp] = m;
      int r = 0;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if ((r++ & 1) != half) continue;
        float G = 0.0f;
        if (valid && start + b < stop) {
          float w, Gv;
          if (pixel_weight(g, sR[2 * b], sR[2 * b + 1], i, jj, fi, fj, &w, &Gv)) G = Gv;
        }
        sW[b * kP + p] = G;  // 0: not composited by this pixel
      }
    }
    __syncthreads();
    if (warp < 8) {
      // 2a. the recurrence over the chunk, back to front
      if (!tc::mbar_wait(barG, n & 1, kWaitLimit)) fail();
      tc::fence_after_sync();
      float gam[32];
      tc::tmem_ld32(tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 32 * (warp >> 2), gam);
      if (n > 0 && !tc::mbar_wait(barD, (n - 1) & 1, kWaitLimit)) fail();  // a is free again
      const unsigned m = sMask[warp];
      float* tauw = sTau + (n & 1) * kCH * 8;
#pragma unroll
      for (int b = kCH - 1; b >= 0; --b) {
        float Tw = 0.0f;
        if (m & (1u << b)) {
          const float G = sW[b * kP + p];
          float dt = 0.0f;
          if (G != 0.0f) {
            const float w = __fmul_rn(sR[2 * b + 1].y, G);
            const float one_m_w = 1.0f - w;
            T = __fdividef(T, one_m_w);  // transmittance in front of entry b
            Tw = T * w;
            dt = T * (gam[b] - Q) * G;
            Q = fmaf(w, gam[b], one_m_w * Q);
          }
          if (__any_sync(0xffffffffu, dt != 0.0f)) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) dt += __shfl_xor_sync(0xffffffffu, dt, o);
          }
          if (lane == 0) tauw[b * 8 + warp] = dt;
        } else if (lane == 0) {
          tauw[b * 8 + warp] = 0.0f;
        }
        __nv_bfloat16 hi, lo;
        tc::split_bf16(Tw, hi, lo);
        const uint32_t off = (b >> 3) * kSboA + (p >> 3) * kLboA + (b & 7) * 16 + (p & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffA1 + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffA2 + off) = lo;
      }
    } else {
      // 2b. next chunk's radiance; previous chunk's dL/ds and dL/dtau
      float x[16];
      const bool more = n + 1 < nchunks;
      if (more) load_rad(n + 1, x);
      if (!tc::mbar_wait(barG, n & 1, kWaitLimit)) fail();  // gamma(n) has read s
      if (more) store_rad(x);
      if (n > 0 && warp < 12) {
        if (!tc::mbar_wait(barD, (n - 1) & 1, kWaitLimit)) fail();
        tc::fence_after_sync();
        drain_dlds(n - 1);
      }
      if (n > 0 && warp == 12) drain_tau(n - 1);
    }
    // 3. issue dL/ds(n) and gamma(n + 1)
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 256 && sMisc[1] == 0) {
      tc::fence_after_sync();
      issue_dlds(tmem);
      tc::mma_commit(barD);
      sMisc[3] = n + 1;
      if (n + 1 < nchunks) {
        issue_gamma(tmem);
        tc::mma_commit(barG);
        sMisc[2] = n + 2;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const bool aborted = sMisc[1] != 0;
  if (!aborted && nchunks > 0) {
    const int nl = nchunks - 1;
    if (warp >= 8 && warp < 12) {
      if (tc::mbar_wait(barD, nl & 1, kWaitLimit)) {
        tc::fence_after_sync();
        drain_dlds(nl);
      } else {
        fail();
      }
    }
    if (warp == 12) drain_tau(nl);
  }
  if (aborted && t == 256) {
    // let MMAs still in flight finish (bounded) before their memory goes
    const uint32_t ng = sMisc[2], nd = sMisc[3];
    if (ng > 0) tc::mbar_wait(barG, (ng - 1) & 1, kWaitLimit);
    if (nd > 0) tc::mbar_wait(barD, (nd - 1) & 1, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

void launch_render_bwd_tc(const BackwardArgs& A, cudaStream_t s) {
  const RenderArgs& a = A.f;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmem));
    configured = true;
  }
  dim3 grid(a.g.T, (a.ncols + kNB - 1) / kNB, a.M);
  render_bwd_tc_kernel<<<grid, kThreads, kSmem, s>>>(A);
  note_launches(1);
}

}  // namespace rxgs
