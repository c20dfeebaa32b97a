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
// 512 threads, 16 warps; pixel p = t % 256 belongs to warps w and w + 8
// (w = p / 32), and its TMEM row (gamma) is lane 32 (w % 4) + p % 32 of
// column block (w % 8) / 4, which both warps may read.  Per chunk n:
//   1. gamma(n) is issued (its radiance s(n) was staged at the end of the
//      previous chunk); all threads evaluate the weights G[b][p] of the
//      entries meeting each 32-pixel strip, the two warps of a strip taking
//      its even and its odd entries, eight at a time;
//   2. the recurrence runs on two threads per pixel: warps 0-7 take entries
//      31..16, warps 8-15 entries 15..0 after deriving the transmittance and
//      Q in the middle of the chunk from entries 31..16 (a product of
//      (1 - w) and the Q recurrence alone); each writes T w (bf16 x 2) and
//      its dL/dtau terms in place of the weights; then all warps drain
//      dL/ds(n-1) from TMEM into the gradient with float atomics (warp w:
//      lanes 32 (w % 4) = columns, entries 8 (w / 4) .. +7);
//   3. one barrier, dL/ds(n) is issued; all threads sum the chunk's dL/dtau
//      terms over the pixels (fixed order, one float atomic per entry) and
//      stage s(n+1) (prefetched into registers during step 2).
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
//   a[b][p]: MN-major (8 entries of one pixel are one 16-byte core row):
//            core (p/8, b/8) at (p/8) * kKsA + (b/8) * kMnA
// (s is written every chunk; its 144-byte core pitch along K spreads a warp's
// stores over all banks; a is written 8 entries per 16-byte store, 8 lanes
// of a quarter warp on one 128-byte span).
constexpr uint32_t kLboG = 128, kSboG = 16 * 128;
constexpr uint32_t kLboS = 144, kSboS = 16 * kLboS;
constexpr uint32_t kMnA = 128, kKsA = 4 * kMnA;
constexpr uint32_t kGBytes = kP * kNB * 2;
constexpr uint32_t kSBytes = 4 * kSboS;
constexpr uint32_t kABytes = (kP / 8) * kKsA;
constexpr uint32_t kOffG1 = 0, kOffG2 = kGBytes;
constexpr uint32_t kOffS1 = 2 * kGBytes, kOffS2 = kOffS1 + kSBytes;
constexpr uint32_t kOffA1 = kOffS2 + kSBytes, kOffA2 = kOffA1 + kABytes;
constexpr uint32_t kOffW = kOffA2 + kABytes;              // float G[32][256]
constexpr uint32_t kOffRec = kOffW + kCH * kP * 4;        // float4 [2][32][2]
constexpr uint32_t kOffIdx = kOffRec + 2 * kCH * 2 * 16;  // u32 [4][32] list indices
constexpr uint32_t kOffTQ = kOffIdx + 4 * kCH * 4;        // float2 [256] T, Q per pixel
constexpr uint32_t kOffMask = kOffTQ + kP * 8;            // u32 [8] strip masks
constexpr uint32_t kOffBar = kOffMask + 64;               // u64 [3] mbarriers
constexpr uint32_t kOffMisc = kOffBar + 24;               // u32 TMEM base, abort, #gamma, #dlds
constexpr uint32_t kSmem = kOffMisc + 16;
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kOffW % 16 == 0 && kOffA1 % 16 == 0 && kOffA2 % 16 == 0, "16-byte operand rows");

constexpr int kWq = 8;  // weights evaluated at once per thread (independent chains)
constexpr uint32_t kTmemCols = 128;  // gamma: columns 0-63 (two M tiles), dL/ds: 64-95
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kIdescGamma = tc::idesc_bf16(128, 32, 0, 0);
constexpr uint32_t kIdescDlds = tc::idesc_bf16(128, 32, 1, 1);

__device__ __forceinline__ uint32_t g_off(int p, int c) {
  return ((p >> 3) * 16 + (c >> 3)) * 128 + (p & 7) * 16 + (c & 7) * 2;
}

__global__ void __launch_bounds__(kThreads, 1)
    render_bwd_tc_kernel(const BackwardArgs A, int next_stride, int g_tma,
                         const __grid_constant__ CUtensorMap gmap) {
  extern __shared__ __align__(128) unsigned char sm[];
  float* sW = reinterpret_cast<float*>(sm + kOffW);
  float4* sRec0 = reinterpret_cast<float4*>(sm + kOffRec);
  uint32_t* sIdx = reinterpret_cast<uint32_t*>(sm + kOffIdx);
  float2* sTQ = reinterpret_cast<float2*>(sm + kOffTQ);
  uint32_t* sMask = reinterpret_cast<uint32_t*>(sm + kOffMask);
  uint64_t* barG = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint64_t* barD = barG + 1;
  uint64_t* barT = barG + 2;  // the cotangent tile's TMA copy
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

  // this thread's pixel; warps w and w + 8 share the pixels of strip w % 8
  const int p = t & (kP - 1);
  const int wp = warp & 7, half = warp >> 3;
  const int i = tr * g.TH + p / g.TW, jj = tcol * g.TW + p % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  // 1 / T and Q at the back end of the next chunk: the recovery
  // T_m = T_{m+1} / (1 - w_m) runs on the reciprocal, iT_m = iT_{m+1} (1 - w_m),
  // a multiply on the serial chain (the reciprocal T_m is off it)
  float iT = 1.0f, Q = 0.0f;
  uint32_t stop = rg.x;
  if (valid) {
    const size_t o = static_cast<size_t>(v) * HW + static_cast<size_t>(i) * g.W + jj;
    iT = A.tfin[o];  // T here; inverted before the sweep
    stop = A.stops[o];
  }
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
  // all threads: radiance of chunk n, entry t / 16, 8 columns from 8 (t % 16);
  // past the chunk the loads read entry 0's row (always in the array) and
  // store_rad writes zeros, so nothing waits for the loads before the
  // recurrence has run
  auto load_rad = [&](int n, float (&x)[8]) -> bool {
    const int b = t >> 4, cg = t & 15;
    const bool ok = b < chunk_len(n);
    const uint32_t k = ok ? sIdx[(n & 3) * kCH + b] : 0u;
    const float4* src =
        reinterpret_cast<const float4*>(radv + static_cast<size_t>(k) * a.stride + col0 + cg * 8);
    const float4 r0 = src[0], r1 = src[1];
    x[0] = r0.x; x[1] = r0.y; x[2] = r0.z; x[3] = r0.w;
    x[4] = r1.x; x[5] = r1.y; x[6] = r1.z; x[7] = r1.w;
    return ok;
  };
  auto store_rad = [&](float (&x)[8], bool ok) {
    const int b = t >> 4, cg = t & 15;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (!ok || col0 + cg * 8 + e >= a.ncols) x[e] = 0.0f;
    uint4 hi, lo;
    tc::split8(x, hi, lo);
    const uint32_t off = (b >> 3) * kSboS + cg * kLboS + (b & 7) * 16;
    *reinterpret_cast<uint4*>(sm + kOffS1 + off) = hi;
    *reinterpret_cast<uint4*>(sm + kOffS2 + off) = lo;
  };
  // all warps: dL/ds of chunk n from TMEM; warp w reads lanes 32 (w % 4)
  // (columns) and entries 8 (w / 4) .. +7
  auto drain_dlds = [&](uint32_t tmem, int n) {
    const int e0 = 8 * (warp >> 2);
    float d[8];
    tc::tmem_ld8(tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 64 + e0, d);
    const int col = col0 + 32 * (warp & 3) + lane;
    const int nb = chunk_len(n);
    const uint32_t* ks = sIdx + (n & 3) * kCH + e0;
    if (col < a.ncols) {
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (e0 + b < nb && d[b] != 0.0f)
          atomicAdd(&drad[static_cast<size_t>(ks[b]) * a.stride + col], d[b]);
    }
  };
  // thread 256: the MMAs of gamma(n) (g x s) and dL/ds(n) (g^T x a);
  // descriptors: a base per operand buffer, the start address (bits 0-13,
  // in 16-byte units) moved by adding the byte offset >> 4
  auto issue_gamma = [&](uint32_t tmem) {
    const uint64_t dg[2] = {tc::smem_desc(sbase + kOffG1, kLboG, kSboG),
                            tc::smem_desc(sbase + kOffG2, kLboG, kSboG)};
    const uint64_t ds[2] = {tc::smem_desc(sbase + kOffS1, kLboS, kSboS),
                            tc::smem_desc(sbase + kOffS2, kLboS, kSboS)};
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int k = 0; k < kNB / 16; ++k)
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint64_t a_d = dg[term == 2] + ((((16 * m) * 16 + 2 * k) * 128) >> 4);
          const uint64_t b_d = ds[term == 1] + ((2 * k * kLboS) >> 4);
          tc::mma_bf16(tmem + 32 * m, a_d, b_d, kIdescGamma, (k | term) != 0);
        }
  };
  auto issue_dlds = [&](uint32_t tmem) {
    // g read MN-major: M = columns (core pitch 128 B), K = pixels (core pitch 2048 B)
    const uint64_t dg[2] = {tc::smem_desc(sbase + kOffG1, kSboG, kLboG),
                            tc::smem_desc(sbase + kOffG2, kSboG, kLboG)};
    // a read MN-major: N = entries (core pitch 128 B), K = pixels (512 B)
    const uint64_t da[2] = {tc::smem_desc(sbase + kOffA1, kKsA, kMnA),
                            tc::smem_desc(sbase + kOffA2, kKsA, kMnA)};
#pragma unroll
    for (int k = 0; k < kP / 16; ++k)
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const uint64_t a_d = dg[term == 2] + ((k * 2 * kSboG) >> 4);
        const uint64_t b_d = da[term == 1] + ((2 * k * kKsA) >> 4);
        tc::mma_bf16(tmem + 64, a_d, b_d, kIdescDlds, (k | term) != 0);
      }
  };

  // ---- set-up: tensor memory, mbarriers, first indices
  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (t == 256) {
    tc::mbar_init(barG, 1);
    tc::mbar_init(barD, 1);
    tc::mbar_init(barT, 1);
    tc::mbar_fence_init();
    sMisc[1] = 0;
    sMisc[2] = 0;
    sMisc[3] = 0;
    if (g_tma) {
      // the tile's cotangent as float32 [kNB / 2C receivers][TH rows][TW
      // pixels x 2C] into the g buffers (one box; out-of-range rows,
      // pixels and receivers read as zero), split in place below; it needs
      // nothing loaded first, so it overlaps the list-index chain
      tc::mbar_arrive_expect_tx(barT, 2 * kGBytes);
      tc::tma_load_4d(sm + kOffG1, &gmap, tcol * g.TW * twoC, tr * g.TH, col0 / twoC, v, barT);
    }
  }
  if (warp == 8 && nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
  }
  // cotangent tile -> g (bf16 x 2): thread t takes pixel p and the 8-column
  // octets (t >> 8) + 2r; every (re, im) column pair is one 8-byte load, all
  // 32 of a thread in flight before the split (without the TMA copy)
  if (!g_tma) {
    float2 xv[8][4];
    const size_t pix = static_cast<size_t>(i) * g.W + jj;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int oc = (t >> 8) + 2 * r;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = col0 + oc * 8 + 2 * e;  // even: (re, im) of one channel
        float2 val = make_float2(0.0f, 0.0f);
        if (valid && col < a.ncols) {
          const int j = col / twoC, ec = col - j * twoC;
          if (A.g_spec)
            val = *reinterpret_cast<const float2*>(
                &A.g_spec[((static_cast<size_t>(v) * a.N + j) * HW + pix) * twoC + ec]);
          if (A.g_uniform) {
            const float2 u =
                *reinterpret_cast<const float2*>(&A.g_uniform[static_cast<size_t>(v) * a.ncols + col]);
            val.x += u.x;
            val.y += u.y;
          }
        }
        xv[r][e] = val;
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int oc = (t >> 8) + 2 * r;
      const float x[8] = {xv[r][0].x, xv[r][0].y, xv[r][1].x, xv[r][1].y,
                          xv[r][2].x, xv[r][2].y, xv[r][3].x, xv[r][3].y};
      uint4 hi, lo;
      tc::split8(x, hi, lo);
      const uint32_t off = g_off(p, oc * 8);
      *reinterpret_cast<uint4*>(sm + kOffG1 + off) = hi;
      *reinterpret_cast<uint4*>(sm + kOffG2 + off) = lo;
    }
  }
  if (warp == 8 && nchunks > 0) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  __syncthreads();  // indices of chunk 0, mbarriers, TMEM address
  if (warp == 8 && nchunks > 0) {
    gather_rec(0);
    cp_async_commit();
  }
  {
    float x[8];
    const bool ok = nchunks > 0 && load_rad(0, x);
    if (g_tma) {
      // the copied tile: thread t reads pixel p's (re, im) pairs of octets
      // (t >> 8) + 2r, then (every read done) writes them split in place
      if (!tc::mbar_wait(barT, 0, kWaitLimit)) fail();
      const float* stg = reinterpret_cast<const float*>(sm + kOffG1);
      const int y = p / g.TW, px = p % g.TW, rowf = g.TW * twoC;
      float2 xv[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int oc = (t >> 8) + 2 * r;
        // column c = 2C z + ec of the block's receiver z (one division per octet)
        int z = (oc * 8) / twoC, ec = oc * 8 - z * twoC;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int c = oc * 8 + 2 * e;
          float2 val = *reinterpret_cast<const float2*>(&stg[(z * g.TH + y) * rowf + px * twoC + ec]);
          ec += 2;
          if (ec == twoC) {
            ec = 0;
            ++z;
          }
          if (A.g_uniform && valid && col0 + c < a.ncols) {
            const float2 u = *reinterpret_cast<const float2*>(
                &A.g_uniform[static_cast<size_t>(v) * a.ncols + col0 + c]);
            val.x += u.x;
            val.y += u.y;
          }
          xv[r][e] = val;
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int oc = (t >> 8) + 2 * r;
        const float xs[8] = {xv[r][0].x, xv[r][0].y, xv[r][1].x, xv[r][1].y,
                             xv[r][2].x, xv[r][2].y, xv[r][3].x, xv[r][3].y};
        uint4 hi, lo;
        tc::split8(xs, hi, lo);
        const uint32_t off = g_off(p, oc * 8);
        *reinterpret_cast<uint4*>(sm + kOffG1 + off) = hi;
        *reinterpret_cast<uint4*>(sm + kOffG2 + off) = lo;
      }
    }
    if (nchunks > 0) store_rad(x, ok);
  }
  const uint32_t tmem = sMisc[0];

  // The cotangent tile of the CTA likely to start next on this SM (linear
  // index + the CTAs resident at once) into L2, so that its prologue reads
  // hit L2 instead of waiting on HBM: one thread per (receiver, tile row)
  // segment, one prefetch per 128-byte line.
  if (A.g_spec && next_stride > 0) {
    const long long total = static_cast<long long>(gridDim.x) * gridDim.y * gridDim.z;
    const long long nxt =
        blockIdx.x + static_cast<long long>(gridDim.x) * (blockIdx.y + static_cast<long long>(gridDim.y) * blockIdx.z) +
        next_stride;
    if (nxt < total) {
      const int tile2 = static_cast<int>(nxt % gridDim.x);
      const long long r2 = nxt / gridDim.x;
      const int v2 = static_cast<int>(r2 / gridDim.y);
      const int c0 = static_cast<int>(r2 % gridDim.y) * kNB, c1 = min(a.ncols, c0 + kNB) - 1;
      const int j0 = c0 / twoC, nj = c1 / twoC - j0 + 1;
      const int i0 = (tile2 / g.tiles_w) * g.TH, jj0 = (tile2 % g.tiles_w) * g.TW;
      const int rows = min(g.TH, g.H - i0), ncol = min(g.TW, g.W - jj0);
      for (int q = t; q < nj * rows; q += kThreads) {
        const int j = j0 + q / rows, i = i0 + q % rows;
        const float* row = A.g_spec + ((static_cast<size_t>(v2) * a.N + j) * HW +
                                       static_cast<size_t>(i) * g.W + jj0) * twoC;
        const uintptr_t e = reinterpret_cast<uintptr_t>(row + static_cast<size_t>(ncol) * twoC);
        for (uintptr_t ln = reinterpret_cast<uintptr_t>(row) & ~static_cast<uintptr_t>(127); ln < e;
             ln += 128)
          asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ln));
      }
    }
  }

  iT = 1.0f / iT;
  const uint32_t strip_stop = __reduce_max_sync(0xffffffffu, stop);  // the warp's 32 pixels
  // ---- the sweep, back to front
  for (int n = 0; n < nchunks; ++n) {
    tc::fence_smem_to_async();  // s(n) (and g for n = 0) for the tensor core
    tc::fence_before_sync();
    cp_async_wait_all();  // records of chunk n, indices of chunk n + 1
    __syncthreads();
    tc::fence_after_sync();
    if (sMisc[1]) break;
    if (t == 256) {
      issue_gamma(tmem);
      tc::mma_commit(barG);
      sMisc[2] = n + 1;
    }
    const uint32_t start = chunk_start(n);
    const int nb = chunk_len(n);
    if (warp == 8) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      if (n + 1 < nchunks) gather_rec(n + 1);
      cp_async_commit();
    }
    const float4* sR = sRec0 + (n & 1) * 2 * kCH;
    // 1. weights G[b][p] (0: not composited) of the entries meeting this
    //    warp's strip; the two warps of a strip take its even and odd entries
    {
      const bool rel = lane < nb && touches_strip(g, sR[2 * lane + 1], strip);
      unsigned m = __ballot_sync(0xffffffffu, rel);
      // entries at or past the strip's last stop position are composited by
      // none of its pixels
      if (strip_stop <= start)
        m = 0;
      else if (strip_stop - start < 32u)
        m &= (1u << (strip_stop - start)) - 1u;
      if (half == 0 && lane == 0) sMask[wp] = m;
      unsigned mine = m & (half ? 0xaaaaaaaau : 0x55555555u);  // odd / even entries
      while (mine) {
        int bq[kWq];
#pragma unroll
        for (int q = 0; q < kWq; ++q) {
          bq[q] = mine ? __ffs(mine) - 1 : -1;
          mine &= mine - 1;
        }
        float G[kWq];
#pragma unroll
        for (int q = 0; q < kWq; ++q) {
          const int b = bq[q] >= 0 ? bq[q] : bq[0];
          G[q] = pixel_G_grad(g, sR[2 * b], sR[2 * b + 1], i, fi, jj, fj);
        }
#pragma unroll
        for (int q = 0; q < kWq; ++q)
          if (bq[q] >= 0)
            sW[bq[q] * kP + p] = (valid && start + bq[q] < stop && G[q] > 0.0f) ? G[q] : 0.0f;
      }
    }
    // the weights and mask of a strip are read only by its two warps: their
    // barrier, not the CTA's (everything else the recurrence reads was
    // ordered by the chunk's first barrier or arrives through mbarriers)
    tc::named_barrier(1 + wp, 64);
    // 2. the recurrence, two threads per pixel
    float x[8];
    const bool more = n + 1 < nchunks;
    bool x_ok = false;
    if (more) x_ok = load_rad(n + 1, x);  // in flight during the recurrence
    if (!tc::mbar_wait(barG, n & 1, kWaitLimit)) fail();
    tc::fence_after_sync();
    float gam[32];
    tc::tmem_ld32(tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 32 * (wp >> 2), gam);
    if (n > 0 && !tc::mbar_wait(barD, (n - 1) & 1, kWaitLimit)) fail();  // a is free again
    tc::fence_after_sync();
    const unsigned m = sMask[wp];
    auto step = [&](int b, float& dt) -> float {
      float Tw = 0.0f;
      dt = 0.0f;
      if (m & (1u << b)) {
        const float G = sW[b * kP + p];
        if (G != 0.0f) {
          const float w = __fmul_rn(sR[2 * b + 1].y, G);
          const float one_m_w = 1.0f - w;
          iT *= one_m_w;
          const float T = __fdividef(1.0f, iT);  // transmittance in front of entry b
          Tw = T * w;
          dt = T * (gam[b] - Q) * G;
          Q = fmaf(w, gam[b], one_m_w * Q);
        }
      }
      return Tw;
    };
    // T w of entries 8e .. 8e + 7 of this pixel: one 16-byte core row per term
    auto put_a = [&](int e, const float (&tw)[8]) {
      uint4 hi, lo;
      tc::split8(tw, hi, lo);
      const uint32_t off = (p >> 3) * kKsA + e * kMnA + (p & 7) * 16;
      *reinterpret_cast<uint4*>(sm + kOffA1 + off) = hi;
      *reinterpret_cast<uint4*>(sm + kOffA2 + off) = lo;
    };
    if (half == 0) {
      // entries 31..16 from the back end; their dL/dtau terms are written
      // after the front thread has read these entries' weights
      float dts[16], tw0[8], tw1[8];
#pragma unroll
      for (int b = kCH - 1; b >= 24; --b) tw1[b - 24] = step(b, dts[b - 16]);
#pragma unroll
      for (int b = 23; b >= 16; --b) tw0[b - 16] = step(b, dts[b - 16]);
      tc::named_barrier(1 + wp, 64);
#pragma unroll
      for (int b = 16; b < kCH; ++b) sW[b * kP + p] = dts[b - 16];
      put_a(2, tw0);
      put_a(3, tw1);
    } else {
      // T and Q in the middle of the chunk: the transmittance product and
      // the Q recurrence over entries 31..16
      float P = 1.0f;
#pragma unroll
      for (int b = kCH - 1; b >= 16; --b) {
        if (m & (1u << b)) {
          const float G = sW[b * kP + p];
          if (G != 0.0f) {
            const float w = __fmul_rn(sR[2 * b + 1].y, G);
            const float one_m_w = 1.0f - w;
            P *= one_m_w;
            Q = fmaf(w, gam[b], one_m_w * Q);
          }
        }
      }
      iT *= P;
      tc::named_barrier(1 + wp, 64);
      float tw0[8], tw1[8];
#pragma unroll
      for (int b = 15; b >= 8; --b) {
        float dt;
        tw1[b - 8] = step(b, dt);
        sW[b * kP + p] = dt;
      }
#pragma unroll
      for (int b = 7; b >= 0; --b) {
        float dt;
        tw0[b] = step(b, dt);
        sW[b * kP + p] = dt;
      }
      put_a(0, tw0);
      put_a(1, tw1);
      sTQ[p] = make_float2(iT, Q);  // the state at the front end of chunk n
    }
    if (n > 0) drain_dlds(tmem, n - 1);
    // 3. issue dL/ds(n); dL/dtau of chunk n; stage s(n + 1)
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (t == 256 && sMisc[1] == 0) {
      tc::fence_after_sync();
      issue_dlds(tmem);
      tc::mma_commit(barD);
      sMisc[3] = n + 1;
    }
    {
      // entry b = t / 16: 16 lanes sum its 256 pixels, 16-byte loads (a
      // quarter warp on 128 contiguous bytes), then a shuffle tree
      const int b = t >> 4, q = t & 15;
      const float4* w4 = reinterpret_cast<const float4*>(sW + b * kP);
      float y = 0.0f;
#pragma unroll
      for (int r = 0; r < kP / 64; ++r) {
        const float4 u = w4[q + 16 * r];
        y += (u.x + u.y) + (u.z + u.w);
      }
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
      if (q == 0 && b < nb && y != 0.0f) atomicAdd(&A.d_tau[sIdx[(n & 3) * kCH + b]], y);
    }
    if (more) store_rad(x, x_ok);  // gamma(n) is complete: s is free
    if (half == 0) {
      const float2 tq = sTQ[p];
      iT = tq.x;
      Q = tq.y;
    }
  }
  cp_async_wait_all();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool aborted = sMisc[1] != 0;
  if (!aborted && nchunks > 0) {
    const int nl = nchunks - 1;
    if (tc::mbar_wait(barD, nl & 1, kWaitLimit)) {
      tc::fence_after_sync();
      drain_dlds(tmem, nl);
    } else {
      fail();
    }
  }
  if (aborted && t == 256) {
    // let copies and MMAs still in flight finish (bounded) before their
    // memory goes
    if (g_tma) tc::mbar_wait(barT, 0, kWaitLimit);
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
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  // the cotangent tile by TMA when a box covers it: 2C divides the block's
  // columns and a tile row of pixels x 2C fits one box extent
  CUtensorMap gmap{};
  const int twoC = 2 * a.C, rowf = a.g.TW * twoC;
  bool tma = A.g_spec && kNB % twoC == 0 && rowf <= 256 && rowf % 4 == 0;
  if (tma) {
    const uint64_t W2 = static_cast<uint64_t>(a.g.W) * twoC;
    const uint64_t dims[4] = {W2, static_cast<uint64_t>(a.g.H), static_cast<uint64_t>(a.N),
                              static_cast<uint64_t>(a.M)};
    const uint64_t strides[3] = {W2 * 4, W2 * a.g.H * 4, W2 * a.g.H * a.N * 4};
    const uint32_t box[4] = {static_cast<uint32_t>(rowf), static_cast<uint32_t>(a.g.TH),
                             static_cast<uint32_t>(kNB / twoC), 1};
    tma = tc::encode_f32_tiled(&gmap, A.g_spec, 4, dims, strides, box);
  }
  dim3 grid(a.g.T, (a.ncols + kNB - 1) / kNB, a.M);
  render_bwd_tc_kernel<<<grid, kThreads, kSmem, s>>>(A, nsm, tma ? 1 : 0, gmap);
  note_launches(1);
}

}  // namespace rxgs
