// render_fwd_tc.cu -- front-to-back compositing (Algorithm 1, Stage 3) of one
// (view, tile, 128-column block) with the chunk products on the tcgen05
// tensor cores and the tile's spectra accumulated in tensor memory.
//
// The tile list is consumed in chunks of 32 Gaussians.  For chunk n each
// pixel p walks the entries that meet its warp's strip in depth order and
// forms A[p][b] = T_b w_b (zero where Gaussian b is not composited by p); the
// chunk's contribution to all 128 columns is the product
//   C[p][c] += sum_b A[p][b] s[b][c]        (M = 256 pixels, N = 128, K = 32)
// accumulated over the whole list in TMEM (two 128-row tiles x 128 float32
// columns).  A and s enter the MMA split into two bf16 terms each (three MMAs
// per product, about 1.2e-5 relative error per term, tc_common.cuh).  The
// weights and the transmittance follow the float32 decision specification
// exactly as the CUDA-core kernel does, so the per-pixel stop positions and
// final transmittances are bit-identical to it.
//
// 256 threads, one per pixel (thread = TMEM lane of its pixel row), two CTAs
// per SM.  Per chunk n: wait for the MMA of chunk n - 1 (it read A and the
// radiance buffer that chunk n + 1 will fill), write A for chunk n, stage
// the radiance of chunk n + 1 (double-buffered), one barrier, issue the MMA
// of chunk n.  The tile stops after the chunk in which its last pixel
// stopped.  Epilogue: the accumulator comes back 32 columns at a time
// (tcgen05.ld), is written as spectra, and its column sums over the tile
// (a warp reduce-scatter, then eight warps in order) go to the per-tile
// partial sums of CSI / RSSI.  Every mbarrier wait is bounded (kErrTimeout).
#include <cuda_bf16.h>

#include "render_common.cuh"
#include "rxgs_internal.h"
#include "tc_common.cuh"

namespace rxgs {
namespace {

constexpr int kP = kTilePixels;  // 256
constexpr int kNB = 128;
constexpr int kCH = kChunk;      // 32
constexpr int kThreads = kP;

// s[b][c]: core (b/8, c/8) at (b/8) * kSboS + (c/8) * kLboS, read MN-major
//          (N = columns, core pitch kLboS; K = entries, core pitch kSboS)
// A[b][p]: core (b/8, p/8) at (b/8) * kSboA + (p/8) * kLboA, read MN-major
//          (M = pixels, core pitch kLboA; K = entries, core pitch kSboA)
constexpr uint32_t kLboS = 144, kSboS = 16 * kLboS;
constexpr uint32_t kLboA = 144, kSboA = 32 * kLboA;
constexpr uint32_t kSBytes = 4 * kSboS;
constexpr uint32_t kABytes = 4 * kSboA;
constexpr uint32_t kOffS = 0;                               // [2 buffers][hi, lo]
constexpr uint32_t kOffA1 = 4 * kSBytes, kOffA2 = kOffA1 + kABytes;
constexpr uint32_t kOffRec = kOffA2 + kABytes;              // float4 [2][32][2]
constexpr uint32_t kOffIdx = kOffRec + 2 * kCH * 2 * 16;    // u32 [3][32]
constexpr uint32_t kOffMask = kOffIdx + 3 * kCH * 4;        // u32 [8]
constexpr uint32_t kOffBar = kOffMask + 32;                 // u64
constexpr uint32_t kOffMisc = kOffBar + 8;                  // u32 TMEM base, abort, tile stop
constexpr uint32_t kSmemUsed = kOffMisc + 12;
// requested: more than a third of an SM's shared memory, so at most two CTAs
// (2 x 256 TMEM columns, all of it) share an SM and an allocation never waits
constexpr uint32_t kSmem = 80 * 1024;
static_assert(kSmemUsed <= kSmem, "shared memory");
// the epilogue reuses the operand buffers (the MMAs are done): two staging
// buffers of 32 spectra columns for the TMA stores, then the column sums
// float [8 warps][128]
constexpr uint32_t kStage = kP * 32 * 4;
constexpr uint32_t kOffPart = 2 * kStage;
static_assert(kOffPart + 8 * kNB * 4 <= kOffRec, "staging and partial sums fit in the operands");
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(2 * kSmem <= 232448, "two CTAs per SM");

constexpr int kWq = 3;  // weights evaluated at once per thread (independent chains)
constexpr uint32_t kTmemCols = 256;  // two M tiles x 128 float32 columns
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr uint32_t kIdesc = tc::idesc_bf16(128, 128, 1, 1);

__global__ void __launch_bounds__(kThreads, 2)
    render_fwd_tc_kernel(const RenderArgs a, int s_tma, const __grid_constant__ CUtensorMap smap) {
  extern __shared__ __align__(128) unsigned char sm[];
  float4* sRec0 = reinterpret_cast<float4*>(sm + kOffRec);
  uint32_t* sIdx = reinterpret_cast<uint32_t*>(sm + kOffIdx);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(sm + kOffMisc);

  const GridConst& g = a.g;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int col0 = blockIdx.y * kNB;
  const int tr = tile / g.tiles_w, tcol = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tcol * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = a.ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = a.rec + static_cast<size_t>(v) * a.K * 2;
  const float* radv = a.rad + static_cast<size_t>(v) * a.rad_view;
  const int nchunks = static_cast<int>((rg.y - rg.x + kCH - 1) / kCH);
  const uint32_t sbase = tc::smem_u32(sm);
  const Strip strip = warp_strip(g, tr, tcol, warp);

  auto chunk_len = [&](int n) {
    return min(kCH, static_cast<int>(rg.y - rg.x - static_cast<uint32_t>(n) * kCH));
  };
  auto copy_indices = [&](int n) {  // warp 0
    const bool ok = lane < chunk_len(n);
    cp_async4(&sIdx[(n % 3) * kCH + lane], ok ? &a.vals[rg.x + n * kCH + lane] : a.vals, ok);
  };
  auto gather_rec = [&](int n) {  // warp 0
    const bool ok = lane < chunk_len(n);
    const uint32_t k = ok ? sIdx[(n % 3) * kCH + lane] : 0u;
    float4* rb = sRec0 + (n & 1) * 2 * kCH;
    cp_async16(&rb[2 * lane + 0], &rec[2 * k + 0], ok);
    cp_async16(&rb[2 * lane + 1], &rec[2 * k + 1], ok);
  };
  // radiance of chunk n: thread t takes entry t / 8 and 16 columns; past the
  // chunk the loads read entry 0's row (always in the array) and store_rad
  // writes zeros, so nothing waits for the loads before the weights have run
  auto load_rad = [&](int n, float (&x)[16]) -> bool {
    const int b = t >> 3, cg = t & 7;
    const bool ok = b < chunk_len(n);
    const uint32_t k = ok ? sIdx[(n % 3) * kCH + b] : 0u;
    const float4* src =
        reinterpret_cast<const float4*>(radv + static_cast<size_t>(k) * a.stride + col0 + cg * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 r = src[q];
      x[4 * q + 0] = r.x;
      x[4 * q + 1] = r.y;
      x[4 * q + 2] = r.z;
      x[4 * q + 3] = r.w;
    }
    return ok;
  };
  auto store_rad = [&](int buf, float (&x)[16], bool ok) {
    const int b = t >> 3, cg = t & 7;
#pragma unroll
    for (int e = 0; e < 16; ++e)
      if (!ok || col0 + cg * 16 + e >= a.ncols) x[e] = 0.0f;
    float x0[8], x1[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      x0[e] = x[e];
      x1[e] = x[8 + e];
    }
    const uint32_t hi_off = kOffS + (2 * buf) * kSBytes, lo_off = hi_off + kSBytes;
    const uint32_t row = (b >> 3) * kSboS + (b & 7) * 16;
    uint4 hi, lo;
    tc::split8(x0, hi, lo);
    *reinterpret_cast<uint4*>(sm + hi_off + row + (2 * cg) * kLboS) = hi;
    *reinterpret_cast<uint4*>(sm + lo_off + row + (2 * cg) * kLboS) = lo;
    tc::split8(x1, hi, lo);
    *reinterpret_cast<uint4*>(sm + hi_off + row + (2 * cg + 1) * kLboS) = hi;
    *reinterpret_cast<uint4*>(sm + lo_off + row + (2 * cg + 1) * kLboS) = lo;
  };
  auto issue_mma = [&](uint32_t tmem, int n) {
    const uint32_t s_hi = sbase + kOffS + (2 * (n & 1)) * kSBytes, s_lo = s_hi + kSBytes;
#pragma unroll 1
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int k = 0; k < kCH / 16; ++k)
#pragma unroll
        for (int term = 0; term < 3; ++term) {
          const uint32_t aa = sbase + (term == 2 ? kOffA2 : kOffA1) + 16 * m * kLboA + 2 * k * kSboA;
          const uint32_t bb = (term == 1 ? s_lo : s_hi) + 2 * k * kSboS;
          tc::mma_bf16(tmem + 128 * m, tc::smem_desc(aa, kSboA, kLboA),
                       tc::smem_desc(bb, kSboS, kLboS), kIdesc, (n | k | term) != 0);
        }
  };

  // ---- set-up
  if (warp == 0) tc::tmem_alloc(&sMisc[0], kTmemCols);
  if (t == 32) {
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
    sMisc[1] = 0;
  }
  if (warp == 0 && nchunks > 0) {
    copy_indices(0);
    cp_async_commit();
    if (nchunks > 1) copy_indices(1);
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();  // indices of chunk 0, mbarrier, TMEM address
  tc::fence_after_sync();
  const uint32_t tmem = sMisc[0];
  if (warp == 0 && nchunks > 0) {
    gather_rec(0);
    cp_async_commit();
  }
  if (nchunks > 0) {
    float x[16];
    const bool ok = load_rad(0, x);
    store_rad(0, x, ok);
  }

  float T = 1.0f;
  bool alive = valid;
  int ncon = 0, issued = 0;
  uint32_t stop = valid ? rg.y : rg.x;  // list position after the stopping entry
  for (int n = 0; n < nchunks; ++n) {
    cp_async_wait_all();  // records of chunk n, indices of chunk n + 1
    __syncthreads();
    if (sMisc[1]) break;
    const int nb = chunk_len(n);
    if (warp == 0) {
      if (n + 2 < nchunks) copy_indices(n + 2);
      if (n + 1 < nchunks) gather_rec(n + 1);
      cp_async_commit();
    }
    float x[16];
    const bool more = n + 1 < nchunks;
    bool x_ok = false;
    if (more) x_ok = load_rad(n + 1, x);
    // the MMA of chunk n - 1 has read A and radiance buffer (n + 1) & 1
    if (n > 0 && !tc::mbar_wait(bar, (n - 1) & 1, kWaitLimit)) {
      atomicOr(&sMisc[1], 1u);
      if (a.err) atomicOr(a.err, kErrTimeout);
    }
    // A[p][b] = T w for the entries of this warp's strip, in depth order:
    // weights three entries at a time (independent, branch-free), then the
    // transmittance updates in list order
    const float4* sR = sRec0 + (n & 1) * 2 * kCH;
    const bool rel = lane < nb && touches_strip(g, sR[2 * lane + 1], strip);
    const unsigned mask = __any_sync(0xffffffffu, alive) ? __ballot_sync(0xffffffffu, rel) : 0u;
    auto put_a = [&](int b, float Tw) {
      __nv_bfloat16 hi, lo;
      tc::split_bf16(Tw, hi, lo);
      const uint32_t off = (b >> 3) * kSboA + (t >> 3) * kLboA + (b & 7) * 16 + (t & 7) * 2;
      *reinterpret_cast<__nv_bfloat16*>(sm + kOffA1 + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(sm + kOffA2 + off) = lo;
    };
    // entries that meet no pixel of the strip: A = 0 (both terms, no split)
    for (unsigned z = ~mask; z; z &= z - 1) {
      const int b = __ffs(z) - 1;
      const uint32_t off = (b >> 3) * kSboA + (t >> 3) * kLboA + (b & 7) * 16 + (t & 7) * 2;
      *reinterpret_cast<uint16_t*>(sm + kOffA1 + off) = 0;
      *reinterpret_cast<uint16_t*>(sm + kOffA2 + off) = 0;
    }
    for (unsigned m = mask; m;) {
      int bq[kWq];
#pragma unroll
      for (int q = 0; q < kWq; ++q) {
        bq[q] = m ? __ffs(m) - 1 : -1;
        m &= m - 1;
      }
      float G[kWq];
#pragma unroll
      for (int q = 0; q < kWq; ++q) {
        const int b = bq[q] >= 0 ? bq[q] : bq[0];
        G[q] = pixel_G(g, sR[2 * b], sR[2 * b + 1], i, fi, jj, fj);
      }
#pragma unroll
      for (int q = 0; q < kWq; ++q) {
        if (bq[q] < 0) break;
        float Tw = 0.0f;
        if (alive && G[q] >= 0.0f) {
          const float w = __fmul_rn(sR[2 * bq[q] + 1].y, G[q]);
          Tw = __fmul_rn(T, w);
          T = __fmul_rn(T, __fsub_rn(1.0f, w));
          ++ncon;
          if (T < g.eps_T) {
            alive = false;
            stop = rg.x + static_cast<uint32_t>(n * kCH + bq[q] + 1);
          }
        }
        put_a(bq[q], Tw);
      }
    }
    if (more) store_rad((n + 1) & 1, x, x_ok);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    const int n_alive = __syncthreads_count(alive);
    if (t == 0 && sMisc[1] == 0) {
      tc::fence_after_sync();
      issue_mma(tmem, n);
      tc::mma_commit(bar);
    }
    issued = n + 1;
    if (n_alive == 0) break;
  }
  cp_async_wait_all();
  __syncthreads();
  const bool ok = sMisc[1] == 0;
  bool have = issued > 0 && ok;
  if (have && !tc::mbar_wait(bar, (issued - 1) & 1, kWaitLimit)) {
    atomicOr(&sMisc[1], 1u);
    if (a.err) atomicOr(a.err, kErrTimeout);
  }
  __syncthreads();
  have = have && sMisc[1] == 0;
  tc::fence_after_sync();

  // ---- epilogue: spectra, per-tile column sums, stop counts
  const size_t HW = static_cast<size_t>(g.H) * g.W;
  const int twoC = 2 * a.C;
  const size_t po = static_cast<size_t>(i) * g.W + jj;
  float* sPart = reinterpret_cast<float*>(sm + kOffPart);  // [8][128]; the MMAs are done
  const int y = t / g.TW, px = t % g.TW, rowf = g.TW * twoC;
#pragma unroll 1
  for (int q = 0; q < kNB / 32; ++q) {
    float d[32];
    if (have) {
      tc::tmem_ld32(tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 128 * (warp >> 2) + 32 * q,
                    d);
    } else {
#pragma unroll
      for (int e = 0; e < 32; ++e) d[e] = 0.0f;
    }
    if (s_tma) {
      // 32 columns as one box [32 / 2C receivers][TH rows][TW pixels x 2C]
      // staged in shared memory and stored by TMA (out-of-range pixels and
      // receivers are not written); two staging buffers
      float* stg = reinterpret_cast<float*>(sm + (q & 1) * kStage);
      if (q >= 2) {
        if (t == 0) tc::bulk_wait_read<1>();  // the store of q - 2 has read its buffer
        __syncthreads();
      }
      int z = 0, ec = 0;
#pragma unroll
      for (int e = 0; e < 32; e += 2) {
        *reinterpret_cast<float2*>(&stg[(z * g.TH + y) * rowf + px * twoC + ec]) =
            make_float2(d[e], d[e + 1]);
        ec += 2;
        if (ec == twoC) {
          ec = 0;
          ++z;
        }
      }
      tc::fence_smem_to_async();
      __syncthreads();
      if (t == 0) {
        tc::tma_store_4d(&smap, tcol * g.TW * twoC, tr * g.TH, (col0 + 32 * q) / twoC, v, stg);
        tc::bulk_commit();
      }
    } else if (a.spectra && valid) {
      // column c = 2C j + ec of receiver j: the (re, im) pairs of this
      // pixel advance by 2 within a receiver and by H W 2C floats to the
      // next one (one division per 32 columns)
      const int c0 = col0 + 32 * q;
      int ec = c0 % twoC;
      float* dst = a.spectra + ((static_cast<size_t>(v) * a.N + c0 / twoC) * HW + po) * twoC + ec;
      const size_t jstep = HW * twoC - twoC;
#pragma unroll
      for (int e = 0; e < 32; e += 2) {
        if (c0 + e < a.ncols) *reinterpret_cast<float2*>(dst) = make_float2(d[e], d[e + 1]);
        ec += 2;
        dst += 2;
        if (ec == twoC) {
          ec = 0;
          dst += jstep;
        }
      }
    }
    if (a.partial) {
      // reduce-scatter over the warp's 32 pixels: lane l ends with column l
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int e = 0; e < s; ++e) {
          const float send = upper ? d[e] : d[e + s];
          const float keep = upper ? d[e + s] : d[e];
          d[e] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
      }
      sPart[warp * kNB + 32 * q + lane] = d[0];
    }
  }
  if (col0 == 0 && valid) {
    const size_t o = static_cast<size_t>(v) * HW + po;
    if (a.ncontrib) a.ncontrib[o] = ncon;
    if (a.tfinal) a.tfinal[o] = T;
    if (a.keep_tfin) {
      a.keep_tfin[o] = T;
      a.keep_stops[o] = stop;
    }
  }
  // the tile's largest stop (reuses the abort word's neighbour: the MMAs and
  // every wait are over)
  if (col0 == 0 && a.keep_tile_stop) {
    if (t == 0) sMisc[2] = rg.x;
    __syncthreads();
    atomicMax(&sMisc[2], stop);
    __syncthreads();
    if (t == 0) a.keep_tile_stop[static_cast<size_t>(v) * g.T + tile] = sMisc[2];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (a.partial && t < kNB && col0 + t < a.ncols) {
    float y = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) y += sPart[w * kNB + t];
    a.partial[(static_cast<size_t>(v) * g.T + tile) * a.ncols + col0 + t] = y;
  }
  if (s_tma && t == 0) tc::bulk_wait_read<0>();  // staging read before the CTA leaves
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace

void launch_render_fwd_tc(const RenderArgs& a, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(kSmem));
    configured = true;
  }
  // spectra by TMA stores when a box of 32 columns covers whole receivers
  // and a tile row of pixels x 2C fits one box extent
  CUtensorMap smap{};
  const int twoC = 2 * a.C, rowf = a.g.TW * twoC;
  bool tma = a.spectra && 32 % twoC == 0 && rowf <= 256 && rowf % 4 == 0;
  if (tma) {
    const uint64_t W2 = static_cast<uint64_t>(a.g.W) * twoC;
    const uint64_t dims[4] = {W2, static_cast<uint64_t>(a.g.H), static_cast<uint64_t>(a.N),
                              static_cast<uint64_t>(a.M)};
    const uint64_t strides[3] = {W2 * 4, W2 * a.g.H * 4, W2 * a.g.H * a.N * 4};
    const uint32_t box[4] = {static_cast<uint32_t>(rowf), static_cast<uint32_t>(a.g.TH),
                             static_cast<uint32_t>(32 / twoC), 1};
    tma = tc::encode_f32_tiled(&smap, a.spectra, 4, dims, strides, box);
  }
  dim3 grid(a.g.T, (a.ncols + kNB - 1) / kNB, a.M);
  render_fwd_tc_kernel<<<grid, kThreads, kSmem, s>>>(a, tma ? 1 : 0, smap);
  note_launches(1);
}

}  // namespace rxgs
