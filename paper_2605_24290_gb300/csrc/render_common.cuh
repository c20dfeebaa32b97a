// render_common.cuh -- pieces shared by the forward and backward compositing
// kernels: the per-pixel weight (the decision specification of Algorithm 1,
// Stage 3) and cp.async helpers.
#pragma once
#include "rxgs_internal.h"
#include "rxgs_math.cuh"

namespace rxgs {

constexpr int kTilePixels = 256;
constexpr int kChunk = 32;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Per-pixel weight of one Gaussian record (the decision specification:
// footprint test, q in float32 with this exact operation order, q <= q_max,
// w = tau * exp(-q/2)).  Returns false when the Gaussian does not contribute.
__device__ __forceinline__ bool pixel_weight(const GridConst& g, const float4 r0, const float4 r1,
                                             int i, int jj, float fi, float fj, float* w_out,
                                             float* G_out) {
  const int rows = __float_as_int(r1.z), cols = __float_as_int(r1.w);
  if (i < (rows & 0xffff) || i > (rows >> 16)) return false;
  int dj = jj - (cols & 0xffff);
  if (dj < 0) dj += g.W;
  if (dj > (cols >> 16)) return false;
  const float dt = __fsub_rn(fi, r0.x);
  float dp = __fsub_rn(fj, r0.y);
  if (dp >= g.halfW)
    dp = __fsub_rn(dp, g.Wf);
  else if (dp < -g.halfW)
    dp = __fadd_rn(dp, g.Wf);
  const float t1 = __fmul_rn(r0.w, dp);
  const float t2 = __fmaf_rn(r0.z, dt, t1);
  const float t3 = __fmul_rn(r1.x, dp);
  const float t4 = __fmul_rn(t3, dp);
  const float q = __fmaf_rn(dt, t2, t4);
  if (!(q <= g.q_max)) return false;
  const float G = exp32(__fmul_rn(-0.5f, q));
  *G_out = G;
  *w_out = __fmul_rn(r1.y, G);
  return true;
}

// The same decision without branches: G = exp(-q/2) >= 0 when the Gaussian
// contributes to pixel (i, jj) (footprint, q <= q_max), else -1.  Identical
// operations to pixel_weight (so identical bits, exp32's underflow to 0
// included), evaluated whether or not the pixel is inside, so that several
// entries can be in flight at once.
__device__ __forceinline__ float pixel_G(const GridConst& g, const float4 r0, const float4 r1,
                                         int i, float fi, int jj, float fj) {
  const int rows = __float_as_int(r1.z), cols = __float_as_int(r1.w);
  int dj = jj - (cols & 0xffff);
  dj += dj < 0 ? g.W : 0;
  const bool inside = i >= (rows & 0xffff) && i <= (rows >> 16) && dj <= (cols >> 16);
  const float dt = __fsub_rn(fi, r0.x);
  float dp = __fsub_rn(fj, r0.y);
  dp = dp >= g.halfW ? __fsub_rn(dp, g.Wf) : (dp < -g.halfW ? __fadd_rn(dp, g.Wf) : dp);
  const float t1 = __fmul_rn(r0.w, dp);
  const float t2 = __fmaf_rn(r0.z, dt, t1);
  const float t3 = __fmul_rn(r1.x, dp);
  const float t4 = __fmul_rn(t3, dp);
  const float q = __fmaf_rn(dt, t2, t4);
  const float x = __fmul_rn(-0.5f, q);
  const float G = x > -87.0f ? exp32_inrange(x) : 0.0f;
  return (inside && q <= g.q_max) ? G : -1.0f;
}

// The backward's weight: the same decision as pixel_G (footprint, q in the
// specification's operation order, q <= q_max, so the same entries count as
// composited) with the value exp(-q/2) from the hardware exponential
// (__expf: a few ulp, well inside the gradients' tolerance).  The forward
// keeps pixel_G, whose exact value decides the transmittance cut-off.
__device__ __forceinline__ float pixel_G_grad(const GridConst& g, const float4 r0,
                                              const float4 r1, int i, float fi, int jj,
                                              float fj) {
  const int rows = __float_as_int(r1.z), cols = __float_as_int(r1.w);
  int dj = jj - (cols & 0xffff);
  dj += dj < 0 ? g.W : 0;
  const bool inside = i >= (rows & 0xffff) && i <= (rows >> 16) && dj <= (cols >> 16);
  const float dt = __fsub_rn(fi, r0.x);
  float dp = __fsub_rn(fj, r0.y);
  dp = dp >= g.halfW ? __fsub_rn(dp, g.Wf) : (dp < -g.halfW ? __fadd_rn(dp, g.Wf) : dp);
  const float t1 = __fmul_rn(r0.w, dp);
  const float t2 = __fmaf_rn(r0.z, dt, t1);
  const float t3 = __fmul_rn(r1.x, dp);
  const float t4 = __fmul_rn(t3, dp);
  const float q = __fmaf_rn(dt, t2, t4);
  const float x = __fmul_rn(-0.5f, q);
  const float G = x > -87.0f ? __expf(x) : 0.0f;
  return (inside && q <= g.q_max) ? G : -1.0f;
}

// The pixels of warp `w` of a tile (threads 32w .. 32w+31, row-major over the
// TH x TW tile) lie in grid rows [r0, r1] and columns [c0, c1].
struct Strip {
  int r0, r1, c0, c1;
};

// Pixels p0 .. p0+np-1 of a tile (row-major over TH x TW; np is 16 or 32
// and divides or is a multiple of TW, which is 8, 16 or 32).
__device__ __forceinline__ Strip pixel_strip(const GridConst& g, int tr, int tc, int p0, int np) {
  Strip s;
  const int t1 = p0 + np - 1;
  s.r0 = tr * g.TH + p0 / g.TW;
  s.r1 = tr * g.TH + t1 / g.TW;
  if (g.TW >= np) {
    s.c0 = tc * g.TW + p0 % g.TW;
    s.c1 = s.c0 + np - 1;
  } else {
    s.c0 = tc * g.TW;
    s.c1 = s.c0 + g.TW - 1;
  }
  if (s.r1 > g.H - 1) s.r1 = g.H - 1;
  if (s.c1 > g.W - 1) s.c1 = g.W - 1;
  return s;
}

__device__ __forceinline__ Strip warp_strip(const GridConst& g, int tr, int tc, int w) {
  return pixel_strip(g, tr, tc, 32 * w, 32);
}

// Does a footprint (record word r1: rows i_lo..i_hi, columns j_lo..j_lo+span
// modulo W) meet the strip?  A superset test: every pixel of the strip that
// lies in the footprint makes it true.
__device__ __forceinline__ bool touches_strip(const GridConst& g, const float4 r1, const Strip& s) {
  if (s.r0 > s.r1 || s.c0 > s.c1) return false;
  const int rows = __float_as_int(r1.z), cols = __float_as_int(r1.w);
  const int i_lo = rows & 0xffff, i_hi = rows >> 16, j_lo = cols & 0xffff, span = cols >> 16;
  if (i_hi < s.r0 || i_lo > s.r1) return false;
  int a = s.c0 - j_lo;
  if (a < 0) a += g.W;
  if (a <= span) return true;
  int b = j_lo - s.c0;
  if (b < 0) b += g.W;
  return b <= s.c1 - s.c0;
}

}  // namespace rxgs
