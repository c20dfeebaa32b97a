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

}  // namespace rxgs
