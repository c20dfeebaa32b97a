// rxgs_math.cuh -- float32 arithmetic that takes the renderer's discrete
// decisions (culling, footprint, tile set, depth order, q <= q_max, T < eps).
//
// Every operation here is an explicitly rounded IEEE binary32 intrinsic
// (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn) so the compiler
// cannot contract or reorder it; the order of operations is the decision
// specification of the library, and a CPU program that follows the same
// order reproduces every decision bit for bit.
//
// exp and atan2 are written from their textbook definitions instead of
// calling expf/atan2f, whose float results are implementation-specific:
//   exp   Cody & Waite (1980) reduction x = n ln2 + r with ln 2 split into
//         two floats, Taylor polynomial of e^r to degree 7, exact 2^n scale.
//   atan2 reduction to t = min/max in [0,1], then t > tan(pi/8) mapped by
//         atan t = pi/4 + atan((t-1)/(t+1)), Gregory series to t^19, then
//         the octant is restored.
#pragma once
#include <cstdint>

namespace rxgs {

// Correctly rounded binary32 values of mathematical constants.
constexpr float kLog2e = 0x1.715476p+0f;    // 1/ln 2
constexpr float kLn2Hi = 0x1.62e430p-1f;    // ln 2
constexpr float kLn2Lo = -0x1.05c610p-29f;  // ln 2 - kLn2Hi
constexpr float kPi = 0x1.921fb6p+1f;
constexpr float kPi2 = 0x1.921fb6p+0f;
constexpr float kPi4 = 0x1.921fb6p-1f;
constexpr float kTwoPi = 0x1.921fb6p+2f;
constexpr float kTanPi8 = 0x1.a8279ap-2f;

__device__ __forceinline__ float exp32(float x) {
  if (!(x > -87.0f)) return 0.0f;
  if (x > 88.0f) return __int_as_float(0x7f800000);
  const float t = __fmul_rn(x, kLog2e);
  const float n = rintf(t);
  float r = __fmaf_rn(-n, kLn2Hi, x);
  r = __fmaf_rn(-n, kLn2Lo, r);
  float p = 1.0f / 5040.0f;
  p = __fmaf_rn(p, r, 1.0f / 720.0f);
  p = __fmaf_rn(p, r, 1.0f / 120.0f);
  p = __fmaf_rn(p, r, 1.0f / 24.0f);
  p = __fmaf_rn(p, r, 1.0f / 6.0f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const float s = __int_as_float((static_cast<int>(n) + 127) << 23);
  return __fmul_rn(p, s);
}

// exp32 without its range checks, for -87 < x <= 88 (the compositing weight
// exp(-q/2) with q in [0, q_max]): the same operations, so the same result
// bits there; outside that range the value is meaningless and callers
// discard it.
__device__ __forceinline__ float exp32_inrange(float x) {
  const float t = __fmul_rn(x, kLog2e);
  const float n = rintf(t);
  float r = __fmaf_rn(-n, kLn2Hi, x);
  r = __fmaf_rn(-n, kLn2Lo, r);
  float p = 1.0f / 5040.0f;
  p = __fmaf_rn(p, r, 1.0f / 720.0f);
  p = __fmaf_rn(p, r, 1.0f / 120.0f);
  p = __fmaf_rn(p, r, 1.0f / 24.0f);
  p = __fmaf_rn(p, r, 1.0f / 6.0f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  const float s = __int_as_float((static_cast<int>(n) + 127) << 23);
  return __fmul_rn(p, s);
}

__device__ __forceinline__ float atan2_32(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = ax > ay ? ax : ay;
  const float mn = ax > ay ? ay : ax;
  if (mx == 0.0f) return 0.0f;
  float t = __fdiv_rn(mn, mx);
  float base = 0.0f;
  if (t > kTanPi8) {
    t = __fdiv_rn(__fsub_rn(t, 1.0f), __fadd_rn(t, 1.0f));
    base = kPi4;
  }
  const float z = __fmul_rn(t, t);
  float p = -1.0f / 19.0f;
  p = __fmaf_rn(p, z, 1.0f / 17.0f);
  p = __fmaf_rn(p, z, -1.0f / 15.0f);
  p = __fmaf_rn(p, z, 1.0f / 13.0f);
  p = __fmaf_rn(p, z, -1.0f / 11.0f);
  p = __fmaf_rn(p, z, 1.0f / 9.0f);
  p = __fmaf_rn(p, z, -1.0f / 7.0f);
  p = __fmaf_rn(p, z, 1.0f / 5.0f);
  p = __fmaf_rn(p, z, -1.0f / 3.0f);
  p = __fmaf_rn(p, z, 1.0f);
  float a = __fmaf_rn(t, p, base);
  if (ay > ax) a = __fsub_rn(kPi2, a);
  if (x < 0.0f) a = __fsub_rn(kPi, a);
  if (y < 0.0f) a = -a;
  return a;
}

}  // namespace rxgs
