// geom.cu -- transmitter-side kernels: scene upload (covariance), projection
// onto the angular grid, tile counting and key emission, tile ranges.
// (Algorithm 1, Stage 1; App. E.1; App. D "Transmitter-Side Preprocessing")
#include "rxgs_internal.h"
#include "rxgs_math.cuh"

namespace rxgs {

// ------------------------------------------------------------------ upload
// Sigma = R S S^T R^T, R from the normalised quaternion (w,x,y,z),
// S = diag(exp(s))  (App. E.1).  Operation order is part of the decision
// specification (Sigma feeds the footprint).
__global__ void scene_upload_kernel(const float* __restrict__ means,
                                    const float* __restrict__ log_scales,
                                    const float* __restrict__ quats,
                                    const float* __restrict__ opacity, int K,
                                    float4* __restrict__ geom) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const float q0 = quats[4 * k + 0], q1 = quats[4 * k + 1], q2 = quats[4 * k + 2],
              q3 = quats[4 * k + 3];
  const float n2 = __fmaf_rn(q0, q0, __fmaf_rn(q1, q1, __fmaf_rn(q2, q2, __fmul_rn(q3, q3))));
  float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
  if (n2 > 0.0f) {
    const float nr = __fsqrt_rn(n2);
    w = __fdiv_rn(q0, nr);
    x = __fdiv_rn(q1, nr);
    y = __fdiv_rn(q2, nr);
    z = __fdiv_rn(q3, nr);
  }
  const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  float R[3][3];
  R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
  const float sg[3] = {exp32(log_scales[3 * k + 0]), exp32(log_scales[3 * k + 1]),
                       exp32(log_scales[3 * k + 2])};
  float M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = __fmul_rn(R[a][b], sg[b]);
  auto dot3 = [&](int a, int b) {
    return __fmaf_rn(M[a][2], M[b][2], __fmaf_rn(M[a][1], M[b][1], __fmul_rn(M[a][0], M[b][0])));
  };
  geom[3 * k + 0] = make_float4(means[3 * k + 0], means[3 * k + 1], means[3 * k + 2], opacity[k]);
  geom[3 * k + 1] = make_float4(dot3(0, 0), dot3(0, 1), dot3(0, 2), dot3(1, 1));
  geom[3 * k + 2] = make_float4(dot3(1, 2), dot3(2, 2), 0.0f, 0.0f);
}

void launch_scene_upload(const float* means, const float* log_scales, const float* quats,
                         const float* opacity, int K, float4* geom, cudaStream_t s) {
  if (K <= 0) return;
  scene_upload_kernel<<<(K + 255) / 256, 256, 0, s>>>(means, log_scales, quats, opacity, K, geom);
  note_launches(1);
}

__global__ void set_opacity_kernel(const float* __restrict__ opacity, int K, float4* geom) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) geom[3 * k].w = opacity[k];
}

void launch_set_opacity(const float* opacity, int K, float4* geom, cudaStream_t s) {
  if (K <= 0) return;
  set_opacity_kernel<<<(K + 255) / 256, 256, 0, s>>>(opacity, K, geom);
  note_launches(1);
}

// -------------------------------------------------------------- projection
// Footprint of Gaussian k in view v (transmitter c):
//   u = p - c, rho = |u|, h = |u_xy|; culled if rho < r_near or h <= 1e-6 rho;
//   (theta, phi) in pixel units; Sigma2D = J Sigma J^T with J the Jacobian
//   of (elevation, azimuth) in pixel units; conic = Sigma2D^-1;
//   rows [ceil(theta - ksig sqrt(a)), floor(theta + ksig sqrt(a))] clipped to
//   the grid; columns [ceil(phi - ksig sqrt(c)), floor(phi + ksig sqrt(c))]
//   modulo W (all columns when that span reaches W); culled when either
//   range holds no pixel.
// Record: {theta_px, phi_px, conic_a, 2 conic_b}, {conic_c, tau, rows, cols}
// with rows = i_lo | i_hi << 16 and cols = j_lo | span << 16.
struct Footprint {
  bool vis;
  float theta_px, phi_px, ca, cb2, cc, rho;
  int i_lo, i_hi, j_lo, span;
};

__device__ __forceinline__ Footprint project_one(const GridConst& g, const float4 g0,
                                                 const float4 g1, const float4 g2, float cx,
                                                 float cy, float cz) {
  Footprint o;
  o.vis = false;
  const float ux = __fsub_rn(g0.x, cx), uy = __fsub_rn(g0.y, cy), uz = __fsub_rn(g0.z, cz);
  const float hh = __fmaf_rn(uy, uy, __fmul_rn(ux, ux));
  const float rr = __fmaf_rn(uz, uz, hh);
  const float rho = __fsqrt_rn(rr), h = __fsqrt_rn(hh);
  o.rho = rho;
  if (!(rho >= g.r_near) || !(h > __fmul_rn(1e-6f, rho))) return o;
  float phi = atan2_32(uy, ux);
  if (phi < 0.0f) phi = __fadd_rn(phi, kTwoPi);
  float phi_px = __fmul_rn(phi, g.inv_step);
  if (phi_px >= g.Wf) phi_px = __fsub_rn(phi_px, g.Wf);
  const float th = atan2_32(uz, h);
  const float theta_px = __fsub_rn(__fmul_rn(th, g.inv_step), g.theta0_px);
  const float gt = __fdiv_rn(g.inv_step, __fmul_rn(rr, h));
  const float gp = __fdiv_rn(g.inv_step, hh);
  const float J00 = __fmul_rn(-__fmul_rn(ux, uz), gt), J01 = __fmul_rn(-__fmul_rn(uy, uz), gt),
              J02 = __fmul_rn(hh, gt);
  const float J10 = __fmul_rn(-uy, gp), J11 = __fmul_rn(ux, gp);
  const float S00 = g1.x, S01 = g1.y, S02 = g1.z, S11 = g1.w, S12 = g2.x, S22 = g2.y;
  const float t0x = __fmaf_rn(S02, J02, __fmaf_rn(S01, J01, __fmul_rn(S00, J00)));
  const float t0y = __fmaf_rn(S12, J02, __fmaf_rn(S11, J01, __fmul_rn(S01, J00)));
  const float t0z = __fmaf_rn(S22, J02, __fmaf_rn(S12, J01, __fmul_rn(S02, J00)));
  const float t1x = __fmaf_rn(S01, J11, __fmul_rn(S00, J10));
  const float t1y = __fmaf_rn(S11, J11, __fmul_rn(S01, J10));
  const float a = __fmaf_rn(J02, t0z, __fmaf_rn(J01, t0y, __fmul_rn(J00, t0x)));
  const float b = __fmaf_rn(J11, t0y, __fmul_rn(J10, t0x));
  const float c = __fmaf_rn(J11, t1y, __fmul_rn(J10, t1x));
  const float det = __fmaf_rn(a, c, -__fmul_rn(b, b));
  if (!(a > 0.0f) || !(c > 0.0f) || !(det > 0.0f)) return o;
  const float et = __fmul_rn(g.ksig, __fsqrt_rn(a)), ep = __fmul_rn(g.ksig, __fsqrt_rn(c));
  float lo = ceilf(__fsub_rn(theta_px, et)), hi = floorf(__fadd_rn(theta_px, et));
  if (lo < 0.0f) lo = 0.0f;
  if (hi > g.Hm1f) hi = g.Hm1f;
  if (!(lo <= hi)) return o;
  const float clo = ceilf(__fsub_rn(phi_px, ep)), chi = floorf(__fadd_rn(phi_px, ep));
  if (!(clo <= chi)) return o;  // no column centre inside the footprint
  if (__fsub_rn(chi, clo) >= __fsub_rn(g.Wf, 1.0f)) {
    o.j_lo = 0;
    o.span = g.W - 1;
  } else {
    const int jl = static_cast<int>(clo), jh = static_cast<int>(chi);
    o.span = jh - jl;
    o.j_lo = jl < 0 ? jl + g.W : (jl >= g.W ? jl - g.W : jl);  // into [0, W)
  }
  o.vis = true;
  o.theta_px = theta_px;
  o.phi_px = phi_px;
  o.ca = __fdiv_rn(c, det);
  o.cb2 = __fmul_rn(2.0f, __fdiv_rn(-b, det));
  o.cc = __fdiv_rn(a, det);
  o.i_lo = static_cast<int>(lo);
  o.i_hi = static_cast<int>(hi);
  return o;
}

// Tile columns touched by columns j_lo .. j_lo+span (mod W): up to two
// intervals [c0a, c0b] and [c1a, c1b] of tile columns (c1a > c1b = empty).
struct TileCols {
  int c0a, c0b, c1a, c1b;
};

__device__ __forceinline__ TileCols tile_cols(const GridConst& g, int j_lo, int span) {
  TileCols t;
  t.c1a = 1;
  t.c1b = 0;
  if (span >= g.W - 1) {
    t.c0a = 0;
    t.c0b = g.tiles_w - 1;
    return t;
  }
  const int j_hi = j_lo + span;
  if (j_hi < g.W) {
    t.c0a = j_lo / g.TW;
    t.c0b = j_hi / g.TW;
    return t;
  }
  t.c0a = j_lo / g.TW;
  t.c0b = g.tiles_w - 1;
  t.c1a = 0;
  t.c1b = (j_hi - g.W) / g.TW;
  if (t.c1b >= t.c0a) {  // the two pieces meet in tile space: all columns
    t.c0a = 0;
    t.c0b = g.tiles_w - 1;
    t.c1a = 1;
    t.c1b = 0;
  }
  return t;
}

// One (view, Gaussian) pair of the projection; returns its tile count and
// its depth key.
__device__ __forceinline__ uint32_t preprocess_one(GridConst g, const float4* __restrict__ geom,
                                                   int K, const float* __restrict__ tx,
                                                   float4* __restrict__ rec,
                                                   uint32_t* __restrict__ depth,
                                                   uint32_t* __restrict__ count,
                                                   const int* __restrict__ nviews_dev, int k,
                                                   int v, uint32_t& dkey) {
  const float4 g0 = geom[3 * k + 0], g1 = geom[3 * k + 1], g2 = geom[3 * k + 2];
  Footprint f;
  if (nviews_dev && v >= *nviews_dev) {
    f.vis = false;  // view slot unused in this batch
    f.rho = 0.0f;
  } else {
    f = project_one(g, g0, g1, g2, tx[3 * v + 0], tx[3 * v + 1], tx[3 * v + 2]);
  }
  const size_t idx = static_cast<size_t>(v) * K + k;
  uint32_t n = 0;
  if (f.vis) {
    const int rows = f.i_hi / g.TH - f.i_lo / g.TH + 1;
    const TileCols tc = tile_cols(g, f.j_lo, f.span);
    const int cols = (tc.c0b - tc.c0a + 1) + (tc.c1b >= tc.c1a ? tc.c1b - tc.c1a + 1 : 0);
    n = static_cast<uint32_t>(rows * cols);
    rec[2 * idx + 0] = make_float4(f.theta_px, f.phi_px, f.ca, f.cb2);
    rec[2 * idx + 1] = make_float4(f.cc, g0.w, __int_as_float(f.i_lo | (f.i_hi << 16)),
                                   __int_as_float(f.j_lo | (f.span << 16)));
  } else {
    rec[2 * idx + 0] = make_float4(0.f, 0.f, 0.f, 0.f);
    rec[2 * idx + 1] = make_float4(0.f, 0.f, __int_as_float(1), __int_as_float(0));  // empty rows
  }
  dkey = __float_as_uint(f.rho);
  depth[idx] = dkey;
  count[idx] = n;
  return n;
}

// stats (optional, [M][4] zeroed before the launch), per view: [0..1] the
// total tile count (uint64), [2] the largest ~depth key and [3] the largest
// depth key of the visible pairs (their smallest key is ~stats[2]); one
// atomic per block and quantity, into the view's own slot.
__global__ void preprocess_kernel(GridConst g, const float4* __restrict__ geom, int K,
                                  const float* __restrict__ tx, float4* __restrict__ rec,
                                  uint32_t* __restrict__ depth, uint32_t* __restrict__ count,
                                  const int* __restrict__ nviews_dev, uint32_t* __restrict__ stats) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  uint32_t n = 0, dkey = 0;
  if (k < K) {
    n = preprocess_one(g, geom, K, tx, rec, depth, count, nviews_dev, k, v, dkey);
  }
  if (stats) {
    // all lanes reach this point: warp reductions, then the block's
    __shared__ uint32_t red[3][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t tot = __reduce_add_sync(0xffffffffu, n);
    uint32_t nmin = __reduce_max_sync(0xffffffffu, n ? ~dkey : 0u);
    uint32_t dmax = __reduce_max_sync(0xffffffffu, n ? dkey : 0u);
    if (lane == 0) {
      red[0][w] = tot;
      red[1][w] = nmin;
      red[2][w] = dmax;
    }
    __syncthreads();
    if (w == 0) {
      const bool in = lane < static_cast<int>(blockDim.x >> 5);
      tot = __reduce_add_sync(0xffffffffu, in ? red[0][lane] : 0u);
      nmin = __reduce_max_sync(0xffffffffu, in ? red[1][lane] : 0u);
      dmax = __reduce_max_sync(0xffffffffu, in ? red[2][lane] : 0u);
      if (lane == 0 && tot) {
        uint32_t* st = stats + 4 * static_cast<size_t>(v);
        atomicAdd(reinterpret_cast<unsigned long long*>(st), static_cast<unsigned long long>(tot));
        atomicMax(&st[2], nmin);
        atomicMax(&st[3], dmax);
      }
    }
  }
}

// The per-view stats [M][4] of preprocess_kernel combined into dst[4] (one
// block; dst may be mapped pinned host memory).
__global__ void combine_stats_kernel(const uint32_t* __restrict__ stats, int M,
                                     uint32_t* __restrict__ dst) {
  __shared__ unsigned long long s_tot[256];
  __shared__ uint32_t s_min[256], s_max[256];
  unsigned long long tot = 0;
  uint32_t nmin = 0, dmax = 0;
  for (int v = threadIdx.x; v < M; v += blockDim.x) {
    const uint32_t* st = stats + 4 * static_cast<size_t>(v);
    tot += static_cast<unsigned long long>(st[0]) | (static_cast<unsigned long long>(st[1]) << 32);
    nmin = max(nmin, st[2]);
    dmax = max(dmax, st[3]);
  }
  s_tot[threadIdx.x] = tot;
  s_min[threadIdx.x] = nmin;
  s_max[threadIdx.x] = dmax;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (static_cast<int>(threadIdx.x) < h) {
      s_tot[threadIdx.x] += s_tot[threadIdx.x + h];
      s_min[threadIdx.x] = max(s_min[threadIdx.x], s_min[threadIdx.x + h]);
      s_max[threadIdx.x] = max(s_max[threadIdx.x], s_max[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dst[0] = static_cast<uint32_t>(s_tot[0]);
    dst[1] = static_cast<uint32_t>(s_tot[0] >> 32);
    dst[2] = s_min[0];
    dst[3] = s_max[0];
  }
}

void launch_combine_stats(const uint32_t* stats, int M, uint32_t* dst, cudaStream_t s) {
  combine_stats_kernel<<<1, 256, 0, s>>>(stats, M, dst);
  note_launches(1);
}

void launch_preprocess(const GridConst& g, const float4* geom, int K, const float* tx, int M,
                       float4* rec, uint32_t* depth, uint32_t* count, cudaStream_t s,
                       const int* nviews_dev, uint32_t* stats) {
  if (K <= 0 || M <= 0) return;
  dim3 grid((K + 255) / 256, M);
  preprocess_kernel<<<grid, 256, 0, s>>>(g, geom, K, tx, rec, depth, count, nviews_dev, stats);
  note_launches(1);
}

// ---------------------------------------------- instances in depth order
// The per-tile lists (Algorithm 1, Stage 1) in two sorts instead of one over
// 64-bit (view | tile | depth) instance keys: every view's Gaussians by
// depth (a segmented sort of the depth keys, one segment per view, values
// the view-major pair index; the stable sort keeps equal depths in
// ascending Gaussian index), then the instances, emitted in that order, by
// (view, tile) with 32-bit keys (the stable sort keeps each tile's
// instances in depth order).  The result is the order of the single sort:
// by (view, tile, depth, Gaussian index).
__global__ void gather_words_kernel(const uint32_t* __restrict__ src,
                                    const uint32_t* __restrict__ idx, size_t n,
                                    uint32_t* __restrict__ dst) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

void launch_gather_words(const uint32_t* src, const uint32_t* idx, size_t n, uint32_t* dst,
                         cudaStream_t s) {
  if (n == 0) return;
  gather_words_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(src, idx, n, dst);
  note_launches(1);
}

// Instances of the depth-ordered pairs: pair i (view-major index ord[i])
// writes its tiles at offsets[i] .. offsets[i + 1] - 1 with key
// view << tile_bits | tile and value the Gaussian index.  A warp takes 32
// consecutive pairs; their instances form one contiguous range, lane l
// writes positions start + l, start + l + 32, ... (coalesced), the owner
// found by binary search over the warp's offsets as in emit_kernel.
__global__ void __launch_bounds__(256) emit_sorted_kernel(
    GridConst g, const float4* __restrict__ rec, const uint32_t* __restrict__ ord,
    const uint32_t* __restrict__ offsets, size_t MK, int K, int tile_bits,
    uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t cap,
    unsigned* __restrict__ err) {
  __shared__ uint32_t sO[8][33];  // per warp: first position of each lane's pair, end
  __shared__ int4 sD[8][32];      // (tr0, ncols, n0 | c0a << 16, c1a)
  __shared__ uint2 sB[8][32];     // (view << tile_bits, Gaussian index)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint32_t o, end;
  int4 d = make_int4(0, 1, 0, 0);
  uint2 b = make_uint2(0u, 0u);
  if (i < MK) {
    o = offsets[i];
    end = offsets[i + 1];
    if (end > cap && err) atomicOr(err, kErrCapacity);  // nothing past cap is written
    if (end > o) {
      const uint32_t idx = ord[i];
      const uint32_t m = idx / static_cast<uint32_t>(K);
      const float4 r1 = rec[2 * static_cast<size_t>(idx) + 1];
      const int rows = __float_as_int(r1.z), cols = __float_as_int(r1.w);
      const int i_lo = rows & 0xffff, j_lo = cols & 0xffff, span = cols >> 16;
      const TileCols tc = tile_cols(g, j_lo, span);
      const int n0 = tc.c0b - tc.c0a + 1, n1 = tc.c1b >= tc.c1a ? tc.c1b - tc.c1a + 1 : 0;
      d = make_int4(i_lo / g.TH, n0 + n1, n0 | (tc.c0a << 16), tc.c1a);
      b = make_uint2(m << tile_bits, idx - m * static_cast<uint32_t>(K));
    }
  } else {
    o = end = offsets[MK];  // past the last pair
  }
  sO[w][lane] = o;
  if (lane == 31) sO[w][32] = end;
  sD[w][lane] = d;
  sB[w][lane] = b;
  __syncwarp();
  const uint32_t start = sO[w][0], stop = min(sO[w][32], cap);
  for (uint32_t q = start + lane; q < stop; q += 32) {
    // the owner: the last lane whose first position is <= q (a lane with
    // no instances shares its first position with the next lane)
    int lo = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
      if (sO[w][lo + step] <= q) lo += step;
    const int4 dd = sD[w][lo];
    const uint2 bb = sB[w][lo];
    const int j = static_cast<int>(q - sO[w][lo]);
    const int row = j / dd.y, ci = j - row * dd.y;
    const int n0 = dd.z & 0xffff;
    const int c = ci < n0 ? (dd.z >> 16) + ci : dd.w + (ci - n0);
    keys[q] = bb.x | static_cast<uint32_t>((dd.x + row) * g.tiles_w + c);
    vals[q] = bb.y;
  }
}

void launch_emit_sorted(const GridConst& g, const float4* rec, const uint32_t* ord,
                        const uint32_t* offsets, size_t MK, int K, int tile_bits, uint32_t* keys,
                        uint32_t* vals, cudaStream_t s, uint32_t cap, unsigned* err) {
  if (MK == 0) return;
  emit_sorted_kernel<<<static_cast<unsigned>((MK + 255) / 256), 256, 0, s>>>(
      g, rec, ord, offsets, MK, K, tile_bits, keys, vals, cap, err);
  note_launches(1);
}

// (view | tile) keys and Gaussian indices -> (view | tile | depth) keys
__global__ void expand_keys_kernel(const uint32_t* __restrict__ vt, const uint32_t* __restrict__ vals,
                                   size_t n, const uint32_t* __restrict__ depth, int K,
                                   int tile_bits, uint64_t* __restrict__ out) {
  const size_t q = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint32_t key = vt[q];
  const size_t m = key >> tile_bits;
  out[q] = (static_cast<uint64_t>(key) << 31) | depth[m * K + vals[q]];
}

void launch_expand_keys(const uint32_t* vt, const uint32_t* vals, size_t n, const uint32_t* depth,
                        int K, int tile_bits, uint64_t* out, cudaStream_t s) {
  if (n == 0) return;
  expand_keys_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(vt, vals, n, depth, K,
                                                                            tile_bits, out);
  note_launches(1);
}

// ------------------------------------------------------------ small copies
// n 32-bit words from src to dst by the SMs (device memory, or pinned host
// memory mapped into the device's address space): small transfers that
// must not wait behind large copies queued on the copy engines.
__global__ void copy_words_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                  size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

void launch_copy_words(const uint32_t* src, uint32_t* dst, size_t n, cudaStream_t s) {
  if (n == 0) return;
  const size_t blocks = std::min<size_t>((n + 255) / 256, 64);
  copy_words_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(src, dst, n);
  note_launches(1);
}

// -------------------------------------------------------------- tile ranges
// Keys (view | tile): 32 bits (64-bit keys would carry the depth in their
// low 31 bits).
template <typename Key>
__global__ void tile_ranges_kernel(const Key* __restrict__ keys, size_t n, int tile_bits,
                                   int T, uint2* __restrict__ ranges,
                                   const uint32_t* __restrict__ n_dev) {
  if (n_dev && *n_dev < n) n = *n_dev;
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto slot = [&](Key key) {
    const uint64_t vt = sizeof(Key) == 8 ? static_cast<uint64_t>(key) >> 31 : key;
    const uint64_t v = vt >> tile_bits, t = vt & ((1ull << tile_bits) - 1);
    return v * T + t;
  };
  const uint64_t cur = slot(keys[i]);
  if (i == 0 || slot(keys[i - 1]) != cur) ranges[cur].x = static_cast<unsigned>(i);
  if (i + 1 == n || slot(keys[i + 1]) != cur) ranges[cur].y = static_cast<unsigned>(i + 1);
}

template <typename Key>
static void tile_ranges(const Key* keys, size_t n, int tile_bits, int T, uint2* ranges, int M,
                        cudaStream_t s, const uint32_t* n_dev) {
  cudaMemsetAsync(ranges, 0, sizeof(uint2) * static_cast<size_t>(M) * T, s);
  if (n == 0) return;
  tile_ranges_kernel<Key><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
      keys, n, tile_bits, T, ranges, n_dev);
  note_launches(1);
}

void launch_tile_ranges(const uint32_t* keys, size_t n, int tile_bits, int T, uint2* ranges,
                        int M, cudaStream_t s, const uint32_t* n_dev) {
  tile_ranges<uint32_t>(keys, n, tile_bits, T, ranges, M, s, n_dev);
}

// -------------------------------------------------------------------- scan
// Three-phase exclusive scan: per-block sums, a one-block scan of the sums,
// then per-block scans with the block offsets.  2048 items per block.
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = w;
  }
  __syncthreads();
  const uint32_t before = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, size_t n,
                                   uint32_t* __restrict__ sums) {
  const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile;
  uint32_t s = 0;
  for (int e = 0; e < kScanItems; ++e) {
    const size_t i = base + static_cast<size_t>(e) * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(uint32_t* sums, int nb) {
  // one block; nb may exceed the block's items, loop in tiles
  uint32_t carry = 0;
  for (int base = 0; base < nb; base += kScanThreads) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nb ? sums[i] : 0;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_apply_kernel(const uint32_t* __restrict__ in, size_t n,
                                  const uint32_t* __restrict__ sums, uint32_t* __restrict__ out) {
  const size_t base = static_cast<size_t>(blockIdx.x) * kScanTile;
  // blocked arrangement: thread t owns items base + t*8 .. +7
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int e = 0; e < kScanItems; ++e) {
    const size_t i = base + static_cast<size_t>(threadIdx.x) * kScanItems + e;
    v[e] = i < n ? in[i] : 0;
    s += v[e];
  }
  uint32_t total;
  uint32_t ex = block_exclusive_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int e = 0; e < kScanItems; ++e) {
    const size_t i = base + static_cast<size_t>(threadIdx.x) * kScanItems + e;
    if (i < n) out[i] = ex;
    ex += v[e];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

size_t scan_tmp_words(size_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

void launch_exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp,
                           cudaStream_t s) {
  if (n == 0) {
    cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    return;
  }
  const int nb = static_cast<int>((n + kScanTile - 1) / kScanTile);
  scan_reduce_kernel<<<nb, kScanThreads, 0, s>>>(in, n, tmp);
  note_launches(1);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(tmp, nb);
  note_launches(1);
  scan_apply_kernel<<<nb, kScanThreads, 0, s>>>(in, n, tmp, out);
  note_launches(1);
}

// ---------------------------------------------------------------- radiance
__global__ void radiance_transpose_kernel(const float* __restrict__ rad, int N, int K, int C,
                                          int stride, float* __restrict__ out) {
  // out[k][j*2C + e] = rad[j][k][e], e < 2C; zero pad columns
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t total = static_cast<size_t>(K) * stride;
  if (idx >= total) return;
  const int k = static_cast<int>(idx / stride);
  const int col = static_cast<int>(idx % stride);
  const int twoC = 2 * C;
  float v = 0.0f;
  if (col < N * twoC) {
    const int j = col / twoC, e = col % twoC;
    v = rad[(static_cast<size_t>(j) * K + k) * twoC + e];
  }
  out[idx] = v;
}

void launch_radiance_transpose(const float* rad, int N, int K, int C, int stride, float* out,
                               cudaStream_t s) {
  const size_t total = static_cast<size_t>(K) * stride;
  if (total == 0) return;
  radiance_transpose_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      rad, N, K, C, stride, out);
  note_launches(1);
}

__global__ void radiance_untranspose_add_kernel(const float* __restrict__ in, int N, int K,
                                                int C, int stride, float* __restrict__ out) {
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int twoC = 2 * C;
  const size_t total = static_cast<size_t>(N) * K * twoC;
  if (idx >= total) return;
  const int e = static_cast<int>(idx % twoC);
  const size_t jk = idx / twoC;
  const int k = static_cast<int>(jk % K);
  const int j = static_cast<int>(jk / K);
  out[idx] += in[static_cast<size_t>(k) * stride + j * twoC + e];
}

void launch_radiance_untranspose_add(const float* in, int N, int K, int C, int stride,
                                     float* out, cudaStream_t s) {
  const size_t total = static_cast<size_t>(N) * K * 2 * C;
  if (total == 0) return;
  radiance_untranspose_add_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
      in, N, K, C, stride, out);
  note_launches(1);
}

}  // namespace rxgs
