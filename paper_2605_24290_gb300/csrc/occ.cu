// occ.cu -- occupancy grid and occlusion probes of the local conditioning
// branch (App. E.5): a res^3 density grid splatted once from the frozen
// Gaussians, probed along each (Gaussian, receiver) segment for the local
// MLP's inputs T_k = prod_s (1 - rho_s) and rho_bar_k = mean_s rho_s.
//
// Grid: over the bounding box [lo, hi] of the means, voxel size
// D = (hi - lo) / res per axis (1e-3 m for an axis of zero extent), voxel
// centre lo + (i + 0.5) D.  Gaussian k adds tau_k exp(-1/2 sum_a
// ((c_a - p_a) / s_a)^2) with s_a = sqrt(Sigma_aa) to every voxel centre
// within 2 s_a of p_a on every axis (float32 atomics; densities clamp to
// [0, 1] when probed).  Probes at t_s = float32(0.05 + 0.06 s), s = 0..15:
// x = p + t_s (r - p), voxel floor((x - lo) / D), density 0 outside.
// Voxel ranges and indices are decided in float32 with the operation order
// written here; the densities themselves are values, not decisions.
#include <cmath>

#include "rxgs_internal.h"

namespace rxgs {

constexpr int kOccProbes = 16;

struct OccProbeT {
  float t[kOccProbes];
};

// box[0..2] = lo, box[3..5] = D
__global__ void occ_bounds_kernel(const float4* __restrict__ geom, int K, int res,
                                  float* __restrict__ box) {
  __shared__ float smin[3][256], smax[3][256];
  const int t = threadIdx.x;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = t; k < K; k += blockDim.x) {
    const float4 p = geom[3 * k];
    mn[0] = fminf(mn[0], p.x);
    mn[1] = fminf(mn[1], p.y);
    mn[2] = fminf(mn[2], p.z);
    mx[0] = fmaxf(mx[0], p.x);
    mx[1] = fmaxf(mx[1], p.y);
    mx[2] = fmaxf(mx[2], p.z);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    smin[a][t] = mn[a];
    smax[a][t] = mx[a];
  }
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (t < o) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        smin[a][t] = fminf(smin[a][t], smin[a][t + o]);
        smax[a][t] = fmaxf(smax[a][t], smax[a][t + o]);
      }
    }
    __syncthreads();
  }
  if (t < 3) {
    const float lo = smin[t][0];
    float ext = __fsub_rn(smax[t][0], lo);
    if (!(ext > 0.0f)) ext = 1e-3f;
    box[t] = lo;
    box[3 + t] = __fdiv_rn(ext, static_cast<float>(res));
  }
}

// One warp per Gaussian: the lanes cover the voxels of its 2-sigma box.
__global__ void occ_splat_kernel(const float4* __restrict__ geom, int K, int res,
                                 const float* __restrict__ box, float* __restrict__ grid) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= K) return;
  const float4 p = geom[3 * warp], c1 = geom[3 * warp + 1], c2 = geom[3 * warp + 2];
  const float pos[3] = {p.x, p.y, p.z};
  const float sd[3] = {__fsqrt_rn(c1.x), __fsqrt_rn(c1.w), __fsqrt_rn(c2.y)};
  int lo_i[3], n_i[3];
  for (int a = 0; a < 3; ++a) {
    const float two = __fmul_rn(2.0f, sd[a]);
    const float alo = __fsub_rn(__fdiv_rn(__fsub_rn(__fsub_rn(pos[a], two), box[a]), box[3 + a]), 0.5f);
    const float ahi = __fsub_rn(__fdiv_rn(__fsub_rn(__fadd_rn(pos[a], two), box[a]), box[3 + a]), 0.5f);
    const int i0 = max(static_cast<int>(ceilf(alo)), 0);
    const int i1 = min(static_cast<int>(floorf(ahi)), res - 1);
    lo_i[a] = i0;
    n_i[a] = i1 - i0 + 1;
  }
  if (n_i[0] <= 0 || n_i[1] <= 0 || n_i[2] <= 0 || !(p.w > 0.0f)) return;
  const int total = n_i[0] * n_i[1] * n_i[2];
  for (int e = lane; e < total; e += 32) {
    const int iz = lo_i[2] + e % n_i[2], iy = lo_i[1] + (e / n_i[2]) % n_i[1],
              ix = lo_i[0] + e / (n_i[2] * n_i[1]);
    const int id[3] = {ix, iy, iz};
    float q = 0.0f;
    for (int a = 0; a < 3; ++a) {
      const float c = box[a] + (static_cast<float>(id[a]) + 0.5f) * box[3 + a];
      const float u = (c - pos[a]) / sd[a];
      q += u * u;
    }
    atomicAdd(&grid[(static_cast<size_t>(ix) * res + iy) * res + iz], p.w * expf(-0.5f * q));
  }
}

// feat[j][k] = (T, rho_bar) for every (receiver, Gaussian) pair.
__global__ void occ_probe_kernel(const float4* __restrict__ geom, int K,
                                 const float* __restrict__ rx, int N, int res,
                                 const float* __restrict__ box, const float* __restrict__ grid,
                                 OccProbeT tp, float2* __restrict__ feat) {
  const size_t pair = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (pair >= static_cast<size_t>(N) * K) return;
  const int j = static_cast<int>(pair / K), k = static_cast<int>(pair % K);
  const float4 p = geom[3 * k];
  const float pos[3] = {p.x, p.y, p.z};
  float dv[3];
  for (int a = 0; a < 3; ++a) dv[a] = __fsub_rn(rx[3 * j + a], pos[a]);
  float T = 1.0f, acc = 0.0f;
#pragma unroll
  for (int s = 0; s < kOccProbes; ++s) {
    int id[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float x = __fadd_rn(pos[a], __fmul_rn(tp.t[s], dv[a]));
      const float u = __fdiv_rn(__fsub_rn(x, box[a]), box[3 + a]);
      const float fl = floorf(u);
      inside = inside && fl >= 0.0f && fl < static_cast<float>(res);
      id[a] = inside ? static_cast<int>(fl) : 0;
    }
    const float rho =
        inside ? fminf(grid[(static_cast<size_t>(id[0]) * res + id[1]) * res + id[2]], 1.0f) : 0.0f;
    T *= 1.0f - rho;
    acc += rho;
  }
  feat[pair] = make_float2(T, acc * (1.0f / kOccProbes));
}

void launch_occ_build(const float4* geom, int K, int res, float* box, float* grid,
                      cudaStream_t s) {
  cudaMemsetAsync(grid, 0, sizeof(float) * static_cast<size_t>(res) * res * res, s);
  if (K <= 0) return;
  occ_bounds_kernel<<<1, 256, 0, s>>>(geom, K, res, box);
  note_launches(1);
  const size_t threads = static_cast<size_t>(K) * 32;
  occ_splat_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(geom, K, res, box,
                                                                               grid);
  note_launches(1);
}

void launch_occ_probes(const float4* geom, int K, const float* rx, int N, int res,
                       const float* box, const float* grid, float2* feat, cudaStream_t s) {
  const size_t pairs = static_cast<size_t>(N) * K;
  if (pairs == 0) return;
  OccProbeT tp;
  for (int i = 0; i < kOccProbes; ++i) tp.t[i] = static_cast<float>(0.05 + 0.06 * i);
  occ_probe_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, 0, s>>>(
      geom, K, rx, N, res, box, grid, tp, feat);
  note_launches(1);
}

}  // namespace rxgs
