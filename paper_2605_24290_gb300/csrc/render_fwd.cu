// render_fwd.cu -- multi-receiver front-to-back compositing (Algorithm 1,
// Stage 3) over a (tile, column block, view) grid, and its reduction to CSI /
// RSSI (Def. 2).  The per-tile work is render_tile (render_tile.cuh).
#include <cstdio>

#include "rxgs_internal.h"
#include "rxgs_math.cuh"
#include "render_common.cuh"
#include "render_tile.cuh"

namespace rxgs {

// 128-column blocks run with two threads per pixel (512 threads).
template <int NB>
constexpr int fwd_tpp() {
  return NB >= 128 ? 2 : 1;
}

template <int NB>
__global__ void __launch_bounds__(fwd_tpp<NB>() * kTilePixels, NB >= 128 ? 1 : 2)
    render_fwd_kernel(const RenderArgs a) {
  using S = FwdShape<NB, fwd_tpp<NB>()>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);              // [kChunk][256]
  float* sR = sA + kChunk * kTilePixels;                        // [kChunk][NB]
  float4* sRec = reinterpret_cast<float4*>(sR + 2 * kChunk * NB);  // [2][kChunk][2]
  __shared__ float sRed[S::kThreads / 32][8];
  TileJob job;
  job.v = blockIdx.z;
  job.tile = blockIdx.x;
  job.col0 = blockIdx.y * NB;
  job.col_base = 0;
  job.ncols_v = a.ncols;
  job.out_rx0 = job.v * a.N;
  job.partial_row =
      a.partial ? a.partial + (static_cast<size_t>(job.v) * a.g.T + job.tile) * a.ncols : nullptr;
  render_tile<NB, fwd_tpp<NB>()>(a, job, sA, sR, sRec, sRed);
}

template <int NB>
static void launch_fwd_nb(const RenderArgs& a, cudaStream_t s) {
  using S = FwdShape<NB, fwd_tpp<NB>()>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(render_fwd_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(S::smem));
    configured = true;
  }
  dim3 grid(a.g.T, (a.ncols + NB - 1) / NB, a.M);
  render_fwd_kernel<NB><<<grid, S::kThreads, S::smem, s>>>(a);
  note_launches(1);
}

void launch_render_fwd_tc(const RenderArgs& a, cudaStream_t s);  // render_fwd_tc.cu

// Blocks of 16-64 columns composite on the CUDA cores; blocks of 128 columns
// run their chunk products on the tensor cores (render_fwd_tc.cu).
void launch_render_fwd(const RenderArgs& a, int cols_per_cta, cudaStream_t s) {
  if (a.M <= 0 || a.ncols <= 0) return;
  switch (cols_per_cta) {
    case 16: launch_fwd_nb<16>(a, s); break;
    case 32: launch_fwd_nb<32>(a, s); break;
    case 128: launch_render_fwd_tc(a, s); break;
    default: launch_fwd_nb<64>(a, s); break;
  }
}

// csi[v][j][c][2] = sum over tiles of partial[v][t][col] (fixed order);
// rssi[v][j] = |csi[v][j][0]| when C == 1.
__global__ void reduce_tiles_kernel(const float* __restrict__ partial, int M, int T, int ncols,
                                    int C, float* __restrict__ csi, float* __restrict__ rssi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // (v, j, c) complex entry
  const int ncplx = ncols / 2;
  if (idx >= M * ncplx) return;
  const int v = idx / ncplx, cc = idx % ncplx;
  const float* p = partial + static_cast<size_t>(v) * T * ncols + 2 * cc;
  float re = 0.0f, im = 0.0f;
  for (int t = 0; t < T; ++t) {
    re += p[static_cast<size_t>(t) * ncols];
    im += p[static_cast<size_t>(t) * ncols + 1];
  }
  if (csi) {
    csi[2 * static_cast<size_t>(idx)] = re;
    csi[2 * static_cast<size_t>(idx) + 1] = im;
  }
  if (rssi && C == 1) rssi[idx] = sqrtf(re * re + im * im);
}

void launch_reduce_tiles(const float* partial, int M, int T, int N, int C, float* csi,
                         float* rssi, cudaStream_t s) {
  const int n = M * N * C;
  if (n <= 0) return;
  reduce_tiles_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, M, T, 2 * N * C, C, csi, rssi);
  note_launches(1);
}

}  // namespace rxgs
