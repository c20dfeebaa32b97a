// noalloc.cu -- rxgs_render_csi_noalloc: CSI / RSSI of prepared views without
// any device allocation.
//
// Who needs it: callers that must not allocate device memory while they
// render -- a serving thread running under a hard latency budget (an
// allocation can block on the driver or on the memory pool's locks), a host
// program whose device memory is entirely owned by another allocator or
// budgeted up front, or code running where the CUDA allocator must not be
// touched.  The regular rxgs_render_views takes its per-tile partial sums
// and its Gaussian-major radiance copy from CUDA's stream-ordered pool; this
// variant reads the caller's receiver-major radiance in place and keeps the
// per-tile partial sums in one fixed, file-scope device array instead.
//
// The array holds kNoAllocFloats floats (16 MiB).  Its device address is
// looked up when a context is created on a device (rxgs_create calls
// noalloc_scratch_address with that device current); that lookup also loads
// the module that holds the array, so from the first rxgs_create on a device
// the array occupies 16 MiB there until the process exits.  Every call
// shares it: the kernel writes every entry it later reads, so no clearing is
// needed, but two calls whose work overlaps on the same GPU (for example on
// two streams) race on it and give wrong results.
#include <cstdio>
#include <mutex>

#include "rxgs.h"
#include "ctx_internal.h"
#include "render_common.cuh"
#include "rxgs_internal.h"

namespace rxgs {

constexpr size_t kNoAllocFloats = size_t(1) << 22;  // 16 MiB of per-tile partial sums
constexpr int kNoAllocCols = 64;                    // output columns per CTA

static __device__ __align__(256) float g_noalloc_partial[kNoAllocFloats];

// Device address of g_noalloc_partial on `device`, which must be the current
// device; looked up once per device (a host-side reference to the symbol is
// not a device address).
cudaError_t noalloc_scratch_address(int device, float** out) {
  constexpr int kMaxDevices = 64;
  static float* addr[kMaxDevices] = {};
  static std::mutex mu;
  *out = nullptr;
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    addr[device] = static_cast<float*>(p);
  }
  *out = addr[device];
  return cudaSuccess;
}

// Same two-phase compositing as the regular forward kernel (phase A: the
// transmittance-weighted alphas of a chunk; phase B: their product with the
// chunk's radiance), restricted to the per-tile column sums, with the
// radiance read from the caller's receiver-major [N][K][C][2] array.
__global__ void __launch_bounds__(kTilePixels, 2)
    render_csi_noalloc_kernel(const GridConst g, const float4* __restrict__ rec_all,
                              const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
                              const float* __restrict__ rad, int K, int N, int C,
                              float* __restrict__ partial) {
  constexpr int NB = kNoAllocCols, CG = NB / 8, PG = kTilePixels / CG, PX = kTilePixels / PG;
  __shared__ float sA[kChunk * kTilePixels];
  __shared__ __align__(16) float sR[kChunk * NB];
  __shared__ float4 sRec[2 * kChunk];
  const int t = threadIdx.x;
  const int tile = blockIdx.x, v = blockIdx.z;
  const int col0 = blockIdx.y * NB;
  const int ncols = 2 * N * C, twoC = 2 * C;
  const int tr = tile / g.tiles_w, tc = tile % g.tiles_w;
  const int i = tr * g.TH + t / g.TW, jj = tc * g.TW + t % g.TW;
  const bool valid = i < g.H && jj < g.W;
  const float fi = static_cast<float>(i), fj = static_cast<float>(jj);
  const uint2 rg = ranges[static_cast<size_t>(v) * g.T + tile];
  const float4* rec = rec_all + static_cast<size_t>(v) * K * 2;
  const int pg = t % PG, cg = t / PG;
  float acc[PX][8];
#pragma unroll
  for (int p = 0; p < PX; ++p)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[p][c] = 0.0f;
  float T = 1.0f;
  bool alive = valid;
  for (uint32_t start = rg.x; start < rg.y; start += kChunk) {
    const int nb = min(kChunk, static_cast<int>(rg.y - start));
    __syncthreads();
    if (t < kChunk) {
      const bool ok = t < nb;
      const uint32_t k = ok ? vals[start + t] : 0u;
      sRec[2 * t + 0] = ok ? rec[2 * k + 0] : make_float4(0.f, 0.f, 0.f, 0.f);
      sRec[2 * t + 1] = ok ? rec[2 * k + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int e = t; e < kChunk * NB; e += kTilePixels) {
      const int b = e / NB, c = e % NB;
      const int col = col0 + c;
      float x = 0.0f;
      if (b < nb && col < ncols) {
        const uint32_t k = vals[start + b];
        const int j = col / twoC, q = col - j * twoC;
        x = rad[(static_cast<size_t>(j) * K + k) * twoC + q];
      }
      sR[e] = x;
    }
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      float Tw = 0.0f;
      if (alive) {
        float w, G;
        if (pixel_weight(g, sRec[2 * b], sRec[2 * b + 1], i, jj, fi, fj, &w, &G)) {
          Tw = __fmul_rn(T, w);
          T = __fmul_rn(T, __fsub_rn(1.0f, w));
          if (T < g.eps_T) alive = false;
        }
      }
      sA[b * kTilePixels + t] = Tw;
    }
    const int n_alive = __syncthreads_count(alive);
    for (int b = 0; b < nb; ++b) {
      float av[PX];
#pragma unroll
      for (int p = 0; p < PX; ++p) av[p] = sA[b * kTilePixels + p * PG + pg];
      const float4 b0 = *reinterpret_cast<const float4*>(&sR[b * NB + cg * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sR[b * NB + cg * 8 + 4]);
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int p = 0; p < PX; ++p)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[p][c] = fmaf(av[p], bv[c], acc[p][c]);
    }
    if (n_alive == 0) break;
  }
  // per-tile column sums (PG == 32: one column group per warp)
  float s[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float x = 0.0f;
#pragma unroll
    for (int p = 0; p < PX; ++p) x += acc[p][c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    s[c] = x;
  }
  if (pg == 0) {
    float* dst = partial + (static_cast<size_t>(v) * g.T + tile) * ncols;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = col0 + cg * 8 + c;
      if (col < ncols) dst[col] = s[c];
    }
  }
}

}  // namespace rxgs

using namespace rxgs;

namespace {
// Makes `device` current for the scope and restores the caller's device.
struct DeviceScope {
  int prev = -1;
  cudaError_t e = cudaSuccess;
  explicit DeviceScope(int device) {
    e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};
}  // namespace

extern "C" rxgs_status rxgs_render_csi_noalloc(rxgs_ctx* ctx, rxgs_views_t views,
                                               const float* radiance, int N, float* csi,
                                               float* rssi, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  if (!radiance || (!csi && !rssi) || N <= 0)
    return fail(ctx, RXGS_E_INVALID, "render_csi_noalloc: null radiance, no output, or N <= 0");
  // the views stay locked from the lookup through both launches, so a
  // concurrent rxgs_release_views cannot free them in between
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "render_csi_noalloc: unknown views");
  const ViewsState* v = it->second;
  const int C = ctx->scenes.at(v->scene)->C;
  if (rssi && C != 1)
    return fail(ctx, RXGS_E_INVALID, "render_csi_noalloc: RSSI needs one channel (C = %d)", C);
  const GridConst& g = ctx->g;
  const size_t need = static_cast<size_t>(v->M) * g.T * 2 * static_cast<size_t>(N) * C;
  if (need > kNoAllocFloats)
    return fail(ctx, RXGS_E_INVALID,
                "render_csi_noalloc: %zu partial sums (views x tiles x 2NC) exceed the fixed "
                "scratch of %zu floats",
                need, kNoAllocFloats);
  const size_t ncols = 2 * static_cast<size_t>(N) * C;
  const size_t blocks_y = (ncols + kNoAllocCols - 1) / kNoAllocCols;
  if (blocks_y > 65535 || v->M > 65535)
    return fail(ctx, RXGS_E_INVALID,
                "render_csi_noalloc: %zu column blocks x %d views exceed the launch grid", blocks_y,
                v->M);
  float* partial = ctx->noalloc_partial;
  if (!partial) return fail(ctx, RXGS_E_CUDA, "render_csi_noalloc: no scratch address");
  DeviceScope dev(ctx->device);
  if (dev.e != cudaSuccess)
    return fail(ctx, RXGS_E_CUDA, "render_csi_noalloc: %s", cudaGetErrorString(dev.e));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dim3 grid(g.T, static_cast<unsigned>(blocks_y), v->M);
  render_csi_noalloc_kernel<<<grid, kTilePixels, 0, st>>>(g, v->rec, v->vals, v->ranges, radiance,
                                                          v->K, N, C, partial);
  note_launches(1);
  launch_reduce_tiles(partial, v->M, g.T, N, C, csi, rssi, st);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(ctx, RXGS_E_CUDA, "render_csi_noalloc: %s", cudaGetErrorString(e));
  return RXGS_OK;
}
