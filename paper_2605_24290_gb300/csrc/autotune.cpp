// autotune.cpp -- picks the tile shape and the output columns per CTA for a
// workload by timing the candidates (rxgs_autotune).  The choice only moves
// work between CTAs: every candidate composites each pixel's Gaussians in the
// same order, so spectra are bit-identical across candidates and CSI/RSSI
// differ only in the rounding order of their sums over tiles.
#include <algorithm>
#include <cstring>
#include <string>

#include "ctx_internal.h"

namespace rxgs {
bool make_grid_options(const rxgs_options& o, GridConst* g);
}

using namespace rxgs;

extern "C" rxgs_status rxgs_autotune(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                                     const float* rx, int N, const rxgs_render_desc* d, int iters,
                                     char* json, size_t cap) {
  if (!ctx || !tx || !d || M <= 0 || N <= 0) return fail(ctx, RXGS_E_INVALID, "bad arguments");
  if (iters <= 0) iters = 3;
  int C = 0;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->scenes.find(scene);
    if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
    C = it->second->C;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = nullptr;
  CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  const size_t HW = static_cast<size_t>(ctx->opts.H) * ctx->opts.W;
  float *spec = nullptr, *csi = nullptr, *rssi = nullptr;
  cudaError_t e = cudaSuccess;
  if (d->kind & RXGS_OUT_SPECTRA) e = cudaMalloc(&spec, sizeof(float) * M * N * HW * 2 * C);
  if (e == cudaSuccess) e = cudaMalloc(&csi, sizeof(float) * M * N * 2 * C);
  if (e == cudaSuccess) e = cudaMalloc(&rssi, sizeof(float) * M * N);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const rxgs_options saved = ctx->opts;
  const GridConst saved_g = ctx->g;
  std::string out = "{\"candidates\": [";
  float best_ms = 1e30f;
  int best_th = saved.tile_h, best_tw = saved.tile_w, best_cols = 64;
  const int tiles[3][2] = {{16, 16}, {8, 32}, {32, 8}};
  const int cols[4] = {16, 32, 64, 128};
  bool first = true;
  rxgs_status rs = e == cudaSuccess ? RXGS_OK : RXGS_E_OOM;
  for (int ti = 0; ti < 3 && rs == RXGS_OK; ++ti)
    for (int ci = 0; ci < 4 && rs == RXGS_OK; ++ci) {
      if (cols[ci] > 16 && cols[ci] / 2 >= 2 * N * C) continue;  // wider than the work
      {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->opts.tile_h = tiles[ti][0];
        ctx->opts.tile_w = tiles[ti][1];
        ctx->opts.cols_per_cta = cols[ci];
        make_grid_options(ctx->opts, &ctx->g);
      }
      rxgs_outputs o{spec, (d->kind & RXGS_OUT_RSSI) ? rssi : nullptr, csi, nullptr, nullptr};
      rxgs_render_desc dd = *d;
      dd.kind = d->kind | RXGS_OUT_CSI;
      float ms = 0.0f;
      for (int it = 0; it <= iters && rs == RXGS_OK; ++it) {
        if (it == 1) cudaEventRecord(a, st);
        rs = rxgs_render(ctx, scene, tx, M, rx, N, &dd, &o, st);
      }
      if (rs != RXGS_OK) break;
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      ms /= iters;
      char buf[128];
      snprintf(buf, sizeof buf, "%s{\"tile\": [%d, %d], \"cols\": %d, \"ms\": %.4f}",
               first ? "" : ", ", tiles[ti][0], tiles[ti][1], cols[ci], ms);
      out += buf;
      first = false;
      if (ms < best_ms) {
        best_ms = ms;
        best_th = tiles[ti][0];
        best_tw = tiles[ti][1];
        best_cols = cols[ci];
      }
    }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->opts = saved;
    if (rs == RXGS_OK) {
      ctx->opts.tile_h = best_th;
      ctx->opts.tile_w = best_tw;
      ctx->opts.cols_per_cta = best_cols;
    }
    make_grid_options(ctx->opts, &ctx->g);
    if (rs != RXGS_OK) ctx->g = saved_g;
  }
  char buf[160];
  snprintf(buf, sizeof buf, "], \"chosen\": {\"tile\": [%d, %d], \"cols\": %d, \"ms\": %.4f}}", best_th,
           best_tw, best_cols, best_ms);
  out += buf;
  cudaStreamSynchronize(st);
  if (spec) cudaFree(spec);
  if (csi) cudaFree(csi);
  if (rssi) cudaFree(rssi);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaStreamDestroy(st);
  if (rs != RXGS_OK) return rs;
  if (json && cap) {
    if (out.size() + 1 > cap) return fail(ctx, RXGS_E_INVALID, "json buffer too small");
    std::memcpy(json, out.c_str(), out.size() + 1);
  }
  return RXGS_OK;
}
