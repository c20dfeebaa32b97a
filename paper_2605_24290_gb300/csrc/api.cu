// api.cu -- the C ABI (include/rxgs.h): contexts, scenes, transmitter-side
// views, forward and backward renders.  Device memory comes from CUDA's
// stream-ordered pool (cudaMallocAsync / cudaFreeAsync on the caller's
// stream); nothing here synchronises except rxgs_prepare (one readback of
// the instance count) and rxgs_sync.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rxgs.h"
#include "ctx_internal.h"
#include "rxgs_internal.h"

namespace rxgs {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
static std::atomic<unsigned long long> g_dallocs{0};
void note_dalloc() { g_dallocs.fetch_add(1, std::memory_order_relaxed); }
unsigned long long dalloc_count() { return g_dallocs.load(std::memory_order_relaxed); }
}  // namespace rxgs

using namespace rxgs;

namespace {

rxgs_status check_last(rxgs_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, RXGS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return RXGS_OK;
}

bool make_grid(const rxgs_options& o, GridConst* g, std::string* why) {
  if (o.H <= 0 || o.W <= 0 || o.H > 32767 || o.W > 32767) return *why = "H, W out of range", false;
  if (!(o.step_deg > 0.0f) || std::fabs(o.W * static_cast<double>(o.step_deg) - 360.0) > 1e-3)
    return *why = "W * step_deg must be 360", false;
  if (o.H * static_cast<double>(o.step_deg) > 180.0 + 1e-3) return *why = "H * step_deg > 180", false;
  if (o.tile_h <= 0 || o.tile_w <= 0 || o.tile_h * o.tile_w != 256)
    return *why = "tile_h * tile_w must be 256", false;
  if (!(o.q_max > 0.0f) || !(o.eps_T >= 0.0f) || !(o.r_near > 0.0f))
    return *why = "q_max, eps_T, r_near out of range", false;
  if (o.deterministic != 0) return *why = "deterministic backward is not provided", false;
  if (o.cols_per_cta != 0 && o.cols_per_cta != 16 && o.cols_per_cta != 32 &&
      o.cols_per_cta != 64 && o.cols_per_cta != 128)
    return *why = "cols_per_cta must be 0, 16, 32, 64 or 128", false;
  g->H = o.H;
  g->W = o.W;
  g->TH = o.tile_h;
  g->TW = o.tile_w;
  g->tiles_h = (o.H + o.tile_h - 1) / o.tile_h;
  g->tiles_w = (o.W + o.tile_w - 1) / o.tile_w;
  g->T = g->tiles_h * g->tiles_w;
  g->inv_step = static_cast<float>(180.0 / (3.14159265358979323846 * static_cast<double>(o.step_deg)));
  g->theta0_px = static_cast<float>(static_cast<double>(o.theta0_deg) / static_cast<double>(o.step_deg));
  g->Wf = static_cast<float>(o.W);
  g->halfW = 0.5f * static_cast<float>(o.W);
  g->Hm1f = static_cast<float>(o.H - 1);
  g->eps_T = o.eps_T;
  g->q_max = o.q_max;
  g->ksig = sqrtf(o.q_max);
  g->r_near = o.r_near;
  return true;
}

}  // namespace

// Cotangent that is uniform over the pixels of a (view, receiver, channel):
// dL/dCSI directly, plus dL/dRSSI * S/|S| for RSSI = |S| (C == 1).
__global__ void uniform_cot_kernel(const float* __restrict__ gcsi, const float* __restrict__ grssi,
                                   const float* __restrict__ fcsi, int M, int N, int C,
                                   float* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // (v, j, c)
  if (idx >= M * N * C) return;
  float re = gcsi ? gcsi[2 * idx] : 0.0f, im = gcsi ? gcsi[2 * idx + 1] : 0.0f;
  if (grssi && C == 1) {
    const float sr = fcsi[2 * idx], si = fcsi[2 * idx + 1];
    const float mag = sqrtf(sr * sr + si * si);
    if (mag > 0.0f) {
      re += grssi[idx] * sr / mag;
      im += grssi[idx] * si / mag;
    }
  }
  out[2 * idx] = re;
  out[2 * idx + 1] = im;
}

void launch_uniform_cotangent(const float* gcsi, const float* grssi, const float* fcsi, int M,
                              int N, int C, float* out, cudaStream_t s) {
  const int n = M * N * C;
  uniform_cot_kernel<<<(n + 255) / 256, 256, 0, s>>>(gcsi, grssi, fcsi, M, N, C, out);
  note_launches(1);
}

namespace rxgs {
bool make_grid_options(const rxgs_options& o, GridConst* g) {
  std::string why;
  return make_grid(o, g, &why);
}

cudaEvent_t take_event(rxgs_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int pick_cols(const rxgs_ctx* ctx, int ncols) {
  if (ctx->opts.cols_per_cta) return ctx->opts.cols_per_cta;
  if (ncols <= 16) return 16;
  if (ncols <= 32) return 32;
  if (ncols <= 64) return 64;
  return 128;
}

bool lookup_views(void* c, uint64_t views, ViewsRef* out, const char** err) {
  rxgs_ctx* ctx = static_cast<rxgs_ctx*>(c);
  if (!ctx) {
    *err = "null context";
    return false;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) {
    *err = "unknown views";
    return false;
  }
  const ViewsState* v = it->second;
  const SceneState* s = ctx->scenes.at(v->scene);
  out->device = ctx->device;
  out->g = ctx->g;
  out->M = v->M;
  out->K = v->K;
  out->C = s->C;
  out->rec = v->rec;
  out->vals = v->vals;
  out->ranges = v->ranges;
  return true;
}
}  // namespace rxgs

// ====================================================================== ABI
extern "C" {

void rxgs_default_options(rxgs_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->H = 90;
  o->W = 360;
  o->theta0_deg = 0.0f;
  o->step_deg = 1.0f;
  o->tile_h = 16;
  o->tile_w = 16;
  o->eps_T = 1e-4f;
  o->q_max = 9.0f;
  o->r_near = 0.05f;
  o->cols_per_cta = 0;
  o->deterministic = 0;
  o->mem_budget = 0;
}

rxgs_status rxgs_create(const rxgs_options* opts, int device, rxgs_ctx** out) {
  rxgs_ctx* ctx = nullptr;
  if (!out) return RXGS_E_INVALID;
  *out = nullptr;
  ctx = new rxgs_ctx();
  if (opts)
    ctx->opts = *opts;
  else
    rxgs_default_options(&ctx->opts);
  std::string why;
  if (!make_grid(ctx->opts, &ctx->g, &why)) {
    delete ctx;
    return RXGS_E_INVALID;
  }
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->d_pinned),
                                                     ctx->h_pinned, 0);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_stats, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t thr = ~0ull;  // keep freed blocks cached in the pool
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  // the allocation-free entry point's scratch address on this device (this
  // also loads the module that holds the array, so it exists from here on)
  if (e == cudaSuccess) e = noalloc_scratch_address(device, &ctx->noalloc_partial);
  if (e != cudaSuccess) {
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? RXGS_E_OOM : RXGS_E_CUDA;
  }
  *out = ctx;
  return RXGS_OK;
}

rxgs_status rxgs_destroy(rxgs_ctx* ctx) {
  if (!ctx) return RXGS_E_INVALID;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->views) {
    ViewsState* v = kv.second;
    cudaFree(v->tx); cudaFree(v->rec); cudaFree(v->depth); cudaFree(v->counts);
    cudaFree(v->offsets); cudaFree(v->keys); cudaFree(v->vals); cudaFree(v->ranges);
    cudaFree(v->rad); cudaFree(v->glob);
    delete v;
  }
  for (auto& kv : ctx->scenes) {
    SceneState* s = kv.second;
    cudaFree(s->geom); cudaFree(s->base); cudaFree(s->mlp);
    cudaFree(s->occ); cudaFree(s->occ_box);
    delete s;
  }
  if (ctx->serve) destroy_serve(ctx->serve);
  for (BatchPlan* p : ctx->plans) destroy_plan(p);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_pinned);
  if (ctx->ev_stats) cudaEventDestroy(ctx->ev_stats);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
  return RXGS_OK;
}

const char* rxgs_last_error(rxgs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

rxgs_status rxgs_upload_scene(rxgs_ctx* ctx, const rxgs_scene_desc* d, rxgs_scene_t* out) {
  if (!ctx || !d || !out) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (d->K <= 0 || d->K > (1ll << 30)) return fail(ctx, RXGS_E_INVALID, "K out of range");
  if (d->C <= 0 || d->C > 512) return fail(ctx, RXGS_E_INVALID, "C out of range");
  if (!d->means || !d->log_scales || !d->quats || !d->opacity)
    return fail(ctx, RXGS_E_INVALID, "missing scene array");
  if (d->mlp_params && (!d->base_radiance || d->mlp_hidden != 64))
    return fail(ctx, RXGS_E_INVALID, "the MLP needs base_radiance and hidden == 64");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const int K = static_cast<int>(d->K), C = d->C;
  const cudaMemcpyKind kind = d->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!d->on_device) {
    // host-side validation: finite positions and opacity in (0, 1)
    for (int k = 0; k < K; ++k) {
      for (int a = 0; a < 3; ++a)
        if (!std::isfinite(d->means[3 * k + a]) || !std::isfinite(d->log_scales[3 * k + a]))
          return fail(ctx, RXGS_E_INVALID, "non-finite mean or scale at %d", k);
      if (!(d->opacity[k] > 0.0f && d->opacity[k] < 1.0f))
        return fail(ctx, RXGS_E_INVALID, "opacity out of (0,1) at %d", k);
    }
  }
  SceneState* s = new SceneState();
  s->K = K;
  s->C = C;
  float *m = nullptr, *ls = nullptr, *q = nullptr, *op = nullptr;
  cudaStream_t st = 0;
  cudaError_t e = cudaSuccess;
  auto alloc_copy = [&](float** dst, const float* src, size_t n) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(*dst, src, n * sizeof(float), kind, st);
  };
  alloc_copy(&m, d->means, 3ull * K);
  alloc_copy(&ls, d->log_scales, 3ull * K);
  alloc_copy(&q, d->quats, 4ull * K);
  alloc_copy(&op, d->opacity, static_cast<size_t>(K));
  if (e == cudaSuccess) e = cudaMalloc(&s->geom, sizeof(float4) * 3ull * K);
  if (e == cudaSuccess) {
    launch_scene_upload(m, ls, q, op, K, s->geom, st);
    e = cudaGetLastError();
  }
  if (d->base_radiance) alloc_copy(&s->base, d->base_radiance, 2ull * K * C);
  if (d->mlp_params) {
    const size_t h = static_cast<size_t>(d->mlp_hidden);
    s->mlp_floats = h * 3 + h + 4 * C * h + 4 * C + h * 6 + h + 4 * C * h + 4 * C;
    s->hidden = d->mlp_hidden;
    s->bf16 = d->mlp_bf16;
    alloc_copy(&s->mlp, d->mlp_params, s->mlp_floats);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(m);
  cudaFree(ls);
  cudaFree(q);
  cudaFree(op);
  if (e != cudaSuccess) {
    cudaFree(s->geom); cudaFree(s->base); cudaFree(s->mlp);
    delete s;
    return fail(ctx, e == cudaErrorMemoryAllocation ? RXGS_E_OOM : RXGS_E_CUDA, "upload: %s",
                cudaGetErrorString(e));
  }
  const uint64_t id = ctx->next_id++;
  ctx->scenes[id] = s;
  *out = id;
  return RXGS_OK;
}

rxgs_status rxgs_release_scene(rxgs_ctx* ctx, rxgs_scene_t scene) {
  if (!ctx) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->scenes.find(scene);
  if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  SceneState* s = it->second;
  cudaFree(s->geom); cudaFree(s->base); cudaFree(s->mlp);
  cudaFree(s->occ); cudaFree(s->occ_box);
  delete s;
  ctx->scenes.erase(it);
  return RXGS_OK;
}

rxgs_status rxgs_build_occupancy(rxgs_ctx* ctx, rxgs_scene_t scene, int res, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  if (res < 0 || res > 512) return fail(ctx, RXGS_E_INVALID, "res must be 0..512");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->scenes.find(scene);
  if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
  SceneState* s = it->second;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->occ) {
    CK(cudaStreamSynchronize(st));
    cudaFree(s->occ);
    cudaFree(s->occ_box);
    s->occ = nullptr;
    s->occ_box = nullptr;
    s->occ_res = 0;
  }
  s->generation++;  // cached radiance of earlier renders is stale
  if (res == 0) return RXGS_OK;
  const size_t n = static_cast<size_t>(res) * res * res;
  if (cudaMalloc(&s->occ, sizeof(float) * n) != cudaSuccess ||
      cudaMalloc(&s->occ_box, sizeof(float) * 6) != cudaSuccess) {
    cudaFree(s->occ);
    s->occ = nullptr;
    return fail(ctx, RXGS_E_OOM, "occupancy grid of %d^3", res);
  }
  s->occ_res = res;
  launch_occ_build(s->geom, s->K, res, s->occ_box, s->occ, st);
  return check_last(ctx, "build_occupancy");
}

rxgs_status rxgs_update_scene(rxgs_ctx* ctx, rxgs_scene_t scene, const float* opacity,
                              const float* base_radiance, const float* mlp_params,
                              void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->scenes.find(scene);
  if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
  SceneState* s = it->second;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  s->generation++;
  if (opacity) launch_set_opacity(opacity, s->K, s->geom, st);
  if (base_radiance) {
    if (!s->base) return fail(ctx, RXGS_E_INVALID, "scene has no base radiance");
    CK(cudaMemcpyAsync(s->base, base_radiance, sizeof(float) * 2ull * s->K * s->C,
                       cudaMemcpyDeviceToDevice, st));
  }
  if (mlp_params) {
    if (!s->mlp) return fail(ctx, RXGS_E_INVALID, "scene has no MLP");
    CK(cudaMemcpyAsync(s->mlp, mlp_params, sizeof(float) * s->mlp_floats,
                       cudaMemcpyDeviceToDevice, st));
  }
  return check_last(ctx, "update_scene");
}

rxgs_status rxgs_prepare(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                         rxgs_views_t* out, void* stream) {
  if (!ctx || !tx || !out) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (M <= 0 || M > (1 << 16)) return fail(ctx, RXGS_E_INVALID, "M out of range");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->scenes.find(scene);
  if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
  const SceneState* s = it->second;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const GridConst& g = ctx->g;
  ViewsState* v = new ViewsState();
  v->scene = scene;
  v->M = M;
  v->K = s->K;
  v->tile_bits = bits_for(static_cast<uint64_t>(g.T));
  v->view_bits = bits_for(static_cast<uint64_t>(M));
  if (v->tile_bits + v->view_bits > 32) {
    delete v;
    return fail(ctx, RXGS_E_INVALID, "too many views x tiles for a 32-bit (view, tile) key");
  }
  const size_t MK = static_cast<size_t>(M) * s->K;
  if (MK >= 0xffffffffull) {
    delete v;
    return fail(ctx, RXGS_E_INVALID, "views x Gaussians must stay below 2^32");
  }
  uint32_t* scan_tmp = nullptr;
  // the depth order of every view's Gaussians: key and index buffers of
  // the segmented sort, the counts in that order
  uint32_t *dkeys = nullptr, *dkeys_alt = nullptr, *ord_a = nullptr, *ord_b = nullptr;
  uint32_t *dsort_tmp = nullptr, *scounts = nullptr;
  const uint32_t* ord = nullptr;
  auto free_order = [&]() {
    dfree(dkeys, st); dfree(dkeys_alt, st); dfree(ord_a, st); dfree(ord_b, st);
    dfree(dsort_tmp, st); dfree(scounts, st);
  };
  auto cleanup = [&]() {
    dfree(v->tx, st); dfree(v->rec, st); dfree(v->depth, st); dfree(v->counts, st);
    dfree(v->offsets, st); dfree(v->keys, st); dfree(v->vals, st); dfree(v->ranges, st);
    dfree(scan_tmp, st);
    free_order();
    delete v;
  };
  cudaError_t e = dalloc(&v->tx, 3ull * M, st);
  if (e == cudaSuccess) {
    // transmitters already on the device are copied by a kernel, so the
    // step does not wait behind copies the caller queued on the copy engines
    cudaPointerAttributes pa{};
    const cudaError_t pe = cudaPointerGetAttributes(&pa, tx);
    if (pe != cudaSuccess) cudaGetLastError();  // not a device pointer: clear and copy
    const bool on_device =
        pe == cudaSuccess && (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    if (on_device)
      launch_copy_words(reinterpret_cast<const uint32_t*>(tx), reinterpret_cast<uint32_t*>(v->tx),
                        3ull * M, st);
    else
      e = cudaMemcpyAsync(v->tx, tx, sizeof(float) * 3 * M, cudaMemcpyDefault, st);
  }
  if (e == cudaSuccess) e = dalloc(&v->rec, 2 * MK, st);
  if (e == cudaSuccess) e = dalloc(&v->depth, MK, st);
  if (e == cudaSuccess) e = dalloc(&v->counts, MK, st);
  if (e == cudaSuccess) e = dalloc(&v->offsets, MK + 1, st);
  if (e == cudaSuccess) e = dalloc(&scan_tmp, scan_tmp_words(MK), st);
  if (e == cudaSuccess) e = dalloc(&v->ranges, static_cast<size_t>(M) * g.T, st);
  if (e == cudaSuccess) e = dalloc(&dkeys, MK, st);
  if (e == cudaSuccess) e = dalloc(&dkeys_alt, MK, st);
  if (e == cudaSuccess) e = dalloc(&ord_a, MK, st);
  if (e == cudaSuccess) e = dalloc(&ord_b, MK, st);
  if (e == cudaSuccess) e = dalloc(&dsort_tmp, radix_segments_tmp_words(s->K, M), st);
  if (e == cudaSuccess) e = dalloc(&scounts, std::max<size_t>(MK, 4ull * M), st);  // also the stats
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, RXGS_E_OOM, "prepare: %s", cudaGetErrorString(e));
  }
  {
    // stats: the instance count and the visible pairs' depth-key range
    Stage sg(ctx, "preprocess", st);
    cudaMemsetAsync(scounts, 0, 4 * sizeof(uint32_t) * M, st);
    launch_preprocess(g, s->geom, s->K, v->tx, M, v->rec, v->depth, v->counts, st, nullptr,
                      scounts);
  }
  // read back by a kernel into the pinned slot (a copy-engine transfer
  // would queue behind the caller's large copies); the depth sort's first
  // pass (the low 9 bits, independent of the depth range) is queued behind
  // it and runs while the host waits for the slot
  launch_combine_stats(scounts, M, ctx->d_pinned, st);
  e = cudaEventRecord(ctx->ev_stats, st);
  {
    Stage sg(ctx, "depth_sort", st);
    radix_sort_segments_first(v->depth, s->K, M, dkeys, ord_a, dsort_tmp, st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(ctx->ev_stats);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, RXGS_E_CUDA, "prepare: %s", cudaGetErrorString(e));
  }
  const uint64_t I64 = static_cast<uint64_t>(ctx->h_pinned[0]) |
                       (static_cast<uint64_t>(ctx->h_pinned[1]) << 32);
  if (I64 > 0x7fffffffu) {
    cleanup();
    return fail(ctx, RXGS_E_INVALID, "instance count overflow");
  }
  const uint32_t I = static_cast<uint32_t>(I64);
  // visible depth keys lie in [dmin, dmax]: the sort needs the bits of
  // dmax - bias only, bias = dmin rounded down to a multiple of 512 (culled
  // pairs emit nothing; their order is immaterial)
  const uint32_t dmin = I ? ~ctx->h_pinned[2] : 0u, dmax = I ? ctx->h_pinned[3] : 0u;
  const uint32_t dbias = dmin & ~511u;
  const int dbits = bits_for(static_cast<uint64_t>(dmax - dbias) + 1);
  {
    // every view's Gaussians by depth (ties: ascending Gaussian index), and
    // their tile counts in that order
    Stage sg(ctx, "depth_sort", st);
    ord = radix_sort_segments_rest(s->K, M, dbits, dbias, dkeys, dkeys_alt, ord_a, ord_b, dsort_tmp,
                                   v->counts, scounts, st);
  }
  {
    Stage sg(ctx, "scan", st);
    launch_exclusive_scan(scounts, v->offsets, MK, scan_tmp, st);
  }
  dfree(scan_tmp, st);
  v->n_inst = I;
  uint32_t* keys_alt = nullptr;
  uint32_t* vals_alt = nullptr;
  uint32_t* sort_tmp = nullptr;
  e = dalloc(&v->keys, I, st);
  if (e == cudaSuccess) e = dalloc(&v->vals, I, st);
  if (e == cudaSuccess) e = dalloc(&keys_alt, I, st);
  if (e == cudaSuccess) e = dalloc(&vals_alt, I, st);
  // one pass by tile within each view's run when the tile fits one digit
  const bool one_pass = v->tile_bits <= 9;
  if (e == cudaSuccess)
    e = dalloc(&sort_tmp, one_pass ? radix_views_tmp_words(I, M) : radix_tmp_words(I), st);
  if (e != cudaSuccess) {
    dfree(keys_alt, st); dfree(vals_alt, st); dfree(sort_tmp, st);
    cleanup();
    return fail(ctx, RXGS_E_OOM, "prepare (sort buffers): %s", cudaGetErrorString(e));
  }
  {
    Stage sg(ctx, "emit", st);
    launch_emit_sorted(g, v->rec, ord, v->offsets, MK, s->K, v->tile_bits, v->keys, v->vals, st);
  }
  free_order();
  bool in_alt = false;
  if (one_pass) {
    // stable: each (view, tile) keeps the depth order of the emission; the
    // pass writes the ranges as well
    Stage sg(ctx, "sort", st);
    radix_sort_views(v->keys, v->vals, keys_alt, vals_alt, I, v->offsets, s->K, M, v->tile_bits,
                     v->ranges, g.T, sort_tmp, st);
    in_alt = true;
  } else {
    {
      Stage sg(ctx, "sort", st);
      radix_sort_pairs(v->keys, v->vals, keys_alt, vals_alt, I, v->tile_bits + v->view_bits,
                       sort_tmp, &in_alt, st, nullptr, ctx->d_err);
    }
    Stage sg(ctx, "ranges", st);
    launch_tile_ranges(in_alt ? keys_alt : v->keys, I, v->tile_bits, g.T, v->ranges, M, st);
  }
  if (in_alt) {
    std::swap(v->keys, keys_alt);
    std::swap(v->vals, vals_alt);
  }
  dfree(keys_alt, st);
  dfree(vals_alt, st);
  dfree(sort_tmp, st);
  rxgs_status rs = check_last(ctx, "prepare kernels");
  if (rs != RXGS_OK) {
    cleanup();
    return rs;
  }
  const uint64_t id = ctx->next_id++;
  ctx->views[id] = v;
  *out = id;
  return RXGS_OK;
}

rxgs_status rxgs_release_views(rxgs_ctx* ctx, rxgs_views_t views, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "unknown views");
  cudaSetDevice(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ViewsState* v = it->second;
  dfree(v->tx, st); dfree(v->rec, st); dfree(v->depth, st); dfree(v->counts, st);
  dfree(v->offsets, st); dfree(v->keys, st); dfree(v->vals, st); dfree(v->ranges, st);
  dfree(v->rad, st); dfree(v->glob, st);
  dfree(v->tfin, st); dfree(v->stops, st); dfree(v->tile_stop, st);
  delete v;
  ctx->views.erase(it);
  return RXGS_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ render
namespace {

// Checks of the FLE radiance arguments (explicit or FiLM-conditioned).
rxgs_status check_fle(rxgs_ctx* ctx, const SceneState* s, const rxgs_render_desc* d) {
  if (d->film_local && !d->fle_base)
    return fail(ctx, RXGS_E_INVALID, "film_local needs fle_base (the FiLM-conditioned FLE path)");
  if (!d->fle_coeffs && !d->fle_base) return RXGS_OK;
  if (d->fle_coeffs && d->fle_base)
    return fail(ctx, RXGS_E_INVALID, "fle_coeffs and fle_base exclude each other");
  if (d->radiance) return fail(ctx, RXGS_E_INVALID, "radiance and FLE coefficients exclude each other");
  if (s->C != 1) return fail(ctx, RXGS_E_INVALID, "FLE radiance needs C == 1");
  if (d->fle_lmax < 0 || d->fle_lmax > 9) return fail(ctx, RXGS_E_INVALID, "fle_lmax must be 0..9");
  if (d->reduce_path == 1) return fail(ctx, RXGS_E_INVALID, "reduce_path 1 does not take FLE radiance");
  if (d->film_local && !d->fle_base)
    return fail(ctx, RXGS_E_INVALID, "film_local needs fle_base (the FiLM-conditioned FLE path)");
  if (d->film_local && (!s->mlp || !local_branch_supported(s->hidden, s->C)))
    return fail(ctx, RXGS_E_INVALID,
                "film_local needs a scene with conditioning MLP weights (64 hidden units, C == 1)");
  if (d->fle_base) {
    if (!d->film) return fail(ctx, RXGS_E_INVALID, "fle_base needs the FiLM parameters (film)");
    if (rxgs_film_param_count(d->film_nfreq, d->film_embed, d->film_hidden, d->fle_lmax) <= 0)
      return fail(ctx, RXGS_E_INVALID, "FiLM sizes out of range (nfreq 1..%d, embed 0..%d, hidden 1..%d)",
                  kFilmMaxFreq, kFilmMaxEmbed, kFilmMaxHidden);
  }
  return RXGS_OK;
}

FilmDims desc_film_dims(const rxgs_render_desc* d) {
  return film_dims(d->film_nfreq, d->film_embed, d->film_hidden, d->fle_lmax);
}

// The FLE contraction writes columns [0, used) of every row; the pad columns
// [used, stride) are read by the compositing as zero radiance.
void clear_pad_columns(float* rad, size_t rows, int stride, int used, cudaStream_t st) {
  if (stride > used)
    cudaMemset2DAsync(rad + used, sizeof(float) * stride, 0, sizeof(float) * (stride - used), rows,
                      st);
}

// Produces the Gaussian-major radiance [K][stride] for receivers rx[N]; with
// FLE coefficients, one such array per view of v ([M][K][stride]).
rxgs_status make_radiance(rxgs_ctx* ctx, const SceneState* s, const ViewsState* v,
                          const float* rx, int N, const rxgs_render_desc* d, int stride,
                          float* rad, float* glob, cudaStream_t st) {
  Stage sg(ctx, d->radiance ? "radiance_transpose"
                            : (d->fle_coeffs ? "fle" : (d->fle_base ? "fle_film" : "mlp")), st);
  if (d->fle_base) {
    const FilmDims f = desc_film_dims(d);
    float4* ab = nullptr;
    if (dalloc(&ab, static_cast<size_t>(N) * f.L, st) != cudaSuccess)
      return fail(ctx, RXGS_E_OOM, "FiLM outputs");
    // the conditioned coefficients (Eq. film_apply; with the local branch,
    // Eq. combined_local) are formed inside the contraction from the base
    // coefficients, the modulations ab and the local factors loc
    float4* loc = nullptr;
    float2* feat = nullptr;
    cudaError_t e = cudaSuccess;
    if (d->film_local) e = dalloc(&loc, static_cast<size_t>(N) * s->K, st);
    if (e == cudaSuccess && d->film_local && s->occ)
      e = dalloc(&feat, static_cast<size_t>(N) * s->K, st);
    unsigned char* image = nullptr;
    if (e == cudaSuccess) e = dalloc(&image, fle_basis_image_bytes(s->K, v->M), st);
    if (e != cudaSuccess) {
      dfree(ab, st); dfree(loc, st); dfree(feat, st); dfree(image, st);
      return fail(ctx, RXGS_E_OOM, "FiLM radiance");
    }
    launch_film_global(d->film, f, rx, N, ab, st);
    if (d->film_local) {
      if (feat) launch_occ_probes(s->geom, s->K, rx, N, s->occ_res, s->occ_box, s->occ, feat, st);
      launch_local_factors(s->mlp, rx, N, s->geom, s->K, feat, loc, st);
    }
    {
      Stage sb(ctx, "fle_basis", st);  // within the radiance stage
      launch_fle_basis_image(s->geom, v->tx, s->K, v->M, d->fle_lmax, image, st);
    }
    clear_pad_columns(rad, static_cast<size_t>(v->M) * s->K, stride, 2 * N, st);
    launch_fle_radiance_film_tc(d->fle_base, ab, loc, N, s->K, d->fle_lmax, image, v->M, stride,
                                static_cast<size_t>(s->K) * stride, rad, st, ctx->d_err);
    dfree(image, st);
    dfree(ab, st);
    dfree(loc, st);
    dfree(feat, st);
  } else if (d->fle_coeffs) {
    unsigned char* image = nullptr;
    if (dalloc(&image, fle_basis_image_bytes(s->K, v->M), st) != cudaSuccess)
      return fail(ctx, RXGS_E_OOM, "FLE basis image");
    {
      Stage sb(ctx, "fle_basis", st);  // within the radiance stage
      launch_fle_basis_image(s->geom, v->tx, s->K, v->M, d->fle_lmax, image, st);
    }
    clear_pad_columns(rad, static_cast<size_t>(v->M) * s->K, stride, 2 * N, st);
    launch_fle_radiance_tc(d->fle_coeffs, N, s->K, d->fle_lmax, image, v->M, stride,
                           static_cast<size_t>(s->K) * stride, rad, st, ctx->d_err);
    dfree(image, st);
  } else if (d->radiance) {
    launch_radiance_transpose(d->radiance, N, s->K, s->C, stride, rad, st);
  } else {
    if (!s->mlp) return fail(ctx, RXGS_E_INVALID, "no radiance given and the scene has no MLP");
    MlpParams m{s->mlp, s->hidden, s->C, s->bf16};
    float2* feat = nullptr;
    if (s->occ) {
      if (dalloc(&feat, static_cast<size_t>(N) * s->K, st) != cudaSuccess)
        return fail(ctx, RXGS_E_OOM, "occlusion inputs");
      launch_occ_probes(s->geom, s->K, rx, N, s->occ_res, s->occ_box, s->occ, feat, st);
      m.feat = feat;
    }
    // every (Gaussian, receiver) column is written: only the pad columns
    // past 2 N C are cleared
    clear_pad_columns(rad, s->K, stride, 2 * N * s->C, st);
    launch_mlp_radiance(m, rx, N, s->geom, s->base, s->K, stride, rad, glob, st, nullptr,
                        nullptr, false);
    dfree(feat, st);
  }
  return check_last(ctx, "radiance");
}

}  // namespace

extern "C" {

rxgs_status rxgs_render_views(rxgs_ctx* ctx, rxgs_views_t views, const float* rx, int N,
                              const rxgs_render_desc* d, rxgs_outputs* out, void* stream) {
  if (!ctx || !d || !out) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (N <= 0 || N > (1 << 20)) return fail(ctx, RXGS_E_INVALID, "N out of range");
  const int kind = d->kind;
  if (!kind) return fail(ctx, RXGS_E_INVALID, "empty output kind");
  if ((kind & RXGS_OUT_SPECTRA) && !out->spectra) return fail(ctx, RXGS_E_INVALID, "spectra == NULL");
  if ((kind & RXGS_OUT_RSSI) && !out->rssi) return fail(ctx, RXGS_E_INVALID, "rssi == NULL");
  if ((kind & RXGS_OUT_CSI) && !out->csi) return fail(ctx, RXGS_E_INVALID, "csi == NULL");
  if (!d->radiance && !d->fle_coeffs && !rx) return fail(ctx, RXGS_E_INVALID, "rx == NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "unknown views");
  ViewsState* v = it->second;
  const SceneState* s = ctx->scenes.at(v->scene);
  if ((kind & RXGS_OUT_RSSI) && s->C != 1) return fail(ctx, RXGS_E_INVALID, "RSSI needs C == 1");
  if (rxgs_status fs = check_fle(ctx, s, d); fs != RXGS_OK) return fs;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const GridConst& g = ctx->g;
  if (d->reduce_path == 1) {
    // CSI / RSSI through visibility weights (Eq. render_reorder)
    if (kind & RXGS_OUT_SPECTRA)
      return fail(ctx, RXGS_E_INVALID, "reduce_path 1 gives CSI / RSSI only, not spectra");
    if (d->radiance && !weighted_sum_supported(s->C))
      return fail(ctx, RXGS_E_INVALID, "reduce_path 1 with explicit radiance needs 2C to divide 256");
    if (!d->radiance && !s->mlp)
      return fail(ctx, RXGS_E_INVALID, "no radiance given and the scene has no MLP");
    if (!d->radiance && s->C > 52) return fail(ctx, RXGS_E_INVALID, "reduce_path 1 supports C <= 52");
    if (!d->radiance && s->occ)
      return fail(ctx, RXGS_E_INVALID, "reduce_path 1 does not take occlusion inputs (occupancy grid)");
    float *W = nullptr, *tmp = nullptr, *glob = nullptr, *csi_t = nullptr;
    const size_t ntmp = d->radiance ? weighted_sum_tmp_floats(v->M, s->K, N, s->C)
                                    : mlp_weighted_tmp_floats(v->M, s->K, N, s->C);
    cudaError_t e = dalloc(&W, static_cast<size_t>(v->M) * s->K, st);
    if (e == cudaSuccess) e = dalloc(&tmp, ntmp, st);
    if (e == cudaSuccess && !d->radiance) e = dalloc(&glob, static_cast<size_t>(N) * 4 * s->C, st);
    float* csi = (kind & RXGS_OUT_CSI) ? out->csi : nullptr;
    if (e == cudaSuccess && !csi) e = dalloc(&csi_t, static_cast<size_t>(v->M) * N * 2 * s->C, st);
    if (e != cudaSuccess) {
      dfree(W, st); dfree(tmp, st); dfree(glob, st); dfree(csi_t, st);
      return fail(ctx, RXGS_E_OOM, "render (visibility): %s", cudaGetErrorString(e));
    }
    if (!csi) csi = csi_t;
    RenderArgs a{};
    a.g = g;
    a.rec = v->rec;
    a.vals = v->vals;
    a.ranges = v->ranges;
    a.K = s->K;
    a.M = v->M;
    {
      Stage sg(ctx, "visibility", st);
      launch_visibility(a, W, st);
    }
    float* rssi = (kind & RXGS_OUT_RSSI) ? out->rssi : nullptr;
    if (d->radiance) {
      Stage sg(ctx, "weighted_sum", st);
      launch_weighted_sum(d->radiance, N, s->K, s->C, W, v->M, tmp, csi, rssi, st);
    } else {
      Stage sg(ctx, "mlp_weighted", st);
      MlpParams m{s->mlp, s->hidden, s->C, s->bf16};
      launch_mlp_global(m, rx, N, glob, st);
      launch_mlp_weighted(m, rx, N, s->geom, s->base, s->K, W, v->M, nullptr, glob, tmp, csi, rssi,
                          nullptr, st);
    }
    rxgs_status rs = check_last(ctx, "render (visibility)");
    dfree(W, st); dfree(tmp, st); dfree(glob, st); dfree(csi_t, st);
    return rs;
  }
  const int ncols = 2 * N * s->C;
  const int stride = round_up(ncols, 128);
  const bool fle = d->fle_coeffs != nullptr || d->fle_base != nullptr;
  const size_t rad_view = fle ? static_cast<size_t>(s->K) * stride : 0;
  float* rad = nullptr;
  float* partial = nullptr;
  float* glob = nullptr;
  CK(dalloc(&rad, static_cast<size_t>(s->K) * stride * (fle ? v->M : 1), st));
  const bool reduce = (kind & (RXGS_OUT_RSSI | RXGS_OUT_CSI)) != 0;
  cudaError_t e = cudaSuccess;
  if (reduce) e = dalloc(&partial, static_cast<size_t>(v->M) * g.T * ncols, st);
  if (e == cudaSuccess && !d->radiance && !fle)
    e = dalloc(&glob, static_cast<size_t>(N) * 4 * s->C, st);
  if (e != cudaSuccess) {
    dfree(rad, st); dfree(partial, st);
    return fail(ctx, RXGS_E_OOM, "render: %s", cudaGetErrorString(e));
  }
  rxgs_status rs = make_radiance(ctx, s, v, rx, N, d, stride, rad, glob, st);
  if (rs == RXGS_OK) {
    // keep this radiance for a backward on the same views
    dfree(v->rad, st);
    dfree(v->glob, st);
    v->rad = rad;
    v->glob = glob;
    v->key_rx = rx;
    v->key_radiance = d->radiance;
    v->key_fle = d->fle_coeffs ? d->fle_coeffs : d->fle_base;
    v->key_film = d->fle_base ? d->film : nullptr;
    v->key_film_dims[0] = d->fle_base ? d->film_nfreq : 0;
    v->key_film_dims[1] = d->fle_base ? d->film_embed : 0;
    v->key_film_dims[2] = d->fle_base ? d->film_hidden : 0;
    v->key_film_local = d->fle_base ? d->film_local : 0;
    v->key_lmax = fle ? d->fle_lmax : -1;
    v->key_N = N;
    v->key_stride = stride;
    v->key_gen = s->generation;
    rad = nullptr;
    glob = nullptr;
    RenderArgs a{};
    a.g = g;
    a.rec = v->rec;
    a.vals = v->vals;
    a.ranges = v->ranges;
    a.rad = v->rad;
    a.rad_view = rad_view;
    a.K = s->K;
    a.M = v->M;
    a.N = N;
    a.C = s->C;
    a.stride = stride;
    a.ncols = ncols;
    a.spectra = (kind & RXGS_OUT_SPECTRA) ? out->spectra : nullptr;
    a.partial = partial;
    a.ncontrib = out->ncontrib;
    a.tfinal = out->tfinal;
    a.err = ctx->d_err;
    const int cols = pick_cols(ctx, ncols);
    // the tensor-core forward also leaves the backward's per-pixel state on
    // the views (kept for their lifetime; without the buffers it is skipped)
    if (render_fwd_keeps_stops(cols) && !v->stops_valid) {
      const size_t MHW = static_cast<size_t>(v->M) * g.H * g.W;
      if (!v->tfin && dalloc(&v->tfin, MHW, st) != cudaSuccess) v->tfin = nullptr;
      if (!v->stops && dalloc(&v->stops, MHW, st) != cudaSuccess) v->stops = nullptr;
      if (!v->tile_stop && dalloc(&v->tile_stop, static_cast<size_t>(v->M) * g.T, st) != cudaSuccess)
        v->tile_stop = nullptr;
      if (v->tfin && v->stops && v->tile_stop) {
        a.keep_tfin = v->tfin;
        a.keep_stops = v->stops;
        a.keep_tile_stop = v->tile_stop;
      }
    }
    {
      Stage sg(ctx, "render_fwd", st);
      launch_render_fwd(a, cols, st);
    }
    if (a.keep_tfin) v->stops_valid = true;
    if (reduce) {
      Stage sg(ctx, "reduce", st);
      launch_reduce_tiles(partial, v->M, g.T, N, s->C, (kind & RXGS_OUT_CSI) ? out->csi : nullptr,
                          (kind & RXGS_OUT_RSSI) ? out->rssi : nullptr, st);
    }
    rs = check_last(ctx, "render");
  }
  dfree(rad, st);
  dfree(partial, st);
  dfree(glob, st);
  return rs;
}

rxgs_status rxgs_render(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                        const float* rx, int N, const rxgs_render_desc* d, rxgs_outputs* out,
                        void* stream) {
  rxgs_views_t v = 0;
  rxgs_status st = rxgs_prepare(ctx, scene, tx, M, &v, stream);
  if (st != RXGS_OK) return st;
  st = rxgs_render_views(ctx, v, rx, N, d, out, stream);
  rxgs_status st2 = rxgs_release_views(ctx, v, stream);
  return st != RXGS_OK ? st : st2;
}

rxgs_status rxgs_views_info(rxgs_ctx* ctx, rxgs_views_t views, int64_t* n_inst) {
  if (!ctx || !n_inst) return fail(ctx, RXGS_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "unknown views");
  *n_inst = it->second->n_inst;
  return RXGS_OK;
}

rxgs_status rxgs_views_export(rxgs_ctx* ctx, rxgs_views_t views, float* rec, uint32_t* counts,
                              uint64_t* keys, uint32_t* vals, uint32_t* ranges, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "unknown views");
  const ViewsState* v = it->second;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  const size_t MK = static_cast<size_t>(v->M) * v->K;
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  if (rec) CK(cudaMemcpyAsync(rec, v->rec, sizeof(float4) * 2 * MK, dd, st));
  if (counts) CK(cudaMemcpyAsync(counts, v->counts, sizeof(uint32_t) * MK, dd, st));
  if (keys && v->n_inst) {
    launch_expand_keys(v->keys, v->vals, v->n_inst, v->depth, v->K, v->tile_bits, keys, st);
    CK(cudaGetLastError());
  }
  if (vals && v->n_inst) CK(cudaMemcpyAsync(vals, v->vals, sizeof(uint32_t) * v->n_inst, dd, st));
  if (ranges)
    CK(cudaMemcpyAsync(ranges, v->ranges, sizeof(uint2) * static_cast<size_t>(v->M) * ctx->g.T, dd,
                       st));
  return RXGS_OK;
}

// CSI / RSSI cotangents with explicit radiance: the visibility-weight
// backward (vis_bwd.cu) -- no Gaussian-major radiance copy and no
// [K][N*2C] gradient buffer.
static rxgs_status backward_visibility(rxgs_ctx* ctx, const SceneState* s, const ViewsState* v,
                                       int N, const rxgs_render_desc* d,
                                       const rxgs_cotangents* cot, rxgs_grads* gr,
                                       cudaStream_t st) {
  const GridConst& g = ctx->g;
  const int C = s->C, K = s->K, M = v->M;
  const size_t MK = static_cast<size_t>(M) * K;
  const size_t MHW = static_cast<size_t>(M) * g.H * g.W;
  float *g_uni = nullptr, *gamma = nullptr, *W = nullptr, *tfin = nullptr, *d_tau = nullptr;
  uint32_t *stops = nullptr, *tstop = nullptr;
  auto cleanup = [&]() {
    dfree(g_uni, st); dfree(gamma, st); dfree(W, st); dfree(tfin, st); dfree(stops, st);
    dfree(tstop, st);
    if (!gr->grad_opacity) dfree(d_tau, st);
  };
  cudaError_t e = dalloc(&g_uni, static_cast<size_t>(M) * 2 * N * C, st);
  if (e == cudaSuccess) e = dalloc(&gamma, MK, st);
  if (e == cudaSuccess && gr->grad_radiance) e = dalloc(&W, MK, st);
  if (e == cudaSuccess && W) e = cudaMemsetAsync(W, 0, sizeof(float) * MK, st);
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&tfin, MHW, st);
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&stops, MHW, st);
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&tstop, static_cast<size_t>(M) * g.T, st);
  d_tau = gr->grad_opacity;
  if (e == cudaSuccess && !d_tau) e = dalloc(&d_tau, static_cast<size_t>(K), st);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, RXGS_E_OOM, "backward: %s", cudaGetErrorString(e));
  }
  launch_uniform_cotangent(cot->grad_csi, cot->grad_rssi, cot->fwd_csi, M, N, C, g_uni, st);
  BackwardArgs A{};
  A.f.g = g;
  A.f.rec = v->rec;
  A.f.vals = v->vals;
  A.f.ranges = v->ranges;
  A.f.K = K;
  A.f.M = M;
  A.f.N = N;
  A.f.C = C;
  A.f.ncols = 2 * N * C;
  A.d_tau = d_tau;
  A.n_inst = v->n_inst;
  if (v->stops_valid) {
    // kept by the tensor-core forward on these views
    A.tfin = v->tfin;
    A.stops = v->stops;
    A.tile_stop = v->tile_stop;
  } else {
    A.tfin = tfin;
    A.stops = stops;
    A.tile_stop = tstop;
    Stage sg(ctx, "bwd_prepass", st);
    launch_bwd_prepass(A, st);
  }
  {
    Stage sg(ctx, "vis_bwd", st);
    launch_vis_backward(A, d->radiance, g_uni, gamma, W, gr->grad_radiance, st);
  }
  rxgs_status rs = check_last(ctx, "backward");
  cleanup();
  return rs;
}

rxgs_status rxgs_render_backward(rxgs_ctx* ctx, rxgs_views_t views, const float* rx, int N,
                                 const rxgs_render_desc* d, const rxgs_cotangents* cot,
                                 rxgs_grads* gr, void* stream) {
  if (!ctx || !d || !cot || !gr) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (N <= 0 || N > (1 << 20)) return fail(ctx, RXGS_E_INVALID, "N out of range");
  if (!cot->grad_spectra && !cot->grad_csi && !cot->grad_rssi)
    return fail(ctx, RXGS_E_INVALID, "no cotangent");
  if (cot->grad_rssi && !cot->fwd_csi)
    return fail(ctx, RXGS_E_INVALID, "grad_rssi needs the forward CSI (fwd_csi)");
  if (!d->radiance && !d->fle_coeffs && !rx) return fail(ctx, RXGS_E_INVALID, "rx == NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->views.find(views);
  if (it == ctx->views.end()) return fail(ctx, RXGS_E_INVALID, "unknown views");
  const ViewsState* v = it->second;
  const SceneState* s = ctx->scenes.at(v->scene);
  if (cot->grad_rssi && s->C != 1) return fail(ctx, RXGS_E_INVALID, "RSSI needs C == 1");
  if (rxgs_status fs = check_fle(ctx, s, d); fs != RXGS_OK) return fs;
  if (!d->radiance && !d->fle_coeffs && !d->fle_base) {
    if (!s->mlp) return fail(ctx, RXGS_E_INVALID, "no radiance given and the scene has no MLP");
    if (s->bf16) return fail(ctx, RXGS_E_INVALID, "backward through a bf16 MLP is not supported");

  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (d->radiance && !cot->grad_spectra) return backward_visibility(ctx, s, v, N, d, cot, gr, st);
  const GridConst& g = ctx->g;
  const int C = s->C, K = s->K, M = v->M;
  const int ncols = 2 * N * C;
  const int stride = round_up(ncols, 128);
  const bool film = d->fle_base != nullptr;
  const bool fle = d->fle_coeffs != nullptr || film;
  const size_t rad_view = fle ? static_cast<size_t>(K) * stride : 0;
  const size_t nrad = static_cast<size_t>(K) * stride * (fle ? M : 1);
  float *rad = nullptr, *glob = nullptr, *d_rad = nullptr, *g_uni = nullptr, *d_tau = nullptr;
  float *g_base = nullptr, *g_mlp = nullptr, *mlp_tmp = nullptr, *tfin = nullptr;
  uint32_t *stops = nullptr, *tstop = nullptr;
  const bool cached = v->rad && v->key_rx == rx && v->key_radiance == d->radiance &&
                      v->key_fle == (d->fle_coeffs ? d->fle_coeffs : d->fle_base) &&
                      v->key_film == (film ? d->film : nullptr) &&
                      v->key_film_dims[0] == (film ? d->film_nfreq : 0) &&
                      v->key_film_dims[1] == (film ? d->film_embed : 0) &&
                      v->key_film_dims[2] == (film ? d->film_hidden : 0) &&
                      v->key_film_local == (film ? d->film_local : 0) &&
                      v->key_lmax == (fle ? d->fle_lmax : -1) &&
                      v->key_N == N && v->key_stride == stride && v->key_gen == s->generation;
  auto cleanup = [&]() {
    if (cached) {
      rad = nullptr;
      glob = nullptr;
    }
    dfree(rad, st); dfree(glob, st); dfree(d_rad, st); dfree(g_uni, st); dfree(mlp_tmp, st);
    dfree(tfin, st); dfree(stops, st); dfree(tstop, st);
    if (!gr->grad_opacity) dfree(d_tau, st);
    if (!gr->grad_base) dfree(g_base, st);
    if (!gr->grad_mlp) dfree(g_mlp, st);
  };
  cudaError_t e = cudaSuccess;
  if (cached) {
    rad = v->rad;
    glob = v->glob;
  } else {
    e = dalloc(&rad, nrad, st);
    if (e == cudaSuccess && !d->radiance && !fle)
      e = dalloc(&glob, static_cast<size_t>(N) * 4 * C, st);
  }
  if (e == cudaSuccess) e = dalloc(&d_rad, nrad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_rad, 0, sizeof(float) * nrad, st);
  const size_t MHW = static_cast<size_t>(M) * g.H * g.W;
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&tfin, MHW, st);
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&stops, MHW, st);
  if (e == cudaSuccess && !v->stops_valid) e = dalloc(&tstop, static_cast<size_t>(M) * g.T, st);
  if (e == cudaSuccess && (cot->grad_csi || cot->grad_rssi))
    e = dalloc(&g_uni, static_cast<size_t>(M) * ncols, st);
  d_tau = gr->grad_opacity;
  if (e == cudaSuccess && !d_tau) e = dalloc(&d_tau, static_cast<size_t>(K), st);
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, RXGS_E_OOM, "backward: %s", cudaGetErrorString(e));
  }
  rxgs_status rs = cached ? RXGS_OK : make_radiance(ctx, s, v, rx, N, d, stride, rad, glob, st);
  if (rs != RXGS_OK) {
    cleanup();
    return rs;
  }
  if (g_uni) launch_uniform_cotangent(cot->grad_csi, cot->grad_rssi, cot->fwd_csi, M, N, C, g_uni, st);
  BackwardArgs A{};
  A.f.g = g;
  A.f.rec = v->rec;
  A.f.vals = v->vals;
  A.f.ranges = v->ranges;
  A.f.rad = rad;
  A.f.rad_view = rad_view;
  A.f.K = K;
  A.f.M = M;
  A.f.N = N;
  A.f.C = C;
  A.f.stride = stride;
  A.f.ncols = ncols;
  A.f.spectra = nullptr;
  A.g_spec = cot->grad_spectra;
  A.g_uniform = g_uni;
  A.d_rad = d_rad;
  A.d_tau = d_tau;
  A.n_inst = v->n_inst;
  A.err = ctx->d_err;
  if (v->stops_valid) {
    // kept by the tensor-core forward on these views
    A.tfin = v->tfin;
    A.stops = v->stops;
    A.tile_stop = v->tile_stop;
  } else {
    A.tfin = tfin;
    A.stops = stops;
    A.tile_stop = tstop;
    Stage sg(ctx, "bwd_prepass", st);
    launch_bwd_prepass(A, st);
  }
  {
    Stage sg(ctx, "render_bwd", st);
    launch_render_bwd(A, st);
  }
  if (d->radiance) {
    Stage sg(ctx, "radiance_grad", st);
    if (gr->grad_radiance) launch_radiance_untranspose_add(d_rad, N, K, C, stride, gr->grad_radiance, st);
  } else if (film) {
    const FilmDims f = desc_film_dims(d);
    float4 *ab = nullptr, *d_ab = nullptr, *loc = nullptr, *d_loc = nullptr;
    float *ftmp = nullptr, *G = nullptr;
    unsigned char* image = nullptr;
    float2* feat = nullptr;
    const size_t S = static_cast<size_t>(N) * f.L;
    const size_t NK = static_cast<size_t>(N) * K;
    e = dalloc(&ab, S, st);
    if (e == cudaSuccess) e = dalloc(&d_ab, S, st);
    if (e == cudaSuccess && gr->grad_film) e = dalloc(&ftmp, film_backward_tmp_floats(f, N), st);
    // the conditioned coefficients' gradient [N][K][2][L], written (not
    // accumulated) by the tensor-core contraction, then folded
    if (e == cudaSuccess) e = dalloc(&G, S * K * 2, st);
    if (e == cudaSuccess) e = dalloc(&image, fle_basis_image_bytes(K, M), st);
    if (e == cudaSuccess && d->film_local) e = dalloc(&loc, NK, st);
    if (e == cudaSuccess && d->film_local) e = dalloc(&d_loc, NK, st);
    if (e == cudaSuccess && d->film_local && s->occ) e = dalloc(&feat, NK, st);
    auto free_film = [&]() {
      dfree(ab, st); dfree(d_ab, st); dfree(ftmp, st); dfree(G, st);
      dfree(loc, st); dfree(d_loc, st); dfree(feat, st); dfree(image, st);
    };
    if (e != cudaSuccess) {
      free_film();
      cleanup();
      return fail(ctx, RXGS_E_OOM, "backward (FiLM): %s", cudaGetErrorString(e));
    }
    {
      Stage sg(ctx, "fle_film_bwd", st);
      cudaMemsetAsync(d_ab, 0, sizeof(float4) * S, st);
      launch_film_global(d->film, f, rx, N, ab, st);
      {
        Stage sb(ctx, "fle_basis", st);  // within the backward stage
        launch_fle_basis_image(s->geom, v->tx, K, M, d->fle_lmax, image, st);
      }
      launch_fle_backward_tc(d_rad, N, K, d->fle_lmax, image, M, stride, rad_view, G, false, st,
                             ctx->d_err);
      if (d->film_local) {
        // the local branch (Eq. combined_local): its gradient, and G becomes
        // the FiLM-modulated coefficients' gradient
        if (feat) launch_occ_probes(s->geom, K, rx, N, s->occ_res, s->occ_box, s->occ, feat, st);
        launch_local_factors(s->mlp, rx, N, s->geom, K, feat, loc, st);
        launch_film_local_backward(G, d->fle_base, ab, loc, s->mlp, rx, N, s->geom, K,
                                   d->fle_lmax, feat, d_loc, gr->grad_mlp, st);
      }
      launch_film_fold(G, N, K, d->fle_lmax, d->fle_base, ab, gr->grad_fle_base,
                       reinterpret_cast<float*>(d_ab), st);
    }
    if (gr->grad_film) {
      Stage sg(ctx, "film_mlp_bwd", st);
      launch_film_backward(d->film, f, rx, N, d_ab, ftmp, gr->grad_film, st);
    }
    free_film();
  } else if (fle) {
    Stage sg(ctx, "fle_bwd", st);
    if (gr->grad_fle) {
      unsigned char* image = nullptr;
      if (dalloc(&image, fle_basis_image_bytes(K, M), st) != cudaSuccess) {
        cleanup();
        return fail(ctx, RXGS_E_OOM, "backward (FLE basis image)");
      }
      {
        Stage sb(ctx, "fle_basis", st);  // within the backward stage
        launch_fle_basis_image(s->geom, v->tx, K, M, d->fle_lmax, image, st);
      }
      launch_fle_backward_tc(d_rad, N, K, d->fle_lmax, image, M, stride, rad_view, gr->grad_fle,
                             true, st, ctx->d_err);
      dfree(image, st);
    }
  } else {
    MlpParams m{s->mlp, s->hidden, C, 0};
    g_base = gr->grad_base;
    g_mlp = gr->grad_mlp;
    e = cudaSuccess;
    float2* feat = nullptr;
    if (!g_base) e = dalloc(&g_base, 2ull * K * C, st);
    if (e == cudaSuccess && !g_mlp) e = dalloc(&g_mlp, s->mlp_floats, st);
    if (e == cudaSuccess) e = dalloc(&mlp_tmp, mlp_backward_tmp_floats(m, N, K), st);
    if (e == cudaSuccess && s->occ) {
      e = dalloc(&feat, static_cast<size_t>(N) * K, st);
      if (e == cudaSuccess) {
        launch_occ_probes(s->geom, K, rx, N, s->occ_res, s->occ_box, s->occ, feat, st);
        m.feat = feat;
      }
    }
    if (e != cudaSuccess) {
      cleanup();
      return fail(ctx, RXGS_E_OOM, "backward (MLP): %s", cudaGetErrorString(e));
    }
    Stage sg(ctx, "mlp_bwd", st);
    launch_mlp_backward(m, rx, N, s->geom, s->base, K, stride, d_rad, glob, g_base, g_mlp,
                        mlp_tmp, st);
    dfree(feat, st);
  }
  rs = check_last(ctx, "backward");
  cleanup();
  return rs;
}

int64_t rxgs_film_param_count(int nfreq, int embed, int hidden, int lmax) {
  if (nfreq < 1 || nfreq > kFilmMaxFreq || embed < 0 || embed > kFilmMaxEmbed || hidden < 1 ||
      hidden > kFilmMaxHidden || lmax < 0 || lmax > 9)
    return 0;
  return static_cast<int64_t>(film_dims(nfreq, embed, hidden, lmax).total);
}

rxgs_status rxgs_film_eval(rxgs_ctx* ctx, const float* film, int nfreq, int embed, int hidden,
                           int lmax, const float* rx, int N, float* ab, void* stream) {
  if (!ctx || !film || !rx || !ab) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (N <= 0 || N > (1 << 20)) return fail(ctx, RXGS_E_INVALID, "N out of range");
  if (rxgs_film_param_count(nfreq, embed, hidden, lmax) <= 0)
    return fail(ctx, RXGS_E_INVALID, "FiLM sizes out of range");
  CK(cudaSetDevice(ctx->device));
  launch_film_global(film, film_dims(nfreq, embed, hidden, lmax), rx, N,
                     reinterpret_cast<float4*>(ab), static_cast<cudaStream_t>(stream));
  return check_last(ctx, "film_eval");
}

rxgs_status rxgs_profile(rxgs_ctx* ctx, int enable) {
  if (!ctx) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->prof = enable != 0;
  return RXGS_OK;
}

rxgs_status rxgs_profile_read(rxgs_ctx* ctx, char* json, size_t cap, int reset) {
  if (!ctx || !json || cap == 0) return fail(ctx, RXGS_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  for (auto& p : ctx->pending) {
    CK(cudaEventSynchronize(p.b));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    auto& e = ctx->stage_ms[p.name];
    e.first += ms;
    e.second += 1;
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.clear();
  // allocation evidence: the library's stream-ordered allocations so far and
  // the device's default memory pool (which those allocations draw on)
  size_t used = 0, reserved = 0;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
    uint64_t u = 0, r = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &u) == cudaSuccess) used = u;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r) == cudaSuccess)
      reserved = r;
  }
  std::string out = "{\"kernel_launches\": " + std::to_string(launch_count()) +
                    ", \"device_allocs\": " + std::to_string(dalloc_count()) +
                    ", \"pool_used_bytes\": " + std::to_string(used) +
                    ", \"pool_reserved_bytes\": " + std::to_string(reserved) + ", \"stages\": {";
  bool first = true;
  for (auto& kv : ctx->stage_ms) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s\"%s\": {\"ms\": %.6f, \"calls\": %ld}", first ? "" : ", ",
             kv.first.c_str(), kv.second.first, kv.second.second);
    out += buf;
    first = false;
  }
  out += "}}";
  if (reset) ctx->stage_ms.clear();
  if (out.size() + 1 > cap) return fail(ctx, RXGS_E_INVALID, "buffer too small (%zu)", out.size() + 1);
  std::memcpy(json, out.c_str(), out.size() + 1);
  return RXGS_OK;
}

rxgs_status rxgs_l1_loss(rxgs_ctx* ctx, int kind, const float* values, const float* target,
                         size_t n, float* loss, float* grad, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  if (!values || !target || !loss || !grad) return fail(ctx, RXGS_E_INVALID, "l1_loss: null argument");
  if (kind != RXGS_OUT_SPECTRA && kind != RXGS_OUT_RSSI)
    return fail(ctx, RXGS_E_INVALID, "l1_loss: kind must be RXGS_OUT_SPECTRA or RXGS_OUT_RSSI");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nparts = l1_loss_blocks();
  float* part = nullptr;
  CK(dalloc(&part, static_cast<size_t>(nparts), st));
  launch_l1_loss(kind == RXGS_OUT_SPECTRA, values, target, n, loss, grad, part, nparts, st);
  dfree(part, st);
  return check_last(ctx, "l1_loss");
}

rxgs_status rxgs_sync(rxgs_ctx* ctx, void* stream) {
  if (!ctx) return RXGS_E_INVALID;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  unsigned h = 0;
  CK(cudaMemcpy(&h, ctx->d_err, sizeof h, cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(ctx->d_err, 0, sizeof(unsigned));
    return fail(ctx, RXGS_E_DEVICE, "device error word 0x%x", h);
  }
  return RXGS_OK;
}

}  // extern "C"
