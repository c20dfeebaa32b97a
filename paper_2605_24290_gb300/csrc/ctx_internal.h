// ctx_internal.h -- host-side state of a context (scenes, views, batch
// plans, serving) shared by the library's translation units.  Not part of
// the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rxgs.h"
#include "rxgs_internal.h"

namespace rxgs {

struct SceneState {
  int K = 0, C = 0;
  uint64_t generation = 0;  // bumped by rxgs_update_scene
  float4* geom = nullptr;   // [K][3]
  float* base = nullptr;    // [K][C][2]
  float* mlp = nullptr;     // flat
  size_t mlp_floats = 0;
  int hidden = 0, bf16 = 0;
  // occupancy grid of the local branch's occlusion inputs (null: clear)
  float* occ = nullptr;      // [res^3]
  float* occ_box = nullptr;  // lo[3], D[3]
  int occ_res = 0;
};

struct ViewsState {
  rxgs_scene_t scene = 0;
  int M = 0, K = 0;
  float* tx = nullptr;        // [M][3]
  float4* rec = nullptr;      // [M][K][2]
  uint32_t* depth = nullptr;  // [M][K]
  uint32_t* counts = nullptr; // [M*K] tile counts, view-major
  uint32_t* offsets = nullptr;// [M*K+1] scan of the counts in (view, depth) order
  uint32_t* keys = nullptr;   // [I] (view << tile_bits | tile), sorted
  uint32_t* vals = nullptr;   // [I]
  uint2* ranges = nullptr;    // [M][T]
  uint32_t n_inst = 0;
  int tile_bits = 0, view_bits = 0;
  // radiance of the last rxgs_render_views on these views, kept for the
  // backward: valid for the same rx pointer, N, radiance pointer and scene
  // generation
  float* rad = nullptr;
  float* glob = nullptr;
  const float* key_rx = nullptr;
  const float* key_radiance = nullptr;
  const float* key_fle = nullptr;   // fle_coeffs, or fle_base with the FiLM below
  const float* key_film = nullptr;
  int key_film_dims[3] = {0, 0, 0};
  int key_film_local = 0;
  int key_lmax = -1;
  int key_N = 0, key_stride = 0;
  uint64_t key_gen = ~0ull;
  // per-pixel final T and stop position and per-tile largest stop, written
  // by a tensor-core forward on these views (they depend on the views only),
  // so that the backward can skip its pre-pass
  float* tfin = nullptr;
  uint32_t* stops = nullptr;
  uint32_t* tile_stop = nullptr;
  bool stops_valid = false;
};

struct BatchPlan;    // batch.cu
struct ServeState;   // serve.cpp
void destroy_plan(BatchPlan* p);
void destroy_serve(ServeState* s);

}  // namespace rxgs

struct rxgs_ctx {
  int device = 0;
  rxgs_options opts{};
  rxgs::GridConst g{};
  std::mutex mu;
  std::string err;
  uint64_t next_id = 1;
  std::map<uint64_t, rxgs::SceneState*> scenes;
  std::map<uint64_t, rxgs::ViewsState*> views;
  std::vector<rxgs::BatchPlan*> plans;
  long plans_built = 0;           // batch plans built (graph captures) so far
  rxgs::ServeState* serve = nullptr;
  unsigned* d_err = nullptr;      // device error word
  uint32_t* h_pinned = nullptr;   // pinned readback slot
  cudaEvent_t ev_stats = nullptr;  // prepare: the readback slot is written
  uint32_t* d_pinned = nullptr;   // ... its device-side address (kernels write it)
  // stage profiler: CUDA events recorded on the call's stream around each
  // stage while enabled, folded into per-stage totals by rxgs_profile_read
  bool prof = false;
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::map<std::string, std::pair<double, long>> stage_ms;
  // device address of the allocation-free entry point's fixed scratch array
  // on `device` (noalloc.cu), taken when the context is created
  float* noalloc_partial = nullptr;
};

namespace rxgs {

inline rxgs_status fail(rxgs_ctx* c, rxgs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? RXGS_E_OOM : RXGS_E_CUDA,      \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// Number of stream-ordered device allocations the library has made (all
// render, backward and prepare scratch goes through dalloc).
void note_dalloc();
unsigned long long dalloc_count();

template <typename T>
cudaError_t dalloc(T** p, size_t n, cudaStream_t s) {
  if (n == 0) n = 1;
  note_dalloc();
  return cudaMallocAsync(reinterpret_cast<void**>(p), n * sizeof(T), s);
}

// Looks up (once per device, with that device current) the device address
// of the allocation-free entry point's scratch array (noalloc.cu).
cudaError_t noalloc_scratch_address(int device, float** out);

template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

inline int bits_for(uint64_t n) {  // bits to hold values 0..n-1
  int b = 0;
  while ((1ull << b) < n) ++b;
  return b;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

cudaEvent_t take_event(rxgs_ctx* c);

// Times one stage of a call on `stream` when the profiler is on.
struct Stage {
  rxgs_ctx* c;
  cudaStream_t s;
  std::string name;
  cudaEvent_t a = nullptr;
  Stage(rxgs_ctx* ctx, const char* n, cudaStream_t st) : c(ctx), s(st), name(n) {
    if (c->prof) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~Stage() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back({name, a, b});
    }
  }
};

int pick_cols(const rxgs_ctx* ctx, int ncols);

// rxgs_render_batched with a plan owner tag (serving slots own their plans)
// and the instance-capacity margin over the measured batch.
rxgs_status render_batched_tagged(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int B,
                                  const float* rx, const int32_t* rx_counts,
                                  const rxgs_render_desc* d, rxgs_outputs* out, void* stream,
                                  int tag, double inst_margin, const void** plan_used = nullptr);
void drop_plans(rxgs_ctx* ctx, int tag);
// Drops one plan (a batch overflowed its instance capacity); the caller has
// synchronised the stream the plan ran on.
void drop_plan(rxgs_ctx* ctx, const void* plan);

}  // namespace rxgs
