// serve.cpp -- continuous-batching request loop over a device-resident scene
// (rxgs_serve_*).
//
// Clients submit (transmitter, receiver set) queries of any size from any
// thread; a scheduler thread owned by the context admits queued requests in
// arrival order into the next free slot while the batch fits the slot's
// receiver/view capacity and the memory budget still has room next to the
// batches already on the GPU, renders the slot's batch with the batched
// pipeline (one CUDA graph replay per batch, on the slot's own stream), and
// moves on: with several slots, batches overlap on the device and requests
// that arrive meanwhile wait only for the next free slot.  Completions are
// detected with events; results are copied to pinned memory and handed to
// rxgs_serve_poll.  Latency = submit to completion, per request.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ctx_internal.h"

namespace rxgs {

using Clock = std::chrono::steady_clock;

struct ServeRequest {
  rxgs_ticket_t ticket = 0;
  float tx[3] = {0, 0, 0};
  std::vector<float> rx;  // [n][3]
  int n = 0;
  size_t bytes = 0;       // admission estimate
  Clock::time_point t_submit, t_done;
  int status = RXGS_E_NOT_READY;
  bool done = false;
  std::vector<float> out;
};

struct Slot {
  int tag = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  size_t bytes = 0;
  std::vector<ServeRequest*> reqs;
  std::vector<int32_t> counts;
  float *h_tx = nullptr, *h_rx = nullptr, *h_out = nullptr;  // pinned
  unsigned* h_err = nullptr;                                 // pinned
  float* d_out = nullptr;
  int cap_views = 0, cap_rx = 0, out_per_rx = 0;
  const void* plan = nullptr;  // the batch plan of the batch in flight
};

struct ServeState {
  rxgs_ctx* ctx = nullptr;
  rxgs_scene_t scene = 0;
  rxgs_serve_options o{};
  int K = 0, C = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeRequest*> queue;
  std::map<rxgs_ticket_t, ServeRequest*> reqs;
  rxgs_ticket_t next_ticket = 1;
  std::vector<Slot> slots;
  size_t inflight_bytes = 0;
  std::thread worker;
  bool stop = false;
  int fault_next = 0;  // test hook: fail the next N batches on the host
  // statistics
  std::vector<double> lat_ms;
  long batches = 0, batch_rx = 0, failed = 0, retried = 0, cancelled = 0;
  long plans_base = 0;  // ctx->plans_built at the last statistics reset
  Clock::time_point t_start;
};

static size_t estimate_bytes(const ServeState& s, int n) {
  // batches run the visibility path: per receiver its position, output and
  // per-chunk partial sums; per request (view) its projected records, tile
  // counts and offsets, (Gaussian, tile) instances with sort buffers (about
  // four tiles per Gaussian, keys and values twice) and its weights W
  const size_t per_rx = (static_cast<size_t>(s.K) / 4096 + 2) * 2 * s.C * 4 + 64;
  const size_t per_view = static_cast<size_t>(s.K) * (32 + 12 + 4 + 4 * 2 * 12);
  return static_cast<size_t>(n) * per_rx + per_view;
}

static void complete_slot(ServeState* S, Slot& sl, bool ok) {
  // caller holds S->mu
  const Clock::time_point now = Clock::now();
  size_t off = 0;
  for (ServeRequest* r : sl.reqs) {
    const size_t cnt = static_cast<size_t>(r->n) * sl.out_per_rx;
    if (ok) {
      r->out.assign(sl.h_out + off, sl.h_out + off + cnt);
      r->status = RXGS_OK;
      S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
    } else {
      r->status = RXGS_E_DEVICE;
      S->failed++;
    }
    r->t_done = now;
    r->done = true;
    off += cnt;
  }
  S->inflight_bytes -= sl.bytes;
  sl.bytes = 0;
  sl.busy = false;
  sl.reqs.clear();
  S->cv_done.notify_all();
}

static void worker_main(ServeState* S) {
  rxgs_ctx* ctx = S->ctx;
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    // ---- completions
    for (Slot& sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        complete_slot(S, sl, false);
        continue;
      }
      if (*sl.h_err & kErrCapacity) {
        // the batch overflowed its plan's instance capacity: grow and retry
        *sl.h_err = 0;
        cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), sl.st);
        cudaStreamSynchronize(sl.st);
        lk.unlock();
        drop_plan(ctx, sl.plan);  // only the plan that overflowed is rebuilt
        lk.lock();
        sl.plan = nullptr;
        for (auto it = sl.reqs.rbegin(); it != sl.reqs.rend(); ++it) S->queue.push_front(*it);
        S->retried += static_cast<long>(sl.reqs.size());
        S->inflight_bytes -= sl.bytes;
        sl.bytes = 0;
        sl.busy = false;
        sl.reqs.clear();
        continue;
      }
      complete_slot(S, sl, true);
    }
    // ---- admission into a free slot
    Slot* free_slot = nullptr;
    for (Slot& sl : S->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    if (!free_slot || S->queue.empty()) {
      bool any_busy = false;
      for (Slot& sl : S->slots) any_busy |= sl.busy;
      // poll completions every 50 us while work is on the GPU, else sleep
      S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 2000));
      continue;
    }
    Slot& sl = *free_slot;
    int nrx = 0;
    size_t bytes = 0;
    while (!S->queue.empty() && static_cast<int>(sl.reqs.size()) < sl.cap_views) {
      ServeRequest* r = S->queue.front();
      if (nrx + r->n > sl.cap_rx) break;
      if (!sl.reqs.empty() && S->inflight_bytes + bytes + r->bytes > S->o.mem_budget) break;
      if (sl.reqs.empty() && S->inflight_bytes + r->bytes > S->o.mem_budget &&
          S->inflight_bytes > 0)
        break;  // wait for memory to free up
      S->queue.pop_front();
      sl.reqs.push_back(r);
      nrx += r->n;
      bytes += r->bytes;
    }
    if (sl.reqs.empty()) {
      S->cv_work.wait_for(lk, std::chrono::microseconds(50));
      continue;
    }
    sl.counts.clear();
    int off = 0;
    for (size_t b = 0; b < sl.reqs.size(); ++b) {
      ServeRequest* r = sl.reqs[b];
      std::memcpy(sl.h_tx + 3 * b, r->tx, sizeof(float) * 3);
      std::memcpy(sl.h_rx + 3 * off, r->rx.data(), sizeof(float) * 3 * r->n);
      sl.counts.push_back(r->n);
      off += r->n;
    }
    sl.bytes = bytes;
    S->inflight_bytes += bytes;
    sl.busy = true;
    S->batches++;
    S->batch_rx += nrx;
    const bool inject = S->fault_next > 0;
    if (inject) S->fault_next--;
    lk.unlock();
    rxgs_status st = RXGS_E_CUDA;
    if (!inject) {
      rxgs_render_desc d{};
      d.kind = S->o.kind;
      d.reduce_path = 1;  // CSI / RSSI through visibility weights
      rxgs_outputs out{};
      if (S->o.kind == RXGS_OUT_RSSI)
        out.rssi = sl.d_out;
      else
        out.csi = sl.d_out;
      st = render_batched_tagged(ctx, S->scene, sl.h_tx, static_cast<int>(sl.reqs.size()), sl.h_rx,
                                 sl.counts.data(), &d, &out, sl.st, sl.tag, 2.0, &sl.plan);
      if (st == RXGS_OK) {
        cudaMemcpyAsync(sl.h_out, sl.d_out, sizeof(float) * static_cast<size_t>(nrx) * sl.out_per_rx,
                        cudaMemcpyDeviceToHost, sl.st);
        cudaMemcpyAsync(sl.h_err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, sl.st);
        cudaEventRecord(sl.ev, sl.st);
      }
    }
    lk.lock();
    if (st != RXGS_OK) complete_slot(S, sl, false);
  }
  // drain: wait for batches in flight
  for (Slot& sl : S->slots)
    if (sl.busy) {
      cudaEventSynchronize(sl.ev);
      complete_slot(S, sl, !(*sl.h_err & kErrCapacity));
    }
}

void destroy_serve(ServeState* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (Slot& sl : S->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
    cudaFreeHost(sl.h_tx);
    cudaFreeHost(sl.h_rx);
    cudaFreeHost(sl.h_out);
    cudaFreeHost(sl.h_err);
    cudaFree(sl.d_out);
  }
  for (auto& kv : S->reqs) delete kv.second;
  for (const Slot& sl : S->slots) drop_plans(S->ctx, sl.tag);
  delete S;
}

}  // namespace rxgs

using namespace rxgs;

extern "C" {

void rxgs_serve_default_options(rxgs_serve_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->kind = RXGS_OUT_RSSI;
  o->max_batch_receivers = 4096;
  o->max_batch_views = 64;
  o->mem_budget = 16ull << 30;
  o->slots = 2;
}

rxgs_status rxgs_serve_start(rxgs_ctx* ctx, rxgs_scene_t scene, const rxgs_serve_options* opts) {
  if (!ctx) return RXGS_E_INVALID;
  rxgs_serve_options o;
  if (opts)
    o = *opts;
  else
    rxgs_serve_default_options(&o);
  if (o.kind != RXGS_OUT_RSSI && o.kind != RXGS_OUT_CSI)
    return fail(ctx, RXGS_E_INVALID, "serving returns RSSI or CSI");
  if (o.max_batch_receivers < 1 || o.max_batch_views < 1 || o.slots < 1 || o.slots > 8 ||
      o.mem_budget == 0)
    return fail(ctx, RXGS_E_INVALID, "bad serving options");
  SceneState* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serve) return fail(ctx, RXGS_E_INVALID, "serving already started");
    auto it = ctx->scenes.find(scene);
    if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
    s = it->second;
  }
  if (!s->mlp) return fail(ctx, RXGS_E_INVALID, "serving needs a scene with a conditioning MLP");
  if (s->occ) return fail(ctx, RXGS_E_INVALID, "serving does not take occlusion inputs (occupancy grid)");
  if (o.kind == RXGS_OUT_RSSI && s->C != 1) return fail(ctx, RXGS_E_INVALID, "RSSI needs C == 1");
  CK(cudaSetDevice(ctx->device));
  ServeState* S = new ServeState();
  S->ctx = ctx;
  S->scene = scene;
  S->o = o;
  S->K = s->K;
  S->C = s->C;
  S->t_start = Clock::now();
  const int out_per_rx = o.kind == RXGS_OUT_RSSI ? 1 : 2 * s->C;
  S->slots.resize(o.slots);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < o.slots; ++i) {
    Slot& sl = S->slots[i];
    sl.tag = 1000 + i;
    sl.cap_views = o.max_batch_views;
    sl.cap_rx = o.max_batch_receivers;
    sl.out_per_rx = out_per_rx;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_tx, sizeof(float) * 3 * sl.cap_views);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_rx, sizeof(float) * 3 * sl.cap_rx);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_out, sizeof(float) * out_per_rx * sl.cap_rx);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.h_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, sizeof(float) * out_per_rx * sl.cap_rx);
    if (sl.h_err) *sl.h_err = 0;
  }
  if (e != cudaSuccess) {
    destroy_serve(S);
    return fail(ctx, RXGS_E_OOM, "serving buffers: %s", cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->serve = S;
  }
  S->worker = std::thread(worker_main, S);
  return RXGS_OK;
}

rxgs_status rxgs_serve_submit(rxgs_ctx* ctx, const float* tx, const float* rx, int n,
                              rxgs_ticket_t* ticket) {
  if (!ctx || !tx || !rx || !ticket || n <= 0) return fail(ctx, RXGS_E_INVALID, "bad request");
  ServeState* S = ctx->serve;
  if (!S) return fail(ctx, RXGS_E_INVALID, "serving not started");
  if (n > S->o.max_batch_receivers)
    return fail(ctx, RXGS_E_ADMISSION, "request of %d receivers exceeds the batch capacity %d", n,
                S->o.max_batch_receivers);
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(tx[a])) return fail(ctx, RXGS_E_INVALID, "non-finite transmitter");
  for (int q = 0; q < 3 * n; ++q)
    if (!std::isfinite(rx[q])) return fail(ctx, RXGS_E_INVALID, "non-finite receiver");
  const size_t bytes = estimate_bytes(*S, n);
  if (bytes > S->o.mem_budget)
    return fail(ctx, RXGS_E_ADMISSION, "request needs ~%zu bytes, budget is %zu", bytes,
                S->o.mem_budget);
  ServeRequest* r = new ServeRequest();
  std::memcpy(r->tx, tx, sizeof r->tx);
  r->rx.assign(rx, rx + 3 * static_cast<size_t>(n));
  r->n = n;
  r->bytes = bytes;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
  }
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return RXGS_OK;
}

rxgs_status rxgs_serve_poll(rxgs_ctx* ctx, rxgs_ticket_t ticket, float* out, int timeout_us) {
  if (!ctx) return RXGS_E_INVALID;
  ServeState* S = ctx->serve;
  if (!S) return fail(ctx, RXGS_E_INVALID, "serving not started");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(ctx, RXGS_E_INVALID, "unknown ticket");
  ServeRequest* r = it->second;
  if (!r->done && timeout_us != 0) {
    auto pred = [&] { return r->done; };
    if (timeout_us < 0)
      S->cv_done.wait(lk, pred);
    else
      S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
  }
  if (!r->done) return timeout_us == 0 ? RXGS_E_NOT_READY : RXGS_E_TIMEOUT;
  const int st = r->status;
  if (st == RXGS_OK && out) std::memcpy(out, r->out.data(), sizeof(float) * r->out.size());
  S->reqs.erase(it);
  delete r;
  if (st != RXGS_OK) return fail(ctx, static_cast<rxgs_status>(st), "request failed on the device");
  return RXGS_OK;
}

rxgs_status rxgs_serve_cancel(rxgs_ctx* ctx, rxgs_ticket_t ticket) {
  if (!ctx || !ctx->serve) return RXGS_E_INVALID;
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(ctx, RXGS_E_INVALID, "unknown ticket");
  ServeRequest* r = it->second;
  auto q = std::find(S->queue.begin(), S->queue.end(), r);
  if (q == S->queue.end()) return fail(ctx, RXGS_E_NOT_READY, "request already on the GPU");
  S->queue.erase(q);
  r->status = RXGS_E_CANCELLED;
  r->done = true;
  S->cancelled++;
  S->cv_done.notify_all();
  return RXGS_OK;
}

rxgs_status rxgs_serve_stats(rxgs_ctx* ctx, char* json, size_t cap) {
  if (!ctx || !json || !ctx->serve) return RXGS_E_INVALID;
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat_ms;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) {
    if (v.empty()) return 0.0;
    const size_t i = std::min(v.size() - 1, static_cast<size_t>(std::ceil(p * v.size())) - 1);
    return v[i];
  };
  const double el = std::chrono::duration<double>(Clock::now() - S->t_start).count();
  const double mean = v.empty() ? 0.0 : std::accumulate(v.begin(), v.end(), 0.0) / v.size();
  long built = 0;
  {
    std::lock_guard<std::mutex> lc(ctx->mu);
    built = ctx->plans_built - S->plans_base;
  }
  char buf[800];
  snprintf(buf, sizeof buf,
           "{\"completed\": %zu, \"failed\": %ld, \"retried\": %ld, \"cancelled\": %ld, "
           "\"plans_built\": %ld, "
           "\"batches\": %ld, \"mean_batch_receivers\": %.2f, \"p50_ms\": %.4f, \"p90_ms\": %.4f, "
           "\"p99_ms\": %.4f, \"max_ms\": %.4f, \"mean_ms\": %.4f, \"queued\": %zu, "
           "\"inflight_bytes\": %zu, \"elapsed_s\": %.3f}",
           v.size(), S->failed, S->retried, S->cancelled, built, S->batches,
           S->batches ? static_cast<double>(S->batch_rx) / S->batches : 0.0, pct(0.5), pct(0.9),
           pct(0.99), v.empty() ? 0.0 : v.back(), mean, S->queue.size(), S->inflight_bytes, el);
  if (strlen(buf) + 1 > cap) return RXGS_E_INVALID;
  std::memcpy(json, buf, strlen(buf) + 1);
  return RXGS_OK;
}

rxgs_status rxgs_serve_reset_stats(rxgs_ctx* ctx) {
  if (!ctx || !ctx->serve) return RXGS_E_INVALID;
  ServeState* S = ctx->serve;
  std::lock_guard<std::mutex> lk(S->mu);
  S->lat_ms.clear();
  S->batches = S->batch_rx = S->failed = S->retried = S->cancelled = 0;
  {
    std::lock_guard<std::mutex> lc(ctx->mu);
    S->plans_base = ctx->plans_built;
  }
  S->t_start = Clock::now();
  return RXGS_OK;
}

rxgs_status rxgs_serve_inject_fault(rxgs_ctx* ctx, int batches) {
  if (!ctx || !ctx->serve || batches < 0) return RXGS_E_INVALID;
  std::lock_guard<std::mutex> lk(ctx->serve->mu);
  ctx->serve->fault_next = batches;
  return RXGS_OK;
}

rxgs_status rxgs_serve_stop(rxgs_ctx* ctx) {
  if (!ctx || !ctx->serve) return RXGS_E_INVALID;
  ServeState* S = ctx->serve;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->serve = nullptr;
  }
  destroy_serve(S);
  return RXGS_OK;
}

}  // extern "C"
