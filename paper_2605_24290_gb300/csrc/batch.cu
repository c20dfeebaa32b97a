// batch.cu -- uneven receiver batches in one persistent launch under a CUDA
// graph (rxgs_render_batched, rxgs_autotune).
//
// A batch is B transmitters (views), each with its own receivers (ragged
// counts).  A plan owns fixed-capacity device buffers for up to B_max views,
// R_max receivers and I_cap (Gaussian, tile) instances, and a CUDA graph of
// the whole pipeline captured once:
//   preprocess (view slots >= B culled) -> scan -> emit (capacity-checked) ->
//   radix sort and tile ranges on the device-side instance count -> radiance
//   (MLP or a transpose of the given radiance, into per-view column groups) ->
//   ONE persistent render launch whose CTAs take (view, tile, column block)
//   jobs from an atomic counter -> per-receiver reduction to CSI / RSSI.
// Every size a kernel needs is read from a device descriptor the host fills
// per batch, so one graph serves every batch within the capacities; the
// host copies tx/rx/descriptor in, launches the graph and copies outputs out.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx_internal.h"
#include "render_common.cuh"
#include "render_tile.cuh"
#include "rxgs_internal.h"

namespace rxgs {

// Device descriptor layout (int32):
//   [0] nviews   [1] nrx   [2] njobs   [3] ncols_total (padded)
//   rx_off[B_max+1], colbase[B_max+1], job_off[B_max+1], rx_view[R_max], col_of[R_max]
struct DescLayout {
  int B, R;
  __host__ __device__ int rx_off() const { return 4; }
  __host__ __device__ int colbase() const { return 4 + (B + 1); }
  __host__ __device__ int job_off() const { return 4 + 2 * (B + 1); }
  __host__ __device__ int rx_view() const { return 4 + 3 * (B + 1); }
  __host__ __device__ int col_of() const { return 4 + 3 * (B + 1) + R; }
  __host__ __device__ int size() const { return 4 + 3 * (B + 1) + 2 * R; }
};

struct BatchPlan {
  rxgs_scene_t scene = 0;
  int tag = 0;  // owner (0 = rxgs_render_batched, >0 = a serving slot)
  int B_max = 0, R_max = 0, C = 0, NB = 64, kind = 0;
  bool mlp = false;
  bool vis = false;  // CSI / RSSI through visibility weights (MLP radiance)
  float* W = nullptr;       // [B_max][K]
  float* wtmp = nullptr;    // chunk partial sums
  uint32_t I_cap = 0;
  int cols_cap = 0, stride = 0;
  int tile_bits = 0, view_bits = 0;
  GridConst g{};
  DescLayout L{};
  // device buffers
  float *tx = nullptr, *rx = nullptr, *rad_in = nullptr, *rad = nullptr, *glob = nullptr;
  int* desc = nullptr;
  float4* rec = nullptr;
  uint32_t *depth = nullptr, *counts = nullptr, *offsets = nullptr, *scan_tmp = nullptr;
  // the depth order of every view slot's Gaussians: key and index buffers,
  // sort scratch, the tile counts in that order
  uint32_t *dkeys = nullptr, *dkeys_alt = nullptr, *ord_a = nullptr, *ord_b = nullptr;
  uint32_t *dsort_tmp = nullptr, *scounts = nullptr;
  uint32_t *keys = nullptr, *keys_alt = nullptr;  // (view << tile_bits | tile)
  uint32_t *vals = nullptr, *vals_alt = nullptr, *sort_tmp = nullptr;
  uint2* ranges = nullptr;
  float *partial = nullptr, *spectra = nullptr, *csi = nullptr, *rssi = nullptr;
  unsigned* counter = nullptr;
  bool sorted_in_alt = false;
  // host staging (pinned)
  int* h_desc = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  cudaEvent_t desc_done = nullptr;  // the pinned descriptor has been copied
  size_t bytes = 0;
};

void destroy_plan(BatchPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  if (p->desc_done) cudaEventDestroy(p->desc_done);
  void* bufs[] = {p->tx, p->rx, p->rad_in, p->rad, p->glob, p->desc, p->rec, p->depth,
                  p->counts, p->offsets, p->scan_tmp, p->dkeys, p->dkeys_alt, p->ord_a,
                  p->ord_b, p->dsort_tmp, p->scounts, p->keys, p->keys_alt, p->vals,
                  p->vals_alt, p->sort_tmp, p->ranges, p->partial, p->spectra, p->csi,
                  p->rssi, p->counter, p->W, p->wtmp};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->h_desc) cudaFreeHost(p->h_desc);
  delete p;
}

// ------------------------------------------------------------------ kernels
// Receiver-major [R][K][C][2] -> Gaussian-major rows with per-receiver
// column starts col_of[j]; pad columns are zero (the buffer is cleared).
__global__ void batch_transpose_kernel(const float* __restrict__ in, int R_max, int K, int C,
                                       int stride, const int* __restrict__ desc, int col_of_off,
                                       float* __restrict__ out) {
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int twoC = 2 * C;
  const int nrx = desc[1];
  if (idx >= static_cast<size_t>(nrx) * K * twoC) return;
  const int e = static_cast<int>(idx % twoC);
  const size_t jk = idx / twoC;
  const int k = static_cast<int>(jk % K), j = static_cast<int>(jk / K);
  out[static_cast<size_t>(k) * stride + desc[col_of_off + j] + e] = in[idx];
}

// Persistent render: CTAs take (view, tile, column block) jobs in order from
// an atomic counter until the batch's jobs are done.
template <int NB>
__global__ void __launch_bounds__(kTilePixels, NB >= 128 ? 1 : 2)
    batch_render_kernel(const RenderArgs a, const int* __restrict__ desc, DescLayout L,
                        unsigned* __restrict__ counter, int cols_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);
  float* sR = sA + kChunk * kTilePixels;
  float4* sRec = reinterpret_cast<float4*>(sR + 2 * kChunk * NB);
  __shared__ float sRed[kTilePixels / 32][8];
  __shared__ int sJob;
  const int nviews = desc[0];
  const int njobs = desc[2];
  const int* rx_off = desc + L.rx_off();
  const int* colbase = desc + L.colbase();
  const int* job_off = desc + L.job_off();
  const int T = a.g.T;
  for (;;) {
    __syncthreads();  // the previous job is done with sJob and shared memory
    if (threadIdx.x == 0) sJob = static_cast<int>(atomicAdd(counter, 1u));
    __syncthreads();
    const int item = sJob;
    if (item >= njobs) break;
    int lo = 0, hi = nviews;  // find v with job_off[v] <= item < job_off[v+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (job_off[mid] <= item) lo = mid; else hi = mid;
    }
    const int v = lo;
    const int nrx_v = rx_off[v + 1] - rx_off[v];
    const int ncols_v = 2 * nrx_v * a.C;
    const int ncb = (ncols_v + NB - 1) / NB;
    const int local = item - job_off[v];
    TileJob job;
    job.v = v;
    job.tile = local / ncb;
    job.col0 = (local % ncb) * NB;
    job.col_base = colbase[v];
    job.ncols_v = ncols_v;
    job.out_rx0 = rx_off[v];
    job.partial_row = a.partial ? a.partial + static_cast<size_t>(job.tile) * cols_cap + colbase[v]
                                : nullptr;
    (void)T;
    render_tile<NB>(a, job, sA, sR, sRec, sRed);
  }
}

// csi[j][c] = sum over tiles of partial[t][col_of[j] + 2c .. +1]; rssi = |csi|.
__global__ void batch_reduce_kernel(const float* __restrict__ partial, int T, int cols_cap, int C,
                                    const int* __restrict__ desc, int col_of_off,
                                    float* __restrict__ csi, float* __restrict__ rssi) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // (j, c)
  const int nrx = desc[1];
  if (idx >= nrx * C) return;
  const int j = idx / C, c = idx % C;
  const float* p = partial + desc[col_of_off + j] + 2 * c;
  float re = 0.0f, im = 0.0f;
  for (int t = 0; t < T; ++t) {
    re += p[static_cast<size_t>(t) * cols_cap];
    im += p[static_cast<size_t>(t) * cols_cap + 1];
  }
  if (csi) {
    csi[2 * static_cast<size_t>(idx)] = re;
    csi[2 * static_cast<size_t>(idx) + 1] = im;
  }
  if (rssi && C == 1) rssi[j] = sqrtf(re * re + im * im);
}

template <int NB>
static void launch_batch_render(const RenderArgs& a, const int* desc, const DescLayout& L,
                                unsigned* counter, int cols_cap, cudaStream_t s) {
  constexpr size_t smem = FwdShape<NB>::smem;
  cudaFuncSetAttribute(batch_render_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_render_kernel<NB>, kTilePixels,
                                                smem);
  const int grid = sms * std::max(1, per_sm);
  batch_render_kernel<NB><<<grid, kTilePixels, smem, s>>>(a, desc, L, counter, cols_cap);
  note_launches(1);
}

// ------------------------------------------------------------ plan set-up
static size_t plan_bytes(const BatchPlan& p, int K) {
  const size_t MK = static_cast<size_t>(p.B_max) * K;
  size_t b = 0;
  b += sizeof(float4) * 2 * MK + 3 * sizeof(uint32_t) * MK;
  b += 5 * sizeof(uint32_t) * MK;  // depth-order keys and indices (x2), counts in that order
  b += 2 * sizeof(uint32_t) * 2ull * p.I_cap;
  b += sizeof(float) * static_cast<size_t>(K) * p.stride;
  b += sizeof(float) * static_cast<size_t>(p.g.T) * p.cols_cap;
  if (p.kind & RXGS_OUT_SPECTRA)
    b += sizeof(float) * static_cast<size_t>(p.R_max) * p.g.H * p.g.W * 2 * p.C;
  if (!p.mlp) b += sizeof(float) * static_cast<size_t>(p.R_max) * K * 2 * p.C;
  return b;
}

static rxgs_status build_plan(rxgs_ctx* ctx, const SceneState* s, BatchPlan* p) {
  const int K = s->K, C = s->C;
  const GridConst& g = p->g;
  const size_t MK = static_cast<size_t>(p->B_max) * K;
  p->L = DescLayout{p->B_max, p->R_max};
  // every view's column group starts on a multiple of 4 floats (16 B)
  p->cols_cap = round_up(2 * p->R_max * C + 4 * p->B_max, 4);
  p->stride = round_up(p->cols_cap, 128) + 128;
  p->tile_bits = bits_for(static_cast<uint64_t>(g.T));
  p->view_bits = bits_for(static_cast<uint64_t>(p->B_max));
  if (p->tile_bits + p->view_bits > 32)
    return fail(ctx, RXGS_E_INVALID, "too many views x tiles for a 32-bit (view, tile) key");
  p->bytes = plan_bytes(*p, K);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** ptr, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(ptr), std::max<size_t>(n, 1) * sizeof(**ptr));
  };
  A(&p->tx, 3ull * p->B_max);
  A(&p->rx, 3ull * p->R_max);
  A(&p->desc, static_cast<size_t>(p->L.size()));
  A(&p->rec, 2 * MK);
  A(&p->depth, MK);
  A(&p->counts, MK);
  A(&p->offsets, MK + 1);
  A(&p->scan_tmp, scan_tmp_words(MK));
  A(&p->dkeys, MK);
  A(&p->dkeys_alt, MK);
  A(&p->ord_a, MK);
  A(&p->ord_b, MK);
  A(&p->dsort_tmp, radix_segments_tmp_words(K, p->B_max));
  A(&p->scounts, MK);
  A(&p->keys, p->I_cap);
  A(&p->keys_alt, p->I_cap);
  A(&p->vals, p->I_cap);
  A(&p->vals_alt, p->I_cap);
  A(&p->sort_tmp, p->tile_bits <= 9 ? radix_views_tmp_words(p->I_cap, p->B_max)
                                    : radix_tmp_words(p->I_cap));
  A(&p->ranges, static_cast<size_t>(p->B_max) * g.T);
  if (p->vis) {
    A(&p->W, static_cast<size_t>(p->B_max) * K);
    A(&p->wtmp, mlp_weighted_tmp_floats(1, K, p->R_max, C));
  } else {
    A(&p->rad, static_cast<size_t>(K) * p->stride);
    A(&p->partial, static_cast<size_t>(g.T) * p->cols_cap);
  }
  A(&p->counter, 1);
  if (p->mlp)
    A(&p->glob, static_cast<size_t>(p->R_max) * 4 * C);
  else
    A(&p->rad_in, static_cast<size_t>(p->R_max) * K * 2 * C);
  if (p->kind & RXGS_OUT_SPECTRA) A(&p->spectra, static_cast<size_t>(p->R_max) * g.H * g.W * 2 * C);
  A(&p->csi, static_cast<size_t>(p->R_max) * 2 * C);
  A(&p->rssi, static_cast<size_t>(p->R_max));
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_desc, sizeof(int) * p->L.size());
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->desc_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(p->desc_done, p->cap);
  if (e != cudaSuccess)
    return fail(ctx, e == cudaErrorMemoryAllocation ? RXGS_E_OOM : RXGS_E_CUDA,
                "batch plan buffers (%.1f MB): %s", p->bytes / 1e6, cudaGetErrorString(e));
  // ---- capture the pipeline
  cudaStream_t st = p->cap;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(ctx, RXGS_E_CUDA, "capture: %s", cudaGetErrorString(e));
  const int* nviews_dev = p->desc;
  launch_preprocess(g, s->geom, K, p->tx, p->B_max, p->rec, p->depth, p->counts, st, nviews_dev);
  // the per-tile lists as in prepare: every view slot's Gaussians by depth
  // (all 31 bits: nothing is read back inside the graph), the instances
  // emitted in that order (none past the capacity), then one stable pass by
  // tile within each view's run, which writes the ranges
  radix_sort_segments_first(p->depth, K, p->B_max, p->dkeys, p->ord_a, p->dsort_tmp, st);
  const uint32_t* ord = radix_sort_segments_rest(K, p->B_max, 31, 0u, p->dkeys, p->dkeys_alt,
                                                 p->ord_a, p->ord_b, p->dsort_tmp, p->counts,
                                                 p->scounts, st);
  launch_exclusive_scan(p->scounts, p->offsets, MK, p->scan_tmp, st);
  launch_emit_sorted(g, p->rec, ord, p->offsets, MK, K, p->tile_bits, p->keys, p->vals, st,
                     p->I_cap, ctx->d_err);
  const uint32_t* n_dev = p->offsets + MK;
  bool in_alt = true;
  if (p->tile_bits <= 9) {
    radix_sort_views(p->keys, p->vals, p->keys_alt, p->vals_alt, p->I_cap, p->offsets, K,
                     p->B_max, p->tile_bits, p->ranges, g.T, p->sort_tmp, st);
  } else {
    radix_sort_pairs(p->keys, p->vals, p->keys_alt, p->vals_alt, p->I_cap,
                     p->tile_bits + p->view_bits, p->sort_tmp, &in_alt, st, n_dev, ctx->d_err);
    launch_tile_ranges(in_alt ? p->keys_alt : p->keys, p->I_cap, p->tile_bits, g.T, p->ranges,
                       p->B_max, st, n_dev);
  }
  p->sorted_in_alt = in_alt;
  uint32_t* vals = in_alt ? p->vals_alt : p->vals;
  if (p->vis) {
    // CSI / RSSI = sum_k W[v(j)][k] s(j, k): one receiver-independent pass
    // per view, then the MLP evaluated only where the weight is non-zero
    RenderArgs va{};
    va.g = g;
    va.rec = p->rec;
    va.vals = in_alt ? p->vals_alt : p->vals;
    va.ranges = p->ranges;
    va.K = K;
    va.M = p->B_max;
    launch_visibility(va, p->W, st);
    MlpParams m{s->mlp, s->hidden, C, s->bf16};
    launch_mlp_global(m, p->rx, p->R_max, p->glob, st, p->desc + 1);
    launch_mlp_weighted(m, p->rx, p->R_max, s->geom, s->base, K, p->W, p->B_max,
                        p->desc + p->L.rx_view(), p->glob, p->wtmp, p->csi,
                        C == 1 ? p->rssi : nullptr, p->desc + 1, st);
    e = cudaStreamEndCapture(st, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, RXGS_E_CUDA, "graph: %s", cudaGetErrorString(e));
    return RXGS_OK;
  }
  // no clearing of the radiance: a column block may read columns past its
  // view's last one, but those only feed accumulators that are never stored
  if (p->mlp) {
    MlpParams m{s->mlp, s->hidden, C, s->bf16};
    launch_mlp_radiance(m, p->rx, p->R_max, s->geom, s->base, K, p->stride, p->rad, p->glob, st,
                        p->desc + 1, p->desc + p->L.col_of(), false);
  } else {
    const size_t n = static_cast<size_t>(p->R_max) * K * 2 * C;
    batch_transpose_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
        p->rad_in, p->R_max, K, C, p->stride, p->desc, p->L.col_of(), p->rad);
    note_launches(1);
  }
  cudaMemsetAsync(p->counter, 0, sizeof(unsigned), st);
  RenderArgs a{};
  a.g = g;
  a.rec = p->rec;
  a.vals = vals;
  a.ranges = p->ranges;
  a.rad = p->rad;
  a.K = K;
  a.M = p->B_max;
  a.N = 0;
  a.C = C;
  a.stride = p->stride;
  a.ncols = 0;
  a.spectra = p->spectra;
  a.partial = (p->kind & (RXGS_OUT_CSI | RXGS_OUT_RSSI)) ? p->partial : nullptr;
  switch (p->NB) {
    case 16: launch_batch_render<16>(a, p->desc, p->L, p->counter, p->cols_cap, st); break;
    case 32: launch_batch_render<32>(a, p->desc, p->L, p->counter, p->cols_cap, st); break;
    case 128: launch_batch_render<128>(a, p->desc, p->L, p->counter, p->cols_cap, st); break;
    default: launch_batch_render<64>(a, p->desc, p->L, p->counter, p->cols_cap, st); break;
  }
  if (a.partial) {
    const int n = p->R_max * C;
    batch_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(p->partial, g.T, p->cols_cap, C, p->desc,
                                                         p->L.col_of(), p->csi,
                                                         C == 1 ? p->rssi : nullptr);
    note_launches(1);
  }
  e = cudaStreamEndCapture(st, &graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(ctx, RXGS_E_CUDA, "graph: %s", cudaGetErrorString(e));
  return RXGS_OK;
}

// Host-side descriptor of one batch: view offsets, 16-byte aligned column
// groups, job prefix, receiver -> view and receiver -> first column.
static void fill_desc(const BatchPlan& p, int B, const int32_t* counts, int* d) {
  const DescLayout& L = p.L;
  std::memset(d, 0, sizeof(int) * L.size());
  int R = 0, col = 0, jobs = 0;
  for (int v = 0; v < B; ++v) {
    d[L.rx_off() + v] = R;
    d[L.colbase() + v] = col;
    d[L.job_off() + v] = jobs;
    const int ncols_v = 2 * counts[v] * p.C;
    for (int q = 0; q < counts[v]; ++q) {
      d[L.rx_view() + R + q] = v;
      d[L.col_of() + R + q] = col + 2 * p.C * q;
    }
    R += counts[v];
    col = round_up(col + ncols_v, 4);
    jobs += p.g.T * ((ncols_v + p.NB - 1) / p.NB);
  }
  d[L.rx_off() + B] = R;
  d[L.colbase() + B] = col;
  d[L.job_off() + B] = jobs;
  d[0] = B;
  d[1] = R;
  d[2] = jobs;
  d[3] = col;
}

static int next_pow2(int x, int lo) {
  int p = lo;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace rxgs

using namespace rxgs;

// Builds a plan for (scene, kind, radiance mode) holding B views, R
// receivers and inst_need instances.
static rxgs_status new_plan(rxgs_ctx* ctx, rxgs_scene_t scene, const SceneState* s, int kind,
                            bool mlp, bool vis, int B, int R, uint32_t inst_need, int tag,
                            BatchPlan** out) {
  BatchPlan* p = new BatchPlan();
  p->scene = scene;
  p->tag = tag;
  p->vis = vis;
  p->kind = kind;
  p->mlp = mlp;
  p->C = s->C;
  p->B_max = next_pow2(B, 4);
  p->R_max = next_pow2(R, 32);
  p->I_cap = std::max<uint32_t>(inst_need, 1u << 16);
  p->g = ctx->g;
  p->NB = ctx->opts.cols_per_cta ? ctx->opts.cols_per_cta : 64;
  rxgs_status st = build_plan(ctx, s, p);
  if (st != RXGS_OK) {
    destroy_plan(p);
    return st;
  }
  ctx->plans.push_back(p);
  ctx->plans_built++;
  *out = p;
  return RXGS_OK;
}

// The smallest existing plan that fits, so launch sizes stay within 2x of
// the batch (plans come in power-of-two size classes of views and receivers).
static BatchPlan* find_plan(rxgs_ctx* ctx, rxgs_scene_t scene, int kind, bool mlp, bool vis, int B,
                            int R, int tag) {
  const int NB = ctx->opts.cols_per_cta ? ctx->opts.cols_per_cta : 64;
  const int Bc = next_pow2(B, 4), Rc = next_pow2(R, 32);
  BatchPlan* best = nullptr;
  for (BatchPlan* q : ctx->plans)
    if (q->scene == scene && q->tag == tag && q->kind == kind && q->mlp == mlp && q->vis == vis &&
        q->B_max >= B && q->R_max >= R && q->B_max <= 2 * Bc && q->R_max <= 2 * Rc &&
        q->g.TH == ctx->g.TH && q->g.TW == ctx->g.TW && q->NB == NB &&
        (!best || static_cast<size_t>(q->B_max) * q->R_max <
                      static_cast<size_t>(best->B_max) * best->R_max))
      best = q;
  return best;
}

// Drops the plans of one owner (after a capacity overflow, to grow them).
void rxgs::drop_plans(rxgs_ctx* ctx, int tag) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::vector<BatchPlan*> keep;
  for (BatchPlan* q : ctx->plans) {
    if (q->tag == tag) {
      cudaDeviceSynchronize();
      destroy_plan(q);
    } else {
      keep.push_back(q);
    }
  }
  ctx->plans.swap(keep);
}

void rxgs::drop_plan(rxgs_ctx* ctx, const void* plan) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::vector<BatchPlan*> keep;
  for (BatchPlan* q : ctx->plans) {
    if (q == plan)
      destroy_plan(q);
    else
      keep.push_back(q);
  }
  ctx->plans.swap(keep);
}

// Exact instance count of a batch's views (one synchronising readback);
// used to size a new plan.
static rxgs_status count_instances(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int B,
                                   uint32_t* max_per_view, cudaStream_t st);

namespace rxgs {
rxgs_status render_batched_tagged(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int B,
                                  const float* rx, const int32_t* rx_counts,
                                  const rxgs_render_desc* d, rxgs_outputs* out, void* stream,
                                  int tag, double inst_margin, const void** plan_used) {
  if (!ctx || !tx || !rx_counts || !d || !out) return fail(ctx, RXGS_E_INVALID, "null argument");
  if (B <= 0 || B > 4096) return fail(ctx, RXGS_E_INVALID, "B out of range");
  int R = 0;
  for (int v = 0; v < B; ++v) {
    if (rx_counts[v] <= 0) return fail(ctx, RXGS_E_INVALID, "empty receiver batch %d", v);
    R += rx_counts[v];
  }
  const int kind = d->kind;
  if (!kind) return fail(ctx, RXGS_E_INVALID, "empty output kind");
  if ((kind & RXGS_OUT_SPECTRA) && !out->spectra) return fail(ctx, RXGS_E_INVALID, "spectra == NULL");
  if ((kind & RXGS_OUT_RSSI) && !out->rssi) return fail(ctx, RXGS_E_INVALID, "rssi == NULL");
  if ((kind & RXGS_OUT_CSI) && !out->csi) return fail(ctx, RXGS_E_INVALID, "csi == NULL");
  if (!d->radiance && !rx) return fail(ctx, RXGS_E_INVALID, "rx == NULL");
  if (d->fle_coeffs || d->fle_base)
    return fail(ctx, RXGS_E_INVALID, "batched rendering does not take FLE radiance");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SceneState* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->scenes.find(scene);
    if (it == ctx->scenes.end()) return fail(ctx, RXGS_E_INVALID, "unknown scene");
    s = it->second;
  }
  if ((kind & RXGS_OUT_RSSI) && s->C != 1) return fail(ctx, RXGS_E_INVALID, "RSSI needs C == 1");
  if (!d->radiance && s->occ)
    return fail(ctx, RXGS_E_INVALID, "batched rendering does not take occlusion inputs (occupancy grid)");
  if (!d->radiance && !s->mlp)
    return fail(ctx, RXGS_E_INVALID, "no radiance given and the scene has no MLP");
  CK(cudaSetDevice(ctx->device));
  // size a plan: reuse one that fits, else measure this batch's instances
  const bool mlp = d->radiance == nullptr;
  const bool vis = d->reduce_path == 1;
  if (vis && (!mlp || (kind & RXGS_OUT_SPECTRA) || s->C > 52))
    return fail(ctx, RXGS_E_INVALID,
                "batched reduce_path 1 needs MLP radiance, CSI/RSSI only and C <= 52");
  BatchPlan* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    p = find_plan(ctx, scene, kind, mlp, vis, B, R, tag);
  }
  if (!p) {
    uint32_t per_view = 0;
    rxgs_status rs = count_instances(ctx, scene, tx, B, &per_view, st);
    if (rs != RXGS_OK) return rs;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const double need_d = static_cast<double>(per_view) * next_pow2(B, 4) * inst_margin + 4096.0;
    if (need_d > 2147483647.0) return fail(ctx, RXGS_E_INVALID, "instance capacity overflow");
    rs = new_plan(ctx, scene, s, kind, mlp, vis, B, R, static_cast<uint32_t>(need_d), tag, &p);
    if (rs != RXGS_OK) return rs;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  Stage sg(ctx, "batched", st);
  // the previous call's copy of the pinned descriptor must have finished
  // before it is overwritten; the device buffers are ordered on `st`
  CK(cudaEventSynchronize(p->desc_done));
  fill_desc(*p, B, rx_counts, p->h_desc);
  CK(cudaMemcpyAsync(p->desc, p->h_desc, sizeof(int) * p->L.size(), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(p->desc_done, st));
  CK(cudaMemcpyAsync(p->tx, tx, sizeof(float) * 3 * B, cudaMemcpyDefault, st));
  if (rx) CK(cudaMemcpyAsync(p->rx, rx, sizeof(float) * 3 * R, cudaMemcpyDefault, st));
  if (!mlp)
    CK(cudaMemcpyAsync(p->rad_in, d->radiance, sizeof(float) * static_cast<size_t>(R) * s->K * 2 * s->C,
                       cudaMemcpyDefault, st));
  // the pinned descriptor is consumed by the copy above before we return
  CK(cudaGraphLaunch(p->exec, st));
  if (plan_used) *plan_used = p;
  const size_t HW2C = static_cast<size_t>(p->g.H) * p->g.W * 2 * s->C;
  if (kind & RXGS_OUT_SPECTRA)
    CK(cudaMemcpyAsync(out->spectra, p->spectra, sizeof(float) * R * HW2C, cudaMemcpyDeviceToDevice, st));
  if (kind & RXGS_OUT_CSI)
    CK(cudaMemcpyAsync(out->csi, p->csi, sizeof(float) * R * 2 * s->C, cudaMemcpyDeviceToDevice, st));
  if (kind & RXGS_OUT_RSSI)
    CK(cudaMemcpyAsync(out->rssi, p->rssi, sizeof(float) * R, cudaMemcpyDeviceToDevice, st));
  return RXGS_OK;
}
}  // namespace rxgs

extern "C" rxgs_status rxgs_render_batched(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx,
                                           int B, const float* rx, const int32_t* rx_counts,
                                           const rxgs_render_desc* d, rxgs_outputs* out,
                                           void* stream) {
  return render_batched_tagged(ctx, scene, tx, B, rx, rx_counts, d, out, stream, 0, 1.25);
}

static rxgs_status count_instances(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int B,
                                   uint32_t* max_per_view, cudaStream_t st) {
  *max_per_view = 0;
  for (int v = 0; v < B; ++v) {
    rxgs_views_t h = 0;
    rxgs_status rs = rxgs_prepare(ctx, scene, tx + 3 * v, 1, &h, st);
    if (rs != RXGS_OK) return rs;
    int64_t n = 0;
    rxgs_views_info(ctx, h, &n);
    rxgs_release_views(ctx, h, st);
    *max_per_view = std::max<uint32_t>(*max_per_view, static_cast<uint32_t>(n));
  }
  return RXGS_OK;
}
