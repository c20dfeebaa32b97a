/*
 * rxgs.h -- C ABI of the GB300 multi-receiver RF Gaussian renderer.
 *
 * The library renders a frozen set of 3D Gaussians, as seen from one or
 * more transmitters, at many receivers at once.  For every transmitter it
 * projects the Gaussians onto an elevation x azimuth grid centred at the
 * transmitter, bins them into tiles and depth-sorts each tile once; all
 * receivers of that transmitter share this work and differ only in their
 * radiance, which is alpha-composited front to back into a complex spectrum
 * per receiver and optionally reduced to RSSI or per-subcarrier CSI.
 *
 *   Problem statement  S(t, r) = f(t, r; Theta)           (Sec. 3, Eq. 3)
 *   Transmitter side   projection, tiles, depth sort       (Algorithm 1, Stage 1)
 *   Receiver side      per-receiver radiance s_k^(j)       (Algorithm 1, Stage 2;
 *                      Sec. 3.3.2, Eq. film, local, combined_local)
 *                      or Fourier-Legendre coefficients,   (App. E.2)
 *                      explicit or conditioned by the      (Eq. rx_enc, film,
 *                      global FiLM branch                   film_apply; App. E.4)
 *   Compositing        w = tau exp(-q/2), C += T w s,
 *                      T *= (1 - w), stop when T < eps     (Algorithm 1, Stage 3)
 *   Amplitude          |R| = sqrt(Re^2 + Im^2 + 1e-8)      (App. E.2)
 *   RSSI / CSI         coherent sum over directions        (Def. 2, Eq. render)
 *   Backward           dL/d radiance, dL/d opacity         (App. D)
 *
 * Conventions shared by every call.
 *   - Grid: row i has elevation theta0 + i*step, column j has azimuth j*step
 *     (degrees); W*step must equal 360.  Pixels are the left/bottom grid
 *     points.
 *   - Complex numbers are two consecutive float32 (real, imaginary).
 *   - Unless a field says otherwise, pointers are DEVICE pointers on the
 *     current CUDA device, owned by the caller, and must stay valid until
 *     the work on `stream` has finished.  `stream` is a cudaStream_t (NULL =
 *     legacy default stream).  Calls enqueue work and return; device-side
 *     problems surface as RXGS_E_DEVICE from the next call that
 *     synchronises (rxgs_prepare, rxgs_sync, the serving calls).
 *   - A status other than RXGS_OK means nothing was enqueued, except for
 *     RXGS_E_CUDA / RXGS_E_DEVICE, which report an error of the CUDA
 *     context; rxgs_last_error() gives a message.
 *   - Forward outputs are deterministic: the same inputs and options give
 *     bit-identical results.  A receiver's spectrum does not depend on the
 *     other receivers of its batch beyond the width of the column block it
 *     falls in: blocks of 16-64 columns composite on the CUDA cores in list
 *     order, blocks of 128 columns (2 N C > 64) run the chunk products on
 *     the tensor cores in split bf16 with float32 accumulation; the two
 *     agree to about 1e-5 of each value's absolute chain.
 *   - Backward outputs accumulate over tiles and views with float atomics:
 *     repeated runs agree to within float32 rounding, not bit for bit.
 */
#ifndef RXGS_H
#define RXGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rxgs_ctx rxgs_ctx;
typedef uint64_t rxgs_scene_t;   /* handle to a device-resident scene         */
typedef uint64_t rxgs_views_t;   /* handle to transmitter-side (shared) state */
typedef uint64_t rxgs_ticket_t;  /* handle to a serving request               */

typedef enum {
  RXGS_OK = 0,
  RXGS_E_INVALID = 1,    /* bad argument; nothing enqueued                  */
  RXGS_E_OOM = 2,        /* device allocation failed                        */
  RXGS_E_CUDA = 3,       /* a CUDA call failed                              */
  RXGS_E_ADMISSION = 4,  /* serving: request larger than the memory budget  */
  RXGS_E_NOT_READY = 5,  /* serving: result not ready yet                   */
  RXGS_E_TIMEOUT = 6,    /* serving: poll timed out                         */
  RXGS_E_DEVICE = 7,     /* a kernel reported an error (capacity, bounds)   */
  RXGS_E_CANCELLED = 8   /* serving: request cancelled                      */
} rxgs_status;

enum { RXGS_OUT_SPECTRA = 1, RXGS_OUT_RSSI = 2, RXGS_OUT_CSI = 4 };

/* Grid and numerical options (Table 5 grids; Algorithm 1 constants). */
typedef struct {
  int H, W;            /* grid rows (elevation) x columns (azimuth)          */
  float theta0_deg;    /* elevation of row 0 in degrees (0 or -90)           */
  float step_deg;      /* angular step in degrees; W*step_deg == 360         */
  int tile_h, tile_w;  /* tile shape; tile_h*tile_w == 256                   */
  float eps_T;         /* stop threshold on transmittance (1e-4)             */
  float q_max;         /* Mahalanobis cut-off q <= q_max (9 = 3 sigma)       */
  float r_near;        /* Gaussians nearer than this to the transmitter are
                          culled (0.05 m)                                    */
  int cols_per_cta;    /* receiver*channel*2 columns per render CTA:
                          16, 32, 64 or 128; 0 = chosen by the autotuner     */
  int deterministic;   /* must be 0: a bit-reproducible backward is not
                          provided (it would need a fixed-order reduction of
                          per-instance dL/ds rows, 5 GB at 10M instances x
                          128 columns); rxgs_create refuses other values     */
  size_t mem_budget;   /* serving admission budget in bytes; 0 = 8 GiB      */
} rxgs_options;

/* Fills `o` with the defaults: 90x360 grid from 0 deg at 1 deg, 16x16
 * tiles, eps 1e-4, q_max 9, r_near 0.05, autotuned columns. */
void rxgs_default_options(rxgs_options* o);

/* Creates a context on CUDA device `device`.  The context owns the scenes,
 * views and serving state created through it.  Not thread-safe except for
 * the serving calls.  Returns RXGS_E_INVALID for a bad option set. */
rxgs_status rxgs_create(const rxgs_options* opts, int device, rxgs_ctx** out);
rxgs_status rxgs_destroy(rxgs_ctx* ctx);
const char* rxgs_last_error(rxgs_ctx* ctx);

/* Scene upload (App. E.1 state: mean p, log-scale s, quaternion q = (w,x,y,z)
 * not necessarily normalised, opacity tau in (0,1)).  The library copies the
 * arrays into memory it owns and builds Sigma = R S S^T R^T once.
 *   means[K,3], log_scales[K,3], quats[K,4], opacity[K]          float32
 *   base_radiance[K,C,2]  phi_base, required when mlp_params != NULL
 *   mlp_params            flat float32 parameters of the two conditioning
 *                         MLPs (global: Linear(3,h) ReLU Linear(h,4C);
 *                         local: Linear(6,h) ReLU Linear(h,4C)), in the order
 *                         g_w1[h,3] g_b1[h] g_w2[4C,h] g_b2[4C] l_w1[h,6]
 *                         l_b1[h] l_w2[4C,h] l_b2[4C]; NULL = no MLP
 *   mlp_hidden            h (64)
 *   mlp_bf16              1: matmul operands rounded to bf16, fp32 accumulate
 *   on_device             1: pointers are device pointers; 0: host pointers */
typedef struct {
  int64_t K;
  int C;
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity;
  const float* base_radiance;
  const float* mlp_params;
  int mlp_hidden;
  int mlp_bf16;
  int on_device;
} rxgs_scene_desc;

rxgs_status rxgs_upload_scene(rxgs_ctx* ctx, const rxgs_scene_desc* desc, rxgs_scene_t* out);
rxgs_status rxgs_release_scene(rxgs_ctx* ctx, rxgs_scene_t scene);

/* Occlusion inputs of the local conditioning branch (App. E.5): splats the
 * scene's Gaussians as they are now (positions, covariances, opacities)
 * into a res^3 density grid over the bounding box of the means (Gaussian k
 * adds tau_k exp(-1/2 sum_a ((c_a - p_a) / s_a)^2), s_a = sqrt(Sigma_aa), to
 * voxel centres within 2 s_a on every axis; densities clamp to [0, 1]).
 * Later MLP renders and backwards of the scene (per-pixel reduce path)
 * feed the local MLP T_k = prod_s (1 - rho_s) and rho_bar_k = mean_s rho_s
 * over 16 probes x = p + t (r - p), t = 0.05 + 0.06 s, instead of the clear
 * (1, 0).  res = 0 removes the grid.  1 <= res <= 512.  Batched rendering,
 * serving and reduce_path 1 refuse a scene with a grid. */
rxgs_status rxgs_build_occupancy(rxgs_ctx* ctx, rxgs_scene_t scene, int res, void* stream);
/* Replaces the opacity and/or phi_base / MLP parameters of a scene in place
 * (device pointers, same shapes; NULL = keep).  Geometry stays frozen. */
rxgs_status rxgs_update_scene(rxgs_ctx* ctx, rxgs_scene_t scene, const float* opacity,
                              const float* base_radiance, const float* mlp_params, void* stream);

/* Transmitter-side state (Algorithm 1, Stage 1): projection of every
 * Gaussian for each of the M transmitters tx[M,3], the per-tile lists sorted
 * by (transmitter, tile, depth) and the tile ranges.  It is shared by every
 * receiver rendered against it.  This call reads back one integer (the
 * instance count) and so synchronises `stream` once. */
rxgs_status rxgs_prepare(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                         rxgs_views_t* out, void* stream);
rxgs_status rxgs_release_views(rxgs_ctx* ctx, rxgs_views_t views, void* stream);

/* What to render.
 *   kind       RXGS_OUT_* bitmask
 *   radiance   [N,K,C,2] receiver-major float32 (the paper's (N, K, 2)
 *              signal tensor), shared by all transmitters; NULL = evaluate
 *              the scene's conditioning MLP for the receivers (unless
 *              fle_coeffs is given)
 *   reduce_path for RSSI/CSI without spectra: 0 = per-pixel compositing then
 *              a sum over pixels; 1 = visibility weights W_k (Eq.
 *              render_reorder) then sum_k W_k s_kj.  Both give the same
 *              value up to rounding order.
 *   fle_coeffs [N,K,2,L] float32, L = (fle_lmax + 1)^2, or NULL: the
 *              per-receiver directional coefficients of the Fourier-Legendre
 *              radiance (App. E.2, the tensor Algorithm 1 reduces against the
 *              transmitter-side basis).  Component l*l + l + m holds a_lm
 *              ([..][0][.]) and b_lm ([..][1][.]); for the direction from the
 *              transmitter to Gaussian k (polar angle theta from +z, azimuth
 *              phi) s = sum (a + i b) N_l|m| P_l^|m|(cos theta) e^{i m phi},
 *              P without the Condon-Shortley phase.  Needs C == 1,
 *              radiance == NULL, reduce_path == 0 and 0 <= fle_lmax <= 9; the
 *              radiance then differs per transmitter.
 *   fle_lmax   the degree of fle_coeffs (or of fle_base)
 *   fle_base   [K,2,L] float32 or NULL: base FLE coefficients conditioned on
 *              the receiver by the global FiLM branch (Eq. rx_enc, film,
 *              film_apply): receiver j's coefficient l of Gaussian k is
 *              (1 + a_jl) fle_base_kl + b_jl (complex), with (a_jl, b_jl) from
 *              `film` (see rxgs_film_eval).  Excludes fle_coeffs and radiance;
 *              needs `film`, rx, C == 1, reduce_path == 0, 0 <= fle_lmax <= 9.
 *   film       packed FiLM parameters (rxgs_film_param_count floats, device),
 *              read when fle_base != NULL
 *   film_nfreq, film_embed, film_hidden   the FiLM sizes: frequency vectors
 *              (1..32), embedding width (0..64), hidden width (1..256)
 *   film_local 1: with fle_base, also the local branch (Eq. local): each
 *              (receiver j, Gaussian k) gets (alpha_jk, beta_jk) from the
 *              scene's conditioning MLP's local branch (inputs [v_hat, d, T,
 *              rho_bar], the occlusion probes when the scene has an occupancy
 *              grid), composed per Eq. combined_local:
 *              (1 + alpha_jk) ((1 + a_jl) fle_base_kl + b_jl) + beta_jk.
 *              Needs a scene uploaded with MLP weights (64 hidden units, C ==
 *              1); its backward adds the local branch's gradient to grad_mlp
 *              (the global branch's entries stay untouched).  0: no local
 *              branch. */
typedef struct {
  int kind;
  const float* radiance;
  int reduce_path;
  const float* fle_coeffs;
  int fle_lmax;
  const float* fle_base;
  const float* film;
  int film_nfreq;
  int film_embed;
  int film_hidden;
  int film_local;
} rxgs_render_desc;

/* The global FiLM branch over FLE components (Eq. rx_enc, film; App. E.4).
 * Packed parameters, float32, in this order:
 *   omega[nfreq][3]   frequency vectors of the receiver encoding
 *                     gamma(r) = [sin(w_1.r), cos(w_1.r), ..., sin(w_F.r), cos(w_F.r)]
 *   embed[L][embed]   component embeddings e_l, L = (lmax + 1)^2
 *   w1[hidden][din], b1[hidden], w2[hidden][hidden], b2[hidden],
 *   w3[4][hidden], b3[4]   three linear layers, ReLU between them,
 *                     din = 2 nfreq + 2 + embed
 * The input of component l*l + l + m for receiver r is
 * [gamma(r); l / max(lmax, 1); m / max(lmax, 1); e_l]; the four outputs are
 * (a.re, a.im, b.re, b.im).
 * rxgs_film_param_count returns the packed length, or 0 for sizes out of range.
 * rxgs_film_eval writes ab[N][L][4] for receivers rx[N][3] (device pointers
 * on `stream`, caller-owned); RXGS_E_INVALID for sizes out of range or null
 * pointers. */
int64_t rxgs_film_param_count(int nfreq, int embed, int hidden, int lmax);
rxgs_status rxgs_film_eval(rxgs_ctx* ctx, const float* film, int nfreq, int embed, int hidden,
                           int lmax, const float* rx, int N, float* ab, void* stream);

/* Outputs, all optional except those `kind` asks for:
 *   spectra  [M,N,H,W,C,2]
 *   rssi     [M,N]          |sum over pixels| (C must be 1)
 *   csi      [M,N,C,2]      sum over pixels
 *   ncontrib [M,H,W] int32  number of Gaussians composited per pixel
 *   tfinal   [M,H,W]        transmittance after compositing */
typedef struct {
  float* spectra;
  float* rssi;
  float* csi;
  int32_t* ncontrib;
  float* tfinal;
} rxgs_outputs;

/* Renders every (transmitter, receiver) pair of `views` x rx[N,3]. */
rxgs_status rxgs_render_views(rxgs_ctx* ctx, rxgs_views_t views, const float* rx, int N,
                              const rxgs_render_desc* desc, rxgs_outputs* out, void* stream);

/* rxgs_prepare + rxgs_render_views + rxgs_release_views in one call. */
rxgs_status rxgs_render(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                        const float* rx, int N, const rxgs_render_desc* desc,
                        rxgs_outputs* out, void* stream);

/* Uneven receiver batches (one transmitter per batch, ragged receiver
 * counts) rendered by one persistent launch inside a CUDA graph.
 *   tx[B,3]            one transmitter per batch (device or host pointer)
 *   rx[R,3]            all receivers, batch after batch, R = sum rx_counts
 *   rx_counts[B]       HOST array, each >= 1
 *   desc->radiance     [R,K,C,2] receiver-major, or NULL = scene MLP
 *   out->spectra       [R,H,W,C,2], out->csi [R,C,2], out->rssi [R]
 * The first call for a (scene, kind, radiance mode) whose sizes exceed every
 * existing plan measures the batch's instance counts (one readback per
 * view), allocates a plan with capacity for the next power of two of views
 * and receivers and 1.25x the largest per-view instance count, and captures
 * the pipeline into a CUDA graph; later calls copy the inputs and a small
 * descriptor into the plan and replay the graph.  A batch whose instances
 * exceed the plan's capacity sets RXGS_E_DEVICE at the next rxgs_sync (its
 * results are then invalid).  Calls that share a plan must be ordered (one
 * stream). */
rxgs_status rxgs_render_batched(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int B,
                                const float* rx, const int32_t* rx_counts,
                                const rxgs_render_desc* desc, rxgs_outputs* out, void* stream);

/* Autotuner: renders the given workload (M transmitters x N receivers, as
 * rxgs_render) with every tile shape in {16x16, 8x32, 32x8} and every
 * column block in {16, 32, 64, 128} not wider than the work, `iters` times
 * each after one warm-up, and keeps the fastest pair in the context's
 * options (used by later calls, including new batch plans).  Writes
 *   {"candidates": [{"tile": [h, w], "cols": c, "ms": t}, ...],
 *    "chosen": {...}}
 * into json[cap] when json != NULL.  Spectra do not depend on the choice. */
rxgs_status rxgs_autotune(rxgs_ctx* ctx, rxgs_scene_t scene, const float* tx, int M,
                          const float* rx, int N, const rxgs_render_desc* desc, int iters,
                          char* json, size_t cap);

/* Serving: a request loop that batches (transmitter, receiver set) queries of
 * different sizes against a device-resident scene (continuous batching).  A
 * scheduler thread owned by the context admits queued requests in arrival
 * order into the next free slot while the batch fits the slot's capacity
 * and the memory budget has room next to the batches already on the GPU,
 * renders the batch with the batched pipeline on the slot's stream, and
 * picks the next batch without waiting: with `slots` > 1, batches overlap on
 * the device.  A request's result does not depend on the batch it lands in
 * (see rxgs_render_batched).  The scene needs a conditioning MLP.
 *   kind                 RXGS_OUT_RSSI (C == 1) or RXGS_OUT_CSI
 *   max_batch_receivers  receivers per batch (a larger request is refused
 *                        with RXGS_E_ADMISSION at submit)
 *   max_batch_views      requests per batch
 *   mem_budget           bytes of estimated device memory all batches in
 *                        flight may use (a request estimated above it alone
 *                        is refused with RXGS_E_ADMISSION)
 *   slots                batches that may be in flight at once (1..8) */
typedef struct {
  int kind;
  int max_batch_receivers;
  int max_batch_views;
  size_t mem_budget;
  int slots;
} rxgs_serve_options;

void rxgs_serve_default_options(rxgs_serve_options* o);
rxgs_status rxgs_serve_start(rxgs_ctx* ctx, rxgs_scene_t scene, const rxgs_serve_options* opts);
/* tx[3] and rx[n,3] are HOST pointers, copied before the call returns. */
rxgs_status rxgs_serve_submit(rxgs_ctx* ctx, const float* tx, const float* rx, int n,
                              rxgs_ticket_t* ticket);
/* Waits up to timeout_us (0 = do not wait, < 0 = forever) for the request;
 * on RXGS_OK copies its result to the HOST buffer out (n floats for RSSI,
 * n*C*2 for CSI) and retires the ticket.  RXGS_E_NOT_READY (timeout_us == 0)
 * and RXGS_E_TIMEOUT keep the ticket; RXGS_E_CANCELLED and RXGS_E_DEVICE
 * retire it. */
rxgs_status rxgs_serve_poll(rxgs_ctx* ctx, rxgs_ticket_t ticket, float* out, int timeout_us);
/* Removes a request that is still queued (RXGS_E_NOT_READY once it is on
 * the GPU); a later poll returns RXGS_E_CANCELLED. */
rxgs_status rxgs_serve_cancel(rxgs_ctx* ctx, rxgs_ticket_t ticket);
/* {"completed", "failed", "retried", "cancelled", "batches",
 *  "mean_batch_receivers", "p50_ms", "p90_ms", "p99_ms", "max_ms", "mean_ms",
 *  "queued", "inflight_bytes", "elapsed_s"}; latency = submit to completion. */
rxgs_status rxgs_serve_stats(rxgs_ctx* ctx, char* json, size_t cap);
rxgs_status rxgs_serve_reset_stats(rxgs_ctx* ctx);
/* Failure injection on the host: the next `batches` batches fail before
 * launch and their requests complete with RXGS_E_DEVICE (no GPU fault). */
rxgs_status rxgs_serve_inject_fault(rxgs_ctx* ctx, int batches);
/* Drains the batches in flight, stops the scheduler and frees its state. */
rxgs_status rxgs_serve_stop(rxgs_ctx* ctx);

/* Backward (App. D): gradients of a loss L given dL/d(outputs).
 *   grad_spectra [M,N,H,W,C,2] or NULL
 *   grad_csi     [M,N,C,2] or NULL   (uniform over pixels)
 *   grad_rssi    [M,N] or NULL       (needs fwd_csi)
 *   fwd_csi      the forward CSI [M,N,1,2] when grad_rssi is given
 * Nothing else of the forward is needed: each tile re-walks its list with
 * the forward's decisions, then sweeps it back to front.  `views`, `rx` and
 * `desc->radiance` must be those of the forward.  The radiance the last
 * rxgs_render_views computed on `views` is reused when rx, N, radiance (or
 * fle_coeffs, or fle_base with film and its sizes) and the scene
 * (rxgs_update_scene) are unchanged, compared by pointer; otherwise it is
 * recomputed.  A forward that ran with 128-column blocks (the tensor-core
 * kernel) also leaves on `views` each pixel's stop position and final
 * transmittance (they depend on the views alone); the backward then skips
 * the re-walk.  Both reuses assume the backward is ordered after that
 * forward (same stream, or synchronised).
 * Gradients are accumulated with float atomics (their rounding order is not
 * fixed).
 * Outputs (accumulated: caller zero-fills):
 *   grad_radiance [N,K,C,2]  when desc->radiance != NULL
 *   grad_opacity  [K]
 *   grad_base     [K,C,2] and grad_mlp (flat) when the scene MLP is used
 *   grad_fle      [N,K,2,L] when desc->fle_coeffs != NULL
 *   grad_fle_base [K,2,L] and grad_film (packed) when desc->fle_base != NULL
 * Geometry (means, scales, rotations) is frozen and gets no gradient. */
typedef struct {
  const float* grad_spectra;
  const float* grad_csi;
  const float* grad_rssi;
  const float* fwd_csi;
} rxgs_cotangents;

typedef struct {
  float* grad_radiance;
  float* grad_opacity;
  float* grad_base;
  float* grad_mlp;
  float* grad_fle;       /* [N,K,2,L] += dL/dfle_coeffs (FLE radiance), or NULL */
  float* grad_fle_base;  /* [K,2,L] += dL/dfle_base (FiLM-conditioned FLE), or NULL */
  float* grad_film;      /* packed like `film` += dL/dfilm, or NULL; the MLP's
                            weight gradients are summed in a fixed order, the
                            per-receiver (a, b) gradients with float atomics */
} rxgs_grads;

rxgs_status rxgs_render_backward(rxgs_ctx* ctx, rxgs_views_t views, const float* rx, int N,
                                 const rxgs_render_desc* desc, const rxgs_cotangents* cot,
                                 rxgs_grads* grads, void* stream);

/* Inspection of transmitter-side state (for tests and tools).
 *   n_inst   receives the number of (Gaussian, tile) instances
 * rxgs_views_export copies (device pointers, any may be NULL):
 *   rec[M,K,8]   float32 {theta_px, phi_px, conic_a, 2*conic_b, conic_c, tau,
 *                rows, cols}; rows/cols are int32 bit patterns
 *                i_lo | i_hi << 16 and j_lo | span << 16
 *   counts[M,K]  tiles per Gaussian (0 = culled)
 *   keys[I], vals[I]  sorted (view | tile | depth) keys and Gaussian indices
 *   ranges[M,T,2]     [start, end) of each tile's list in keys/vals */
rxgs_status rxgs_views_info(rxgs_ctx* ctx, rxgs_views_t views, int64_t* n_inst);
rxgs_status rxgs_views_export(rxgs_ctx* ctx, rxgs_views_t views, float* rec, uint32_t* counts,
                              uint64_t* keys, uint32_t* vals, uint32_t* ranges, void* stream);

/* Stage profiler (tracing).  While enabled, every call records a CUDA event
 * pair on its stream around each stage (preprocess, scan, emit, sort, ranges,
 * mlp / radiance_transpose, render_fwd, reduce, render_bwd, mlp_bwd,
 * radiance_grad).  rxgs_profile_read waits for the recorded events, folds
 * them into per-stage totals and writes
 *   {"kernel_launches": L, "device_allocs": A, "pool_used_bytes": U,
 *    "pool_reserved_bytes": R, "stages": {"<stage>": {"ms": t, "calls": n}, ...}}
 * into json[cap] (RXGS_E_INVALID if cap is too small); reset = 1 clears the
 * totals afterwards.  kernel_launches counts every kernel the library has
 * launched in this process, device_allocs every stream-ordered device
 * allocation it has made; U and R are the current used and reserved bytes
 * of the context device's default memory pool, which those allocations
 * draw on. */
rxgs_status rxgs_profile(rxgs_ctx* ctx, int enable);
rxgs_status rxgs_profile_read(rxgs_ctx* ctx, char* json, size_t cap, int reset);

/* CSI (and RSSI when C == 1) of prepared views for the receiver-major
 * radiance[N,K,C,2], WITHOUT allocating any device memory.  The paper has no
 * counterpart: this is for callers that must not allocate while rendering
 * (a latency-bound serving thread, a host program whose device memory is
 * owned by another allocator or budgeted up front).  It computes the same
 * values as rxgs_render_views with RXGS_OUT_CSI / RXGS_OUT_RSSI.
 *   csi[M,N,C,2] and/or rssi[M,N]   outputs (device, caller-owned)
 * The per-tile partial sums live in a fixed 16 MiB device array inside the
 * library.  rxgs_create looks up its device address on the context's device
 * (cudaGetSymbolAddress), which also brings the array into existence there:
 * from the first rxgs_create on a GPU the array occupies 16 MiB of it until
 * the process exits; the calls themselves allocate nothing.
 * M * tiles * 2 * N * C must not exceed 4,194,304, and 2 * N * C / 64 column
 * blocks must fit the launch grid (65,535); larger requests return
 * RXGS_E_INVALID, with the reason in rxgs_last_error, before any launch.
 * The call makes the context's device current for its launches and restores
 * the caller's current device before it returns.  Every call reuses the same
 * array and the last call's contents stay in it (each call writes every
 * entry it reads, so nothing needs clearing): calls whose work overlaps on
 * the GPU race and must be serialised by the caller (one stream, or
 * events). */
rxgs_status rxgs_render_csi_noalloc(rxgs_ctx* ctx, rxgs_views_t views, const float* radiance,
                                    int N, float* csi, float* rssi, void* stream);

/* The L1 term of the Stage II training loss (App. E.3; Sec. 3.1 Stage II)
 * and its cotangent, in one pass over device buffers on `stream`:
 *   kind RXGS_OUT_SPECTRA: values = rendered spectra [n][2] (Re, Im), target
 *     = amplitudes [n]; with a_i = sqrt(Re^2 + Im^2 + 1e-8) (App. E.2)
 *     grad[n][2] = sign(a_i - y_i) / n * (Re, Im) / a_i;
 *   kind RXGS_OUT_RSSI: values = RSSI [n], target [n],
 *     grad[n] = sign(rssi_i - y_i) / n;
 *   loss[0] = (1/n) sum_i |a_i - y_i| (a fixed-order sum: the same from run
 *     to run).
 * All pointers are caller-owned device memory; grad may be passed as the
 * cotangent of rxgs_render_backward.  Null pointers or another kind return
 * RXGS_E_INVALID. */
rxgs_status rxgs_l1_loss(rxgs_ctx* ctx, int kind, const float* values, const float* target,
                         size_t n, float* loss, float* grad, void* stream);

/* Waits for `stream` and converts a recorded device error into a status. */
rxgs_status rxgs_sync(rxgs_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RXGS_H */
