// rxgs_internal.h -- shared declarations of the CUDA library (not part of the
// C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace rxgs {

// Grid constants as the kernels see them (all float32 values derived once on
// the host).
struct GridConst {
  int H, W, TH, TW;
  int tiles_h, tiles_w, T;  // T = tiles_h * tiles_w
  float inv_step;           // 1 / step in radians, rounded to float32
  float theta0_px;          // theta0 / step
  float Wf, halfW, Hm1f;    // W, W/2, H-1 as floats
  float eps_T, q_max, ksig, r_near;  // ksig = sqrt(q_max)
};

// Number of kernel launches issued by the library (all threads, all
// contexts); each launch_* function adds the kernels it launched.
void note_launches(unsigned n);
unsigned long long launch_count();

// Device error word bits (written by kernels, read by the host at syncs).
enum : unsigned {
  kErrCapacity = 1u,   // an instance list was larger than its buffer
  kErrBounds = 2u,     // an index left its buffer (checked builds)
  kErrArgument = 4u,   // a device-side argument check failed
  kErrTimeout = 8u,    // a bounded device-side wait (mbarrier) gave up
};

// ----------------------------------------------------------- geometry (a0-a3)
// Packed scene record: 3 x float4 = {p.xyz, tau}, {S00,S01,S02,S11},
// {S12,S22,0,0}.
void launch_scene_upload(const float* means, const float* log_scales, const float* quats,
                         const float* opacity, int K, float4* geom, cudaStream_t s);
void launch_set_opacity(const float* opacity, int K, float4* geom, cudaStream_t s);

// Projection of K Gaussians for M views.  rec[M][K][2] float4, depth[M][K]
// (float bits of rho), count[M*K] tile counts (0 = culled).
// nviews_dev (optional): number of view slots in use; later slots are culled.
// stats (optional, [M][4] words zeroed before the call), per view: the
// total tile count (uint64 in words 0-1), ~(smallest) and largest depth key
// of the visible pairs (words 2 and 3); launch_combine_stats folds the
// views into dst[4] (device or mapped pinned memory).
void launch_preprocess(const GridConst& g, const float4* geom, int K, const float* tx, int M,
                       float4* rec, uint32_t* depth, uint32_t* count, cudaStream_t s,
                       const int* nviews_dev = nullptr, uint32_t* stats = nullptr);
void launch_combine_stats(const uint32_t* stats, int M, uint32_t* dst, cudaStream_t s);

// Exclusive scan of n uint32 values; out has n+1 entries (out[n] = total).
// tmp must hold scan_tmp_words(n) uint32.
size_t scan_tmp_words(size_t n);
void launch_exclusive_scan(const uint32_t* in, uint32_t* out, size_t n, uint32_t* tmp,
                           cudaStream_t s);

// The two-sort order of the instances (view, tile, depth, Gaussian index):
// every view's Gaussians sorted by depth (radix_sort_segments_first / _rest
// over the depth keys, one segment per view), then dst[i] = src[idx[i]] (the tile
// counts in that order, then scanned) ...
void launch_gather_words(const uint32_t* src, const uint32_t* idx, size_t n, uint32_t* dst,
                         cudaStream_t s);
// ... the instances of the ordered pairs (ord: view-major pair indices,
// offsets: the scan of their counts) with (view << tile_bits | tile) keys
// and Gaussian-index values, then stably sorted by those keys.
// Positions at or past `cap` are not written; a pair whose instances would
// end past it sets kErrCapacity in *err.
void launch_emit_sorted(const GridConst& g, const float4* rec, const uint32_t* ord,
                        const uint32_t* offsets, size_t MK, int K, int tile_bits, uint32_t* keys,
                        uint32_t* vals, cudaStream_t s, uint32_t cap = 0xffffffffu,
                        unsigned* err = nullptr);
// (view | tile) keys and values -> (view | tile | depth) keys (export only).
void launch_expand_keys(const uint32_t* vt, const uint32_t* vals, size_t n, const uint32_t* depth,
                        int K, int tile_bits, uint64_t* out, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// Returns, through *result_in_alt, whether the sorted data ended in the alt
// buffers.  tmp must hold radix_tmp_words(n) uint32.
size_t radix_tmp_words(size_t n);
// n_dev (optional): the actual item count, <= n (launch sizes follow n).
// err (optional): unused (no kernel of the sort waits on another).
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                      size_t n, int bits, uint32_t* tmp, bool* result_in_alt, cudaStream_t s,
                      const uint32_t* n_dev = nullptr, unsigned* err = nullptr);
// Each of nseg segments of len consecutive keys (read only) sorted stably
// on its own, in 9-bit digits of key - bias (uint32 arithmetic, bias a
// multiple of 512 so that the first digit does not depend on it): the
// first pass (radix_sort_segments_first, into keys_a / idx_a, values the
// items' indices in the whole array) can run before the bias is known; the
// rest (radix_sort_segments_rest, `bits` of key - bias in all) returns the
// sorted indices (idx_a or idx_b).  keys_a / keys_b / idx_a / idx_b hold
// len * nseg words.  gather_src (optional): gather_dst[i] = gather_src[index
// i] is written as well.  tmp must hold radix_segments_tmp_words(len, nseg)
// uint32.  Null if nothing was sorted (len * nseg == 0).
size_t radix_segments_tmp_words(size_t len, int nseg);
void radix_sort_segments_first(const uint32_t* keys, size_t len, int nseg, uint32_t* keys_a,
                               uint32_t* idx_a, uint32_t* tmp, cudaStream_t s);
const uint32_t* radix_sort_segments_rest(size_t len, int nseg, int bits, uint32_t bias,
                                         uint32_t* keys_a, uint32_t* keys_b, uint32_t* idx_a,
                                         uint32_t* idx_b, uint32_t* tmp,
                                         const uint32_t* gather_src, uint32_t* gather_dst,
                                         cudaStream_t s);
// The instances of launch_emit_sorted (keys view << tile_bits | tile,
// tile_bits <= 9) in one stable pass by tile within each view's contiguous
// run (offsets: the emission scan, view m's run starts at offsets[m K]);
// writes the sorted keys and values to keys_out / vals_out and ranges[M][T]
// ([start, end) of each (view, tile); zero when empty).  n: the instances,
// or a capacity they do not exceed (the view runs are clamped to it).  tmp
// must hold radix_views_tmp_words(n, M) uint32.
size_t radix_views_tmp_words(size_t n, int M);
void radix_sort_views(const uint32_t* keys, const uint32_t* vals, uint32_t* keys_out,
                      uint32_t* vals_out, size_t n, const uint32_t* offsets, int K, int M,
                      int tile_bits, uint2* ranges, int T, uint32_t* tmp, cudaStream_t s);

// dst[i] = src[i] for n 32-bit words, copied by a kernel (device memory or
// mapped pinned host memory on either side): for small transfers that must
// not queue behind large copies on the copy engines.
void launch_copy_words(const uint32_t* src, uint32_t* dst, size_t n, cudaStream_t s);

// ranges[M*T] = [start, end) of each (view, tile) in the sorted keys.
// ... from (view | tile) keys
void launch_tile_ranges(const uint32_t* keys, size_t n, int tile_bits, int T, uint2* ranges,
                        int M, cudaStream_t s, const uint32_t* n_dev = nullptr);

// ------------------------------------------------------------- radiance (a4)
// receiver-major [N][K][C][2] -> Gaussian-major [K][stride] (columns
// j*2C + 2c + {0,1}; pad columns are zero).
void launch_radiance_transpose(const float* rad, int N, int K, int C, int stride, float* out,
                               cudaStream_t s);
// Gaussian-major [K][stride] -> receiver-major [N][K][C][2] (accumulates).
void launch_radiance_untranspose_add(const float* in, int N, int K, int C, int stride,
                                     float* out, cudaStream_t s);

struct MlpParams {
  const float* p;  // flat parameters (fp32)
  int hidden, C, bf16;
  // occlusion inputs (T, rho_bar) of the local branch per (receiver,
  // Gaussian) pair [N][K], or null: clear (1, 0)
  const float2* feat = nullptr;
};
// Radiance from the conditioning MLP: out[K][stride] Gaussian-major.
// Optional: n_dev = receivers in use (<= N), col_of[j] = first column of
// receiver j (default j*2C); clear = zero the whole buffer first.
void launch_mlp_radiance(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, float* out, float* glob_out,
                         cudaStream_t s, const int* n_dev = nullptr, const int* col_of = nullptr,
                         bool clear = true);
// Backward of the MLP: dS[K][stride] -> grad_base[K][C][2], grad_mlp (flat).
size_t mlp_backward_tmp_floats(const MlpParams& m, int N, int K);
void launch_mlp_backward(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, int stride, const float* dS,
                         const float* glob, float* grad_base, float* grad_mlp, float* tmp,
                         cudaStream_t s);

// ------------------------------------------------------------ render (a5-a7)
struct RenderArgs {
  GridConst g;
  const float4* rec;       // [M][K][2]
  const uint32_t* vals;    // sorted Gaussian ids
  const uint2* ranges;     // [M][T]
  const float* rad;        // [K][stride], or [M][K][stride] when rad_view != 0
  size_t rad_view;         // floats between views' radiance (0: shared by all views)
  int K, M, N, C;
  int stride;              // floats per radiance row
  int ncols;               // N*2C valid columns
  float* spectra;          // [M][N][H][W][C][2] or null
  float* partial;          // [M][T][ncols] per-tile column sums or null
  int32_t* ncontrib;       // [M][H][W] or null
  float* tfinal;           // [M][H][W] or null
  unsigned* err = nullptr; // device error word (kErrTimeout), or null
  // the backward's per-pixel state, written by the tensor-core forward when
  // set (column block 0): final T and stop position per pixel, largest stop
  // per tile, as the backward pre-pass computes them (render_bwd.cu)
  float* keep_tfin = nullptr;          // [M][H][W]
  uint32_t* keep_stops = nullptr;      // [M][H][W]
  uint32_t* keep_tile_stop = nullptr;  // [M][T]
};
// Whether launch_render_fwd writes keep_* for these columns per CTA.
inline bool render_fwd_keeps_stops(int cols_per_cta) { return cols_per_cta == 128; }
void launch_render_fwd(const RenderArgs& a, int cols_per_cta, cudaStream_t s);

// Sums partial[M][T][ncols] over tiles -> csi[M][N][C][2], rssi[M][N].
void launch_reduce_tiles(const float* partial, int M, int T, int N, int C, float* csi,
                         float* rssi, cudaStream_t s);

struct BackwardArgs {
  RenderArgs f;               // forward arguments (spectra = fwd spectra or null)
  const float* g_spec;        // [M][N][H][W][C][2] or null
  const float* g_uniform;     // [M][ncols] cotangent uniform over pixels, or null
  float* d_rad;               // [K][stride] (per view [M][K][stride] when f.rad_view != 0) dL/ds, atomics
  float* d_tau;               // [K] accumulated
  float* tfin;                // scratch [M][H][W]: final transmittance per pixel
  uint32_t* stops;            // scratch [M][H][W]: stop position per pixel
  uint32_t* tile_stop;        // scratch [M][T]: largest stop of each tile
  uint32_t n_inst;
  unsigned* err;              // device error word (kErrTimeout), or null
};
// Walk 1 of the backward (final T and stop per pixel, largest stop per tile)
void launch_bwd_prepass(const BackwardArgs& a, cudaStream_t s);
// Walk 2: the back-to-front sweep producing d_rad and d_tau
void launch_render_bwd(const BackwardArgs& a, cudaStream_t s);
// CSI / RSSI cotangents with explicit receiver-major radiance rad_rm
// [N][K][C][2]: gamma [M][K] and W [M][K] (zeroed by the caller) are
// scratch; d_tau += ..., grad_radiance (or null) += sum_v W g.  Needs the
// pre-pass outputs in A (tfin, stops, tile_stop).
void launch_vis_backward(const BackwardArgs& A, const float* rad_rm, const float* gu,
                         float* gamma, float* W, float* grad_radiance, cudaStream_t s);

// ------------------------------------------------ Stage II L1 term (App. E.3)
// loss[0] = mean |a_i - y_i| over n values (a = |R| of spectra [n][2], or
// RSSI [n]) and grad = its derivative; part holds nparts block sums.
int l1_loss_blocks();
void launch_l1_loss(bool spectra, const float* values, const float* target, size_t n, float* loss,
                    float* grad, float* part, int nparts, cudaStream_t s);
// ------------------------------------------ occupancy grid and probes (App. E.5)
// box[6] = (lo, D) and grid[res^3] from the scene's Gaussians.
void launch_occ_build(const float4* geom, int K, int res, float* box, float* grid, cudaStream_t s);
// feat[N][K] = (T, rho_bar) along each (Gaussian, receiver) segment.
void launch_occ_probes(const float4* geom, int K, const float* rx, int N, int res,
                       const float* box, const float* grid, float2* feat, cudaStream_t s);

// ------------------------------------------ FLE directional radiance (App. E.2)
// The recurrence of the normalised basis y_lm = N_l|m| P_l^m (App. E.2),
// l, m <= 9: r[l][m] = (a, b) with y_lm = a ct y_{l-1,m} - b y_{l-2,m} for
// m < l (b = 0 for m = l - 1), y_ll = a st y_{l-1,l-1} for l >= 1 and
// y_00 = a (ct = cos theta, st = sin theta).
struct FleRec {
  float r[10][10][2];
};
FleRec fle_rec_table();
// The basis operand image (fle_tc.cu): for every (Gaussian, group of 32
// views) the bf16 hi / lo terms of Yr and Yi in the layout the tensor-core
// kernels stage (14,336 bytes each), K * ceil(M / 32) blocks.
size_t fle_basis_image_bytes(int K, int M);
void launch_fle_basis_image(const float4* geom, const float* tx, int K, int M, int lmax,
                            unsigned char* image, cudaStream_t s);
// The tensor-core coefficient gradient (fle_bwd_tc.cu) from the cotangent
// d_rad (the radiance layout below) and the basis image; err receives
// kErrTimeout.  With accumulate false grad is written, not added to.
void launch_fle_backward_tc(const float* d_rad, int N, int K, int lmax,
                            const unsigned char* image, int M, int stride, size_t rad_view,
                            float* grad, bool accumulate, cudaStream_t s, unsigned* err);
// The tensor-core contraction of the FLE radiance (fle_tc.cu) for
// coefficients [N][K][2][L] and the basis image: rad[v][k][stride] columns
// 2j, 2j+1 (v < M, rad_view floats per view); err receives kErrTimeout.
void launch_fle_radiance_tc(const float* coeffs, int N, int K, int lmax,
                            const unsigned char* image, int M, int stride, size_t rad_view,
                            float* rad, cudaStream_t s, unsigned* err);
// The same contraction with the coefficients formed inside it (the global
// FiLM branch, Eq. film_apply): c[j][k][.][l] = (1 + a_jl) base[k][.][l] +
// b_jl (complex) from the base coefficients base[K][2][L] and the
// modulations ab[N][L] = (a.re, a.im, b.re, b.im); when loc is not null,
// the local factors loc[N][K] = (alpha.re, alpha.im, beta.re, beta.im) make
// it (1 + alpha) c + beta (Eq. combined_local).  c is never written to
// memory.
void launch_fle_radiance_film_tc(const float* base, const float4* ab, const float4* loc, int N,
                                 int K, int lmax, const unsigned char* image, int M, int stride,
                                 size_t rad_view, float* rad, cudaStream_t s, unsigned* err);
// The fold of the conditioned coefficients' gradient G[N][K][2][L] (fle_tc.cu)
// into grad_base[K][2][L] += sum_j conj(1 + a) G and d_ab[N][L][4] +=
// sum_k (conj(base) G, G) (either may be NULL).
void launch_film_fold(const float* G, int N, int K, int lmax, const float* base,
                      const float4* ab, float* grad_base, float* d_ab, cudaStream_t s);

// ------------------ local branch composed with the FiLM branch (film_local.cu)
// The scene MLP's local branch supports the composition for 64 hidden units
// and one channel.  loc[N][K] = (alpha.re, alpha.im, beta.re, beta.im) of
// every (receiver, Gaussian) pair (feat = occlusion inputs or NULL).
bool local_branch_supported(int hidden, int C);
void launch_local_factors(const float* mlp, const float* rx, int N, const float4* geom, int K,
                          const float2* feat, float4* loc, cudaStream_t s);
// From the composed coefficients' gradient G[N][K][2][L] (overwritten in
// place by conj(1 + alpha) G, the FiLM-modulated coefficients' gradient):
// d_loc[N][K] (scratch) and grad_mlp's local-branch entries += their
// gradient (grad_mlp may be NULL).
void launch_film_local_backward(float* G, const float* base, const float4* ab, const float4* loc,
                                const float* mlp, const float* rx, int N, const float4* geom,
                                int K, int lmax, const float2* feat, float4* d_loc,
                                float* grad_mlp, cudaStream_t s);
// ------------------------------------------ global FiLM MLP over FLE components
// Packed parameters (float32): omega[nw][3], embed[L][dc], w1[D][din], b1[D],
// w2[D][D], b2[D], w3[4][D], b3[4] with din = 2 nw + 2 + dc (Eq. rx_enc, film).
struct FilmDims {
  int nw, dc, D, lmax, L, din;
  size_t o_omega, o_embed, o_w1, o_b1, o_w2, o_b2, o_w3, o_b3, total;
};
constexpr int kFilmMaxFreq = 32, kFilmMaxEmbed = 64, kFilmMaxHidden = 256;
FilmDims film_dims(int nw, int dc, int D, int lmax);
// ab[N][L] = MLP_global([gamma(r_j); c_l; e_l]) for every receiver and component.
void launch_film_global(const float* film, const FilmDims& f, const float* rx, int N, float4* ab,
                        cudaStream_t s);
// grad_film (packed as above) += the gradient of sum(d_ab * ab) over every
// parameter; tmp holds film_backward_tmp_floats(f, N) floats.
size_t film_backward_tmp_floats(const FilmDims& f, int N);
void launch_film_backward(const float* film, const FilmDims& f, const float* rx, int N,
                          const float4* d_ab, float* tmp, float* grad_film, cudaStream_t s);


// ------------------------------------------ visibility weights (Eq. render_reorder)
// W[M][K] = sum over each view's pixels of T_k w_k (zeroed first).
void launch_visibility(const RenderArgs& a, float* W, cudaStream_t s);
// csi[M][N][C][2] (and rssi[M][N] when C == 1) = sum_k W[v][k] rad[j][k][:],
// rad receiver-major [N][K][C][2].  Needs 256 % (2C) == 0.
bool weighted_sum_supported(int C);
size_t weighted_sum_tmp_floats(int M, int K, int N, int C);
void launch_weighted_sum(const float* rad, int N, int K, int C, const float* W, int M, float* tmp,
                         float* csi, float* rssi, cudaStream_t s);
// The same with the radiance from the conditioning MLP, evaluated on the fly
// (never stored) and only where the weight is non-zero.  rx_view == NULL:
// every receiver with every view, outputs [M][N][C][2]; otherwise receiver j
// with view rx_view[j] only, outputs [N][C][2].  C <= 52.
size_t mlp_weighted_tmp_floats(int M, int K, int N, int C);
void launch_mlp_weighted(const MlpParams& m, const float* rx, int N, const float4* geom,
                         const float* base, int K, const float* W, int M, const int* rx_view,
                         const float* glob, float* tmp, float* csi, float* rssi,
                         const int* n_dev, cudaStream_t s);
// glob[N][4C] = global MLP branch of every receiver (n_dev optional).
void launch_mlp_global(const MlpParams& m, const float* rx, int N, float* glob, cudaStream_t s,
                       const int* n_dev = nullptr);

// Read-only view of a context's prepared transmitter-side state, for entry
// points that live outside api.cu.  Returns false for an unknown handle.
struct ViewsRef {
  int device;
  GridConst g;
  int M, K, C;
  const float4* rec;
  const uint32_t* vals;
  const uint2* ranges;
};
bool lookup_views(void* ctx, uint64_t views, ViewsRef* out, const char** err);

}  // namespace rxgs
