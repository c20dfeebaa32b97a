// film.cu -- the global conditioning branch over the FLE components
// (Eq. rx_enc, film; App. E.4) and its backward.
//
// For receiver j and component l (index l*l + l + m of degree l, order m):
//   x_jl = [gamma(r_j); c_l; e_l],  gamma = [sin(w_1.r), cos(w_1.r), ...],
//          c_l = (l, m) / max(lmax, 1), e_l the learnable embedding,
//   (a.re, a.im, b.re, b.im)_jl = W3 relu(W2 relu(W1 x + b1) + b2) + b3.
// The samples (j, l) are independent and few (N L, a few thousand), so the
// forward takes 16 samples per block with their inputs and both hidden
// layers in shared memory.  The backward recomputes that, writes each
// sample's activations and deltas to scratch, and reduces the weight
// gradients over the samples in a fixed order (chunks of samples, then the
// chunks), so the MLP gradients are deterministic.
#include <algorithm>

#include "rxgs_internal.h"

namespace rxgs {

constexpr int kFilmTS = 16;                                   // samples per block
constexpr int kFilmMaxIn = 2 * kFilmMaxFreq + 2 + kFilmMaxEmbed;  // 130
constexpr int kFilmMaxChunks = 4096;                          // partial sums per gradient

FilmDims film_dims(int nw, int dc, int D, int lmax) {
  FilmDims f{};
  f.nw = nw;
  f.dc = dc;
  f.D = D;
  f.lmax = lmax;
  f.L = (lmax + 1) * (lmax + 1);
  f.din = 2 * nw + 2 + dc;
  size_t o = 0;
  f.o_omega = o; o += 3 * static_cast<size_t>(nw);
  f.o_embed = o; o += static_cast<size_t>(f.L) * dc;
  f.o_w1 = o;    o += static_cast<size_t>(D) * f.din;
  f.o_b1 = o;    o += D;
  f.o_w2 = o;    o += static_cast<size_t>(D) * D;
  f.o_b2 = o;    o += D;
  f.o_w3 = o;    o += 4 * static_cast<size_t>(D);
  f.o_b3 = o;    o += 4;
  f.total = o;
  return f;
}

struct FilmTile {
  float x[kFilmTS][kFilmMaxIn + 1];
  float h1[kFilmTS][kFilmMaxHidden + 1];
  float h2[kFilmTS][kFilmMaxHidden + 1];
};

// Inputs and both hidden layers (after ReLU) of samples s0 .. s0 + 15;
// samples past N L get zero inputs.
__device__ void film_forward_tile(const float* __restrict__ film, const FilmDims& f,
                                  const float* __restrict__ rx, int S, int s0, FilmTile& sm) {
  const int t = threadIdx.x;
  for (int e = t; e < kFilmTS * f.din; e += blockDim.x) {
    const int i = e / f.din, q = e % f.din, s = s0 + i;
    float val = 0.0f;
    if (s < S) {
      const int j = s / f.L, l = s % f.L;
      if (q < 2 * f.nw) {
        const float* w = film + f.o_omega + 3 * (q >> 1);
        const float* r = rx + 3 * j;
        const float ph = fmaf(w[2], r[2], fmaf(w[1], r[1], w[0] * r[0]));
        val = (q & 1) ? cosf(ph) : sinf(ph);
      } else if (q < 2 * f.nw + 2) {
        int deg = 0;
        while ((deg + 1) * (deg + 1) <= l) ++deg;
        const int m = l - deg * deg - deg;
        val = static_cast<float>(q == 2 * f.nw ? deg : m) / static_cast<float>(max(f.lmax, 1));
      } else {
        val = film[f.o_embed + static_cast<size_t>(l) * f.dc + (q - 2 * f.nw - 2)];
      }
    }
    sm.x[i][q] = val;
  }
  __syncthreads();
  for (int e = t; e < kFilmTS * f.D; e += blockDim.x) {
    const int i = e / f.D, o = e % f.D;
    const float* w = film + f.o_w1 + static_cast<size_t>(o) * f.din;
    float acc = film[f.o_b1 + o];
    for (int q = 0; q < f.din; ++q) acc = fmaf(w[q], sm.x[i][q], acc);
    sm.h1[i][o] = fmaxf(acc, 0.0f);
  }
  __syncthreads();
  for (int e = t; e < kFilmTS * f.D; e += blockDim.x) {
    const int i = e / f.D, o = e % f.D;
    const float* w = film + f.o_w2 + static_cast<size_t>(o) * f.D;
    float acc = film[f.o_b2 + o];
    for (int q = 0; q < f.D; ++q) acc = fmaf(w[q], sm.h1[i][q], acc);
    sm.h2[i][o] = fmaxf(acc, 0.0f);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) film_global_kernel(const float* __restrict__ film,
                                                          FilmDims f, const float* __restrict__ rx,
                                                          int N, float* __restrict__ ab) {
  __shared__ FilmTile sm;
  const int S = N * f.L, s0 = blockIdx.x * kFilmTS, t = threadIdx.x;
  film_forward_tile(film, f, rx, S, s0, sm);
  if (t < kFilmTS * 4) {
    const int i = t / 4, p = t % 4, s = s0 + i;
    if (s < S) {
      const float* w = film + f.o_w3 + static_cast<size_t>(p) * f.D;
      float acc = film[f.o_b3 + p];
      for (int o = 0; o < f.D; ++o) acc = fmaf(w[o], sm.h2[i][o], acc);
      ab[static_cast<size_t>(s) * 4 + p] = acc;
    }
  }
}

// Scratch of the backward, per sample s: X[din], H1[D], H2[D] (forward) and
// D3[4], D2[D], D1[D], DX[din] (deltas: output, pre-activation 2 and 1, input).
struct FilmScratch {
  float *X, *H1, *H2, *D3, *D2, *D1, *DX, *part;
};

static FilmScratch film_scratch(const FilmDims& f, int N, float* tmp) {
  const size_t S = static_cast<size_t>(N) * f.L;
  FilmScratch r{};
  r.X = tmp;
  r.H1 = r.X + S * f.din;
  r.H2 = r.H1 + S * f.D;
  r.D3 = r.H2 + S * f.D;
  r.D2 = r.D3 + S * 4;
  r.D1 = r.D2 + S * f.D;
  r.DX = r.D1 + S * f.D;
  r.part = r.DX + S * f.din;
  return r;
}

// Samples per partial sum: at least 512, and at most kFilmMaxChunks chunks.
static int film_chunk_len(int S) { return std::max(512, (S + kFilmMaxChunks - 1) / kFilmMaxChunks); }

static int film_chunks(const FilmDims& f, int N) {
  const int S = N * f.L, len = film_chunk_len(S);
  return (S + len - 1) / len;
}

size_t film_backward_tmp_floats(const FilmDims& f, int N) {
  const size_t S = static_cast<size_t>(N) * f.L;
  const size_t per = 2 * static_cast<size_t>(f.din) + 4 * static_cast<size_t>(f.D) + 4;
  return S * per + static_cast<size_t>(film_chunks(f, N)) * f.total;
}

__global__ void __launch_bounds__(256) film_backward_tile_kernel(
    const float* __restrict__ film, FilmDims f, const float* __restrict__ rx, int N,
    const float4* __restrict__ d_ab, FilmScratch sc) {
  __shared__ FilmTile sm;
  __shared__ float sD3[kFilmTS][4];
  const int S = N * f.L, s0 = blockIdx.x * kFilmTS, t = threadIdx.x;
  film_forward_tile(film, f, rx, S, s0, sm);
  const int ns = min(kFilmTS, S - s0);
  for (int e = t; e < ns * f.din; e += blockDim.x)
    sc.X[static_cast<size_t>(s0) * f.din + e] = sm.x[e / f.din][e % f.din];
  for (int e = t; e < ns * f.D; e += blockDim.x) {
    sc.H1[static_cast<size_t>(s0) * f.D + e] = sm.h1[e / f.D][e % f.D];
    sc.H2[static_cast<size_t>(s0) * f.D + e] = sm.h2[e / f.D][e % f.D];
  }
  if (t < kFilmTS * 4) {
    const int i = t / 4, p = t % 4;
    float v = 0.0f;
    if (i < ns) {
      const float4 g = d_ab[s0 + i];
      v = p == 0 ? g.x : (p == 1 ? g.y : (p == 2 ? g.z : g.w));
      sc.D3[static_cast<size_t>(s0 + i) * 4 + p] = v;
    }
    sD3[i][p] = v;
  }
  __syncthreads();
  // delta of layer 2's pre-activation, in place of h2 (each entry is read
  // and rewritten by the same thread)
  for (int e = t; e < kFilmTS * f.D; e += blockDim.x) {
    const int i = e / f.D, o = e % f.D;
    float v = 0.0f;
    if (sm.h2[i][o] > 0.0f) {
#pragma unroll
      for (int p = 0; p < 4; ++p) v = fmaf(film[f.o_w3 + static_cast<size_t>(p) * f.D + o], sD3[i][p], v);
    }
    sm.h2[i][o] = v;
    if (i < ns) sc.D2[static_cast<size_t>(s0 + i) * f.D + o] = v;
  }
  __syncthreads();
  // delta of layer 1's pre-activation, in place of h1
  for (int e = t; e < kFilmTS * f.D; e += blockDim.x) {
    const int i = e / f.D, o = e % f.D;
    float v = 0.0f;
    if (sm.h1[i][o] > 0.0f) {
      for (int q = 0; q < f.D; ++q)
        v = fmaf(film[f.o_w2 + static_cast<size_t>(q) * f.D + o], sm.h2[i][q], v);
    }
    sm.h1[i][o] = v;
    if (i < ns) sc.D1[static_cast<size_t>(s0 + i) * f.D + o] = v;
  }
  __syncthreads();
  // delta of the inputs
  for (int e = t; e < ns * f.din; e += blockDim.x) {
    const int i = e / f.din, q = e % f.din;
    float v = 0.0f;
    for (int o = 0; o < f.D; ++o)
      v = fmaf(film[f.o_w1 + static_cast<size_t>(o) * f.din + q], sm.h1[i][o], v);
    sc.DX[static_cast<size_t>(s0 + i) * f.din + q] = v;
  }
}

// Partial sums over one chunk of samples of every weight and bias gradient
// (the packed offsets from o_w1 on): part[chunk][total].
__global__ void __launch_bounds__(256) film_wgrad_kernel(FilmDims f, int S, int chunk,
                                                         FilmScratch sc) {
  const size_t nparam = f.total - f.o_w1;
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= nparam) return;
  const size_t pidx = f.o_w1 + idx;
  const int s0 = blockIdx.y * chunk, s1 = min(S, s0 + chunk);
  // which gradient: (delta array, its width, column), (input array, width, column or -1 = bias)
  const float *dl, *in = nullptr;
  int dw, dcol, iw = 0, icol = -1;
  if (pidx < f.o_b1) {
    const size_t r = pidx - f.o_w1;
    dl = sc.D1; dw = f.D; dcol = static_cast<int>(r / f.din);
    in = sc.X; iw = f.din; icol = static_cast<int>(r % f.din);
  } else if (pidx < f.o_w2) {
    dl = sc.D1; dw = f.D; dcol = static_cast<int>(pidx - f.o_b1);
  } else if (pidx < f.o_b2) {
    const size_t r = pidx - f.o_w2;
    dl = sc.D2; dw = f.D; dcol = static_cast<int>(r / f.D);
    in = sc.H1; iw = f.D; icol = static_cast<int>(r % f.D);
  } else if (pidx < f.o_w3) {
    dl = sc.D2; dw = f.D; dcol = static_cast<int>(pidx - f.o_b2);
  } else if (pidx < f.o_b3) {
    const size_t r = pidx - f.o_w3;
    dl = sc.D3; dw = 4; dcol = static_cast<int>(r / f.D);
    in = sc.H2; iw = f.D; icol = static_cast<int>(r % f.D);
  } else {
    dl = sc.D3; dw = 4; dcol = static_cast<int>(pidx - f.o_b3);
  }
  float acc = 0.0f;
  if (in) {
    for (int s = s0; s < s1; ++s)
      acc = fmaf(dl[static_cast<size_t>(s) * dw + dcol], in[static_cast<size_t>(s) * iw + icol], acc);
  } else {
    for (int s = s0; s < s1; ++s) acc += dl[static_cast<size_t>(s) * dw + dcol];
  }
  sc.part[static_cast<size_t>(blockIdx.y) * f.total + pidx] = acc;
}

// grad_film += the chunk partials in chunk order (weights and biases), and
// the embedding gradients summed over the samples in order (the frequency
// vectors: film_freq_grad_kernel).
__global__ void __launch_bounds__(256) film_grad_finish_kernel(const float* __restrict__ film,
                                                               FilmDims f,
                                                               const float* __restrict__ rx, int N,
                                                               int nchunk, FilmScratch sc,
                                                               float* __restrict__ grad) {
  const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= f.total) return;
  float acc = 0.0f;
  if (idx >= f.o_w1) {
    for (int c = 0; c < nchunk; ++c) acc += sc.part[static_cast<size_t>(c) * f.total + idx];
  } else if (idx >= f.o_embed) {
    // dL/de_l[e] = sum_j DX[j L + l][2 nw + 2 + e]
    const size_t r = idx - f.o_embed;
    const int l = static_cast<int>(r / f.dc), e = static_cast<int>(r % f.dc);
    for (int j = 0; j < N; ++j)
      acc += sc.DX[(static_cast<size_t>(j) * f.L + l) * f.din + 2 * f.nw + 2 + e];
  } else {
    return;  // the frequency vectors: film_freq_grad_kernel
  }
  grad[idx] += acc;
}

// dL/dw_f[d] = sum_j r_j[d] sum_l (DX_sin cos(w_f.r_j) - DX_cos sin(w_f.r_j)):
// block f, warp w takes receivers w, w + 8, ... (lanes over components, a
// shuffle sum), then the warps' sums in warp order.
__global__ void __launch_bounds__(256) film_freq_grad_kernel(const float* __restrict__ film,
                                                             FilmDims f,
                                                             const float* __restrict__ rx, int N,
                                                             FilmScratch sc,
                                                             float* __restrict__ grad) {
  __shared__ float part[8][3];
  const int fq = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float* w = film + f.o_omega + 3 * fq;
  float acc[3] = {0.0f, 0.0f, 0.0f};
  for (int j = warp; j < N; j += 8) {
    const float* r = rx + 3 * j;
    const float ph = fmaf(w[2], r[2], fmaf(w[1], r[1], w[0] * r[0]));
    const float cs = cosf(ph), sn = sinf(ph);
    float sj = 0.0f;
    for (int l = lane; l < f.L; l += 32) {
      const float* dx = sc.DX + (static_cast<size_t>(j) * f.L + l) * f.din + 2 * fq;
      sj += fmaf(dx[0], cs, -dx[1] * sn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sj += __shfl_xor_sync(0xffffffffu, sj, o);
#pragma unroll
    for (int d = 0; d < 3; ++d) acc[d] = fmaf(sj, r[d], acc[d]);
  }
  if (lane == 0)
#pragma unroll
    for (int d = 0; d < 3; ++d) part[warp][d] = acc[d];
  __syncthreads();
  if (threadIdx.x < 3) {
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += part[q][threadIdx.x];
    grad[f.o_omega + 3 * fq + threadIdx.x] += t;
  }
}

void launch_film_global(const float* film, const FilmDims& f, const float* rx, int N, float4* ab,
                        cudaStream_t s) {
  const int S = N * f.L;
  if (S <= 0) return;
  film_global_kernel<<<(S + kFilmTS - 1) / kFilmTS, 256, 0, s>>>(film, f, rx, N,
                                                                 reinterpret_cast<float*>(ab));
  note_launches(1);
}

void launch_film_backward(const float* film, const FilmDims& f, const float* rx, int N,
                          const float4* d_ab, float* tmp, float* grad_film, cudaStream_t s) {
  const int S = N * f.L;
  if (S <= 0) return;
  const FilmScratch sc = film_scratch(f, N, tmp);
  film_backward_tile_kernel<<<(S + kFilmTS - 1) / kFilmTS, 256, 0, s>>>(film, f, rx, N, d_ab, sc);
  const int nchunk = film_chunks(f, N);
  const size_t nparam = f.total - f.o_w1;
  const dim3 grid(static_cast<unsigned>((nparam + 255) / 256), static_cast<unsigned>(nchunk));
  film_wgrad_kernel<<<grid, 256, 0, s>>>(f, S, film_chunk_len(S), sc);
  film_grad_finish_kernel<<<static_cast<unsigned>((f.total + 255) / 256), 256, 0, s>>>(
      film, f, rx, N, nchunk, sc, grad_film);
  if (f.nw > 0) film_freq_grad_kernel<<<f.nw, 256, 0, s>>>(film, f, rx, N, sc, grad_film);
  note_launches(f.nw > 0 ? 4 : 3);
}

}  // namespace rxgs
