/*
 * rxgs_oracle.c -- CPU oracle of the multi-receiver RF Gaussian renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  The product
 * path (the CUDA library) never calls it and shares no code with it.
 *
 * It is a plain, slow, obviously correct restatement of the method:
 *   - Gaussian state and covariance Sigma = R S S^T R^T           (App. E.1)
 *   - projection onto the angular grid centred at the transmitter
 *     (Eq. dk; Algorithm 1, Stage 1)
 *   - every pixel composites the Gaussians whose 3-sigma footprint holds it,
 *     in ascending depth order, front to back with
 *     w = tau * exp(-q/2), C += T w s, T *= (1 - w), stop once T < eps
 *                                                     (Algorithm 1, Stage 3)
 *   - amplitude |R| = sqrt(Re^2 + Im^2 + 1e-8)                  (App. E.2)
 *   - RSSI / CSI as the coherent sum over directions (Def. 2, Eq. render;
 *     Eq. render_reorder)
 *   - the exact derivative of the above with respect to the radiance and
 *     the opacity, decisions held fixed (App. D, backward kernel)
 *
 * Values are computed in float64.  Every DISCRETE decision (culling, the
 * footprint, the per-tile depth order, the q <= q_max test and the T < eps
 * stop) is taken by a float32 "shadow" whose operation order is written out
 * below, so that a float32 implementation that follows the same order takes
 * the same decisions.  The shadow's exp and atan2 are written here from
 * their textbook definitions (Cody-Waite reduction + Taylor series; octant
 * reduction + Gregory series) rather than taken from libm, whose float
 * results differ between platforms.
 *
 * Compile with -ffp-contract=off (no silent FMA contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int H, W;           /* rows = elevation, columns = azimuth                 */
  double theta0_deg;  /* elevation of row 0                                  */
  double step_deg;    /* angular step of both axes                           */
  int TH, TW;         /* tile height / width in pixels                       */
  float eps_T;        /* transmittance stop threshold                        */
  float q_max;        /* Mahalanobis cut-off (9 = 3 sigma)                   */
  float r_near;       /* Gaussians closer than this to the centre are culled */
} or_grid;

/* ------------------------------------------------------------------ consts
 * Correctly rounded binary32 values of mathematical constants (hex floats). */
#define F_LOG2E    0x1.715476p+0f   /* 1/ln 2                */
#define F_LN2_HI   0x1.62e430p-1f   /* ln 2                  */
#define F_LN2_LO  -0x1.05c610p-29f  /* ln 2 - F_LN2_HI       */
#define F_PI       0x1.921fb6p+1f
#define F_PI_2     0x1.921fb6p+0f
#define F_PI_4     0x1.921fb6p-1f
#define F_TWO_PI   0x1.921fb6p+2f
#define F_TAN_PI_8 0x1.a8279ap-2f   /* tan(pi/8) = sqrt(2)-1 */

/* ----------------------------------------------------- float32 exp (shadow)
 * Cody & Waite (1980) range reduction x = n ln2 + r, |r| <= ln2/2, with ln 2
 * split in two floats, then the Taylor polynomial of e^r to degree 7
 * (truncation < 1e-8 relative), then an exact scaling by 2^n.              */
float or_exp32(float x) {
  if (!(x > -87.0f)) return 0.0f;
  if (x > 88.0f) return INFINITY;
  float t = x * F_LOG2E;
  float n = rintf(t);
  float r = fmaf(-n, F_LN2_HI, x);
  r = fmaf(-n, F_LN2_LO, r);
  float p = 1.0f / 5040.0f;
  p = fmaf(p, r, 1.0f / 720.0f);
  p = fmaf(p, r, 1.0f / 120.0f);
  p = fmaf(p, r, 1.0f / 24.0f);
  p = fmaf(p, r, 1.0f / 6.0f);
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  uint32_t bits = (uint32_t)((int)n + 127) << 23;
  float s;
  memcpy(&s, &bits, 4);
  return p * s;
}

/* --------------------------------------------------- float32 atan2 (shadow)
 * Reduce to t = min/max in [0,1]; for t > tan(pi/8) use
 * atan t = pi/4 + atan((t-1)/(t+1)) so |t'| <= tan(pi/8); Gregory series
 * atan t' = sum_k (-1)^k t'^(2k+1)/(2k+1), k = 0..9 (truncation < 1e-9);
 * then undo the octant folding.                                             */
float or_atan2_32(float y, float x) {
  float ax = fabsf(x), ay = fabsf(y);
  float mx = ax > ay ? ax : ay;
  float mn = ax > ay ? ay : ax;
  if (mx == 0.0f) return 0.0f;
  float t = mn / mx;
  float base = 0.0f;
  if (t > F_TAN_PI_8) {
    t = (t - 1.0f) / (t + 1.0f);
    base = F_PI_4;
  }
  float z = t * t;
  float p = -1.0f / 19.0f;
  p = fmaf(p, z, 1.0f / 17.0f);
  p = fmaf(p, z, -1.0f / 15.0f);
  p = fmaf(p, z, 1.0f / 13.0f);
  p = fmaf(p, z, -1.0f / 11.0f);
  p = fmaf(p, z, 1.0f / 9.0f);
  p = fmaf(p, z, -1.0f / 7.0f);
  p = fmaf(p, z, 1.0f / 5.0f);
  p = fmaf(p, z, -1.0f / 3.0f);
  p = fmaf(p, z, 1.0f);
  float a = fmaf(t, p, base);
  if (ay > ax) a = F_PI_2 - a;
  if (x < 0.0f) a = F_PI - a;
  if (y < 0.0f) a = -a;
  return a;
}

/* ------------------------------------------------------------- covariance
 * Sigma = R S S^T R^T with R from the normalised quaternion (w,x,y,z) and
 * S = diag(exp(s)) (App. E.1).  Output order: S00 S01 S02 S11 S12 S22.     */
void or_cov32(const float s[3], const float q[4], float S[6]) {
  float n2 = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3])));
  float w = 1.0f, x = 0.0f, y = 0.0f, z = 0.0f;
  if (n2 > 0.0f) {
    float nr = sqrtf(n2);
    w = q[0] / nr; x = q[1] / nr; y = q[2] / nr; z = q[3] / nr;
  }
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (yy + zz);
  R[0][1] = 2.0f * (xy - wz);
  R[0][2] = 2.0f * (xz + wy);
  R[1][0] = 2.0f * (xy + wz);
  R[1][1] = 1.0f - 2.0f * (xx + zz);
  R[1][2] = 2.0f * (yz - wx);
  R[2][0] = 2.0f * (xz - wy);
  R[2][1] = 2.0f * (yz + wx);
  R[2][2] = 1.0f - 2.0f * (xx + yy);
  float sg[3] = {or_exp32(s[0]), or_exp32(s[1]), or_exp32(s[2])};
  float M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M[a][b] = R[a][b] * sg[b];
  static const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int e = 0; e < 6; ++e) {
    int a = ia[e], b = ib[e];
    S[e] = fmaf(M[a][2], M[b][2], fmaf(M[a][1], M[b][1], M[a][0] * M[b][0]));
  }
}

void or_cov64(const float s[3], const float q[4], double S[6]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double n2 = w * w + x * x + y * y + z * z;
  if (n2 > 0.0) {
    double nr = sqrt(n2);
    w /= nr; x /= nr; y /= nr; z /= nr;
  } else {
    w = 1.0; x = y = z = 0.0;
  }
  double R[3][3] = {
      {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
      {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
      {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  double sg[3] = {exp((double)s[0]), exp((double)s[1]), exp((double)s[2])};
  double Sig[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0;
      for (int l = 0; l < 3; ++l) acc += R[a][l] * sg[l] * sg[l] * R[b][l];
      Sig[a][b] = acc;
    }
  S[0] = Sig[0][0]; S[1] = Sig[0][1]; S[2] = Sig[0][2];
  S[3] = Sig[1][1]; S[4] = Sig[1][2]; S[5] = Sig[2][2];
}

/* ------------------------------------------------------------- projection */
typedef struct {
  int vis;                 /* 0 = culled                                     */
  float theta_px, phi_px;  /* centre in pixel units                          */
  float ca, cb2, cc;       /* conic (inverse 2D covariance), cb2 = 2*conic_b */
  float rho;               /* depth = distance to the centre (sort key)      */
  int i_lo, i_hi;          /* footprint rows                                 */
  int j_lo, span;          /* footprint columns j_lo .. j_lo+span (mod W)    */
  int wrap_hi;             /* 1 if the raw azimuth was folded from >= W      */
} or_p32;

typedef struct {
  double theta_px, phi_px; /* centre in pixel units (same branch as shadow)  */
  double ca, cb, cc;       /* conic                                          */
} or_p64;

static float or_inv_step(const or_grid* g) {
  return (float)(180.0 / (3.14159265358979323846 * g->step_deg));
}
static float or_theta0_px(const or_grid* g) { return (float)(g->theta0_deg / g->step_deg); }

/* float32 shadow of the projection (Algorithm 1, Stage 1 / App. D).  The
 * operation order here is the decision specification.                     */
void or_project32(const or_grid* g, const float p[3], float tau, const float S[6],
                  const float c[3], or_p32* o) {
  memset(o, 0, sizeof(*o));
  const float inv_step = or_inv_step(g), th0 = or_theta0_px(g);
  const float Wf = (float)g->W;
  float ux = p[0] - c[0], uy = p[1] - c[1], uz = p[2] - c[2];
  float hh = fmaf(uy, uy, ux * ux);
  float rr = fmaf(uz, uz, hh);
  float rho = sqrtf(rr), h = sqrtf(hh);
  if (!(rho >= g->r_near) || !(h > 1e-6f * rho)) return;
  float phi = or_atan2_32(uy, ux);
  if (phi < 0.0f) phi = phi + F_TWO_PI;
  float phi_px = phi * inv_step;
  int wrap_hi = 0;
  if (phi_px >= Wf) { phi_px = phi_px - Wf; wrap_hi = 1; }
  float th = or_atan2_32(uz, h);
  float theta_px = th * inv_step - th0;
  float gt = inv_step / (rr * h);
  float gp = inv_step / hh;
  float J00 = -(ux * uz) * gt, J01 = -(uy * uz) * gt, J02 = hh * gt;
  float J10 = -uy * gp, J11 = ux * gp;
  float S00 = S[0], S01 = S[1], S02 = S[2], S11 = S[3], S12 = S[4], S22 = S[5];
  float t0x = fmaf(S02, J02, fmaf(S01, J01, S00 * J00));
  float t0y = fmaf(S12, J02, fmaf(S11, J01, S01 * J00));
  float t0z = fmaf(S22, J02, fmaf(S12, J01, S02 * J00));
  float t1x = fmaf(S01, J11, S00 * J10);
  float t1y = fmaf(S11, J11, S01 * J10);
  float a = fmaf(J02, t0z, fmaf(J01, t0y, J00 * t0x));
  float b = fmaf(J11, t0y, J10 * t0x);
  float cc = fmaf(J11, t1y, J10 * t1x);
  float det = fmaf(a, cc, -(b * b));
  if (!(a > 0.0f) || !(cc > 0.0f) || !(det > 0.0f)) return;
  float kq = sqrtf(g->q_max);
  float et = kq * sqrtf(a), ep = kq * sqrtf(cc);
  float lo = ceilf(theta_px - et), hi = floorf(theta_px + et);
  if (lo < 0.0f) lo = 0.0f;
  if (hi > (float)(g->H - 1)) hi = (float)(g->H - 1);
  if (!(lo <= hi)) return;
  float clo = ceilf(phi_px - ep), chi = floorf(phi_px + ep);
  if (!(clo <= chi)) return;   /* no column centre inside the footprint */
  int j_lo, span;
  if (chi - clo >= Wf - 1.0f) {
    j_lo = 0; span = g->W - 1;
  } else {
    int jl = (int)clo, jh = (int)chi;
    span = jh - jl;
    j_lo = jl < 0 ? jl + g->W : (jl >= g->W ? jl - g->W : jl);   /* into [0, W) */
  }
  o->vis = 1;
  o->theta_px = theta_px; o->phi_px = phi_px;
  o->ca = cc / det; o->cb2 = 2.0f * (-b / det); o->cc = a / det;
  o->rho = rho;
  o->i_lo = (int)lo; o->i_hi = (int)hi; o->j_lo = j_lo; o->span = span;
  o->wrap_hi = wrap_hi;
}

/* float64 values of the projection.  The azimuth branch (folding into
 * [0, W)) follows the shadow so both describe the same point.              */
void or_project64(const or_grid* g, const float p[3], const double S[6], const float c[3],
                  const or_p32* s32, or_p64* o) {
  const double inv_step = 180.0 / (3.14159265358979323846 * g->step_deg);
  double ux = (double)p[0] - c[0], uy = (double)p[1] - c[1], uz = (double)p[2] - c[2];
  double hh = ux * ux + uy * uy, rr = hh + uz * uz, h = sqrt(hh);
  double phi_px = atan2(uy, ux) * inv_step;
  /* bring to the shadow's branch: nearest representative to s32->phi_px */
  double d = phi_px - s32->phi_px;
  d -= g->W * floor(d / g->W + 0.5);
  o->phi_px = s32->phi_px + d;
  o->theta_px = atan2(uz, h) * inv_step - g->theta0_deg / g->step_deg;
  double J[2][3] = {{-ux * uz / (rr * h) * inv_step, -uy * uz / (rr * h) * inv_step, hh / (rr * h) * inv_step},
                    {-uy / hh * inv_step, ux / hh * inv_step, 0.0}};
  double Sg[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  double A[2][2];
  for (int r = 0; r < 2; ++r)
    for (int s = 0; s < 2; ++s) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += J[r][i] * Sg[i][j] * J[s][j];
      A[r][s] = acc;
    }
  double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
  o->ca = A[1][1] / det;
  o->cb = -A[0][1] / det;
  o->cc = A[0][0] / det;
}

/* 2D covariance in float64 for the closed-form tests: [a b c] */
void or_sigma2d64(const or_grid* g, const float p[3], const double S[6], const float c[3],
                  double out[3]) {
  const double inv_step = 180.0 / (3.14159265358979323846 * g->step_deg);
  double ux = (double)p[0] - c[0], uy = (double)p[1] - c[1], uz = (double)p[2] - c[2];
  double hh = ux * ux + uy * uy, rr = hh + uz * uz, h = sqrt(hh);
  double J[2][3] = {{-ux * uz / (rr * h) * inv_step, -uy * uz / (rr * h) * inv_step, hh / (rr * h) * inv_step},
                    {-uy / hh * inv_step, ux / hh * inv_step, 0.0}};
  double Sg[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  double A[2][2];
  for (int r = 0; r < 2; ++r)
    for (int s = 0; s < 2; ++s) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += J[r][i] * Sg[i][j] * J[s][j];
      A[r][s] = acc;
    }
  out[0] = A[0][0]; out[1] = A[0][1]; out[2] = A[1][1];
}

/* Is pixel (i, jj) inside the footprint?                                    */
static int or_in_footprint(const or_grid* g, const or_p32* s, int i, int jj) {
  if (i < s->i_lo || i > s->i_hi) return 0;
  int dj = jj - s->j_lo;
  if (dj < 0) dj += g->W;
  return dj <= s->span;
}

/* float32 shadow of the per-pixel weight.  Returns 0 when q > q_max.
 * *wrapm receives the multiple of W subtracted from the azimuth offset.     */
static int or_weight32(const or_grid* g, const or_p32* s, float tau, int i, int jj,
                       float* w_out, int* wrapm) {
  const float Wf = (float)g->W, halfW = 0.5f * (float)g->W;
  float dt = (float)i - s->theta_px;
  float dp = (float)jj - s->phi_px;
  int m = 0;
  if (dp >= halfW) { dp = dp - Wf; m = 1; }
  else if (dp < -halfW) { dp = dp + Wf; m = -1; }
  float t1 = s->cb2 * dp;
  float t2 = fmaf(s->ca, dt, t1);
  float t3 = s->cc * dp;
  float t4 = t3 * dp;
  float q = fmaf(dt, t2, t4);
  if (!(q <= g->q_max)) return 0;
  float G = or_exp32(-0.5f * q);
  *w_out = tau * G;
  *wrapm = m;
  return 1;
}

static double or_weight64(const or_grid* g, const or_p64* v, double tau, int i, int jj, int m,
                          double* G_out) {
  double dt = i - v->theta_px;
  double dp = jj - v->phi_px - (double)m * g->W;
  double q = v->ca * dt * dt + 2.0 * v->cb * dt * dp + v->cc * dp * dp;
  double G = exp(-0.5 * q);
  if (G_out) *G_out = G;
  return tau * G;
}

/* ------------------------------------------------------------ scene state */
typedef struct {
  int K;
  const float *p, *s, *q, *tau;
  float* S32;    /* [K][6] */
  double* S64;   /* [K][6] */
  or_p32* P32;   /* [K]    */
  or_p64* P64;   /* [K]    */
  int* order;    /* visible Gaussians in ascending (rho32, k)            */
  int nvis;
} or_view;

static const or_p32* g_cmp_base;
static int or_cmp_depth(const void* A, const void* B) {
  int a = *(const int*)A, b = *(const int*)B;
  float ra = g_cmp_base[a].rho, rb = g_cmp_base[b].rho;
  if (ra < rb) return -1;
  if (ra > rb) return 1;
  return (a > b) - (a < b);
}

static int or_view_init(or_view* V, const or_grid* g, int K, const float* p, const float* s,
                        const float* q, const float* tau, const float c[3]) {
  V->K = K; V->p = p; V->s = s; V->q = q; V->tau = tau;
  V->S32 = (float*)malloc(sizeof(float) * 6 * (size_t)K);
  V->S64 = (double*)malloc(sizeof(double) * 6 * (size_t)K);
  V->P32 = (or_p32*)malloc(sizeof(or_p32) * (size_t)K);
  V->P64 = (or_p64*)malloc(sizeof(or_p64) * (size_t)K);
  V->order = (int*)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
  if (!V->S32 || !V->S64 || !V->P32 || !V->P64 || !V->order) return -1;
  V->nvis = 0;
  for (int k = 0; k < K; ++k) {
    or_cov32(s + 3 * k, q + 4 * k, V->S32 + 6 * k);
    or_cov64(s + 3 * k, q + 4 * k, V->S64 + 6 * k);
    or_project32(g, p + 3 * k, tau[k], V->S32 + 6 * k, c, V->P32 + k);
    if (V->P32[k].vis) {
      or_project64(g, p + 3 * k, V->S64 + 6 * k, c, V->P32 + k, V->P64 + k);
      V->order[V->nvis++] = k;
    }
  }
  g_cmp_base = V->P32;
  qsort(V->order, (size_t)V->nvis, sizeof(int), or_cmp_depth);
  return 0;
}

static void or_view_free(or_view* V) {
  free(V->S32); free(V->S64); free(V->P32); free(V->P64); free(V->order);
}

/* ------------------------------------------------------ exported: shadows */

/* Projection records of one view, float32 shadow.  rec[K][8] =
 * {theta_px, phi_px, ca, cb2, cc, tau, rho, vis}; box[K][4] = {i_lo, i_hi,
 * j_lo, span}.  Returns the number of visible Gaussians.                    */
int or_project_view32(const or_grid* g, int K, const float* p, const float* s, const float* q,
                      const float* tau, const float* c, float* S6, float* rec, int* box) {
  int nvis = 0;
  for (int k = 0; k < K; ++k) {
    float S[6];
    or_p32 o;
    or_cov32(s + 3 * k, q + 4 * k, S);
    if (S6) memcpy(S6 + 6 * k, S, sizeof S);
    or_project32(g, p + 3 * k, tau[k], S, c, &o);
    float* r = rec + 8 * (size_t)k;
    r[0] = o.theta_px; r[1] = o.phi_px; r[2] = o.ca; r[3] = o.cb2; r[4] = o.cc;
    r[5] = tau[k]; r[6] = o.rho; r[7] = (float)o.vis;
    int* b = box + 4 * (size_t)k;
    b[0] = o.i_lo; b[1] = o.i_hi; b[2] = o.j_lo; b[3] = o.span;
    nvis += o.vis;
  }
  return nvis;
}

/* Tile sets by enumerating every footprint pixel, and per-tile lists sorted
 * by (rho, k) (Algorithm 1, Stage 1: per-tile depth-sorted list).
 * counts[tiles]; lists = concatenation in tile order (capacity cap).
 * ntiles_per_g[K] = size of each Gaussian's tile set.
 * Returns the total number of instances, or -1 if cap is too small.         */
long or_tile_lists(const or_grid* g, int K, const float* p, const float* s, const float* q,
                   const float* tau, const float* c, int* counts, int* lists, long cap,
                   int* ntiles_per_g) {
  or_view V;
  if (or_view_init(&V, g, K, p, s, q, tau, c)) return -2;
  const int th = (g->H + g->TH - 1) / g->TH, tw = (g->W + g->TW - 1) / g->TW;
  const int T = th * tw;
  unsigned char* mark = (unsigned char*)calloc((size_t)T, 1);
  int* cnt = (int*)calloc((size_t)T, sizeof(int));
  /* first pass: count */
  for (int k = 0; k < K; ++k) ntiles_per_g[k] = 0;
  for (int n = 0; n < V.nvis; ++n) {
    int k = V.order[n];
    memset(mark, 0, (size_t)T);
    const or_p32* P = V.P32 + k;
    for (int i = P->i_lo; i <= P->i_hi; ++i)
      for (int d = 0; d <= P->span; ++d) {
        int jj = (P->j_lo + d) % g->W;
        mark[(i / g->TH) * tw + jj / g->TW] = 1;
      }
    for (int t = 0; t < T; ++t)
      if (mark[t]) { cnt[t]++; ntiles_per_g[k]++; }
  }
  long total = 0;
  for (int t = 0; t < T; ++t) { counts[t] = cnt[t]; total += cnt[t]; }
  if (total > cap) { free(mark); free(cnt); or_view_free(&V); return -1; }
  long* off = (long*)malloc(sizeof(long) * (size_t)T);
  long acc = 0;
  for (int t = 0; t < T; ++t) { off[t] = acc; acc += cnt[t]; }
  /* second pass in depth order: appending keeps each list sorted by (rho, k) */
  for (int n = 0; n < V.nvis; ++n) {
    int k = V.order[n];
    memset(mark, 0, (size_t)T);
    const or_p32* P = V.P32 + k;
    for (int i = P->i_lo; i <= P->i_hi; ++i)
      for (int d = 0; d <= P->span; ++d) {
        int jj = (P->j_lo + d) % g->W;
        mark[(i / g->TH) * tw + jj / g->TW] = 1;
      }
    for (int t = 0; t < T; ++t)
      if (mark[t]) lists[off[t]++] = k;
  }
  free(off); free(mark); free(cnt); or_view_free(&V);
  return total;
}

/* ---------------------------------------------------------------- render
 * One view (transmitter c), N receivers, C complex channels.
 * rad[N][K][C][2] (float64), receiver-major like the paper's (N, K, 2).
 * Outputs (any may be NULL):
 *   spectra[N][H][W][C][2]   composited signal per pixel
 *   absacc [N][H][W][C]      sum_k T w |s|  (scale for relative errors)
 *   ncontrib[H][W]           number of Gaussians composited (incl. the last)
 *   Tfinal[H][W]             float32 shadow transmittance after the loop
 *   T64out[H][W]             float64 transmittance after the loop
 *   Wvis[K]                  visibility weight W_k = sum_pixels T_k w_k
 * Brute force: every pixel walks all visible Gaussians in global depth
 * order and skips those whose footprint misses it.  use_eps = 0 disables
 * the early stop (used by the finite-difference tests).
 * Pixels rows are processed in parallel when built with OpenMP.            */
int or_render_view(const or_grid* g, int K, const float* p, const float* s, const float* q,
                   const float* tau, const float* c, int N, int C, const double* rad,
                   double* spectra, double* absacc, int* ncontrib, float* Tfinal, double* T64out,
                   double* Wvis, int use_eps) {
  or_view V;
  if (or_view_init(&V, g, K, p, s, q, tau, c)) return -2;
  const int H = g->H, W = g->W;
  if (Wvis) memset(Wvis, 0, sizeof(double) * (size_t)K);
  double* Wrow = NULL;
  if (Wvis) Wrow = (double*)calloc((size_t)H * (size_t)K, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < H; ++i) {
    double* acc = (double*)malloc(sizeof(double) * (size_t)N * C * 2);
    double* aab = (double*)malloc(sizeof(double) * (size_t)N * C);
    for (int jj = 0; jj < W; ++jj) {
      memset(acc, 0, sizeof(double) * (size_t)N * C * 2);
      memset(aab, 0, sizeof(double) * (size_t)N * C);
      float T32 = 1.0f;
      double T64 = 1.0;
      int n_c = 0;
      for (int n = 0; n < V.nvis; ++n) {
        int k = V.order[n];
        const or_p32* P = V.P32 + k;
        if (!or_in_footprint(g, P, i, jj)) continue;
        float w32;
        int m;
        if (!or_weight32(g, P, tau[k], i, jj, &w32, &m)) continue;
        double w64 = or_weight64(g, V.P64 + k, (double)tau[k], i, jj, m, NULL);
        double Tw = T64 * w64;
        for (int j = 0; j < N; ++j)
          for (int ch = 0; ch < C; ++ch) {
            const double* sv = rad + ((((size_t)j * K + k) * C + ch) * 2);
            acc[(j * C + ch) * 2 + 0] += Tw * sv[0];
            acc[(j * C + ch) * 2 + 1] += Tw * sv[1];
            aab[j * C + ch] += Tw * sqrt(sv[0] * sv[0] + sv[1] * sv[1]);
          }
        if (Wrow) Wrow[(size_t)i * K + k] += Tw;
        T32 = T32 * (1.0f - w32);
        T64 = T64 * (1.0 - w64);
        n_c++;
        if (use_eps && T32 < g->eps_T) break;
      }
      size_t pix = (size_t)i * W + jj;
      if (ncontrib) ncontrib[pix] = n_c;
      if (Tfinal) Tfinal[pix] = T32;
      if (T64out) T64out[pix] = T64;
      for (int j = 0; j < N; ++j)
        for (int ch = 0; ch < C; ++ch) {
          size_t o = (((size_t)j * H * W + pix) * C + ch);
          if (spectra) {
            spectra[o * 2 + 0] = acc[(j * C + ch) * 2 + 0];
            spectra[o * 2 + 1] = acc[(j * C + ch) * 2 + 1];
          }
          if (absacc) absacc[o] = aab[j * C + ch];
        }
    }
    free(acc); free(aab);
  }
  if (Wvis) {
    for (int i = 0; i < H; ++i)
      for (int k = 0; k < K; ++k) Wvis[k] += Wrow[(size_t)i * K + k];
    free(Wrow);
  }
  or_view_free(&V);
  return 0;
}

/* The same render restricted to a list of pixels (for sampled parity checks
 * at full size).  pix[np] = i*W + jj.  Outputs are [np][N][C][2],
 * [np][N][C], [np], [np].                                                   */
int or_render_pixels(const or_grid* g, int K, const float* p, const float* s, const float* q,
                     const float* tau, const float* c, int N, int C, const double* rad,
                     int np, const int* pix, double* out, double* absacc, int* ncontrib,
                     float* Tfinal) {
  or_view V;
  if (or_view_init(&V, g, K, p, s, q, tau, c)) return -2;
  const int W = g->W;
#pragma omp parallel for schedule(dynamic, 4)
  for (int e = 0; e < np; ++e) {
    int i = pix[e] / W, jj = pix[e] % W;
    double* acc = out + (size_t)e * N * C * 2;
    double* aab = absacc + (size_t)e * N * C;
    memset(acc, 0, sizeof(double) * (size_t)N * C * 2);
    memset(aab, 0, sizeof(double) * (size_t)N * C);
    float T32 = 1.0f;
    double T64 = 1.0;
    int n_c = 0;
    for (int n = 0; n < V.nvis; ++n) {
      int k = V.order[n];
      const or_p32* P = V.P32 + k;
      if (!or_in_footprint(g, P, i, jj)) continue;
      float w32;
      int m;
      if (!or_weight32(g, P, tau[k], i, jj, &w32, &m)) continue;
      double w64 = or_weight64(g, V.P64 + k, (double)tau[k], i, jj, m, NULL);
      double Tw = T64 * w64;
      for (int j = 0; j < N; ++j)
        for (int ch = 0; ch < C; ++ch) {
          const double* sv = rad + ((((size_t)j * K + k) * C + ch) * 2);
          acc[(j * C + ch) * 2 + 0] += Tw * sv[0];
          acc[(j * C + ch) * 2 + 1] += Tw * sv[1];
          aab[j * C + ch] += Tw * sqrt(sv[0] * sv[0] + sv[1] * sv[1]);
        }
      T32 = T32 * (1.0f - w32);
      T64 = T64 * (1.0 - w64);
      n_c++;
      if (T32 < g->eps_T) break;
    }
    ncontrib[e] = n_c;
    Tfinal[e] = T32;
  }
  or_view_free(&V);
  return 0;
}


/* Backward of one pixel (i, jj).  gv(j, ch) points at dL/d(Re, Im) of
 * receiver j, channel ch of this pixel.                                     */
typedef struct {
  int* seq;
  double *sw, *sG, *sT, *Sb;
} or_bwd_scratch;

/* cand[0..ncand) (optional): the Gaussians of V->order, in that order,
 * whose footprint rows include row i -- the others fail the footprint test
 * below anyway.                                                             */
static void or_backward_pixel(const or_grid* g, const or_view* V, const float* tau, int i, int jj,
                              int N, int C, const double* rad, const double* gpix,
                              size_t gstride_j, double* grad_rad, double* grad_tau,
                              double* abs_rad, double* abs_tau, int use_eps,
                              or_bwd_scratch* sc, const int* cand, int ncand) {
  const int K = V->K;
  float T32 = 1.0f;
  double T64 = 1.0;
  int n_c = 0;
  const int nloop = cand ? ncand : V->nvis;
  for (int n = 0; n < nloop; ++n) {
    int k = cand ? cand[n] : V->order[n];
    const or_p32* P = V->P32 + k;
    if (!or_in_footprint(g, P, i, jj)) continue;
    float w32;
    int m;
    if (!or_weight32(g, P, tau[k], i, jj, &w32, &m)) continue;
    double G;
    double w64 = or_weight64(g, V->P64 + k, (double)tau[k], i, jj, m, &G);
    sc->seq[n_c] = k; sc->sw[n_c] = w64; sc->sG[n_c] = G; sc->sT[n_c] = T64;
    T32 = T32 * (1.0f - w32);
    T64 = T64 * (1.0 - w64);
    n_c++;
    if (use_eps && T32 < g->eps_T) break;
  }
  memset(sc->Sb, 0, sizeof(double) * (size_t)N * C * 2);
  for (int e = n_c - 1; e >= 0; --e) {
    int k = sc->seq[e];
    double dLdw = 0.0, adw = 0.0;
    for (int j = 0; j < N; ++j)
      for (int ch = 0; ch < C; ++ch) {
        const double* gv = gpix + j * gstride_j + (size_t)ch * 2;
        const double* sv = rad + ((((size_t)j * K + k) * C + ch) * 2);
        double* gr = grad_rad + ((((size_t)j * K + k) * C + ch) * 2);
        double* Sv = sc->Sb + (j * C + ch) * 2;
        gr[0] += sc->sT[e] * sc->sw[e] * gv[0];
        gr[1] += sc->sT[e] * sc->sw[e] * gv[1];
        if (abs_rad) {
          double* ar = abs_rad + ((((size_t)j * K + k) * C + ch) * 2);
          ar[0] += sc->sT[e] * sc->sw[e] * fabs(gv[0]);
          ar[1] += sc->sT[e] * sc->sw[e] * fabs(gv[1]);
        }
        dLdw += sc->sT[e] * (gv[0] * (sv[0] - Sv[0]) + gv[1] * (sv[1] - Sv[1]));
        adw += sc->sT[e] * (fabs(gv[0]) * (fabs(sv[0]) + fabs(Sv[0])) +
                            fabs(gv[1]) * (fabs(sv[1]) + fabs(Sv[1])));
        Sv[0] = sc->sw[e] * sv[0] + (1.0 - sc->sw[e]) * Sv[0];
        Sv[1] = sc->sw[e] * sv[1] + (1.0 - sc->sw[e]) * Sv[1];
      }
    grad_tau[k] += dLdw * sc->sG[e];
    if (abs_tau) abs_tau[k] += adw * sc->sG[e];
  }
}

int or_omp_threads(void);
static int or_thread_num(void);

static int or_scratch_init(or_bwd_scratch* sc, int nvis, int N, int C) {
  size_t n = (size_t)(nvis > 0 ? nvis : 1);
  sc->seq = (int*)malloc(sizeof(int) * n);
  sc->sw = (double*)malloc(sizeof(double) * n);
  sc->sG = (double*)malloc(sizeof(double) * n);
  sc->sT = (double*)malloc(sizeof(double) * n);
  sc->Sb = (double*)malloc(sizeof(double) * (size_t)N * C * 2);
  return (sc->seq && sc->sw && sc->sG && sc->sT && sc->Sb) ? 0 : -1;
}

static void or_scratch_free(or_bwd_scratch* sc) {
  free(sc->seq); free(sc->sw); free(sc->sG); free(sc->sT); free(sc->Sb);
}

/* ---------------------------------------------------------------- backward
 * Exact derivative of the render for fixed decisions (App. D backward).
 * gspec[N][H][W][C][2] = dL/d(Re, Im) of each spectrum pixel.
 * grad_rad[N][K][C][2] += sum_pixels T_k w_k g                (dL/ds)
 * grad_tau[K]          += sum_pixels G_k sum_j <g_j, T_k (s_kj - S_kj)>
 * where S_kj is the normalised colour behind k, swept back to front:
 * S <- w_m s_m + (1 - w_m) S.
 * abs_rad / abs_tau (optional) receive the same sums taken over absolute
 * values of every term: the scale against which a float32 result's
 * rounding error is measured.                                               */
int or_backward_view(const or_grid* g, int K, const float* p, const float* s, const float* q,
                     const float* tau, const float* c, int N, int C, const double* rad,
                     const double* gspec, double* grad_rad, double* grad_tau, double* abs_rad,
                     double* abs_tau, int use_eps) {
  or_view V;
  if (or_view_init(&V, g, K, p, s, q, tau, c)) return -2;
  const int H = g->H, W = g->W;
  const size_t gstride_j = (size_t)H * W * C * 2;
  const size_t nrad = (size_t)N * K * C * 2;
  /* Rows are split over threads; each thread sums into its own arrays, which
   * are added into the outputs in thread order at the end (a fixed order for
   * a given thread count).                                                 */
  const int nthr = or_omp_threads();
  double** part = (double**)calloc((size_t)nthr * 4, sizeof(double*));
  or_bwd_scratch* scs = (or_bwd_scratch*)calloc((size_t)nthr, sizeof(or_bwd_scratch));
  int ok = part && scs;
  for (int t = 0; ok && t < nthr; ++t) {
    part[4 * t + 0] = (double*)calloc(nrad, sizeof(double));
    part[4 * t + 1] = (double*)calloc((size_t)K, sizeof(double));
    part[4 * t + 2] = abs_rad ? (double*)calloc(nrad, sizeof(double)) : NULL;
    part[4 * t + 3] = abs_tau ? (double*)calloc((size_t)K, sizeof(double)) : NULL;
    ok = part[4 * t] && part[4 * t + 1] && (!abs_rad || part[4 * t + 2]) &&
         (!abs_tau || part[4 * t + 3]) && or_scratch_init(&scs[t], V.nvis, N, C) == 0;
  }
  int* cand = ok ? (int*)malloc(sizeof(int) * (size_t)nthr * (V.nvis > 0 ? V.nvis : 1)) : NULL;
  ok = ok && cand;
  if (ok) {
#pragma omp parallel for schedule(static) num_threads(nthr)
    for (int i = 0; i < H; ++i) {
      const int t = or_thread_num();
      /* the depth-ordered Gaussians whose footprint rows include row i */
      int* ci = cand + (size_t)t * (V.nvis > 0 ? V.nvis : 1);
      int nc = 0;
      for (int n = 0; n < V.nvis; ++n) {
        const or_p32* P = V.P32 + V.order[n];
        if (i >= P->i_lo && i <= P->i_hi) ci[nc++] = V.order[n];
      }
      for (int jj = 0; jj < W; ++jj) {
        size_t pix = (size_t)i * W + jj;
        or_backward_pixel(g, &V, tau, i, jj, N, C, rad, gspec + pix * C * 2, gstride_j,
                          part[4 * t + 0], part[4 * t + 1], part[4 * t + 2], part[4 * t + 3],
                          use_eps, &scs[t], ci, nc);
      }
    }
    for (int t = 0; t < nthr; ++t) {
      for (size_t e = 0; e < nrad; ++e) grad_rad[e] += part[4 * t][e];
      for (int k = 0; k < K; ++k) grad_tau[k] += part[4 * t + 1][k];
      if (abs_rad)
        for (size_t e = 0; e < nrad; ++e) abs_rad[e] += part[4 * t + 2][e];
      if (abs_tau)
        for (int k = 0; k < K; ++k) abs_tau[k] += part[4 * t + 3][k];
    }
  }
  for (int t = 0; part && scs && t < nthr; ++t) {
    for (int e = 0; e < 4; ++e) free(part[4 * t + e]);
    if (scs[t].seq || scs[t].sw || scs[t].sG || scs[t].sT || scs[t].Sb) or_scratch_free(&scs[t]);
  }
  free(part);
  free(scs);
  free(cand);
  or_view_free(&V);
  return ok ? 0 : -2;
}

/* The backward restricted to a pixel list pix[np] (= i*W + jj), with the
 * cotangent of those pixels gpix[np][N][C][2]; the early stop is on.       */
int or_backward_pixels(const or_grid* g, int K, const float* p, const float* s, const float* q,
                       const float* tau, const float* c, int N, int C, const double* rad,
                       int np, const int* pix, const double* gpix, double* grad_rad,
                       double* grad_tau) {
  or_view V;
  if (or_view_init(&V, g, K, p, s, q, tau, c)) return -2;
  or_bwd_scratch sc;
  if (or_scratch_init(&sc, V.nvis, N, C)) return -2;
  for (int e = 0; e < np; ++e)
    or_backward_pixel(g, &V, tau, pix[e] / g->W, pix[e] % g->W, N, C, rad,
                      gpix + (size_t)e * N * C * 2, (size_t)C * 2, grad_rad, grad_tau, NULL, NULL,
                      1, &sc, NULL, 0);
  or_scratch_free(&sc);
  or_view_free(&V);
  return 0;
}

int or_omp_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int or_thread_num(void) {
#ifdef _OPENMP
  extern int omp_get_thread_num(void);
  return omp_get_thread_num();
#else
  return 0;
#endif
}
