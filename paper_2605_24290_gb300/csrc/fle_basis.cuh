// fle_basis.cuh -- the FLE directional basis (App. E.2) of one Gaussian for a
// group of up to 32 views, evaluated in float32 into shared memory by the
// tensor-core FLE kernels (fle_tc.cu, fle_bwd_tc.cu).
//
// For view v (transmitter t_v) and the direction u = p - t_v (polar angle
// theta from +z, azimuth phi = atan2(u_y, u_x)):
//   Y[v][l*l + l + m] = N_l|m| P_l^|m|(cos theta) e^{i m phi},  |m| <= l <= lmax
// with P_l^m from the three-term recurrence in l (no Condon-Shortley phase),
// P_m^m = (2m - 1)!! sin^m theta, and e^{i m phi} by repeated complex
// multiplication.  One task per (view, order m >= 0) fills the components
// (l, +m) and (l, -m) for l = m .. lmax; rows of views past the group and
// components past (lmax + 1)^2 are zero.
#pragma once
#include "rxgs_internal.h"

namespace rxgs {

// nrm: N_l|m| by component index (shared memory); Y: [32][pitch] float2.
__device__ __forceinline__ void fle_basis_group(const float4 p, const float* __restrict__ tx,
                                                int v0, int nv, int lmax, const float* nrm,
                                                float2* Y, int pitch, int t, int nthreads) {
  const int L = (lmax + 1) * (lmax + 1);
  for (int e = t; e < 32 * 10; e += nthreads) {
    const int v = e / 10, m = e % 10;
    float2* Yv = Y + v * pitch;
    if (m > lmax) continue;
    if (v >= nv) {
      if (m == 0)
        for (int l = 0; l < pitch; ++l) Yv[l] = make_float2(0.0f, 0.0f);
      continue;
    }
    const float ux = p.x - tx[3 * (v0 + v)], uy = p.y - tx[3 * (v0 + v) + 1],
                uz = p.z - tx[3 * (v0 + v) + 2];
    const float hh2 = ux * ux + uy * uy;
    const float rho2 = hh2 + uz * uz;
    // a centre on the transmitter itself (culled by the projection anyway)
    // takes the +z direction
    const float irho = rho2 > 0.0f ? rsqrtf(rho2) : 0.0f;
    const float ihh = hh2 > 0.0f ? rsqrtf(hh2) : 0.0f;
    const float ct = rho2 > 0.0f ? uz * irho : 1.0f, st = hh2 * ihh * irho;
    const float cp = hh2 > 0.0f ? ux * ihh : 1.0f, sp = uy * ihh;
    float pmm = 1.0f, er = 1.0f, ei = 0.0f;  // P_m^m and e^{i m phi}
    for (int q = 1; q <= m; ++q) {
      pmm *= static_cast<float>(2 * q - 1) * st;
      const float r = er * cp - ei * sp;
      ei = er * sp + ei * cp;
      er = r;
    }
    auto put = [&](int l, float pv) {
      const float val = nrm[l * l + l + m] * pv;
      Yv[l * l + l + m] = make_float2(val * er, val * ei);
      if (m > 0) Yv[l * l + l - m] = make_float2(val * er, -val * ei);
    };
    put(m, pmm);
    if (m + 1 <= lmax) {
      float p0 = pmm, p1 = static_cast<float>(2 * m + 1) * ct * pmm;
      put(m + 1, p1);
      for (int l = m + 2; l <= lmax; ++l) {
        const float p2 = __fdividef(static_cast<float>(2 * l - 1) * ct * p1 -
                                        static_cast<float>(l + m - 1) * p0,
                                    static_cast<float>(l - m));
        put(l, p2);
        p0 = p1;
        p1 = p2;
      }
    }
    if (m == 0)
      for (int l = L; l < pitch; ++l) Yv[l] = make_float2(0.0f, 0.0f);
  }
}

}  // namespace rxgs
