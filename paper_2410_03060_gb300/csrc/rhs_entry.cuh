// One entry of the right-hand side (Eq. (4)) in closed form, shared by the RHS kernel and the
// persistent solve (which forms its rows' entries itself).
//
// For the rooftop of half-width D centred at s_l on wire p (centre c, direction t), incidence
// frame (khat, e):
//   b_{p,l} = (e.t) D sinc^2(k (khat.t) D / 2) exp(-j k khat.c) exp(-j k (khat.t) s_l),
// with sinc(z) = sin z / z and s_l = -L/2 + (l + 1) D, D = L / n_seg.
#pragma once

#include "common.cuh"

namespace swm {

// x mod 2 pi in float64 (two-constant Cody-Waite split), result in [-pi, pi].
__device__ __forceinline__ double reduce_2pi(double x) {
  const double inv2pi = 0.15915494309189535;
  const double c1 = 6.28318530717958623;      // 2 pi rounded to double
  const double c2 = 2.4492935982947064e-16;   // 2 pi - c1
  const double n = rint(x * inv2pi);
  return fma(-n, c2, fma(-n, c1, x));
}

__device__ __forceinline__ double sinc_d(double z) { return fabs(z) < 1e-8 ? 1.0 - z * z / 6.0 : sin(z) / z; }
// sin(z)/z in float: Taylor series to z^6 on |z| <= 0.5 (truncation below 2e-8 relative), else
// sinf(z)/z; the fast __sinf is avoided because its error is absolute, not relative.
__device__ __forceinline__ float sinc_f(float z) {
  const float z2 = z * z;
  if (z2 <= 0.25f) return 1.0f + z2 * (-1.0f / 6.0f + z2 * (1.0f / 120.0f + z2 * (-1.0f / 5040.0f)));
  return sinf(z) / z;
}

// Wire geometry in internal order (structure of arrays).
struct RhsGeo {
  const double *cx, *cy, *cz, *tx, *ty, *tz, *L;
  const int32_t* ns;
};

// b for unknown l of wire p and the incidence frame f = (khat[3], e[3]).  Float64 throughout on the
// complex128 path; on the complex64 path the phase is formed and reduced mod 2 pi in float64 and the
// rest is float32.
template <typename TV>
__device__ __forceinline__ cplx<TV> rhs_entry(const RhsGeo& g, int64_t p, int l, const double* f, double k) {
  const double tx = g.tx[p], ty = g.ty[p], tz = g.tz[p];
  const double kt = f[0] * tx + f[1] * ty + f[2] * tz;
  const double et = f[3] * tx + f[4] * ty + f[5] * tz;
  const double ph0 = -k * (f[0] * g.cx[p] + f[1] * g.cy[p] + f[2] * g.cz[p]);
  const double Lp = g.L[p];
  const double D = Lp / g.ns[p];
  const double beta = -k * kt;  // exp(j beta s)
  const double sl = -0.5 * Lp + (l + 1) * D;
  if constexpr (sizeof(TV) == 8) {
    const double sc = sinc_d(0.5 * beta * D);
    const double amp = et * D * sc * sc;
    double sa, ca;
    sincos(ph0 + beta * sl, &sa, &ca);
    return mkc(amp * ca, amp * sa);
  } else {
    const float sc = sinc_f((float)(0.5 * beta * D));
    const float amp = (float)(et * D) * sc * sc;
    float sa, ca;
    sincosf((float)reduce_2pi(ph0 + beta * sl), &sa, &ca);
    return mkc(amp * ca, amp * sa);
  }
}

}  // namespace swm
