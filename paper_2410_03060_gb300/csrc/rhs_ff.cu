// Right-hand sides (Eq. (4)) and far field / RCS (Sec. III-A, III-B), both in closed form.
//
// For a rooftop of half-width D centred at s_l on wire p (centre c, direction t):
//   int Lambda(s) exp(j beta s) ds = D exp(j beta s_l) sinc^2(beta D / 2),  sinc(z) = sin z / z.
// RHS:  b_{p,l} = (e.t) exp(-j k khat.c) D exp(-j k (khat.t) s_l) sinc^2(k (khat.t) D / 2)
// far:  F(r) = sum_p t_p D_p exp(j k r.c_p) sinc^2(k (r.t_p) D_p / 2) sum_l j_{p,l} exp(j k (r.t_p) s_l)
//       sigma_s = |e_s . F|^2 / (4 pi), e_s = theta_hat or phi_hat at r.
// The exp(j beta s_l) factors along a wire are a geometric progression in l.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ctx.h"
#include "rhs_entry.cuh"

namespace swm {

namespace {

// Right-hand sides, one thread per (wire, incidence; frames: per incidence khat[3], e[3]): the
// wire's incidence-dependent factors once (float64), then its m entries, each with its own phase
// ph0 + beta s_l formed in float64 (and, on the complex64 path, reduced mod 2 pi in float64 before
// the float32 sincos), as rhs_entry does per entry.
template <typename TV>
__global__ void k_rhs_wire(int64_t nw, RhsGeo g, const int64_t* __restrict__ off, double k,
                           const double* __restrict__ frames, int64_t N, cplx<TV>* __restrict__ B) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  const int r = blockIdx.y;
  const double* f = frames + 6 * r;
  const double tx = g.tx[p], ty = g.ty[p], tz = g.tz[p];
  const double kt = f[0] * tx + f[1] * ty + f[2] * tz;
  const double et = f[3] * tx + f[4] * ty + f[5] * tz;
  const double ph0 = -k * (f[0] * g.cx[p] + f[1] * g.cy[p] + f[2] * g.cz[p]);
  const double Lp = g.L[p];
  const int ns = g.ns[p];
  const double D = Lp / ns;
  const double beta = -k * kt;
  const int64_t o = (int64_t)r * N + off[p];
  if constexpr (sizeof(TV) == 8) {
    const double sc = sinc_d(0.5 * beta * D);
    const double amp = et * D * sc * sc;
    for (int l = 0; l + 1 < ns; ++l) {
      double sa, ca;
      sincos(ph0 + beta * (-0.5 * Lp + (l + 1) * D), &sa, &ca);
      B[o + l] = mkc(amp * ca, amp * sa);
    }
  } else {
    const float sc = sinc_f((float)(0.5 * beta * D));
    const float amp = (float)(et * D) * sc * sc;
    for (int l = 0; l + 1 < ns; ++l) {
      float sa, ca;
      sincosf((float)reduce_2pi(ph0 + beta * (-0.5 * Lp + (l + 1) * D)), &sa, &ca);
      B[o + l] = mkc(amp * ca, amp * sa);
    }
  }
}

// Geometry access: structure-of-arrays (internal) or caller arrays (centres/dirs as nw x 3).
struct Geo {
  const double *cx, *cy, *cz, *tx, *ty, *tz;  // SoA when soa
  const double* c3;                           // AoS centres
  const double* t3;                           // AoS dirs
  const double* L;
  const int32_t* ns;
  const int64_t* off;
  int soa;
  __device__ __forceinline__ void get(int64_t p, double c[3], double t[3]) const {
    if (soa) {
      c[0] = cx[p];
      c[1] = cy[p];
      c[2] = cz[p];
      t[0] = tx[p];
      t[1] = ty[p];
      t[2] = tz[p];
    } else {
      c[0] = c3[3 * p];
      c[1] = c3[3 * p + 1];
      c[2] = c3[3 * p + 2];
      t[0] = t3[3 * p];
      t[1] = t3[3 * p + 1];
      t[2] = t3[3 * p + 2];
    }
  }
};

constexpr int kFFThreads = 128;

__device__ __forceinline__ void obs_frame(const double* obs, int stride, int o, double r[3], double th[3], double ph[3]) {
  double st, ct, sp, cp;
  sincos(obs[(int64_t)o * stride], &st, &ct);
  sincos(obs[(int64_t)o * stride + 1], &sp, &cp);
  r[0] = st * cp;
  r[1] = st * sp;
  r[2] = ct;
  th[0] = ct * cp;
  th[1] = ct * sp;
  th[2] = -st;
  ph[0] = -sp;
  ph[1] = cp;
  ph[2] = 0.0;
}

// grid (ceil(npairs / kFFThreads), nchunks).  Pair e: bistatic (r = e / n_obs, o = e % n_obs),
// monostatic (r = o = e).  partial[chunk][e][3] complex128.
template <typename TC, bool F64>
__global__ void __launch_bounds__(kFFThreads) k_far_partial(Geo geo, int64_t nw, int64_t N, double k, int n_rhs,
                                                            const cplx<TC>* __restrict__ cur, int n_obs,
                                                            const double* __restrict__ obs, int obs_stride, int mono,
                                                            int64_t chunk, c128* __restrict__ partial) {
  const int64_t npairs = mono ? n_rhs : (int64_t)n_rhs * n_obs;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p0 = blockIdx.y * chunk, p1 = min(nw, p0 + chunk);
  if (e >= npairs) return;
  const int r = mono ? (int)e : (int)(e / n_obs);
  const int o = mono ? (int)e : (int)(e % n_obs);
  double rh[3], th[3], ph[3];
  obs_frame(obs, obs_stride, o, rh, th, ph);
  const cplx<TC>* J = cur + (int64_t)r * N;
  double F[6] = {0, 0, 0, 0, 0, 0};
  if constexpr (F64) {
    for (int64_t p = p0; p < p1; ++p) {
      double c[3], t[3];
      geo.get(p, c, t);
      const int n = geo.ns[p];
      const double Lp = geo.L[p], D = Lp / n;
      const double beta = k * (rh[0] * t[0] + rh[1] * t[1] + rh[2] * t[2]);
      const double phc = k * (rh[0] * c[0] + rh[1] * c[1] + rh[2] * c[2]);
      const double s1 = -0.5 * Lp + D;
      const cplx<TC>* Jp = J + geo.off[p];
      double sa, ca, sb, cb;
      sincos(phc + beta * s1, &sa, &ca);
      sincos(beta * D, &sb, &cb);
      const double sc = sinc_d(0.5 * beta * D);
      c128 z = mkc(ca, sa), acc = mkc(0.0, 0.0);
      const c128 rat = mkc(cb, sb);
      for (int l = 0; l < n - 1; ++l) {
        cfma(acc, ccast<double>(Jp[l]), z);
        z = z * rat;
      }
      const double amp = D * sc * sc;
      const double Sr = amp * acc.re, Si = amp * acc.im;
      F[0] += t[0] * Sr;
      F[1] += t[0] * Si;
      F[2] += t[1] * Sr;
      F[3] += t[1] * Si;
      F[4] += t[2] * Sr;
      F[5] += t[2] * Si;
    }
  } else {
    // float32 everywhere except the wire-centre phase k r.c, formed and reduced mod 2 pi in float64
    const float kf = (float)k;
    const float rf[3] = {(float)rh[0], (float)rh[1], (float)rh[2]};
    float Ff[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t p = p0; p < p1; ++p) {
      double c[3], t[3];
      geo.get(p, c, t);
      const float tf[3] = {(float)t[0], (float)t[1], (float)t[2]};
      const int n = geo.ns[p];
      const float Lp = (float)geo.L[p], D = Lp / (float)n;
      const float beta = kf * (rf[0] * tf[0] + rf[1] * tf[1] + rf[2] * tf[2]);
      const float phc = (float)reduce_2pi(k * (rh[0] * c[0] + rh[1] * c[1] + rh[2] * c[2]));
      const float s1 = -0.5f * Lp + D;
      const cplx<TC>* Jp = J + geo.off[p];
      float sa, ca, sb, cb;
      sincosf(phc + beta * s1, &sa, &ca);
      sincosf(beta * D, &sb, &cb);
      const float sc = sinc_f(0.5f * beta * D);
      c64 z = mkc(ca, sa), acc = mkc(0.f, 0.f);
      const c64 rat = mkc(cb, sb);
      for (int l = 0; l < n - 1; ++l) {
        cfma(acc, ccast<float>(Jp[l]), z);
        z = z * rat;
      }
      const float amp = D * sc * sc;
      const float Sr = amp * acc.re, Si = amp * acc.im;
      Ff[0] = fmaf(tf[0], Sr, Ff[0]);
      Ff[1] = fmaf(tf[0], Si, Ff[1]);
      Ff[2] = fmaf(tf[1], Sr, Ff[2]);
      Ff[3] = fmaf(tf[1], Si, Ff[3]);
      Ff[4] = fmaf(tf[2], Sr, Ff[4]);
      Ff[5] = fmaf(tf[2], Si, Ff[5]);
    }
    for (int i = 0; i < 6; ++i) F[i] = Ff[i];
  }
  c128* out = partial + ((int64_t)blockIdx.y * npairs + e) * 3;
  out[0] = mkc(F[0], F[1]);
  out[1] = mkc(F[2], F[3]);
  out[2] = mkc(F[4], F[5]);
}

// One warp per (incidence, observation) pair: sum the chunk partials, then sigma (or, with comp,
// the received components theta_hat . F and phi_hat . F as two complex numbers).  Partial (c, e)
// is at partial + (c * cstride + e * estride) * 3.
__global__ void k_far_reduce(int64_t npairs, int nchunks, const c128* __restrict__ partial, int64_t cstride,
                             int64_t estride, int n_obs, const double* __restrict__ obs, int obs_stride, int mono,
                             double* __restrict__ sigma, int comp = 0) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= npairs) return;
  double F[6] = {0, 0, 0, 0, 0, 0};
  for (int c = lane; c < nchunks; c += 32) {
    const c128* in = partial + ((int64_t)c * cstride + e * estride) * 3;
    for (int d = 0; d < 3; ++d) {
      F[2 * d] += in[d].re;
      F[2 * d + 1] += in[d].im;
    }
  }
  for (int d = 0; d < 6; ++d) F[d] = warp_sum(F[d]);
  if (lane != 0) return;
  const int o = mono ? (int)e : (int)(e % n_obs);
  double rh[3], th[3], ph[3];
  obs_frame(obs, obs_stride, o, rh, th, ph);
  const double tr = th[0] * F[0] + th[1] * F[2] + th[2] * F[4], ti = th[0] * F[1] + th[1] * F[3] + th[2] * F[5];
  const double pr = ph[0] * F[0] + ph[1] * F[2] + ph[2] * F[4], pi = ph[0] * F[1] + ph[1] * F[3] + ph[2] * F[5];
  if (comp) {
    sigma[4 * e] = tr;
    sigma[4 * e + 1] = ti;
    sigma[4 * e + 2] = pr;
    sigma[4 * e + 3] = pi;
    return;
  }
  sigma[2 * e] = (tr * tr + ti * ti) / kFourPi;
  sigma[2 * e + 1] = (pr * pr + pi * pi) / kFourPi;
}

// Per-wire data of the float32 far field: the centre in cycles, c k / (2 pi), split into a float
// and its float remainder, the direction, the rooftop half-width D = L / n and the first rooftop
// centre s_1 = -L / 2 + D.
struct FFWire {
  float ch[3], cl[3], t[3], D, s1, pad;
};

__global__ void k_ff_wires(int64_t nw, const double* __restrict__ cx, const double* __restrict__ cy,
                           const double* __restrict__ cz, const double* __restrict__ tx, const double* __restrict__ ty,
                           const double* __restrict__ tz, const double* __restrict__ Ls,
                           const int32_t* __restrict__ ns, double k, FFWire* __restrict__ out) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  const double s = k / (2.0 * kPi);
  const double c[3] = {cx[p] * s, cy[p] * s, cz[p] * s};
  FFWire w;
  for (int i = 0; i < 3; ++i) {
    w.ch[i] = (float)c[i];
    w.cl[i] = (float)(c[i] - (double)w.ch[i]);
  }
  w.t[0] = (float)tx[p];
  w.t[1] = (float)ty[p];
  w.t[2] = (float)tz[p];
  const double D = Ls[p] / ns[p];
  w.D = (float)D;
  w.s1 = (float)(-0.5 * Ls[p] + D);
  w.pad = 0.f;
  out[p] = w;
}

// Observation frame of the float32 far field, formed once per observation: the direction r, split
// into float hi/lo parts for the centre phase and in float64, and theta_hat, phi_hat in float64
// for the final projection.
struct FFObs {
  double r[3], th[3], ph[3];
  float rhi[3], rlo[3];
};

__global__ void k_ff_obs(int n, const double* __restrict__ obs, int obs_stride, FFObs* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  FFObs f;
  obs_frame(obs, obs_stride, o, f.r, f.th, f.ph);
  for (int i = 0; i < 3; ++i) {
    f.rhi[i] = (float)f.r[i];
    f.rlo[i] = (float)(f.r[i] - (double)f.rhi[i]);
  }
  out[o] = f;
}

// Sum of the chunk partials of each (incidence, observation) pair (one warp each, partial[c][e][3],
// complex64: the partials are float32 sums), four float accumulators per lane and component in a
// fixed order, then sigma in float64 with the frames of k_ff_obs.
__global__ void k_far_reduce_f32(int64_t npairs, int nchunks, const c64* __restrict__ partial, int n_obs, int mono,
                                 const FFObs* __restrict__ frames, double* __restrict__ sigma) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= npairs) return;
  float A[4][6];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 6; ++d) A[a][d] = 0.f;
  // a lane's next eight chunks are loaded together (one round trip to L2 per 256 chunks)
  for (int c0 = 0; c0 < nchunks; c0 += 256) {
    c64 v[8][3];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + lane + 32 * u;
      const c64* in = partial + ((int64_t)c * npairs + e) * 3;
#pragma unroll
      for (int d = 0; d < 3; ++d) v[u][d] = c < nchunks ? in[d] : mkc(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        A[u & 3][2 * d] += v[u][d].re;
        A[u & 3][2 * d + 1] += v[u][d].im;
      }
  }
  double F[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) F[d] = (double)warp_sum((A[0][d] + A[1][d]) + (A[2][d] + A[3][d]));
  if (lane != 0) return;
  const FFObs& f = frames[mono ? (int)e : (int)(e % n_obs)];
  const double tr = f.th[0] * F[0] + f.th[1] * F[2] + f.th[2] * F[4];
  const double ti = f.th[0] * F[1] + f.th[1] * F[3] + f.th[2] * F[5];
  const double pr = f.ph[0] * F[0] + f.ph[1] * F[2] + f.ph[2] * F[4];
  const double pi = f.ph[0] * F[1] + f.ph[1] * F[3] + f.ph[2] * F[5];
  sigma[2 * e] = (tr * tr + ti * ti) / kFourPi;
  sigma[2 * e + 1] = (pr * pr + pi * pi) / kFourPi;
}

// float32 far field.  The centre phase k r.c = 2 pi (r . c k / 2 pi) is formed modulo one cycle
// from the hi/lo splits of r and of the centre in cycles: each hi*hi product is split exactly
// into p + e with an FMA, and p - rint(p) is exact, so the phase keeps ~1e-7 cycles however far
// the wire is from the origin.  The currents' progression along a wire is summed in Horner form,
// sum_l J_l z0 q^l = z0 (J_0 + q (J_1 + q (...))).  One thread per (incidence, observation) pair
// and chunk of wires; the CTA stages the chunk's wire data (and, with one incidence, its currents)
// in shared memory.  Partials partial[chunk][e][3], complex64.
// One wire's factors for one observation: the centre phase (split in cycles) and the first
// rooftop's offset as z0 = e^{i(2 pi fr + beta s1)}, the ratio of consecutive rooftops
// e^{i beta D}, and the amplitude D sinc^2(beta D / 2), beta = k r.t.
struct FFTerm {
  c64 z0, rat;
  float amp;
};
__device__ __forceinline__ FFTerm ff_term(const FFWire& w, const float* rhi, const float* rlo, float k) {
  const float two_pi = 6.28318530717958647692f;
  float fr = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float pr = rhi[i] * w.ch[i];
    const float er = fmaf(rhi[i], w.ch[i], -pr);
    fr += pr - rintf(pr);
    fr += er + rhi[i] * w.cl[i] + rlo[i] * w.ch[i];
  }
  fr -= rintf(fr);
  const float beta = k * (rhi[0] * w.t[0] + rhi[1] * w.t[1] + rhi[2] * w.t[2]);
  float sa, ca, sb, cb;
  __sincosf(fmaf(two_pi, fr, beta * w.s1), &sa, &ca);
  __sincosf(beta * w.D, &sb, &cb);
  const float sc = sinc_f(0.5f * beta * w.D);
  FFTerm t;
  t.z0 = mkc(ca, sa);
  t.rat = mkc(cb, sb);
  t.amp = w.D * sc * sc;
  return t;
}
// h = h * rat + J_l (one Horner step of sum_l J_l rat^l)
__device__ __forceinline__ void horner_step(c64& h, c64 rat, c64 Jl) {
  const c64 hv = h;
  h.re = fmaf(hv.re, rat.re, fmaf(-hv.im, rat.im, Jl.re));
  h.im = fmaf(hv.re, rat.im, fmaf(hv.im, rat.re, Jl.im));
}
// F += t_w amp z0 h
__device__ __forceinline__ void ff_accumulate(float* F, const FFWire& w, const FFTerm& t, c64 h) {
  const c64 acc = t.z0 * h;
  const float Sr = t.amp * acc.re, Si = t.amp * acc.im;
  F[0] = fmaf(w.t[0], Sr, F[0]);
  F[1] = fmaf(w.t[0], Si, F[1]);
  F[2] = fmaf(w.t[1], Sr, F[2]);
  F[3] = fmaf(w.t[1], Si, F[3]);
  F[4] = fmaf(w.t[2], Sr, F[4]);
  F[5] = fmaf(w.t[2], Si, F[5]);
}

constexpr int kFFChunkMax = 64;   // wires per chunk of the float32 far field
constexpr int kFFCurMax = 1024;   // staged currents per chunk
__global__ void __launch_bounds__(kFFThreads) k_far_partial_f32(const FFWire* __restrict__ wires,
                                                                const int32_t* __restrict__ ns,
                                                                const int64_t* __restrict__ off, int64_t nw, int64_t N,
                                                                float k, int n_rhs, const c64* __restrict__ cur,
                                                                int n_obs, const FFObs* __restrict__ frames, int mono,
                                                                int64_t chunk, c64* __restrict__ partial) {
  const int64_t npairs = mono ? n_rhs : (int64_t)n_rhs * n_obs;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t p0 = blockIdx.y * chunk, p1 = min(nw, p0 + chunk);
  const int64_t ec = e < npairs ? e : npairs - 1;  // threads past the end help stage, then leave
  const int r = mono ? (int)ec : (int)(ec / n_obs);
  const int o = mono ? (int)ec : (int)(ec % n_obs);
  float rhi[3], rlo[3];
  for (int i = 0; i < 3; ++i) {
    rhi[i] = frames[o].rhi[i];
    rlo[i] = frames[o].rlo[i];
  }
  // the chunk's wires and their currents, staged once per CTA
  __shared__ FFWire sw[kFFChunkMax];
  __shared__ int sn[kFFChunkMax];
  __shared__ int soff[kFFChunkMax + 1];
  __shared__ c64 sJ[kFFCurMax];
  const int nwc = (int)(p1 - p0);
  const int64_t o0 = off[p0];
  const int ncur = (int)(off[p1] - o0);
  const bool stage_cur = mono == 0 && n_rhs == 1 && ncur <= kFFCurMax;
  for (int t = threadIdx.x; t < nwc; t += blockDim.x) {
    sw[t] = wires[p0 + t];
    sn[t] = ns[p0 + t];
    soff[t] = (int)(off[p0 + t] - o0);
  }
  if (stage_cur)
    for (int t = threadIdx.x; t < ncur; t += blockDim.x) sJ[t] = cur[o0 + t];
  __syncthreads();
  if (e >= npairs) return;
  const c64* J = cur + (int64_t)r * N + o0;
  float F[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // two wires per pass: their phases, sincos and Horner sums are independent chains
  int q = 0;
  for (; q + 1 < nwc; q += 2) {
    FFTerm a = ff_term(sw[q], rhi, rlo, k), b = ff_term(sw[q + 1], rhi, rlo, k);
    const int na = sn[q], nb = sn[q + 1];
    const c64* Ja = stage_cur ? sJ + soff[q] : J + soff[q];
    const c64* Jb = stage_cur ? sJ + soff[q + 1] : J + soff[q + 1];
    c64 ha = Ja[na - 2], hb = Jb[nb - 2];
    for (int l = max(na, nb) - 3; l >= 0; --l) {
      if (l <= na - 3) horner_step(ha, a.rat, Ja[l]);
      if (l <= nb - 3) horner_step(hb, b.rat, Jb[l]);
    }
    ff_accumulate(F, sw[q], a, ha);
    ff_accumulate(F, sw[q + 1], b, hb);
  }
  if (q < nwc) {
    const FFTerm a = ff_term(sw[q], rhi, rlo, k);
    const int na = sn[q];
    const c64* Ja = stage_cur ? sJ + soff[q] : J + soff[q];
    c64 ha = Ja[na - 2];
    for (int l = na - 3; l >= 0; --l) horner_step(ha, a.rat, Ja[l]);
    ff_accumulate(F, sw[q], a, ha);
  }
  c64* out = partial + ((int64_t)blockIdx.y * npairs + e) * 3;
  out[0] = mkc(F[0], F[1]);
  out[1] = mkc(F[2], F[3]);
  out[2] = mkc(F[4], F[5]);
}

}  // namespace

// Launch shape shared by the scratch sizing and the launch itself.
static void ff_shape(int64_t nw, int64_t npairs, int64_t& nchunks, int64_t& chunk) {
  // about eight CTAs per SM, chunks of at least 16 wires
  const int64_t gx = ceil_div(npairs, kFFThreads);
  nchunks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nw, 16), ceil_div(8 * 152, gx)));
  nchunks = std::min<int64_t>(nchunks, 65535);
  chunk = ceil_div(nw, nchunks);
  nchunks = ceil_div(nw, chunk);
}

// Launch shape of the float32 far field: one wave of CTAs (`slots` = resident CTAs per SM x SMs,
// whose warps hide each other's sincos and Horner latencies), chunks of at least 8 wires and at
// most kFFChunkMax (the size of the CTA's staging arrays).
static void ff32_shape(int64_t nw, int64_t npairs, int64_t slots, int64_t& nchunks, int64_t& chunk) {
  const int64_t gx = ceil_div(npairs, kFFThreads);
  nchunks = std::max<int64_t>(1, std::min<int64_t>(ceil_div(nw, 8), ceil_div(std::max<int64_t>(slots, 1), gx)));
  nchunks = std::min<int64_t>(nchunks, 65535);
  chunk = std::min<int64_t>(ceil_div(nw, nchunks), kFFChunkMax);
  nchunks = ceil_div(nw, chunk);
}

// Resident CTAs of the float32 far-field kernel on the whole GPU.
static int64_t ff32_slots(const swm_ctx* ctx) {
  int occ = 0;
  if (occupancy_cached((const void*)k_far_partial_f32, kFFThreads, 0, &occ) != cudaSuccess || occ < 1) occ = 8;
  return (int64_t)occ * std::max(ctx->nsm, 1);
}


// The per-wire data of the float32 far field: allocated on the context's stream (before the build
// forks its second stream), filled on stream s.
int far_field_alloc(swm_ctx* ctx) {
  if (ctx->prec != SWM_C64) return SWM_OK;
  SWM_TRY(dalloc(ctx, ctx->build_bufs, &ctx->ffw, sizeof(FFWire) * ctx->nw));
  return SWM_OK;
}

int prepare_far_field(swm_ctx* ctx, cudaStream_t s) {
  if (ctx->prec != SWM_C64) return SWM_OK;
  k_ff_wires<<<(unsigned)ceil_div(ctx->nw, 256), 256, 0, s>>>(ctx->nw, ctx->cx, ctx->cy, ctx->cz, ctx->tx,
                                                                        ctx->ty, ctx->tz, ctx->L, ctx->ns, ctx->k,
                                                                        (FFWire*)ctx->ffw);
  SWM_LAUNCHED();
  return SWM_OK;
}

int far_field_f32_launch(swm_ctx* ctx, int n_obs, const double* obs, int obs_stride, bool mono, double* sigma,
                         void* scratch, size_t scratch_bytes) {
  const int R = ctx->n_rhs;
  const int64_t npairs = mono ? R : (int64_t)R * n_obs;
  int64_t nchunks, chunk;
  ff32_shape(ctx->nw, npairs, ff32_slots(ctx), nchunks, chunk);
  const size_t part_bytes = (size_t)nchunks * npairs * 3 * sizeof(c64);
  if (part_bytes + sizeof(FFObs) * (size_t)n_obs > scratch_bytes)
    return ctx->fail(SWM_EINVAL, "far field: scratch too small");
  c64* part = (c64*)scratch;
  FFObs* frames = reinterpret_cast<FFObs*>((char*)scratch + part_bytes);  // part_bytes is a multiple of 8
  k_ff_obs<<<(unsigned)ceil_div(n_obs, 128), 128, 0, ctx->stream>>>(n_obs, obs, obs_stride, frames);
  SWM_LAUNCHED();
  dim3 grid((unsigned)ceil_div(npairs, kFFThreads), (unsigned)nchunks);
  k_far_partial_f32<<<grid, kFFThreads, 0, ctx->stream>>>((const FFWire*)ctx->ffw, ctx->ns, ctx->off, ctx->nw, ctx->N,
                                                          (float)ctx->k, R, (const c64*)ctx->Xv, n_obs, frames, mono,
                                                          chunk, part);
  SWM_LAUNCHED();
  k_far_reduce_f32<<<(unsigned)ceil_div(npairs * 32, 256), 256, 0, ctx->stream>>>(npairs, (int)nchunks, part, n_obs,
                                                                                  mono, frames, sigma);
  SWM_LAUNCHED();
  return SWM_OK;
}

int compute_rhs(swm_ctx* ctx, int n_inc, const double* frames_dev) {
  SWM_TRY(ensure_rowinfo(ctx));
  const RhsGeo g{ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->ns};
  const dim3 grid((unsigned)ceil_div(ctx->nw, 128), (unsigned)n_inc);
  ctx->prof_begin(SWM_K_RHS);
  if (ctx->prec == SWM_C128)
    k_rhs_wire<double><<<grid, 128, 0, ctx->stream>>>(ctx->nw, g, ctx->off, ctx->k, frames_dev, ctx->N,
                                                      (c128*)ctx->Bv);
  else
    k_rhs_wire<float><<<grid, 128, 0, ctx->stream>>>(ctx->nw, g, ctx->off, ctx->k, frames_dev, ctx->N,
                                                     (c64*)ctx->Bv);
  ctx->prof_end(SWM_K_RHS);
  SWM_LAUNCHED();
  return SWM_OK;
}

int compute_rhs_f64(swm_ctx* ctx, int n_inc, const double* frames_dev, c128* out) {
  SWM_TRY(ensure_rowinfo(ctx));
  const RhsGeo g{ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->ns};
  const dim3 grid((unsigned)ceil_div(ctx->nw, 128), (unsigned)n_inc);
  k_rhs_wire<double><<<grid, 128, 0, ctx->stream>>>(ctx->nw, g, ctx->off, ctx->k, frames_dev, ctx->N, out);
  SWM_LAUNCHED();
  return SWM_OK;
}

size_t far_field_f32_scratch_bytes(const swm_ctx* ctx, int64_t npairs, int n_obs) {
  int64_t nchunks, chunk;
  ff32_shape(ctx->nw, npairs, ff32_slots(ctx), nchunks, chunk);
  return (size_t)nchunks * npairs * 3 * sizeof(c64) + sizeof(FFObs) * (size_t)n_obs;
}

size_t far_field_scratch_bytes(int64_t nw, int64_t npairs) {
  int64_t nchunks, chunk;
  ff_shape(nw, npairs, nchunks, chunk);
  return (size_t)nchunks * npairs * 3 * sizeof(c128);
}

// Far field + RCS.  Scratch must hold at least 3 * npairs complex128; with less than
// far_field_scratch_bytes() the wire range is cut into fewer chunks.
int far_field_launch(cudaStream_t st, int64_t* launches, bool cur_c64, bool f64, const void* cur, int64_t nw,
                     int64_t N, const double* c3, const double* t3, const double* cx, const double* cy,
                     const double* cz, const double* tx, const double* ty, const double* tz, const double* Ls,
                     const int32_t* ns, const int64_t* off, bool soa, double k, int n_rhs, int n_obs,
                     const double* obs, int obs_stride, bool mono, double* sigma, void* scratch, size_t scratch_bytes,
                     std::string* err, bool components) {
  const int64_t npairs = mono ? n_rhs : (int64_t)n_rhs * n_obs;
  int64_t nchunks, chunk;
  ff_shape(nw, npairs, nchunks, chunk);
  const int64_t fit = (int64_t)(scratch_bytes / (3 * sizeof(c128) * (size_t)npairs));
  if (fit < 1) {
    *err = "far field: scratch too small for " + std::to_string(npairs) + " (incidence, observation) pairs";
    return SWM_EINVAL;
  }
  if (nchunks > fit) {
    nchunks = fit;
    chunk = ceil_div(nw, nchunks);
    nchunks = ceil_div(nw, chunk);
  }
  Geo g{cx, cy, cz, tx, ty, tz, c3, t3, Ls, ns, off, soa ? 1 : 0};
  dim3 grid((unsigned)ceil_div(npairs, kFFThreads), (unsigned)nchunks);
  c128* part = (c128*)scratch;
  if (cur_c64) {
    if (f64)
      k_far_partial<float, true><<<grid, kFFThreads, 0, st>>>(g, nw, N, k, n_rhs, (const c64*)cur, n_obs, obs,
                                                             obs_stride, mono, chunk, part);
    else
      k_far_partial<float, false><<<grid, kFFThreads, 0, st>>>(g, nw, N, k, n_rhs, (const c64*)cur, n_obs, obs,
                                                              obs_stride, mono, chunk, part);
  } else {
    if (f64)
      k_far_partial<double, true><<<grid, kFFThreads, 0, st>>>(g, nw, N, k, n_rhs, (const c128*)cur, n_obs, obs,
                                                              obs_stride, mono, chunk, part);
    else
      k_far_partial<double, false><<<grid, kFFThreads, 0, st>>>(g, nw, N, k, n_rhs, (const c128*)cur, n_obs, obs,
                                                               obs_stride, mono, chunk, part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("far field launch: ") + cudaGetErrorString(e);
    return SWM_ECUDA;
  }
  k_far_reduce<<<(unsigned)ceil_div(npairs * 32, 256), 256, 0, st>>>(npairs, (int)nchunks, part, npairs, 1, n_obs,
                                                                     obs, obs_stride, mono, sigma,
                                                                     components ? 1 : 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *err = std::string("far field reduce launch: ") + cudaGetErrorString(e);
    return SWM_ECUDA;
  }
  if (launches) *launches += 2;
  return SWM_OK;
}

}  // namespace swm
