// Fill of the kept blocks of Z (Sec. II-A, Eqs. (5)-(8); analytic singularity extraction and
// Gaussian quadrature as named after Eq. (8)).
//
// Z_pq[i][j] = (t_p.t_q) sum_{u,v} I_{a b}(u, v) - 1/(k^2 D_p D_q) sum_{u,v} s_a s_b I_G(u, v),
// where basis i (vertex i+1) rises on segment i (slope +1/D) and falls on segment i+1 (slope
// -1/D), I_ab(u, v) is the integral of the two linear shapes against G over segments u of p and
// v of q, and I_G = sum of the four.
//
// Self blocks (p = q), float64, one warp per wire: the double integral over two segments of one
// straight wire depends only on s - s', so with offset d = u - v it is exactly
// D^2 int_{-1}^{1} W_ab(w) G(D (d + w)) dw, W_ab the convolution of the two shapes (piecewise
// cubic).  Each half uses 8 Gauss points; for |d| <= 1 the static 1/(4 pi R) part is integrated
// in closed form.  The block is Toeplitz in i - j.
//
// Mutual blocks (p < q), one CTA per batch of blocks: one thread per block sets up the block's
// geometry in float64 (centre difference, near/far decision), then threads share the batch's
// segment pairs (tensor Gauss-Legendre, 4 points per segment, 8 for near wires), accumulate
// their four shape integrals in shared memory, and finally assemble the m_p x m_q entries,
// writing Z_pq and Z_qp = Z_pq^T.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ctx.h"
#include "rhs_entry.cuh"

namespace swm {

struct GLTable {
  double x4[4], w4[4], x8[8], w8[8];
};

// Gauss-Legendre nodes and weights on [0, 1] by Newton iteration on P_n.
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      dp = n * (z * p0 - p1) / (z * z - 1.0);
      const double dz = p0 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // (2/((1-z^2) P'^2)) / 2
  }
}

static GLTable make_gl() {
  GLTable t;
  gauss_legendre01(4, t.x4, t.w4);
  gauss_legendre01(8, t.x8, t.w8);
  return t;
}

// ------------------------------------------------------------------------------------------------
// self blocks

// Convolution W_ab(w) of shape a on the test segment with shape b on the source segment
// (a, b: 0 = rise x, 1 = fall 1 - x), as cubic coefficients in w for half 0 (w in [-1, 0]) and
// half 1 (w in [0, 1]).  Derived from W_ab(w) = int phi_a(x) phi_b(x - w) dx.
__device__ __constant__ double c_self_poly[2][4][4] = {
    // half 0: rr, rf, fr, ff
    {{1.0 / 3.0, 0.5, 0.0, -1.0 / 6.0},
     {1.0 / 6.0, 0.5, 0.5, 1.0 / 6.0},
     {1.0 / 6.0, -0.5, -0.5, 1.0 / 6.0},
     {1.0 / 3.0, 0.5, 0.0, -1.0 / 6.0}},
    // half 1
    {{1.0 / 3.0, -0.5, 0.0, 1.0 / 6.0},
     {1.0 / 6.0, 0.5, -0.5, -1.0 / 6.0},
     {1.0 / 6.0, -0.5, 0.5, -1.0 / 6.0},
     {1.0 / 3.0, -0.5, 0.0, 1.0 / 6.0}},
};

// Antiderivatives of t^n / sqrt(t^2 + al^2), n = 0..3, at t.
template <typename R>
__device__ __forceinline__ void static_prims(R t, R al, R out[4]) {
  const R r = sqrt(t * t + al * al);
  const R as = asinh(t / al);
  out[0] = as;
  out[1] = r;
  out[2] = R(0.5) * (t * r - al * al * as);
  out[3] = (t * t - R(2) * al * al) * r / R(3);
}

// I[ab] for segment offset d >= 0 of a wire with segment length D and radius a (without 1/(4 pi)),
// in precision R.  xg, wg: 8-point Gauss-Legendre rule on [0, 1].
template <typename R>
__device__ void self_offset(int d, R D, R a, R k, const R* xg, const R* wg, cplx<R> out[4]) {
  for (int ab = 0; ab < 4; ++ab) out[ab] = mkc<R>(0, 0);
  const R al = a / D;
  for (int half = 0; half < 2; ++half) {
    const R w0 = half ? R(0) : R(-1);
    for (int g = 0; g < 8; ++g) {
      const R w = w0 + xg[g];
      const R t = R(d) + w;
      const R Rr = sqrt(D * D * t * t + a * a);
      // half-angle form keeps cos(kR) - 1 accurate when kR is small
      R sh, ch;
      sincos(R(0.5) * k * Rr, &sh, &ch);
      const R cm1 = R(-2) * sh * sh, sn = R(2) * sh * ch;
      // full kernel exp(-jkR)/R, or the smooth remainder (exp(-jkR) - 1)/R for |d| <= 1
      const R re = (d <= 1 ? cm1 : R(1) + cm1) / Rr, im = -sn / Rr;
      const R ww = wg[g];
      for (int ab = 0; ab < 4; ++ab) {
        const double* P = c_self_poly[half][ab];
        const R W = ((R(P[3]) * w + R(P[2])) * w + R(P[1])) * w + R(P[0]);
        out[ab].re += ww * W * re;
        out[ab].im += ww * W * im;
      }
    }
    if (d <= 1) {
      // static part: int W(t - d) / (D sqrt(t^2 + al^2)) dt over t in [w0 + d, w0 + 1 + d]
      R A0[4], A1[4];
      static_prims<R>(w0 + R(d), al, A0);
      static_prims<R>(w0 + R(1) + R(d), al, A1);
      for (int ab = 0; ab < 4; ++ab) {
        const double* P = c_self_poly[half][ab];
        // coefficients of W(t - d) in powers of t
        const R dd = (R)d;
        const R q0 = R(P[0]) - R(P[1]) * dd + R(P[2]) * dd * dd - R(P[3]) * dd * dd * dd;
        const R q1 = R(P[1]) - R(2) * R(P[2]) * dd + R(3) * R(P[3]) * dd * dd;
        const R q2 = R(P[2]) - R(3) * R(P[3]) * dd;
        const R q3 = R(P[3]);
        const R st = q0 * (A1[0] - A0[0]) + q1 * (A1[1] - A0[1]) + q2 * (A1[2] - A0[2]) + q3 * (A1[3] - A0[3]);
        out[ab].re += st / D;
      }
    }
  }
  for (int ab = 0; ab < 4; ++ab) out[ab] = (D * D) * out[ab];
}

constexpr int kSelfThreads = 128;

// One thread per (wire, segment offset d >= 0): S slots per wire (S a power of two >= max n_s),
// kSelfThreads / S wires per CTA; then the CTA writes the Toeplitz blocks of its wires.
template <typename R, typename TV>
__global__ void __launch_bounds__(kSelfThreads) k_self_blocks(int64_t nw, const double* __restrict__ Ls,
                                                             const double* __restrict__ as,
                                                             const int32_t* __restrict__ ns, double k, GLTable gl,
                                                             const int64_t* __restrict__ diag_b, Layout lay, int S,
                                                             cplx<TV>* __restrict__ Z) {
  __shared__ cplx<R> sI[kSelfThreads][4];
  __shared__ int obase[kSelfThreads + 1];
  __shared__ R xg[8], wg[8];
  const int wpc = kSelfThreads / S;
  const int64_t p0 = (int64_t)blockIdx.x * wpc;
  const int tid = threadIdx.x;
  if (tid < 8) {
    xg[tid] = (R)gl.x8[tid];
    wg[tid] = (R)gl.w8[tid];
  }
  __syncthreads();
  {
    const int lw = tid / S, d = tid % S;
    const int64_t p = p0 + lw;
    if (p < nw && d < ns[p]) {
      cplx<R> I[4];
      self_offset<R>(d, (R)(Ls[p] / ns[p]), (R)as[p], (R)k, xg, wg, I);
      for (int ab = 0; ab < 4; ++ab) sI[tid][ab] = I[ab];
    }
  }
  if (tid == 0) {
    int acc = 0;
    for (int w = 0; w < wpc; ++w) {
      obase[w] = acc;
      if (p0 + w < nw) acc += (ns[p0 + w] - 1) * (ns[p0 + w] - 1);
    }
    obase[wpc] = acc;
  }
  __syncthreads();
  for (int e = tid; e < obase[wpc]; e += kSelfThreads) {
    int w = 0;
    while (obase[w + 1] <= e) ++w;
    const int64_t p = p0 + w;
    const int n = ns[p], m = n - 1;
    const int local = e - obase[w];
    const int i = local / m, j = local % m;
    const int d = i - j;
    const cplx<R>* T = &sI[w * S][0];
    // I_ab at offset x (any sign): I_ab(-x) = I_ba(x)
    auto get = [&](int x, int ab) -> cplx<R> {
      if (x >= 0) return T[4 * x + ab];
      const int ba = (ab == 1) ? 2 : (ab == 2 ? 1 : ab);
      return T[4 * (-x) + ba];
    };
    auto IG = [&](int x) -> cplx<R> { return get(x, 0) + get(x, 1) + get(x, 2) + get(x, 3); };
    // rise(i) x rise(j): offset d; rise x fall(j+1): d - 1; fall(i+1) x rise: d + 1; fall x fall: d
    const cplx<R> vec = get(d, 0) + get(d - 1, 1) + get(d + 1, 2) + get(d, 3);
    const cplx<R> sca = IG(d) - IG(d - 1) - IG(d + 1) + IG(d);
    const R D = (R)(Ls[p] / n);
    const R sc = R(1) / ((R)k * (R)k * D * D);
    const R f = R(1.0 / kFourPi);
    const cplx<R> z = mkc<R>(f * (vec.re - sc * sca.re), f * (vec.im - sc * sca.im));
    Z[lay.rowbase[p] + lay.colpos[diag_b[p]] + (int64_t)i * lay.K[p] + j] = ccast<TV>(z);
  }
}

// ------------------------------------------------------------------------------------------------
// mutual blocks

struct BlockGeo {
  float D[3], tp[3], tq[3];  // FP32 copies (fast path); the FP64 path re-reads FP64 geometry
  float Lp, Lq, a2, tpq;
  float f, sc;               // D_p D_q / (4 pi) and 1 / (k^2 D_p D_q), formed in float64
  double fd, scd, tpqd;      // the same in float64 for the float64 path
  int nsp, nsq, nq, item0;   // item0: first segment pair of this block in the batch
  int out0;                  // first output entry of this block in the batch
  int p, q;
  int64_t bpq, bqp;          // value offsets of Z_pq[0][0] and Z_qp[0][0]
  int Kp, Kq;
};

// Shortest distance between two finite segments (float64): convex quadratic over a rectangle,
// interior stationary point if it lies inside, else the best clamped optimum on the four edges.
__device__ double seg_dist(const double D[3], const double tp[3], double hp, const double tq[3], double hq) {
  const double b = tp[0] * tq[0] + tp[1] * tq[1] + tp[2] * tq[2];
  const double dp = D[0] * tp[0] + D[1] * tp[1] + D[2] * tp[2];
  const double dq = D[0] * tq[0] + D[1] * tq[1] + D[2] * tq[2];
  auto d2 = [&](double s, double sq) {
    double v0 = D[0] + s * tp[0] - sq * tq[0], v1 = D[1] + s * tp[1] - sq * tq[1], v2 = D[2] + s * tp[2] - sq * tq[2];
    return v0 * v0 + v1 * v1 + v2 * v2;
  };
  double best = INFINITY;
  const double det = 1.0 - b * b;
  if (det > 1e-12) {
    const double s = (b * dq - dp) / det, sq = (dq - b * dp) / det;
    if (fabs(s) <= hp && fabs(sq) <= hq) best = d2(s, sq);
  }
  for (int e = 0; e < 2; ++e) {
    const double s = e ? hp : -hp;
    const double sq = fmin(fmax(dq + b * s, -hq), hq);
    best = fmin(best, d2(s, sq));
  }
  for (int e = 0; e < 2; ++e) {
    const double sq = e ? hq : -hq;
    const double s = fmin(fmax(b * sq - dp, -hp), hp);
    best = fmin(best, d2(s, sq));
  }
  return sqrt(best);
}

template <typename R>
struct SegI {
  cplx<R> rr, rf, fr, ff;
};

// Shape integrals of one segment pair (without the 1/(4 pi) D_p D_q factor).
template <int NQ>
__device__ __forceinline__ void seg_pair_f32(const BlockGeo& G, int u, int v, float k, const float* xg, const float* wg,
                                             SegI<float>& out) {
  float Ex[NQ], Ey[NQ], Ez[NQ], Qx[NQ], Qy[NQ], Qz[NQ];
  const float Dp = G.Lp / G.nsp, Dq = G.Lq / G.nsq;
#pragma unroll
  for (int g = 0; g < NQ; ++g) {
    const float sp = -0.5f * G.Lp + ((float)u + xg[g]) * Dp;
    Ex[g] = G.D[0] + sp * G.tp[0];
    Ey[g] = G.D[1] + sp * G.tp[1];
    Ez[g] = G.D[2] + sp * G.tp[2];
    const float sq = -0.5f * G.Lq + ((float)v + xg[g]) * Dq;
    Qx[g] = sq * G.tq[0];
    Qy[g] = sq * G.tq[1];
    Qz[g] = sq * G.tq[2];
  }
  float rrr = 0.f, rri = 0.f, rfr = 0.f, rfi = 0.f, frr = 0.f, fri = 0.f, ffr = 0.f, ffi = 0.f;
#pragma unroll
  for (int g = 0; g < NQ; ++g) {
    float Ar = 0.f, Ai = 0.f, Br = 0.f, Bi = 0.f;
#pragma unroll
    for (int h = 0; h < NQ; ++h) {
      const float dx = Ex[g] - Qx[h], dy = Ey[g] - Qy[h], dz = Ez[g] - Qz[h];
      const float R2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, G.a2)));
      const float ri = rsqrtf(R2);
      const float Rr = R2 * ri;
      float s, c;
      __sincosf(k * Rr, &s, &c);
      const float gr = c * ri, gi = -s * ri;
      const float wh = wg[h], wxh = wg[h] * xg[h];
      Ar = fmaf(wh, gr, Ar);
      Ai = fmaf(wh, gi, Ai);
      Br = fmaf(wxh, gr, Br);
      Bi = fmaf(wxh, gi, Bi);
    }
    const float wr = wg[g] * xg[g], wf = wg[g] - wr;
    const float Cr = Ar - Br, Ci = Ai - Bi;
    rrr = fmaf(wr, Br, rrr);
    rri = fmaf(wr, Bi, rri);
    rfr = fmaf(wr, Cr, rfr);
    rfi = fmaf(wr, Ci, rfi);
    frr = fmaf(wf, Br, frr);
    fri = fmaf(wf, Bi, fri);
    ffr = fmaf(wf, Cr, ffr);
    ffi = fmaf(wf, Ci, ffi);
  }
  out.rr = mkc(rrr, rri);
  out.rf = mkc(rfr, rfi);
  out.fr = mkc(frr, fri);
  out.ff = mkc(ffr, ffi);
}

template <int NQ>
__device__ __forceinline__ void seg_pair_f64(const double* __restrict__ cx, const double* __restrict__ cy,
                                             const double* __restrict__ cz, const double* __restrict__ tx,
                                             const double* __restrict__ ty, const double* __restrict__ tz,
                                             const double* __restrict__ Ls, const double* __restrict__ as,
                                             const BlockGeo& G, int u, int v, double k, const double* xg,
                                             const double* wg, SegI<double>& out) {
  const int p = G.p, q = G.q;
  const double D[3] = {cx[p] - cx[q], cy[p] - cy[q], cz[p] - cz[q]};
  const double tp[3] = {tx[p], ty[p], tz[p]}, tq[3] = {tx[q], ty[q], tz[q]};
  const double Lp = Ls[p], Lq = Ls[q];
  const double a2 = 0.5 * (as[p] * as[p] + as[q] * as[q]);
  const double Dp = Lp / G.nsp, Dq = Lq / G.nsq;
  double rrr = 0, rri = 0, rfr = 0, rfi = 0, frr = 0, fri = 0, ffr = 0, ffi = 0;
  for (int g = 0; g < NQ; ++g) {
    const double sp = -0.5 * Lp + (u + xg[g]) * Dp;
    const double Ex = D[0] + sp * tp[0], Ey = D[1] + sp * tp[1], Ez = D[2] + sp * tp[2];
    double Ar = 0, Ai = 0, Br = 0, Bi = 0;
    for (int h = 0; h < NQ; ++h) {
      const double sq = -0.5 * Lq + (v + xg[h]) * Dq;
      const double dx = Ex - sq * tq[0], dy = Ey - sq * tq[1], dz = Ez - sq * tq[2];
      const double R = sqrt(dx * dx + dy * dy + dz * dz + a2);
      double s, c;
      sincos(k * R, &s, &c);
      const double gr = c / R, gi = -s / R;
      Ar += wg[h] * gr;
      Ai += wg[h] * gi;
      Br += wg[h] * xg[h] * gr;
      Bi += wg[h] * xg[h] * gi;
    }
    const double wr = wg[g] * xg[g], wf = wg[g] - wr;
    rrr += wr * Br;
    rri += wr * Bi;
    rfr += wr * (Ar - Br);
    rfi += wr * (Ai - Bi);
    frr += wf * Br;
    fri += wf * Bi;
    ffr += wf * (Ar - Br);
    ffi += wf * (Ai - Bi);
  }
  out.rr = mkc(rrr, rri);
  out.rf = mkc(rfr, rfi);
  out.fr = mkc(frr, fri);
  out.ff = mkc(ffr, ffi);
}

constexpr int kFillThreads = 256;

__host__ __device__ constexpr size_t round16(size_t x) { return (x + 15) / 16 * 16; }

// One CTA per batch of `nbatch` upper blocks.  Shared memory: BlockGeo[nbatch], item and output
// prefix arrays, and SegI<R> for every segment pair of the batch (capacity `cap`).
template <typename R, typename TV>
__global__ void __launch_bounds__(kFillThreads, sizeof(R) == 4 ? 3 : 1) k_mutual_blocks(
    int64_t nup, const int64_t* __restrict__ ublk, const int32_t* __restrict__ col, const int64_t* __restrict__ bt,
    const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
    const double* __restrict__ tx, const double* __restrict__ ty, const double* __restrict__ tz,
    const double* __restrict__ Ls, const double* __restrict__ as, const int32_t* __restrict__ ns, double k,
    GLTable gl, Layout lay, int nbatch, cplx<TV>* __restrict__ Z, unsigned long long* __restrict__ evals) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t o_item = round16(sizeof(BlockGeo) * nbatch);
  const size_t o_out = o_item + round16(sizeof(int) * (nbatch + 1));
  const size_t o_seg = o_out + round16(sizeof(int) * (nbatch + 1));
  BlockGeo* geo = reinterpret_cast<BlockGeo*>(smem);
  int* item_pre = reinterpret_cast<int*>(smem + o_item);  // nbatch + 1
  int* out_pre = reinterpret_cast<int*>(smem + o_out);    // nbatch + 1
  SegI<R>* seg = reinterpret_cast<SegI<R>*>(smem + o_seg);
  __shared__ float xs4[4], ws4[4], xs8[8], ws8[8];
  __shared__ unsigned long long cta_evals;

  const int tid = threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * nbatch;
  const int nb_here = (int)min((int64_t)nbatch, nup - b0);
  if (tid < 4) {
    xs4[tid] = (float)gl.x4[tid];
    ws4[tid] = (float)gl.w4[tid];
  }
  if (tid < 8) {
    xs8[tid] = (float)gl.x8[tid];
    ws8[tid] = (float)gl.w8[tid];
  }
  if (tid == 0) cta_evals = 0;
  __syncthreads();
  // --- per-block setup, float64, one thread per block
  if (tid < nb_here) {
    const int64_t b = ublk[b0 + tid];
    const int q = col[b];
    const int64_t bq = bt[b];
    const int p = col[bq];
    BlockGeo G;
    const double D[3] = {cx[p] - cx[q], cy[p] - cy[q], cz[p] - cz[q]};
    const double tp[3] = {tx[p], ty[p], tz[p]}, tq[3] = {tx[q], ty[q], tz[q]};
    const double Lp = Ls[p], Lq = Ls[q];
    const int nsp = ns[p], nsq = ns[q];
    const double dmax = fmax(Lp / nsp, Lq / nsq);
    // near rule: exact segment distance < longer segment length; skipped when the centroid
    // distance already exceeds half the two lengths plus that length
    int nq = 4;
    const double reach = 0.5 * (Lp + Lq) + dmax;
    const double cd2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    if (cd2 < reach * reach * (1.0 + 1e-12)) {
      if (seg_dist(D, tp, 0.5 * Lp, tq, 0.5 * Lq) < dmax) nq = 8;
    }
    for (int c = 0; c < 3; ++c) {
      G.D[c] = (float)D[c];
      G.tp[c] = (float)tp[c];
      G.tq[c] = (float)tq[c];
    }
    G.Lp = (float)Lp;
    G.Lq = (float)Lq;
    G.a2 = (float)(0.5 * (as[p] * as[p] + as[q] * as[q]));
    G.tpqd = tp[0] * tq[0] + tp[1] * tq[1] + tp[2] * tq[2];
    G.tpq = (float)G.tpqd;
    {
      const double Dp = Lp / nsp, Dq = Lq / nsq;
      G.fd = Dp * Dq / kFourPi;
      G.scd = 1.0 / (k * k * Dp * Dq);
      G.f = (float)G.fd;
      G.sc = (float)G.scd;
    }
    G.nsp = nsp;
    G.nsq = nsq;
    G.nq = nq;
    G.p = p;
    G.q = q;
    G.Kp = lay.K[p];
    G.Kq = lay.K[q];
    G.bpq = lay.rowbase[p] + lay.colpos[b];
    G.bqp = lay.rowbase[q] + lay.colpos[bq];
    geo[tid] = G;
    atomicAdd(&cta_evals, (unsigned long long)(nsp * nsq * nq * nq));
  }
  __syncthreads();
  if (tid == 0) {
    int it = 0, ot = 0;
    for (int t = 0; t < nb_here; ++t) {
      item_pre[t] = it;
      out_pre[t] = ot;
      geo[t].item0 = it;
      geo[t].out0 = ot;
      it += geo[t].nsp * geo[t].nsq;
      ot += (geo[t].nsp - 1) * (geo[t].nsq - 1);
    }
    item_pre[nb_here] = it;
    out_pre[nb_here] = ot;
    atomicAdd(evals, cta_evals);
  }
  __syncthreads();

  // --- segment pairs
  const int nitems = item_pre[nb_here];
  for (int it = tid; it < nitems; it += kFillThreads) {
    int lo = 0, hi = nb_here - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (item_pre[mid] <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BlockGeo& G = geo[lo];
    const int local = it - G.item0;
    const int u = local / G.nsq, v = local % G.nsq;
    SegI<R> s;
    if constexpr (sizeof(R) == 4) {
      if (G.nq == 4)
        seg_pair_f32<4>(G, u, v, (float)k, xs4, ws4, s);
      else
        seg_pair_f32<8>(G, u, v, (float)k, xs8, ws8, s);
    } else {
      if (G.nq == 4)
        seg_pair_f64<4>(cx, cy, cz, tx, ty, tz, Ls, as, G, u, v, k, gl.x4, gl.w4, s);
      else
        seg_pair_f64<8>(cx, cy, cz, tx, ty, tz, Ls, as, G, u, v, k, gl.x8, gl.w8, s);
    }
    seg[it] = s;
  }
  __syncthreads();

  // --- assembly of the m_p x m_q entries, written to Z_pq and Z_qp
  const int nout = out_pre[nb_here];
  for (int ot = tid; ot < nout; ot += kFillThreads) {
    int lo = 0, hi = nb_here - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (out_pre[mid] <= ot)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BlockGeo& G = geo[lo];
    const int mq = G.nsq - 1;
    const int local = ot - G.out0;
    const int i = local / mq, j = local % mq;
    const SegI<R>* S = seg + G.item0;
    const int nsq = G.nsq;
    // basis i rises on segment i and falls on segment i + 1 (same for j on wire q)
    const SegI<R> a00 = S[i * nsq + j], a01 = S[i * nsq + j + 1], a10 = S[(i + 1) * nsq + j],
                  a11 = S[(i + 1) * nsq + j + 1];
    const cplx<R> vec = a00.rr + a01.rf + a10.fr + a11.ff;
    auto IG = [](const SegI<R>& x) { return x.rr + x.rf + x.fr + x.ff; };
    const cplx<R> sca = IG(a00) - IG(a01) - IG(a10) + IG(a11);
    R f, sc, tpq;
    if constexpr (sizeof(R) == 4) {
      f = G.f;
      sc = G.sc;
      tpq = G.tpq;
    } else {
      f = G.fd;
      sc = G.scd;
      tpq = G.tpqd;
    }
    const cplx<R> z = mkc<R>(f * (tpq * vec.re - sc * sca.re), f * (tpq * vec.im - sc * sca.im));
    const cplx<TV> zt = ccast<TV>(z);
    Z[G.bpq + (int64_t)i * G.Kp + j] = zt;
    Z[G.bqp + (int64_t)j * G.Kq + i] = zt;
  }
}

// ------------------------------------------------------------------------------------------------
// mutual blocks, float32 path without CTA barriers: each warp takes a batch of kWarpBlocks blocks.
// Lanes 0..kWarpBlocks-1 set up one block each (float32 geometry from a float64 centre difference;
// the exact float64 segment distance only when the wires may be near), then every lane evaluates
// segment pairs and adds each pair's four contributions straight into the block's entries in shared
// memory, and finally the warp writes Z_pq and Z_qp = Z_pq^T.
//
// Split phase: exp(-j k R) = exp(-j k |D|) exp(-j k (R - |D|)) with D the centre difference.  The
// block factor exp(-j k |D|) is formed once per block in float64 and applied to the block's entries
// when they are written; the evaluations take sin and cos of the residual phase k (R - |D|), whose
// magnitude is at most k (L_p + L_q) / 2 + k a (triangle inequality), so the float32 phase carries
// no large multiple of 2 pi.  The evaluations of two quadrature points h, h + 1 of wire q run in
// packed FP32x2 arithmetic.

constexpr int kWarpBlocks = 8;
constexpr int kFillF32Threads = 64;  // two warps: a CTA retires as soon as its two batches are done

struct WarpGeo {
  float D[3], tp[3], tq[3];
  float Lp, Lq, a2, tpq, f, sc;
  float Dp, Dq, rq;  // segment lengths, 1 / n_s(q)
  float kd;          // k |D| in float32: the residual phase is k R - kd
  float2 e0;         // exp(-j k |D|), from float64
  int nsp, nsq, nq, acc0;
  int Kp, Kq;
  int64_t bpq, bqp;
};

// Shape integrals of one segment pair (without the 1/(4 pi) D_p D_q factor and without the block
// factor exp(-j k |D|)).
template <int NQ>
__device__ __forceinline__ void seg_pair_x2(const WarpGeo& G, int u, int v, float k, const float* xg, const float* wg,
                                            SegI<float>& out) {
  constexpr int NH = NQ / 2;
  float2 qx[NH], qy[NH], qz[NH], w2[NH], wx2[NH];
#pragma unroll
  for (int hp = 0; hp < NH; ++hp) {
    const float x0 = xg[2 * hp], x1 = xg[2 * hp + 1];
    const float sq0 = -0.5f * G.Lq + ((float)v + x0) * G.Dq, sq1 = -0.5f * G.Lq + ((float)v + x1) * G.Dq;
    qx[hp] = make_float2(-sq0 * G.tq[0], -sq1 * G.tq[0]);
    qy[hp] = make_float2(-sq0 * G.tq[1], -sq1 * G.tq[1]);
    qz[hp] = make_float2(-sq0 * G.tq[2], -sq1 * G.tq[2]);
    w2[hp] = make_float2(wg[2 * hp], wg[2 * hp + 1]);
    wx2[hp] = make_float2(wg[2 * hp] * x0, wg[2 * hp + 1] * x1);
  }
  const float2 a2 = make_float2(G.a2, G.a2), k2 = make_float2(k, k), nkd = make_float2(-G.kd, -G.kd);
  float rrr = 0.f, rri = 0.f, rfr = 0.f, rfi = 0.f, frr = 0.f, fri = 0.f, ffr = 0.f, ffi = 0.f;
#pragma unroll
  for (int g = 0; g < NQ; ++g) {
    const float sp = -0.5f * G.Lp + ((float)u + xg[g]) * G.Dp;
    const float ex = G.D[0] + sp * G.tp[0], ey = G.D[1] + sp * G.tp[1], ez = G.D[2] + sp * G.tp[2];
    const float2 ex2 = make_float2(ex, ex), ey2 = make_float2(ey, ey), ez2 = make_float2(ez, ez);
    float2 Ar = make_float2(0.f, 0.f), As = Ar, Br = Ar, Bs = Ar;
#pragma unroll
    for (int hp = 0; hp < NH; ++hp) {
      const float2 dx = __fadd2_rn(ex2, qx[hp]), dy = __fadd2_rn(ey2, qy[hp]), dz = __fadd2_rn(ez2, qz[hp]);
      const float2 R2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, a2)));
      const float2 ri = make_float2(rsqrtf(R2.x), rsqrtf(R2.y));
      const float2 th = __ffma2_rn(__fmul2_rn(R2, ri), k2, nkd);
      float s0, c0, s1, c1;
      __sincosf(th.x, &s0, &c0);
      __sincosf(th.y, &s1, &c1);
      const float2 gr = __fmul2_rn(make_float2(c0, c1), ri), gs = __fmul2_rn(make_float2(s0, s1), ri);
      Ar = __ffma2_rn(w2[hp], gr, Ar);
      As = __ffma2_rn(w2[hp], gs, As);
      Br = __ffma2_rn(wx2[hp], gr, Br);
      Bs = __ffma2_rn(wx2[hp], gs, Bs);
    }
    // G = (cos - j sin) / R: the imaginary parts are minus the sine sums
    const float ar = Ar.x + Ar.y, ai = -(As.x + As.y), br = Br.x + Br.y, bi = -(Bs.x + Bs.y);
    const float wr = wg[g] * xg[g], wf = wg[g] - wr;
    const float cr = ar - br, ci = ai - bi;
    rrr = fmaf(wr, br, rrr);
    rri = fmaf(wr, bi, rri);
    rfr = fmaf(wr, cr, rfr);
    rfi = fmaf(wr, ci, rfi);
    frr = fmaf(wf, br, frr);
    fri = fmaf(wf, bi, fri);
    ffr = fmaf(wf, cr, ffr);
    ffi = fmaf(wf, ci, ffi);
  }
  out.rr = mkc(rrr, rri);
  out.rf = mkc(rfr, rfi);
  out.fr = mkc(frr, fri);
  out.ff = mkc(ffr, ffi);
}

__global__ void __launch_bounds__(kFillF32Threads, 16) k_mutual_blocks_f32(
    int64_t nup, const int64_t* __restrict__ ublk, const int32_t* __restrict__ col, const int64_t* __restrict__ bt,
    const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
    const double* __restrict__ tx, const double* __restrict__ ty, const double* __restrict__ tz,
    const double* __restrict__ Ls, const double* __restrict__ as, const int32_t* __restrict__ ns, double k,
    GLTable gl, Layout lay, int acc_per_block, c64* __restrict__ Z, unsigned long long* __restrict__ evals) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float xs4[4], ws4[4], xs8[8], ws8[8];
  __shared__ WarpGeo geo_all[kFillF32Threads / 32][kWarpBlocks];
  __shared__ int pre_all[kFillF32Threads / 32][kWarpBlocks + 1];
  __shared__ int outs_all[kFillF32Threads / 32][kWarpBlocks + 1];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  if (threadIdx.x < 4) {
    xs4[threadIdx.x] = (float)gl.x4[threadIdx.x];
    ws4[threadIdx.x] = (float)gl.w4[threadIdx.x];
  }
  if (threadIdx.x < 8) {
    xs8[threadIdx.x] = (float)gl.x8[threadIdx.x];
    ws8[threadIdx.x] = (float)gl.w8[threadIdx.x];
  }
  __syncthreads();  // the only CTA-wide barrier: the quadrature tables
  WarpGeo* geo = geo_all[wl];
  int* pre = pre_all[wl];
  int* outs = outs_all[wl];
  float2* acc = reinterpret_cast<float2*>(smem) + (size_t)wl * kWarpBlocks * acc_per_block;
  const int64_t b0 = ((int64_t)blockIdx.x * (kFillF32Threads / 32) + wl) * kWarpBlocks;
  if (b0 >= nup) return;  // whole warp
  const int nb_here = (int)min((int64_t)kWarpBlocks, nup - b0);
  const float kf = (float)k;
  // --- set-up, one lane per block
  int items = 0, nout = 0;
  unsigned long long ev = 0;
  if (lane < nb_here) {
    const int64_t b = ublk[b0 + lane];
    const int q = col[b];
    const int64_t bq = bt[b];
    const int p = col[bq];
    WarpGeo G;
    const double Dd[3] = {cx[p] - cx[q], cy[p] - cy[q], cz[p] - cz[q]};
    const double tpd[3] = {tx[p], ty[p], tz[p]}, tqd[3] = {tx[q], ty[q], tz[q]};
    for (int c = 0; c < 3; ++c) {
      G.D[c] = (float)Dd[c];
      G.tp[c] = (float)tpd[c];
      G.tq[c] = (float)tqd[c];
    }
    const int nsp = ns[p], nsq = ns[q];
    G.Lp = (float)Ls[p];
    G.Lq = (float)Ls[q];
    G.Dp = G.Lp / nsp;
    G.Dq = G.Lq / nsq;
    G.rq = 1.0f / nsq;
    const float ap = (float)as[p], aq = (float)as[q];
    G.a2 = 0.5f * (ap * ap + aq * aq);
    G.tpq = G.tp[0] * G.tq[0] + G.tp[1] * G.tq[1] + G.tp[2] * G.tq[2];
    G.f = G.Dp * G.Dq * (float)(1.0 / kFourPi);
    G.sc = 1.0f / (kf * kf * G.Dp * G.Dq);
    // the block's phase k |D| in float64 without a float64 square root or sine (both are long
    // dependent chains here): |D| = |D|^2 y with y the float32 reciprocal square root refined by
    // one Newton step in float64 (relative error ~1e-14), k |D| reduced mod 2 pi in float64, and
    // the factor exp(-j k |D|) from the reduced phase in float32 (|phase| <= pi)
    const double d2 = Dd[0] * Dd[0] + Dd[1] * Dd[1] + Dd[2] * Dd[2];
    double y = (double)rsqrtf((float)d2);
    y = d2 > 0.0 ? y * (1.5 - 0.5 * d2 * y * y) : 0.0;
    const double kd = k * (d2 * y);
    G.kd = (float)kd;
    {
      float sd, cd;
      sincosf((float)reduce_2pi(kd), &sd, &cd);
      G.e0 = make_float2(cd, -sd);
    }
    // near rule, decided in float64 like the reference: only when the wires may come within
    // the longer segment length (the float32 screen has a wide margin)
    const float dmax = fmaxf(G.Dp, G.Dq);
    const float reach = 0.5f * (G.Lp + G.Lq) + dmax;
    const float cd2 = G.D[0] * G.D[0] + G.D[1] * G.D[1] + G.D[2] * G.D[2];
    int nq = 4;
    if (cd2 < reach * reach * 1.001f + 1e-6f) {
      const double Lpd = Ls[p], Lqd = Ls[q];
      const double dmaxd = fmax(Lpd / nsp, Lqd / nsq);
      if (seg_dist(Dd, tpd, 0.5 * Lpd, tqd, 0.5 * Lqd) < dmaxd) nq = 8;
    }
    G.nsp = nsp;
    G.nsq = nsq;
    G.nq = nq;
    G.Kp = lay.K[p];
    G.Kq = lay.K[q];
    G.bpq = lay.rowbase[p] + lay.colpos[b];
    G.bqp = lay.rowbase[q] + lay.colpos[bq];
    items = nsp * nsq;
    nout = (nsp - 1) * (nsq - 1);
    ev = (unsigned long long)items * nq * nq;
    geo[lane] = G;
  }
  // prefixes of items and of output entries over the batch
  int incl = items, oincl = nout;
#pragma unroll
  for (int o = 1; o < kWarpBlocks; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o), w = __shfl_up_sync(0xffffffffu, oincl, o);
    if (lane >= o) {
      incl += v;
      oincl += w;
    }
  }
  if (lane < kWarpBlocks) {
    pre[lane + 1] = incl;
    outs[lane + 1] = oincl;
  }
  if (lane == 0) {
    pre[0] = 0;
    outs[0] = 0;
  }
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
  if (lane == 0) atomicAdd(evals, ev);
  // clear the accumulators of the batch
  for (int e = lane; e < kWarpBlocks * acc_per_block; e += 32) acc[e] = make_float2(0.f, 0.f);
  __syncwarp();
  const int nitems = pre[nb_here];
  int bl = 0;  // a lane's items increase, so its block index only moves forward
  for (int it = lane; it < nitems; it += 32) {
    while (pre[bl + 1] <= it) ++bl;
    const WarpGeo& G = geo[bl];
    const int local = it - pre[bl];
    // local / n_s(q) by the float reciprocal: exact for local < 256
    const int u = (int)(((float)local + 0.5f) * G.rq);
    const int v = local - u * G.nsq;
    SegI<float> S;
    if (G.nq == 4)
      seg_pair_x2<4>(G, u, v, kf, xs4, ws4, S);
    else
      seg_pair_x2<8>(G, u, v, kf, xs8, ws8, S);
    const c64 IG = S.rr + S.rf + S.fr + S.ff;
    // segment u rises for basis u and falls for basis u - 1 (same on wire q with v)
    const int mp = G.nsp - 1, mq = G.nsq - 1;
    float2* A = acc + bl * acc_per_block;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int i = a == 0 ? u : u - 1;
      if (i < 0 || i >= mp) continue;
#pragma unroll
      for (int bb = 0; bb < 2; ++bb) {
        const int jj = bb == 0 ? v : v - 1;
        if (jj < 0 || jj >= mq) continue;
        const c64 I = a == 0 ? (bb == 0 ? S.rr : S.rf) : (bb == 0 ? S.fr : S.ff);
        const float sgn = (a == bb) ? 1.f : -1.f;
        const float re = G.f * (G.tpq * I.re - G.sc * sgn * IG.re);
        const float im = G.f * (G.tpq * I.im - G.sc * sgn * IG.im);
        atomicAdd(&A[i * mq + jj].x, re);
        atomicAdd(&A[i * mq + jj].y, im);
      }
    }
  }
  __syncwarp();
  // write Z_pq and Z_qp = Z_pq^T, each entry times the block factor exp(-j k |D|)
  int ob = 0;
  for (int e = lane; e < outs[nb_here]; e += 32) {
    while (outs[ob + 1] <= e) ++ob;
    const WarpGeo& G = geo[ob];
    const int mq = G.nsq - 1;
    const int local = e - outs[ob];
    const int i = local / mq, jj = local - (local / mq) * mq;
    const float2 z = acc[ob * acc_per_block + i * mq + jj];
    const c64 zc = mkc(z.x * G.e0.x - z.y * G.e0.y, z.x * G.e0.y + z.y * G.e0.x);
    Z[G.bpq + (int64_t)i * G.Kp + jj] = zc;
    Z[G.bqp + (int64_t)jj * G.Kq + i] = zc;
  }
}

template <typename R, typename TV>
int launch_fill(swm_ctx* ctx, const GLTable& gl, unsigned long long* evals) {
  const int ms = ctx->max_ns;
  const int items_per_block = ms * ms;
  // shared budget for segment pairs: 48 KB (float) or 64 KB (double)
  const int cap_bytes = sizeof(R) == 4 ? 48 * 1024 : 64 * 1024;
  int nbatch = std::max(1, cap_bytes / (int)(items_per_block * sizeof(SegI<R>)));
  nbatch = std::min(nbatch, kFillThreads);
  const size_t smem = round16(sizeof(BlockGeo) * nbatch) + 2 * round16(sizeof(int) * (nbatch + 1)) +
                      sizeof(SegI<R>) * nbatch * items_per_block;
  SWM_CK(allow_max_dyn_smem((const void*)k_mutual_blocks<R, TV>, ctx->smem_optin));
  if (ctx->nup > 0) {
    const int64_t grid = ceil_div(ctx->nup, nbatch);
    ctx->prof_begin(SWM_K_FILL_MUTUAL);
    k_mutual_blocks<R, TV><<<(unsigned)grid, kFillThreads, smem, ctx->stream>>>(
        ctx->nup, ctx->ublk, ctx->col, ctx->bt, ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->a,
        ctx->ns, ctx->k, gl, ctx->full, nbatch, reinterpret_cast<cplx<TV>*>(ctx->Z), evals);
    ctx->prof_end(SWM_K_FILL_MUTUAL);
    SWM_LAUNCHED();
  }
  return SWM_OK;
}

// Z and the evaluation counter, allocated and cleared on the context's stream.
int fill_alloc(swm_ctx* ctx) {
  const size_t esz = ctx->prec == SWM_C128 ? sizeof(c128) : sizeof(c64);
  SWM_TRY(dalloc(ctx, ctx->build_bufs, &ctx->Z, esz * std::max<int64_t>(1, ctx->full.nval)));
  SWM_TRY(dalloc(ctx, ctx->build_bufs, (void**)&ctx->d_evals, sizeof(unsigned long long)));
  SWM_CK(cudaMemsetAsync(ctx->d_evals, 0, sizeof(unsigned long long), ctx->stream));
  return SWM_OK;
}

// The self blocks (diagonal of Z), on stream s.
int fill_self(swm_ctx* ctx, cudaStream_t s) {
  static const GLTable gl = make_gl();
  const int64_t nw = ctx->nw;
  int S = 2;
  while (S < ctx->max_ns) S <<= 1;
  const unsigned grid_self = (unsigned)ceil_div(nw, kSelfThreads / S);
  ctx->prof_begin(SWM_K_FILL_SELF);
  if (ctx->prec == SWM_C128)
    k_self_blocks<double, double><<<grid_self, kSelfThreads, 0, s>>>(
        nw, ctx->L, ctx->a, ctx->ns, ctx->k, gl, ctx->diag_b, ctx->full, S, reinterpret_cast<c128*>(ctx->Z));
  else
    k_self_blocks<float, float><<<grid_self, kSelfThreads, 0, s>>>(
        nw, ctx->L, ctx->a, ctx->ns, ctx->k, gl, ctx->diag_b, ctx->full, S, reinterpret_cast<c64*>(ctx->Z));
  ctx->prof_end(SWM_K_FILL_SELF);
  SWM_LAUNCHED();
  return SWM_OK;
}

// The mutual blocks (off-diagonal of Z), on the context's stream.
int fill_mutual(swm_ctx* ctx) {
  static const GLTable gl = make_gl();
  if (ctx->prec == SWM_C128) {
    SWM_TRY((launch_fill<double, double>(ctx, gl, ctx->d_evals)));
  } else if (ctx->nup > 0) {
    const int mm = ctx->max_ns - 1;
    const int acc_per_block = std::max(1, mm * mm);
    const size_t smem = sizeof(float2) * (size_t)(kFillF32Threads / 32) * kWarpBlocks * acc_per_block;
    if (smem > 48 * 1024)
      SWM_CK(allow_max_dyn_smem((const void*)k_mutual_blocks_f32, ctx->smem_optin));
    const int64_t blocks_per_cta = (int64_t)(kFillF32Threads / 32) * kWarpBlocks;
    ctx->prof_begin(SWM_K_FILL_MUTUAL);
    k_mutual_blocks_f32<<<(unsigned)ceil_div(ctx->nup, blocks_per_cta), kFillF32Threads, smem, ctx->stream>>>(
        ctx->nup, ctx->ublk, ctx->col, ctx->bt, ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->a,
        ctx->ns, ctx->k, gl, ctx->full, acc_per_block, reinterpret_cast<c64*>(ctx->Z), ctx->d_evals);
    ctx->prof_end(SWM_K_FILL_MUTUAL);
    SWM_LAUNCHED();
  }
  return SWM_OK;
}

}  // namespace swm
