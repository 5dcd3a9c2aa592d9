// Restarted GMRES on the block-Jacobi right-preconditioned S-NFC system (Sec. II-B, after
// Eq. neardef: iterative solve with block-diagonal preconditioning; the cost per iteration is
// the block-sparse product, O(b_mean N_dof)).
//
// The operator is A = Z M^-1 = I + E (E stored, see precond.cu); GMRES finds y with A y = b and
// the currents are x = M^-1 y.  Several right-hand sides (incidences) run as independent GMRES
// instances that share every pass over E.  One Arnoldi step is three kernels, each over chunks of
// rows:
//   k_step   : v_j = w / |w| (row owners), w' = A v_j, h = V^H w'  (classical Gram-Schmidt, pass 1)
//   k_update : w' -= V h, h2 = V^H w'                              (pass 2)
//   k_finish : w' -= V h2, |w'|, Hessenberg column, Givens rotation, residual estimate
// Reductions end in the last CTA to arrive (no spin-waits).  Every kernel reads the step index
// and the activity flags from device memory, so the host issues identical launches every step;
// it keeps one chunk of steps queued ahead of the convergence flag it is reading, so the GPU
// does not wait for the host inside a restart cycle.  Vectors are stored right-hand-side major:
// V[j][r][n].  Dot products, norms, the Hessenberg matrix and the rotations are float64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {

struct KState {
  int j;          // Arnoldi step inside the cycle
  int cycle_done; // no active right-hand side left in this cycle
  int all_conv;   // every right-hand side met tol at the start of this cycle
  int iters;      // total Arnoldi steps
  int numeric;    // a NaN/Inf appeared
  int pad[3];
};

struct KPtr {
  KState* st;
  unsigned* counter;  // [R]
  int* active;        // [R]
  int* jlast;         // [R]
  double* inv_h;      // [R]
  double* bnorm;      // [R]
  double* resid;      // [R]
  c128* H;            // [R][(restart + 1) * restart]
  double* cs;         // [R][restart]
  c128* sn;           // [R][restart]
  c128* g;            // [R][restart + 1]
  c128* hc;           // [R][restart + 1]
  c128* hc2;          // [R][restart + 1]
  c128* coef;         // [R][restart]
  c128* part;         // [R][nchunk][restart + 1]
  double* partn;      // [R][nchunk]
  int R, restart, nchunk, chunk;
  int64_t N;
  double tol;
};

constexpr int kRows = 256;  // CTA width of the vector kernels
constexpr int kG = 8;       // lanes per scalar row in the block-sparse product

template <typename T>
__device__ __forceinline__ bool finite_c(cplx<T> z) {
  return isfinite((double)z.re) && isfinite((double)z.im);
}

// mode 0 (Arnoldi): x = W_src * inv_h; V[j] = x (row owners); W_dst = x + E x.
// mode 1 (residual): W_dst = B - (Y + E Y).
template <typename TV>
__global__ void __launch_bounds__(kRows) k_apply(int mode, KPtr P, const int32_t* __restrict__ rowwire,
                                                 const int64_t* __restrict__ off, Layout lay,
                                                 const cplx<TV>* __restrict__ E, const cplx<TV>* __restrict__ B,
                                                 cplx<TV>* __restrict__ Y, cplx<TV>* __restrict__ W0,
                                                 cplx<TV>* __restrict__ W1, cplx<TV>* __restrict__ V) {
  if (mode == 0 && P.st->cycle_done) return;
  const int64_t n = (blockIdx.x * (int64_t)kRows + threadIdx.x) / kG;
  const int sub = threadIdx.x % kG;
  const int r = blockIdx.y;
  const int64_t N = P.N;
  const bool row_ok = n < N;
  const int j = mode == 0 ? P.st->j : 0;
  const cplx<TV>* src = mode == 0 ? ((j & 1) ? W1 : W0) + (int64_t)r * N : Y + (int64_t)r * N;
  cplx<TV>* dst = (mode == 0 ? ((j & 1) ? W0 : W1) : W0) + (int64_t)r * N;
  cplx<TV> acc = mkc<TV>(0, 0);
  int64_t p = 0;
  if (row_ok) {
    p = rowwire[n];
    const int i = (int)(n - off[p]);
    const int K = lay.K[p];
    const int64_t vb = lay.rowbase[p] + (int64_t)i * K;
    const int32_t* cm = lay.colmap + lay.cmbase[p];
    for (int c = sub; c < K; c += kG) cfma(acc, E[vb + c], src[cm[c]]);
  }
#pragma unroll
  for (int o = kG / 2; o > 0; o >>= 1) {
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
  }
  if (!row_ok || sub != 0) return;
  if (mode == 0) {
    const bool act = P.active[r];
    const TV s = (TV)P.inv_h[r];
    const cplx<TV> x = act ? s * src[n] : mkc<TV>(0, 0);
    V[((int64_t)j * P.R + r) * N + n] = x;
    dst[n] = act ? x + s * acc : mkc<TV>(0, 0);
  } else {
    dst[n] = B[(int64_t)r * N + n] - (src[n] + acc);
  }
}

// Partial dots conj(V_i) . w over the CTA's rows for i <= j, one warp per i, float64 results.
template <typename TV>
__device__ void cta_dots(const KPtr& P, int j, int r, const cplx<TV>* __restrict__ V, const cplx<TV>* w_sm, int64_t n0,
                         int cnt, c128* __restrict__ out) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int i = wp; i <= j; i += kRows / 32) {
    const cplx<TV>* vi = V + ((int64_t)i * P.R + r) * P.N + n0;
    cplx<TV> acc = mkc<TV>(0, 0);
    for (int t = lane; t < cnt; t += 32) {
      const cplx<TV> v = vi[t], w = w_sm[t];
      acc.re = fma(v.re, w.re, fma(v.im, w.im, acc.re));
      acc.im = fma(v.re, w.im, fma(-v.im, w.re, acc.im));
    }
    const double re = warp_sum((double)acc.re), im = warp_sum((double)acc.im);
    if (lane == 0) out[i] = mkc(re, im);
  }
}

// Last CTA of right-hand side r to arrive sums the partial dots into dst[0..j].
__device__ bool last_cta(const KPtr& P, int r) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&P.counter[r], 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

__device__ void reduce_dots(const KPtr& P, int j, int r, c128* __restrict__ dst) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const c128* part = P.part + (int64_t)r * P.nchunk * (P.restart + 1);
  for (int i = wp; i <= j; i += kRows / 32) {
    double re = 0, im = 0;
    for (int c = lane; c < P.nchunk; c += 32) {
      // written by other CTAs of this launch: read through L2
      const double2 v = __ldcg(reinterpret_cast<const double2*>(part + (int64_t)c * (P.restart + 1) + i));
      re += v.x;
      im += v.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) dst[(int64_t)r * (P.restart + 1) + i] = mkc(re, im);
  }
  if (threadIdx.x == 0) P.counter[r] = 0;
}

// Normalise, multiply by A = I + E and take the first Gram-Schmidt dots, over one chunk of rows.
// Eight lanes share a scalar row; the 32 row groups of the CTA sweep the chunk.
template <typename TV>
__global__ void __launch_bounds__(kRows) k_step(KPtr P, const int32_t* __restrict__ rowwire,
                                                const int64_t* __restrict__ off, Layout lay,
                                                const cplx<TV>* __restrict__ E, cplx<TV>* __restrict__ W0,
                                                cplx<TV>* __restrict__ W1, cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, r = blockIdx.y;
  const int64_t N = P.N;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, N - n0);
  const cplx<TV>* src = ((j & 1) ? W1 : W0) + (int64_t)r * N;
  cplx<TV>* dst = ((j & 1) ? W0 : W1) + (int64_t)r * N;
  const bool act = P.active[r];
  const TV s = (TV)P.inv_h[r];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  const int g = threadIdx.x / kG, sub = threadIdx.x % kG;
  for (int rb = 0; rb < cnt; rb += kRows / kG) {
    const int row = rb + g;
    const bool valid = row < cnt;
    const int64_t n = n0 + row;
    cplx<TV> acc = mkc<TV>(0, 0);
    if (valid && act) {
      const int64_t p = rowwire[n];
      const int i = (int)(n - off[p]);
      const int K = lay.K[p];
      const int64_t vb = lay.rowbase[p] + (int64_t)i * K;
      const int32_t* cm = lay.colmap + lay.cmbase[p];
      for (int c = sub; c < K; c += kG) cfma(acc, E[vb + c], src[cm[c]]);
    }
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (valid && sub == 0) {
      const cplx<TV> x = act ? s * src[n] : mkc<TV>(0, 0);
      const cplx<TV> y = act ? x + s * acc : mkc<TV>(0, 0);
      V[((int64_t)j * P.R + r) * N + n] = x;
      dst[n] = y;
      w_sm[row] = y;
    }
  }
  __syncthreads();
  cta_dots<TV>(P, j, r, V, w_sm, n0, cnt, P.part + ((int64_t)r * P.nchunk + blockIdx.x) * (P.restart + 1));
  if (last_cta(P, r)) reduce_dots(P, j, r, P.hc);
}

// w -= sum_i V_i h_i over the CTA's rows; result kept in shared memory and written back.
template <typename TV>
__device__ void cta_update(const KPtr& P, int j, int r, const cplx<TV>* __restrict__ V, const c128* __restrict__ h,
                           cplx<TV>* __restrict__ w, cplx<TV>* w_sm, int64_t n0, int cnt) {
  __shared__ cplx<TV> hs[SWM_MAX_RESTART + 1];
  for (int i = threadIdx.x; i <= j; i += kRows) hs[i] = ccast<TV>(h[(int64_t)r * (P.restart + 1) + i]);
  __syncthreads();
  for (int t = threadIdx.x; t < cnt; t += kRows) {
    cplx<TV> x = w[t];
    for (int i = 0; i <= j; ++i) {
      const cplx<TV> v = V[((int64_t)i * P.R + r) * P.N + n0 + t];
      const cplx<TV> hh = hs[i];
      x.re = fma(-v.re, hh.re, fma(v.im, hh.im, x.re));
      x.im = fma(-v.re, hh.im, fma(-v.im, hh.re, x.im));
    }
    w[t] = x;
    w_sm[t] = x;
  }
  __syncthreads();
}

template <typename TV>
__global__ void __launch_bounds__(kRows) k_update(KPtr P, cplx<TV>* __restrict__ W0, cplx<TV>* __restrict__ W1,
                                                  const cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  cplx<TV>* w = ((j & 1) ? W0 : W1) + (int64_t)r * P.N + n0;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  cta_update<TV>(P, j, r, V, P.hc, w, w_sm, n0, cnt);
  cta_dots<TV>(P, j, r, V, w_sm, n0, cnt, P.part + ((int64_t)r * P.nchunk + blockIdx.x) * (P.restart + 1));
  if (last_cta(P, r)) reduce_dots(P, j, r, P.hc2);
}

// Second update, norm, and (last CTA) the Hessenberg column, Givens rotation and residual.
template <typename TV>
__global__ void __launch_bounds__(kRows) k_finish(KPtr P, cplx<TV>* __restrict__ W0, cplx<TV>* __restrict__ W1,
                                                  const cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  cplx<TV>* w = ((j & 1) ? W0 : W1) + (int64_t)r * P.N + n0;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  cta_update<TV>(P, j, r, V, P.hc2, w, w_sm, n0, cnt);
  double s = 0.0;
  {
    TV a = 0;
    for (int t = threadIdx.x; t < cnt; t += kRows) a += w_sm[t].re * w_sm[t].re + w_sm[t].im * w_sm[t].im;
    s = (double)a;
  }
  __shared__ double red[kRows / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kRows / 32; ++i) t += red[i];
    P.partn[(int64_t)r * P.nchunk + blockIdx.x] = t;
  }
  if (!last_cta(P, r)) return;
  // ---- last CTA of right-hand side r
  __shared__ double nrm2;
  if (threadIdx.x < 32) {
    double t = 0;
    for (int c = threadIdx.x; c < P.nchunk; c += 32) t += __ldcg(P.partn + (int64_t)r * P.nchunk + c);
    t = warp_sum(t);
    if (threadIdx.x == 0) nrm2 = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    P.counter[r] = 0;
    const int R1 = P.restart + 1;
    if (P.active[r]) {
      const double hn = sqrt(nrm2);
      c128* Hr = P.H + (int64_t)r * R1 * P.restart;  // H[i][j] at i * restart + j
      c128* hc = P.hc + (int64_t)r * R1;
      c128* hc2 = P.hc2 + (int64_t)r * R1;
      double* cs = P.cs + (int64_t)r * P.restart;
      c128* sn = P.sn + (int64_t)r * P.restart;
      c128* g = P.g + (int64_t)r * R1;
      for (int i = 0; i <= j; ++i) Hr[i * P.restart + j] = hc[i] + hc2[i];
      // previous rotations
      for (int i = 0; i < j; ++i) {
        const c128 a = Hr[i * P.restart + j], b = Hr[(i + 1) * P.restart + j];
        const c128 sc = sn[i];
        Hr[i * P.restart + j] = cs[i] * a + sc * b;
        Hr[(i + 1) * P.restart + j] = mkc(-sc.re, sc.im) * a + cs[i] * b;  // -conj(s) a + c b
      }
      // new rotation zeroing the subdiagonal hn (real, >= 0)
      const c128 a = Hr[j * P.restart + j];
      const double aa = hypot(a.re, a.im);
      const double nu = hypot(aa, hn);
      double c;
      c128 sv;
      if (aa == 0.0) {
        c = 0.0;
        sv = mkc(1.0, 0.0);
      } else {
        c = aa / nu;
        sv = mkc(a.re / aa * hn / nu, a.im / aa * hn / nu);
      }
      cs[j] = c;
      sn[j] = sv;
      Hr[j * P.restart + j] = c * a + hn * sv;
      const c128 gj = g[j];
      g[j + 1] = mkc(-sv.re, sv.im) * gj;
      g[j] = c * gj;
      const double res = hypot(g[j + 1].re, g[j + 1].im) / P.bnorm[r];
      P.resid[r] = res;
      P.jlast[r] = j + 1;
      if (!isfinite(hn) || !isfinite(res)) {
        P.st->numeric = 1;
        P.active[r] = 0;
      } else if (res <= P.tol || hn == 0.0) {
        P.active[r] = 0;
      }
      P.inv_h[r] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    // the CTA that finishes the last right-hand side advances the step
    __threadfence();
    const unsigned done = atomicAdd(&P.counter[P.R], 1u);
    if (done == (unsigned)P.R - 1) {
      P.counter[P.R] = 0;
      int any = 0;
      for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
      P.st->j = j + 1;
      P.st->iters += 1;
      if (!any || j + 1 >= P.restart) P.st->cycle_done = 1;
    }
  }
}

// Start of a cycle: norms of the residuals in W0, initial g, activity.
template <typename TV>
__global__ void __launch_bounds__(kRows) k_cycle_start(KPtr P, const cplx<TV>* __restrict__ W0, int first) {
  const int r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  const cplx<TV>* w = W0 + (int64_t)r * P.N + n0;
  double s = 0.0;
  for (int t = threadIdx.x; t < cnt; t += kRows) s += (double)w[t].re * w[t].re + (double)w[t].im * w[t].im;
  __shared__ double red[kRows / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kRows / 32; ++i) t += red[i];
    P.partn[(int64_t)r * P.nchunk + blockIdx.x] = t;
  }
  if (!last_cta(P, r)) return;
  __shared__ double nrm2;
  if (threadIdx.x < 32) {
    double t = 0;
    for (int c = threadIdx.x; c < P.nchunk; c += 32) t += __ldcg(P.partn + (int64_t)r * P.nchunk + c);
    t = warp_sum(t);
    if (threadIdx.x == 0) nrm2 = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    P.counter[r] = 0;
    const double beta = sqrt(nrm2);
    if (first) P.bnorm[r] = beta > 0.0 ? beta : 1.0;
    const double res = beta / P.bnorm[r];
    P.resid[r] = res;
    P.jlast[r] = 0;
    const bool act = isfinite(res) && res > P.tol;
    if (!isfinite(res)) P.st->numeric = 1;
    P.active[r] = act ? 1 : 0;
    P.inv_h[r] = beta > 0.0 ? 1.0 / beta : 0.0;
    P.g[(int64_t)r * (P.restart + 1)] = mkc(beta, 0.0);
    __threadfence();
    const unsigned done = atomicAdd(&P.counter[P.R], 1u);
    if (done == (unsigned)P.R - 1) {
      P.counter[P.R] = 0;
      int any = 0;
      for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
      P.st->j = 0;
      P.st->cycle_done = any ? 0 : 1;
      P.st->all_conv = any ? 0 : 1;
    }
  }
}

// Back substitution H y = g per right-hand side (one thread each).
__global__ void k_backsolve(KPtr P) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P.R) return;
  const int n = P.jlast[r];
  const int R1 = P.restart + 1;
  const c128* Hr = P.H + (int64_t)r * R1 * P.restart;
  const c128* g = P.g + (int64_t)r * R1;
  c128* y = P.coef + (int64_t)r * P.restart;
  for (int i = n - 1; i >= 0; --i) {
    c128 s = g[i];
    for (int l = i + 1; l < n; ++l) s = s - Hr[i * P.restart + l] * y[l];
    const c128 d = Hr[i * P.restart + i];
    const double den = d.re * d.re + d.im * d.im;
    y[i] = den > 0.0 ? mkc((s.re * d.re + s.im * d.im) / den, (s.im * d.re - s.re * d.im) / den) : mkc(0.0, 0.0);
  }
  for (int i = n; i < P.restart; ++i) y[i] = mkc(0.0, 0.0);
}

// Y += V coef.
template <typename TV>
__global__ void k_update_y(KPtr P, const cplx<TV>* __restrict__ V, cplx<TV>* __restrict__ Y) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  const int jl = P.jlast[r];
  if (jl == 0) return;
  const c128* y = P.coef + (int64_t)r * P.restart;
  c128 acc = ccast<double>(Y[(int64_t)r * P.N + n]);
  for (int i = 0; i < jl; ++i) cfma(acc, ccast<double>(V[((int64_t)i * P.R + r) * P.N + n]), y[i]);
  Y[(int64_t)r * P.N + n] = ccast<TV>(acc);
}

// x = M^-1 y, block by block.
template <typename TV>
__global__ void k_apply_minv(int64_t N, int R, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ m, const int64_t* __restrict__ moff,
                             const cplx<TV>* __restrict__ Minv, const cplx<TV>* __restrict__ Y, cplx<TV>* __restrict__ X) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t o = off[p];
  const int i = (int)(n - o), mp = m[p];
  const cplx<TV>* Mi = Minv + moff[p] + (int64_t)i * mp;
  const cplx<TV>* y = Y + (int64_t)r * N + o;
  c128 acc = mkc(0.0, 0.0);
  for (int l = 0; l < mp; ++l) cfma(acc, ccast<double>(Mi[l]), ccast<double>(y[l]));
  X[(int64_t)r * N + n] = ccast<TV>(acc);
}

__global__ void k_rowwire(int64_t nw, const int64_t* __restrict__ off, int32_t* __restrict__ rowwire) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  for (int64_t n = off[p]; n < off[p + 1]; ++n) rowwire[n] = (int32_t)p;
}

template <typename TV>
int gmres_impl(swm_ctx* ctx, double tol, int restart, int max_iter) {
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  std::vector<Buf>& S = ctx->solve_bufs;
  std::vector<Buf> tmp;
  if (!ctx->rowwire) {
    SWM_TRY(dalloc(ctx, ctx->build_bufs, (void**)&ctx->rowwire, sizeof(int32_t) * std::max<int64_t>(1, N)));
    k_rowwire<<<(unsigned)ceil_div(ctx->nw, 256), 256, 0, st>>>(ctx->nw, ctx->off, ctx->rowwire);
    SWM_LAUNCHED();
  }
  KPtr P{};
  P.R = R;
  P.restart = restart;
  P.N = N;
  P.tol = tol;
  P.chunk = (int)std::max<int64_t>(kRows, ceil_div(ceil_div(N, 512), kRows) * kRows);
  P.nchunk = (int)ceil_div(N, P.chunk);
  const int R1 = restart + 1;
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.st, sizeof(KState)));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.counter, sizeof(unsigned) * (R + 1)));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.active, sizeof(int) * R));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.jlast, sizeof(int) * R));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.inv_h, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.bnorm, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.resid, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.H, sizeof(c128) * R * R1 * restart));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.cs, sizeof(double) * R * restart));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.sn, sizeof(c128) * R * restart));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.g, sizeof(c128) * R * R1));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.hc, sizeof(c128) * R * R1));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.hc2, sizeof(c128) * R * R1));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.coef, sizeof(c128) * R * restart));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.part, sizeof(c128) * (size_t)R * P.nchunk * R1));
  SWM_TRY(dalloc(ctx, tmp, (void**)&P.partn, sizeof(double) * (size_t)R * P.nchunk));
  cplx<TV> *Y = nullptr, *W0 = nullptr, *W1 = nullptr, *V = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&Y, sizeof(cplx<TV>) * R * N));
  SWM_TRY(dalloc(ctx, tmp, (void**)&W0, sizeof(cplx<TV>) * R * N));
  SWM_TRY(dalloc(ctx, tmp, (void**)&W1, sizeof(cplx<TV>) * R * N));
  SWM_TRY(dalloc(ctx, tmp, (void**)&V, sizeof(cplx<TV>) * (size_t)R1 * R * N));
  SWM_CK(cudaMemsetAsync(P.st, 0, sizeof(KState), st));
  SWM_CK(cudaMemsetAsync(P.counter, 0, sizeof(unsigned) * (R + 1), st));
  SWM_CK(cudaMemsetAsync(Y, 0, sizeof(cplx<TV>) * R * N, st));
  (void)S;

  const cplx<TV>* E = (const cplx<TV>*)ctx->Zp;
  const cplx<TV>* Bv = (const cplx<TV>*)ctx->Bv;
  const dim3 g_rows((unsigned)ceil_div(N * kG, kRows), R);
  const dim3 g_chunk((unsigned)P.nchunk, R);
  const size_t sm = sizeof(cplx<TV>) * P.chunk;
  if (sm > 48 * 1024) {
    SWM_CK(cudaFuncSetAttribute(k_step<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SWM_CK(cudaFuncSetAttribute(k_update<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SWM_CK(cudaFuncSetAttribute(k_finish<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  }
  KState hs{};
  int cycles = 0;
  bool first = true;
  if (!ctx->pinned_state) {
    SWM_CK(cudaMallocHost(&ctx->pinned_state, 2 * sizeof(KState)));
    SWM_CK(cudaEventCreateWithFlags(&ctx->poll_ev[0], cudaEventDisableTiming));
    SWM_CK(cudaEventCreateWithFlags(&ctx->poll_ev[1], cudaEventDisableTiming));
  }
  KState* slot = reinterpret_cast<KState*>(ctx->pinned_state);
  constexpr int kChunkSteps = 4;
  auto launch_steps = [&](cudaStream_t s, int n) -> int {
    for (int i = 0; i < n; ++i) {
      ctx->prof_begin(SWM_K_APPLY);
      k_step<TV><<<g_chunk, kRows, sm, s>>>(P, ctx->rowwire, ctx->off, ctx->offd, E, W0, W1, V);
      ctx->prof_end(SWM_K_APPLY);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_UPDATE);
      k_update<TV><<<g_chunk, kRows, sm, s>>>(P, W0, W1, V);
      ctx->prof_end(SWM_K_UPDATE);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_FINISH);
      k_finish<TV><<<g_chunk, kRows, sm, s>>>(P, W0, W1, V);
      ctx->prof_end(SWM_K_FINISH);
      SWM_LAUNCHED();
    }
    return SWM_OK;
  };
  // A chunk of Arnoldi steps is a CUDA graph (the launches are identical every step), captured on
  // a private stream and reused while the kernel arguments stay the same.  Profiling a GMRES kernel
  // class uses direct launches so its events time each launch.
  const bool use_graph = ctx->prof_cls != SWM_K_APPLY && ctx->prof_cls != SWM_K_UPDATE &&
                         ctx->prof_cls != SWM_K_FINISH;
  if (use_graph) {
    struct Key {
      KPtr P;
      const void* ptr[6];
      Layout lay;
      size_t sm;
      unsigned gx, gy, bits;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.P = P;
    const void* ptrs[6] = {ctx->rowwire, ctx->off, E, W0, W1, V};
    for (int i = 0; i < 6; ++i) key.ptr[i] = ptrs[i];
    key.lay = ctx->offd;
    key.sm = sm;
    key.gx = g_chunk.x;
    key.gy = g_chunk.y;
    key.bits = sizeof(TV);
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&key);
    std::vector<unsigned char> kv(kb, kb + sizeof(key));
    if (!ctx->gm_exec || kv != ctx->gm_key) {
      if (!ctx->cap_stream) SWM_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      const int64_t launches0 = ctx->launches;
      SWM_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_steps(ctx->cap_stream, kChunkSteps);
      cudaGraph_t graph = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
      ctx->launches = launches0;
      if (rc < 0) return rc;
      SWM_CK(ce);
      if (ctx->gm_exec) {
        cudaGraphExecDestroy(ctx->gm_exec);
        ctx->gm_exec = nullptr;
      }
      const cudaError_t ie = cudaGraphInstantiate(&ctx->gm_exec, graph, 0);
      cudaGraphDestroy(graph);
      SWM_CK(ie);
      ctx->gm_key = kv;
    }
  }
  while (true) {
    // residual of the current y and the start of a cycle
    ctx->prof_begin(SWM_K_APPLY);
    k_apply<TV><<<g_rows, kRows, 0, st>>>(1, P, ctx->rowwire, ctx->off, ctx->offd, E, Bv, Y, W0, W1, V);
    ctx->prof_end(SWM_K_APPLY);
    SWM_LAUNCHED();
    k_cycle_start<TV><<<g_chunk, kRows, 0, st>>>(P, W0, first ? 1 : 0);
    SWM_LAUNCHED();
    first = false;
    SWM_CK(cudaMemcpyAsync(&hs, P.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    if (hs.all_conv || hs.numeric || hs.iters >= max_iter) break;
    const int steps = std::min(restart, max_iter - hs.iters);
    // chunks of steps; the host reads the flag of chunk c - 1 while chunk c is queued
    int c = 0;
    for (int s0 = 0; s0 < steps; s0 += kChunkSteps, ++c) {
      const int n = std::min(steps - s0, kChunkSteps);
      if (use_graph && n == kChunkSteps) {
        SWM_CK(cudaGraphLaunch(ctx->gm_exec, st));
        ctx->launches += 3 * kChunkSteps;
      } else {
        SWM_TRY(launch_steps(st, n));
      }
      SWM_CK(cudaMemcpyAsync(&slot[c & 1], P.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaEventRecord(ctx->poll_ev[c & 1], st));
      if (c >= 1) {
        SWM_CK(cudaEventSynchronize(ctx->poll_ev[(c - 1) & 1]));
        if (slot[(c - 1) & 1].cycle_done) break;
      }
    }
    k_backsolve<<<(unsigned)ceil_div(R, 64), 64, 0, st>>>(P);
    SWM_LAUNCHED();
    k_update_y<TV><<<dim3((unsigned)ceil_div(N, 256), R), 256, 0, st>>>(P, V, Y);
    SWM_LAUNCHED();
    ++cycles;
  }
  // x = M^-1 y
  k_apply_minv<TV><<<dim3((unsigned)ceil_div(N, 256), R), 256, 0, st>>>(N, R, ctx->rowwire, ctx->off, ctx->m,
                                                                        ctx->minv_off, (const cplx<TV>*)ctx->Minv, Y,
                                                                        (cplx<TV>*)ctx->Xv);
  SWM_LAUNCHED();
  std::vector<double> res(R);
  SWM_CK(cudaMemcpyAsync(res.data(), P.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaStreamSynchronize(st));
  dfree_group(ctx, tmp);
  double mx = 0.0;
  for (double v : res) mx = std::max(mx, v);
  ctx->stats.iterations = hs.iters;
  ctx->stats.restarts = cycles;
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = hs.all_conv ? 1 : 0;
  if (hs.numeric) return ctx->fail(SWM_ECUDA, "GMRES produced a non-finite value");
  return hs.all_conv ? SWM_OK : SWM_ENOTCONV;
}

}  // namespace

int gmres_solve(swm_ctx* ctx, double tol, int restart, int max_iter) {
  if (ctx->prec == SWM_C128) return gmres_impl<double>(ctx, tol, restart, max_iter);
  return gmres_impl<float>(ctx, tol, restart, max_iter);
}

}  // namespace swm
