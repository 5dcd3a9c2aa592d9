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
#include <cstdlib>
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
  int cycles;     // restart cycles (persistent solve)
  int pad[2];
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
  int nschunk, schunk;  // chunks of the fused step kernel (finer, for more CTAs)
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
    int t = lane;
    for (; t + 96 < cnt; t += 128) {
      cplx<TV> v[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u] = vi[t + 32 * u];
        w[u] = w_sm[t + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.re = fma(v[u].re, w[u].re, fma(v[u].im, w[u].im, acc.re));
        acc.im = fma(v[u].re, w[u].im, fma(-v[u].im, w[u].re, acc.im));
      }
    }
    for (; t < cnt; t += 32) {
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

// Sum of a strided column of partials, read through L2 with eight loads in flight per lane.
__device__ __forceinline__ c128 sum_partials_c(const c128* __restrict__ base, int stride, int n, int lane) {
  double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
  int c = lane;
  for (; c + 7 * 32 < n; c += 8 * 32) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(reinterpret_cast<const double2*>(base + (int64_t)(c + u * 32) * stride));
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      re[u & 3] += v[u].x;
      im[u & 3] += v[u].y;
    }
  }
  for (; c < n; c += 32) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(base + (int64_t)c * stride));
    re[0] += v.x;
    im[0] += v.y;
  }
  return mkc(warp_sum((re[0] + re[1]) + (re[2] + re[3])), warp_sum((im[0] + im[1]) + (im[2] + im[3])));
}

__device__ __forceinline__ double sum_partials_d(const double* __restrict__ base, int n, int lane) {
  double a[4] = {0, 0, 0, 0};
  int c = lane;
  for (; c + 7 * 32 < n; c += 8 * 32) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(base + c + u * 32);
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u & 3] += v[u];
  }
  for (; c < n; c += 32) a[0] += __ldcg(base + c);
  return warp_sum((a[0] + a[1]) + (a[2] + a[3]));
}

__device__ void reduce_dots(const KPtr& P, int j, int r, c128* __restrict__ dst, int nchunk) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const c128* part = P.part + (int64_t)r * nchunk * (P.restart + 1);
  for (int i = wp; i <= j; i += kRows / 32) {
    const c128 v = sum_partials_c(part + i, P.restart + 1, nchunk, lane);
    if (lane == 0) dst[(int64_t)r * (P.restart + 1) + i] = v;
  }
}

// Normalise, multiply by A = I + E and take the first Gram-Schmidt dots, over one chunk of rows
// (P.schunk rows, a multiple of 32) and a block of RB right-hand sides that share every read of E.
// Eight lanes share a scalar row; the 32 row groups of the CTA take the chunk's rows in turn, with
// their descriptors loaded up front.
template <typename TV, int RB>
__global__ void __launch_bounds__(kRows) k_step(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const cplx<TV>* __restrict__ E,
                                                cplx<TV>* __restrict__ W0, cplx<TV>* __restrict__ W1,
                                                cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, rblk = blockIdx.y;
  const int r0 = rblk * RB;
  const int nr = min(RB, P.R - r0);
  const int64_t N = P.N;
  const int64_t n0 = (int64_t)blockIdx.x * P.schunk;
  const int cnt = (int)min((int64_t)P.schunk, N - n0);
  const cplx<TV>* src = ((j & 1) ? W1 : W0);
  cplx<TV>* dst = ((j & 1) ? W0 : W1);
  bool act[RB];
  TV sc[RB];
  bool any = false;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    act[b] = b < nr && P.active[r0 + b];
    sc[b] = b < nr ? (TV)P.inv_h[r0 + b] : TV(0);
    any |= act[b];
  }
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);  // [RB][schunk]
  const int g = threadIdx.x / kG, sub = threadIdx.x % kG;
  constexpr int kMaxRowsPerGroup = 4;
  RowInfo ri[kMaxRowsPerGroup];
#pragma unroll
  for (int t = 0; t < kMaxRowsPerGroup; ++t) {
    const int row = g + 32 * t;
    ri[t] = (row < cnt) ? rinfo[n0 + row] : RowInfo{0, 0, 0};
  }
#pragma unroll
  for (int t = 0; t < kMaxRowsPerGroup; ++t) {
    const int row = g + 32 * t;
    if (32 * t >= cnt) break;  // uniform across the CTA
    cplx<TV> acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
    if (any) {
      const int32_t* cm = colmap + ri[t].cmb;
      for (int c = sub; c < ri[t].K; c += kG) {
        const cplx<TV> e = E[ri[t].vb + c];
        const int64_t col = cm[c];
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (b < nr) cfma(acc[b], e, src[(int64_t)(r0 + b) * N + col]);
      }
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
#pragma unroll
      for (int o = kG / 2; o > 0; o >>= 1) {
        acc[b].re += __shfl_xor_sync(0xffffffffu, acc[b].re, o);
        acc[b].im += __shfl_xor_sync(0xffffffffu, acc[b].im, o);
      }
    }
    if (row < cnt && sub == 0) {
      const int64_t n = n0 + row;
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        if (b >= nr) break;
        const int64_t off_r = (int64_t)(r0 + b) * N;
        const cplx<TV> x = act[b] ? sc[b] * src[off_r + n] : mkc<TV>(0, 0);
        const cplx<TV> y = act[b] ? x + sc[b] * acc[b] : mkc<TV>(0, 0);
        V[((int64_t)j * P.R + r0 + b) * N + n] = x;
        dst[off_r + n] = y;
        w_sm[b * P.schunk + row] = y;
      }
    }
  }
  __syncthreads();
  for (int b = 0; b < nr; ++b)
    cta_dots<TV>(P, j, r0 + b, V, w_sm + b * P.schunk, n0, cnt,
                 P.part + ((int64_t)(r0 + b) * P.nschunk + blockIdx.x) * (P.restart + 1));
  if (last_cta(P, rblk)) {
    for (int b = 0; b < nr; ++b) reduce_dots(P, j, r0 + b, P.hc, P.nschunk);
    __syncthreads();
    if (threadIdx.x == 0) P.counter[rblk] = 0;
  }
}

// Large-N form of the step, part 1: normalise and multiply by A = I + E, streaming.  One scalar row
// per group of eight lanes, no shared memory and no barrier, so many rows' loads are in flight.
template <typename TV, int RB>
__global__ void __launch_bounds__(kRows) k_spmv(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const cplx<TV>* __restrict__ E,
                                                cplx<TV>* __restrict__ W0, cplx<TV>* __restrict__ W1,
                                                cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j;
  const int r0 = blockIdx.y * RB;
  const int nr = min(RB, P.R - r0);
  const int64_t N = P.N;
  const int64_t n = (blockIdx.x * (int64_t)kRows + threadIdx.x) / kG;
  const int sub = threadIdx.x % kG;
  const cplx<TV>* src = ((j & 1) ? W1 : W0);
  cplx<TV>* dst = ((j & 1) ? W0 : W1);
  bool act[RB];
  TV sc[RB];
  bool any = false;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    act[b] = b < nr && P.active[r0 + b];
    sc[b] = b < nr ? (TV)P.inv_h[r0 + b] : TV(0);
    any |= act[b];
  }
  cplx<TV> acc[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
  if (n < N && any) {
    const RowInfo ri = rinfo[n];
    const int32_t* cm = colmap + ri.cmb;
    int c = sub;
    for (; c + kG < ri.K; c += 2 * kG) {
      const cplx<TV> e0 = E[ri.vb + c], e1 = E[ri.vb + c + kG];
      const int64_t c0 = cm[c], c1 = cm[c + kG];
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (b < nr) {
          const cplx<TV>* x = src + (int64_t)(r0 + b) * N;
          const cplx<TV> x0 = x[c0], x1 = x[c1];
          cfma(acc[b], e0, x0);
          cfma(acc[b], e1, x1);
        }
    }
    if (c < ri.K) {
      const cplx<TV> e0 = E[ri.vb + c];
      const int64_t c0 = cm[c];
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (b < nr) cfma(acc[b], e0, src[(int64_t)(r0 + b) * N + c0]);
    }
  }
#pragma unroll
  for (int b = 0; b < RB; ++b) {
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) {
      acc[b].re += __shfl_xor_sync(0xffffffffu, acc[b].re, o);
      acc[b].im += __shfl_xor_sync(0xffffffffu, acc[b].im, o);
    }
  }
  if (n < N && sub == 0) {
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (b >= nr) break;
      const int64_t off_r = (int64_t)(r0 + b) * N;
      const cplx<TV> x = act[b] ? sc[b] * src[off_r + n] : mkc<TV>(0, 0);
      V[((int64_t)j * P.R + r0 + b) * N + n] = x;
      dst[off_r + n] = act[b] ? x + sc[b] * acc[b] : mkc<TV>(0, 0);
    }
  }
}

// Large-N form of the step, part 2: h = V^H w over chunks of rows (first Gram-Schmidt pass).
template <typename TV>
__global__ void __launch_bounds__(kRows) k_dots_big(KPtr P, cplx<TV>* __restrict__ W0, cplx<TV>* __restrict__ W1,
                                                    const cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  const cplx<TV>* w = ((j & 1) ? W0 : W1) + (int64_t)r * P.N + n0;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  for (int t = threadIdx.x; t < cnt; t += kRows) w_sm[t] = w[t];
  __syncthreads();
  cta_dots<TV>(P, j, r, V, w_sm, n0, cnt, P.part + ((int64_t)r * P.nchunk + blockIdx.x) * (P.restart + 1));
  if (last_cta(P, r)) {
    reduce_dots(P, j, r, P.hc, P.nchunk);
    if (threadIdx.x == 0) P.counter[r] = 0;
  }
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
#pragma unroll 4
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
  if (last_cta(P, r)) {
    reduce_dots(P, j, r, P.hc2, P.nchunk);
    if (threadIdx.x == 0) P.counter[r] = 0;
  }
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
  // ---- last CTA of right-hand side r: the Hessenberg column, its rotations and the residual
  // estimate are worked in shared memory (loaded and stored by all threads) so the one thread
  // that applies the rotations in order never waits on global memory.
  __shared__ double nrm2;
  __shared__ c128 col[SWM_MAX_RESTART + 1];
  __shared__ double scs[SWM_MAX_RESTART];
  __shared__ c128 ssn[SWM_MAX_RESTART];
  __shared__ int act_r;
  __shared__ c128 g_j;
  __shared__ double bnorm_r;
  const int R1 = P.restart + 1;
  c128* Hr = P.H + (int64_t)r * R1 * P.restart;  // H[i][j] at i * restart + j
  if (threadIdx.x < 32) {
    const double t = sum_partials_d(P.partn + (int64_t)r * P.nchunk, P.nchunk, threadIdx.x);
    if (threadIdx.x == 0) {
      nrm2 = t;
      act_r = P.active[r];
      g_j = P.g[(int64_t)r * R1 + j];
      bnorm_r = P.bnorm[r];
    }
  }
  for (int i = threadIdx.x; i <= j; i += kRows)
    col[i] = P.hc[(int64_t)r * R1 + i] + P.hc2[(int64_t)r * R1 + i];
  for (int i = threadIdx.x; i < j; i += kRows) {
    scs[i] = P.cs[(int64_t)r * P.restart + i];
    ssn[i] = P.sn[(int64_t)r * P.restart + i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    P.counter[r] = 0;
    if (act_r) {
      const double hn = sqrt(nrm2);
      // previous rotations
      for (int i = 0; i < j; ++i) {
        const c128 a = col[i], b = col[i + 1];
        const c128 sc = ssn[i];
        col[i] = scs[i] * a + sc * b;
        col[i + 1] = mkc(-sc.re, sc.im) * a + scs[i] * b;  // -conj(s) a + c b
      }
      // new rotation zeroing the subdiagonal hn (real, >= 0)
      const c128 a = col[j];
      const double aa = sqrt(a.re * a.re + a.im * a.im);
      const double nu = sqrt(aa * aa + hn * hn);
      double c;
      c128 sv;
      if (aa == 0.0) {
        c = 0.0;
        sv = mkc(1.0, 0.0);
      } else {
        c = aa / nu;
        sv = mkc(a.re / aa * hn / nu, a.im / aa * hn / nu);
      }
      P.cs[(int64_t)r * P.restart + j] = c;
      P.sn[(int64_t)r * P.restart + j] = sv;
      col[j] = c * a + hn * sv;
      c128* g = P.g + (int64_t)r * R1;
      const c128 gj = g_j;
      const c128 gn = mkc(-sv.re, sv.im) * gj;
      g[j + 1] = gn;
      g[j] = c * gj;
      const double res = sqrt(gn.re * gn.re + gn.im * gn.im) / bnorm_r;
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
  }
  __syncthreads();
  if (act_r)
    for (int i = threadIdx.x; i <= j; i += kRows) Hr[i * P.restart + j] = col[i];
  if (threadIdx.x == 0) {
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
    const double t = sum_partials_d(P.partn + (int64_t)r * P.nchunk, P.nchunk, threadIdx.x);
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

// Back substitution H y = g, one CTA per right-hand side.  The triangle is staged in shared memory
// (dynamic, restart^2 entries) when it fits, the diagonal reciprocals are formed in parallel, and
// warp 0 substitutes upward with a warp reduction per row.
__global__ void __launch_bounds__(kRows) k_backsolve(KPtr P, int smem_tri) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ c128 yv[SWM_MAX_RESTART], gv[SWM_MAX_RESTART], dinv[SWM_MAX_RESTART];
  const int r = blockIdx.x;
  const int n = P.jlast[r];
  const int R1 = P.restart + 1, RS = P.restart;
  const c128* Hg = P.H + (int64_t)r * R1 * RS;
  c128* Hs = reinterpret_cast<c128*>(sm_raw);
  const c128* H = smem_tri ? Hs : Hg;
  if (smem_tri)
    for (int e = threadIdx.x; e < n * n; e += kRows) {
      const int i = e / n, l = e % n;
      if (l >= i) Hs[i * RS + l] = Hg[i * RS + l];
    }
  for (int i = threadIdx.x; i < n; i += kRows) {
    gv[i] = P.g[(int64_t)r * R1 + i];
    const c128 d = Hg[i * RS + i];
    const double den = d.re * d.re + d.im * d.im;
    dinv[i] = den > 0.0 ? mkc(d.re / den, -d.im / den) : mkc(0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = n - 1; i >= 0; --i) {
      double sr = 0.0, si = 0.0;
      for (int l = i + 1 + lane; l < n; l += 32) {
        const c128 h = H[i * RS + l], y = yv[l];
        sr += h.re * y.re - h.im * y.im;
        si += h.re * y.im + h.im * y.re;
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      if (lane == 0) yv[i] = (gv[i] - mkc(sr, si)) * dinv[i];
      __syncwarp();
    }
  }
  __syncthreads();
  c128* y = P.coef + (int64_t)r * RS;
  for (int i = threadIdx.x; i < RS; i += kRows) y[i] = i < n ? yv[i] : mkc(0.0, 0.0);
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

__global__ void k_rowwire(int64_t nw, const int64_t* __restrict__ off, Layout lay, int32_t* __restrict__ rowwire,
                          RowInfo* __restrict__ rinfo) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  const int K = lay.K[p];
  for (int64_t n = off[p]; n < off[p + 1]; ++n) {
    rowwire[n] = (int32_t)p;
    rinfo[n] = RowInfo{lay.rowbase[p] + (n - off[p]) * K, (int32_t)lay.cmbase[p], K};
  }
}

// ------------------------------------------------------------------------------------------------
// Persistent solve: the whole restarted GMRES in one cooperative launch, for systems of up to a
// few hundred thousand unknowns with at most 8 right-hand sides.  There one Arnoldi step moves
// only a few megabytes, so launch gaps, host polls and dependent latencies (L2 round trips,
// float64 divides and square roots) set its time, not bandwidth.  Every CTA owns a contiguous
// chunk of rows and keeps in shared memory, when they fit: its slice of the current Krylov
// vector, its rows of the basis V, and its rows of E with their column map and row descriptors
// (loaded once).  The product first gathers the vector at the CTA's column-map slice (the rows
// of one wire share their block-row's column map) into shared memory, all loads in flight at
// once, and then forms each row's sum from shared memory.  One Arnoldi step has four phases
// separated by three grid barriers:
//   A: v_j = w / |w| (own rows), u = A v_j, first dots V^H u
//   B: sum of the dot partials, u -= V h1, second dots V^H u
//   C: sum, u -= V h2, w = u written for the next gather, |w|^2 partials
//   D: sum of the norms, Hessenberg column, Givens rotation, residual estimate and activity
// Phase D and every partial sum are computed by every CTA from the same partials in the same
// order, so all CTAs reach identical decisions and run identical barrier sequences.  The dot
// products, their sums over the CTAs (in a fixed pairwise order), the rotations and the
// triangular solve run in the precision of the vectors: float64 on the complex128 path, float32 on
// the complex64 path, whose vectors carry float32 rounding anyway (on this GPU a float64 warp
// instruction issues about sixteen times slower than a float32 one, which would otherwise set
// the step time).  The initial residual norm and the relative residual estimate are float64.
// A barrier waits at most kBarrierNs; a CTA that gives up raises an abort flag that the other
// CTAs also poll, every CTA then returns, and the host reports SWM_ETIMEOUT.
constexpr int kPT = 512;              // threads of a persistent-solve CTA
constexpr int kPWarps = kPT / 32;
constexpr int kPersistMaxR = 8;       // right-hand sides of one persistent solve
constexpr int kPersistMaxRowsPerThread = 4;
constexpr unsigned long long kBarrierNs = 1000000000ull;  // 1 s

struct PSync {
  unsigned count;  // arrivals at grid barriers since the launch
  int abort;       // a barrier ran out of time
  int pad[30];
};

struct PArgs {
  KPtr P;                  // st, jlast, resid, H, coef, R, restart, N, tol
  PSync* sync;
  const RowInfo* rinfo;
  const int32_t* colmap;
  const void* E;
  const void* B;
  void* Y;
  void* W;                 // current unnormalised Krylov vector, all rows [R][N]
  void* V;                 // basis [restart + 1][R][N] (unused when it lives in shared memory)
  void* part1;             // [R][restart + 1][G] first dots (vector precision)
  void* part2;             // [R][restart + 1][G] second dots
  void* partn;             // [R][G] squared norms
  int G, rows, max_iter;
  int vsm, esm;            // V / E slices in shared memory
  int64_t emax, cmax;      // largest E and column-map slice of a CTA (entries)
};

// Byte offsets of the shared-memory arrays of the persistent kernel.
struct PLayout {
  size_t h1, h2, yv, gg, sn, col, ri, ys, vs, es, xg, cs, cm, total;
};
__host__ __device__ inline size_t p_align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline PLayout persist_layout(int RB, int R, int restart, int rows, size_t cb, int vsm, int esm,
                                                  int64_t emax, int64_t cmax) {
  PLayout L;
  const size_t R1 = restart + 1;
  size_t o = 0;
  L.yv = o; o += sizeof(c128) * RB * restart;
  L.h1 = o; o += p_align16(cb * RB * R1);  // coefficients and rotations in the vector precision
  L.h2 = o; o += p_align16(cb * RB * R1);
  L.gg = o; o += p_align16(cb * RB * R1);
  L.sn = o; o += p_align16(cb * RB * restart);
  L.col = o; o += p_align16(cb * RB * R1);
  L.ri = o; o += esm ? 16 * (size_t)rows : 0;
  L.ys = o; o += p_align16(cb * RB * rows);
  L.vs = o; o += vsm ? p_align16(cb * R1 * R * rows) : 0;
  L.es = o; o += esm ? p_align16(cb * (size_t)emax) : 0;
  L.xg = o; o += esm ? p_align16(cb * (size_t)R * cmax) : 0;
  L.cs = o; o += p_align16(cb / 2 * RB * restart);
  L.cm = o; o += esm ? 4 * (size_t)cmax : 0;
  L.total = p_align16(o);
  return L;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <typename TV>
__device__ __forceinline__ cplx<TV> ldcg_c(const cplx<TV>* p);
template <>
__device__ __forceinline__ cplx<float> ldcg_c<float>(const cplx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return mkc<float>(v.x, v.y);
}
template <>
__device__ __forceinline__ cplx<double> ldcg_c<double>(const cplx<double>* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return mkc<double>(v.x, v.y);
}

// Grid barrier with a time limit.  Returns false (in every thread of the CTA) if this CTA gave up
// or saw another CTA give up.
__device__ bool grid_sync(PSync* s, unsigned G, unsigned* epoch, int* ok_sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (*epoch + 1u) * G;
    *epoch += 1u;
    __threadfence();
    atomicAdd(&s->count, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while (ld_acquire_u32(&s->count) < target) {
      if (*(volatile int*)&s->abort) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > kBarrierNs) {
        atomicExch(&s->abort, 1);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
    *ok_sm = ok;
  }
  __syncthreads();
  return *ok_sm != 0;
}

// Sum of G partials (contiguous, read through L2), all of a lane's loads issued together, added
// pairwise in the same order in every CTA.
template <typename T>
__device__ __forceinline__ T ldcg_s(const T* p) {
  return __ldcg(p);
}
template <typename T>
__device__ __forceinline__ cplx<T> sum_g_c(const cplx<T>* __restrict__ p, int G, int lane) {
  T re = 0, im = 0;
  for (int c0 = 0; c0 < G; c0 += 256) {
    cplx<T> v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + lane + 32 * u;
      v[u] = c < G ? ldcg_c<T>(p + c) : mkc<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = v[u] + v[u + 4];
    v[0] = v[0] + v[2];
    v[1] = v[1] + v[3];
    re += v[0].re + v[1].re;
    im += v[0].im + v[1].im;
  }
  return mkc<T>(warp_sum(re), warp_sum(im));
}
template <typename T>
__device__ __forceinline__ T sum_g_d(const T* __restrict__ p, int G, int lane) {
  T s = 0;
  for (int c0 = 0; c0 < G; c0 += 256) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + lane + 32 * u;
      v[u] = c < G ? ldcg_s<T>(p + c) : T(0);
    }
    s += ((v[0] + v[4]) + (v[2] + v[6])) + ((v[1] + v[5]) + (v[3] + v[7]));
  }
  return warp_sum(s);
}

// dst[b][i] (shared) = sum over the G CTAs of part[(b * R1 + i) * G + c], for active b, i <= j.
template <typename T>
__device__ void p_reduce(const cplx<T>* __restrict__ part, int G, int R, int R1, int j, const int* act, cplx<T>* dst) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nt = R * (j + 1);
  for (int k = wp; k < nt; k += kPWarps) {
    const int b = k / (j + 1), i = k % (j + 1);
    if (!act[b]) continue;
    const cplx<T> v = sum_g_c<T>(part + (int64_t)(b * R1 + i) * G, G, lane);
    if (lane == 0) dst[b * R1 + i] = v;
  }
}

// Rows of V: row t of basis vector i, right-hand side b is at(i, b)[t].
template <typename TV>
struct VRows {
  cplx<TV>* base;
  int64_t stride;
  int R;
  __device__ __forceinline__ cplx<TV>* at(int i, int b) const { return base + ((int64_t)i * R + b) * stride; }
};

// Partial dots conj(V_i[b]) . ys[b] over the CTA's rows, for active b and i <= j.
template <typename TV>
__device__ void p_dots(const VRows<TV>& V, const cplx<TV>* ys, int rows, int cnt, int R, int R1, int j, int G,
                       const int* act, cplx<TV>* __restrict__ part) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nt = R * (j + 1);
  for (int k = wp; k < nt; k += kPWarps) {
    const int b = k / (j + 1), i = k % (j + 1);
    if (!act[b]) continue;
    const cplx<TV>* vi = V.at(i, b);
    const cplx<TV>* w = ys + b * rows;
    cplx<TV> acc = mkc<TV>(0, 0);
    int t = lane;
    for (; t + 96 < cnt; t += 128) {
      cplx<TV> v[4], x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u] = vi[t + 32 * u];
        x[u] = w[t + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc.re = fma(v[u].re, x[u].re, fma(v[u].im, x[u].im, acc.re));
        acc.im = fma(v[u].re, x[u].im, fma(-v[u].im, x[u].re, acc.im));
      }
    }
    for (; t < cnt; t += 32) {
      const cplx<TV> v = vi[t], x = w[t];
      acc.re = fma(v.re, x.re, fma(v.im, x.im, acc.re));
      acc.im = fma(v.re, x.im, fma(-v.im, x.re, acc.im));
    }
    const TV re = warp_sum(acc.re), im = warp_sum(acc.im);
    if (lane == 0) part[(int64_t)(b * R1 + i) * G + blockIdx.x] = mkc<TV>(re, im);
  }
}

// Block sums of per-thread values nrm[b] to partn[b][blockIdx.x] (warp sums, then warp 0 sums
// the warps' values as a tree).
template <typename T, int RB>
__device__ void p_norm_partials(const T* nrm, int R, int G, T* __restrict__ partn, T (*red)[RB]) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    const T s = warp_sum(nrm[b]);
    if (lane == 0) red[wp][b] = s;
  }
  __syncthreads();
  if (wp == 0) {
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (b >= R) break;
      const T s = warp_sum(lane < kPWarps ? red[lane][b] : T(0));
      if (lane == 0) partn[(int64_t)b * G + blockIdx.x] = s;
    }
  }
}

// ys[b] -= sum_{i <= j} V_i[b] h[b][i] over the CTA's rows, for active b.  With W non-null the
// result also goes to the global vector and the squared norms of the CTA's rows go to partn.
template <typename TV, int RB>
__device__ void p_update(const VRows<TV>& V, cplx<TV>* ys, int rows, int cnt, int64_t n0, int64_t N, int R, int R1,
                         int j, const int* act, const cplx<TV>* h, cplx<TV>* __restrict__ W, TV* __restrict__ partn,
                         int G, TV (*red)[RB]) {
  TV nrm[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) nrm[b] = 0;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    if (b >= R) break;
    if (!act[b]) continue;
    const cplx<TV>* hb = h + b * R1;
    for (int t = threadIdx.x; t < cnt; t += kPT) {
      cplx<TV> x = ys[b * rows + t];
      int i = 0;
      for (; i + 3 <= j; i += 4) {
        cplx<TV> v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = V.at(i + u, b)[t];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const cplx<TV> hh = hb[i + u];
          x.re = fma(-v[u].re, hh.re, fma(v[u].im, hh.im, x.re));
          x.im = fma(-v[u].re, hh.im, fma(-v[u].im, hh.re, x.im));
        }
      }
      for (; i <= j; ++i) {
        const cplx<TV> v0 = V.at(i, b)[t];
        const cplx<TV> hh = hb[i];
        x.re = fma(-v0.re, hh.re, fma(v0.im, hh.im, x.re));
        x.im = fma(-v0.re, hh.im, fma(-v0.im, hh.re, x.im));
      }
      ys[b * rows + t] = x;
      if (W) {
        W[(int64_t)b * N + n0 + t] = x;
        nrm[b] = fma(x.re, x.re, fma(x.im, x.im, nrm[b]));
      }
    }
  }
  if (W) p_norm_partials<TV, RB>(nrm, R, G, partn, red);
}

// The CTA's slice of E: values, column map, row descriptors, and the gathered vector entries.
template <typename TV>
struct ESlice {
  const cplx<TV>* e;
  const int32_t* cm;
  const RowInfo* ri;
  int64_t ebase, cbase;  // subtracted from the descriptors' offsets
  cplx<TV>* xg;          // [R][cstride] gathered vector at the column-map slice (shared) or null
  int clen, cstride;
};

// Rows of the CTA times A = I + E for the R right-hand sides of `src`.
// mode 0 (Arnoldi): x = ys * inv (the normalised v_j, stored in V_j), ys = x + inv * E src.
// mode 1 (residual): ys = W = B - (Y + E Y), squared norms to partn.
template <typename TV, int RB>
__device__ void p_product(int mode, const PArgs& a, const ESlice<TV>& S, const cplx<TV>* __restrict__ src,
                          cplx<TV>* ys, int cnt, int64_t n0, const VRows<TV>& V, int j, const int* act,
                          const TV* inv, const cplx<TV>* __restrict__ B, cplx<TV>* __restrict__ W,
                          TV (*red)[RB]) {
  const int R = a.P.R;
  const int64_t N = a.P.N;
  bool on[RB];
  TV sc[RB];
  TV nrm[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    on[b] = b < R && (mode == 1 || act[b]);
    sc[b] = b < R ? inv[b] : TV(0);
    nrm[b] = 0;
  }
  if (S.xg) {
    // gather src at the column-map slice: every load in flight at once
#pragma unroll 4
    for (int q = threadIdx.x; q < S.clen; q += kPT) {
      const int64_t col = S.cm[q];
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (on[b]) S.xg[b * S.cstride + q] = ldcg_c<TV>(src + (int64_t)b * N + col);
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < cnt; t += kPT) {
    const RowInfo ri = S.ri[t];
    const cplx<TV>* e = S.e + (ri.vb - S.ebase);
    cplx<TV> acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
    if (S.xg) {
      const cplx<TV>* xq = S.xg + (ri.cmb - S.cbase);
      int c = 0;
      for (; c + 1 < ri.K; c += 2) {
        const cplx<TV> e0 = e[c], e1 = e[c + 1];
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (on[b]) {
            cfma(acc[b], e0, xq[b * S.cstride + c]);
            cfma(acc[b], e1, xq[b * S.cstride + c + 1]);
          }
      }
      if (c < ri.K) {
        const cplx<TV> e0 = e[c];
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (on[b]) cfma(acc[b], e0, xq[b * S.cstride + c]);
      }
    } else {
      const int32_t* cm = S.cm + (ri.cmb - S.cbase);
      int c = 0;
      for (; c + 3 < ri.K; c += 4) {
        cplx<TV> ev[4];
        int64_t col[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ev[u] = e[c + u];
          col[u] = cm[c + u];
        }
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (on[b]) {
            cplx<TV> x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = ldcg_c<TV>(src + (int64_t)b * N + col[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) cfma(acc[b], ev[u], x[u]);
          }
      }
      for (; c < ri.K; ++c) {
        const cplx<TV> ev = e[c];
        const int64_t col = cm[c];
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (on[b]) cfma(acc[b], ev, ldcg_c<TV>(src + (int64_t)b * N + col));
      }
    }
    const int64_t n = n0 + t;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (!on[b]) continue;
      if (mode == 0) {
        const cplx<TV> x = sc[b] * ys[b * a.rows + t];
        V.at(j, b)[t] = x;
        ys[b * a.rows + t] = x + sc[b] * acc[b];
      } else {
        const cplx<TV> y = src[(int64_t)b * N + n];  // own row of Y, written by this CTA
        const cplx<TV> r = B[(int64_t)b * N + n] - (y + acc[b]);
        ys[b * a.rows + t] = r;
        W[(int64_t)b * N + n] = r;
        nrm[b] = fma(r.re, r.re, fma(r.im, r.im, nrm[b]));
      }
    }
  }
  if (mode == 1) p_norm_partials<TV, RB>(nrm, R, a.G, (TV*)a.partn, red);
}

template <typename TV, int RB>
__global__ void __launch_bounds__(kPT, 1) k_gmres_persist(PArgs a) {
  using C = cplx<TV>;
  const KPtr& P = a.P;
  const int R = P.R, RS = P.restart, R1 = RS + 1, G = a.G;
  const int64_t N = P.N;
  const int64_t n0 = (int64_t)blockIdx.x * a.rows;
  const int cnt = N > n0 ? (int)(N - n0 < (int64_t)a.rows ? N - n0 : (int64_t)a.rows) : 0;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const C* B = (const C*)a.B;
  C* Y = (C*)a.Y;
  C* W = (C*)a.W;

  extern __shared__ __align__(16) unsigned char sm_raw[];
  const PLayout L = persist_layout(RB, R, RS, a.rows, sizeof(C), a.vsm, a.esm, a.emax, a.cmax);
  C* h1 = reinterpret_cast<C*>(sm_raw + L.h1);         // [RB][R1] first-pass coefficients
  C* h2 = reinterpret_cast<C*>(sm_raw + L.h2);         // [RB][R1] second-pass coefficients
  c128* yv = reinterpret_cast<c128*>(sm_raw + L.yv);   // [RB][RS] back-solve / coefficients
  C* part1 = (C*)a.part1;
  C* part2 = (C*)a.part2;
  TV* partn = (TV*)a.partn;
  C* gg = reinterpret_cast<C*>(sm_raw + L.gg);         // [RB][R1] rotated residual
  C* sn = reinterpret_cast<C*>(sm_raw + L.sn);         // [RB][RS] rotation sines
  C* colv = reinterpret_cast<C*>(sm_raw + L.col);      // [RB][R1] Hessenberg column
  TV* cs = reinterpret_cast<TV*>(sm_raw + L.cs);       // [RB][RS] rotation cosines
  C* ys = reinterpret_cast<C*>(sm_raw + L.ys);         // [RB][rows]
  VRows<TV> V;
  V.R = R;
  if (a.vsm) {
    V.base = reinterpret_cast<C*>(sm_raw + L.vs);
    V.stride = a.rows;
  } else {
    V.base = (C*)a.V + n0;
    V.stride = N;
  }
  ESlice<TV> S;
  S.e = (const C*)a.E;
  S.cm = a.colmap;
  S.ri = a.rinfo + n0;
  S.ebase = 0;
  S.cbase = 0;
  S.xg = nullptr;
  S.clen = 0;
  S.cstride = 0;
  if (a.esm && cnt > 0) {
    RowInfo* ri_s = reinterpret_cast<RowInfo*>(sm_raw + L.ri);
    C* e_s = reinterpret_cast<C*>(sm_raw + L.es);
    int32_t* cm_s = reinterpret_cast<int32_t*>(sm_raw + L.cm);
    const RowInfo first = a.rinfo[n0], last = a.rinfo[n0 + cnt - 1];
    const int64_t elen = last.vb + last.K - first.vb;
    const int64_t clen = (int64_t)last.cmb + last.K - first.cmb;
    if (elen <= a.emax && clen <= a.cmax) {  // always true for the host's slice bounds
      for (int t = threadIdx.x; t < cnt; t += kPT) ri_s[t] = a.rinfo[n0 + t];
      for (int64_t i = threadIdx.x; i < elen; i += kPT) e_s[i] = S.e[first.vb + i];
      for (int64_t i = threadIdx.x; i < clen; i += kPT) cm_s[i] = a.colmap[first.cmb + i];
      S.e = e_s;
      S.cm = cm_s;
      S.ri = ri_s;
      S.ebase = first.vb;
      S.cbase = first.cmb;
      S.xg = reinterpret_cast<C*>(sm_raw + L.xg);
      S.clen = (int)clen;
      S.cstride = (int)a.cmax;
    }
  }
  __shared__ double bnorm[RB], resid[RB];
  __shared__ TV inv[RB], nrm2[RB];
  __shared__ TV red[kPWarps][RB];
  __shared__ int act[RB], jl[RB];
  __shared__ int s_j, s_iters, s_done, s_conv, s_numeric, s_cycles, s_ok;
  __shared__ unsigned s_epoch;
  if (threadIdx.x == 0) {
    s_epoch = 0;
    s_iters = 0;
    s_numeric = 0;
    s_cycles = 0;
    s_conv = 0;
  }
  if (threadIdx.x < RB) {
    act[threadIdx.x] = 0;
    inv[threadIdx.x] = 0;
    jl[threadIdx.x] = 0;
  }
  __syncthreads();
  bool first = true;
  bool ok = true;
  while (true) {
    if (!first) {
      // ---- end of a cycle: CTA 0 solves the triangular systems (one warp per right-hand side)
      if (blockIdx.x == 0 && wp < R) {
        const int b = wp, n = jl[b];
        const c128* Hb = P.H + (int64_t)b * R1 * RS;
        C* y = reinterpret_cast<C*>(yv) + b * RS;
        for (int i = n - 1; i >= 0; --i) {
          TV sr = 0, si = 0;
          for (int l = i + 1 + lane; l < n; l += 32) {
            const C h = ccast<TV>(Hb[i * RS + l]), v = y[l];
            sr += h.re * v.re - h.im * v.im;
            si += h.re * v.im + h.im * v.re;
          }
          sr = warp_sum(sr);
          si = warp_sum(si);
          if (lane == 0) {
            const C d = ccast<TV>(Hb[i * RS + i]);
            const TV den = d.re * d.re + d.im * d.im;
            const TV iden = den > TV(0) ? TV(1) / den : TV(0);
            y[i] = (gg[b * R1 + i] - mkc<TV>(sr, si)) * mkc<TV>(d.re * iden, -d.im * iden);
          }
          __syncwarp();
        }
        for (int i = lane; i < RS; i += 32) P.coef[(int64_t)b * RS + i] = i < n ? ccast<double>(y[i]) : mkc(0.0, 0.0);
      }
      if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
      // ---- Y += V coef on the CTA's rows
      C* yc = reinterpret_cast<C*>(yv);
      for (int k = threadIdx.x; k < R * RS; k += kPT) yc[k] = ccast<TV>(ldcg_c<double>(P.coef + k));
      __syncthreads();
      for (int k = threadIdx.x; cnt > 0 && k < R * cnt; k += kPT) {
        const int b = k / cnt, t = k % cnt;
        const int n = jl[b];
        if (n == 0) continue;
        const int64_t row = (int64_t)b * N + n0 + t;
        C acc = Y[row];
        for (int i = 0; i < n; ++i) cfma(acc, V.at(i, b)[t], yc[b * RS + i]);
        Y[row] = acc;
      }
      if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
    }
    // ---- residual W = B - A Y on the CTA's rows, its squared norms
    p_product<TV, RB>(1, a, S, Y, ys, cnt, n0, V, 0, act, inv, B, W, red);
    if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
    // ---- start of a cycle (every CTA)
    if (wp < R) {
      const TV t = sum_g_d<TV>(partn + (int64_t)wp * G, G, lane);
      if (lane == 0) nrm2[wp] = t;
    }
    __syncthreads();
    if (threadIdx.x < R) {
      const int b = threadIdx.x;
      const double beta = sqrt((double)nrm2[b]);
      if (first) bnorm[b] = beta > 0.0 ? beta : 1.0;
      const double res = beta / bnorm[b];
      resid[b] = res;
      jl[b] = 0;
      const bool ac = isfinite(res) && res > P.tol;
      if (!isfinite(res)) s_numeric = 1;
      act[b] = ac ? 1 : 0;
      inv[b] = beta > 0.0 ? (TV)(1.0 / beta) : TV(0);
      gg[b * R1] = mkc<TV>((TV)beta, TV(0));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int b = 0; b < R; ++b) any |= act[b];
      s_conv = any ? 0 : 1;
      s_j = 0;
      s_done = (!any || s_iters >= a.max_iter) ? 1 : 0;
      if (!first) s_cycles += 1;
    }
    __syncthreads();
    first = false;
    if (s_conv || s_numeric || s_iters >= a.max_iter) break;
    // ---- Arnoldi steps
    while (!s_done) {
      const int j = s_j;
      // A: v_j and u = A v_j on own rows, first dots
      p_product<TV, RB>(0, a, S, W, ys, cnt, n0, V, j, act, inv, B, W, red);
      __syncthreads();
      p_dots<TV>(V, ys, a.rows, cnt, R, R1, j, G, act, part1);
      if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
      // B: h1, u -= V h1, second dots
      p_reduce<TV>(part1, G, R, R1, j, act, h1);
      __syncthreads();
      p_update<TV, RB>(V, ys, a.rows, cnt, n0, N, R, R1, j, act, h1, nullptr, nullptr, G, red);
      __syncthreads();
      p_dots<TV>(V, ys, a.rows, cnt, R, R1, j, G, act, part2);
      if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
      // C: h2, w = u - V h2 to global, squared norms
      p_reduce<TV>(part2, G, R, R1, j, act, h2);
      __syncthreads();
      p_update<TV, RB>(V, ys, a.rows, cnt, n0, N, R, R1, j, act, h2, W, partn, G, red);
      if (!(ok = grid_sync(a.sync, G, &s_epoch, &s_ok))) break;
      // D: norms, Hessenberg column, rotations, residual estimate (every CTA, same values)
      if (wp < R && act[wp]) {
        const TV t = sum_g_d<TV>(partn + (int64_t)wp * G, G, lane);
        if (lane == 0) nrm2[wp] = t;
      }
      for (int k = threadIdx.x; k < R * (j + 1); k += kPT) {
        const int b = k / (j + 1), i = k % (j + 1);
        if (act[b]) colv[b * R1 + i] = h1[b * R1 + i] + h2[b * R1 + i];
      }
      __syncthreads();
      if (threadIdx.x < R && act[threadIdx.x]) {
        const int b = threadIdx.x;
        C* col = colv + b * R1;
        const TV h = sqrt(nrm2[b]);
        for (int i = 0; i < j; ++i) {
          const C x0 = col[i], x1 = col[i + 1];
          const C s = sn[b * RS + i];
          const TV c = cs[b * RS + i];
          col[i] = c * x0 + s * x1;
          col[i + 1] = mkc<TV>(-s.re, s.im) * x0 + c * x1;
        }
        const C x = col[j];
        const TV ax2 = x.re * x.re + x.im * x.im;
        const TV aa = sqrt(ax2);
        const TV nu = sqrt(ax2 + h * h);
        const TV inu = TV(1) / nu;
        TV c;
        C sv;
        if (aa == TV(0)) {
          c = TV(0);
          sv = mkc<TV>(1, 0);
        } else {
          c = aa * inu;
          const TV f = h * inu / aa;
          sv = mkc<TV>(x.re * f, x.im * f);
        }
        cs[b * RS + j] = c;
        sn[b * RS + j] = sv;
        col[j] = c * x + h * sv;
        const C gj = gg[b * R1 + j];
        gg[b * R1 + j + 1] = mkc<TV>(-sv.re, sv.im) * gj;
        gg[b * R1 + j] = c * gj;
        // |g_{j+1}| = |s_j| |g_j| with |s_j| = h / nu
        const double res = resid[b] * (double)(h * inu);
        resid[b] = res;
        jl[b] = j + 1;
        if (!isfinite(h) || !isfinite(res)) {
          s_numeric = 1;
          act[b] = 0;
        } else if (res <= P.tol || h == TV(0)) {
          act[b] = 0;
        }
        inv[b] = h > TV(0) ? TV(1) / h : TV(0);
      }
      __syncthreads();
      if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < R * (j + 1); k += kPT) {
          const int b = k / (j + 1), i = k % (j + 1);
          if (jl[b] == j + 1) P.H[(int64_t)b * R1 * RS + i * RS + j] = ccast<double>(colv[b * R1 + i]);
        }
      if (threadIdx.x == 0) {
        int any = 0;
        for (int b = 0; b < R; ++b) any |= act[b];
        s_j = j + 1;
        s_iters += 1;
        s_done = (!any || j + 1 >= RS || s_iters >= a.max_iter) ? 1 : 0;
      }
      __syncthreads();
    }
    if (!ok) break;
  }
  // ---- results (CTA 0)
  if (blockIdx.x == 0 && ok) {
    if (threadIdx.x < R) {
      P.resid[threadIdx.x] = resid[threadIdx.x];
      P.jlast[threadIdx.x] = jl[threadIdx.x];
    }
    if (threadIdx.x == 0) {
      P.st->iters = s_iters;
      P.st->all_conv = s_conv;
      P.st->numeric = s_numeric;
      P.st->cycles = s_cycles;
    }
  }
}

template <typename TV>
int gmres_impl(swm_ctx* ctx, double tol, int restart, int max_iter) {
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  std::vector<Buf>& S = ctx->solve_bufs;
  std::vector<Buf> tmp;
  SWM_TRY(ensure_rowinfo(ctx));
  KPtr P{};
  P.R = R;
  P.restart = restart;
  P.N = N;
  P.tol = tol;
  P.chunk = (int)std::max<int64_t>(kRows, ceil_div(ceil_div(N, 512), kRows) * kRows);
  P.nchunk = (int)ceil_div(N, P.chunk);
  // the fused step kernel: 64..128 rows per CTA, at most 2048 chunks
  P.schunk = (int)std::min<int64_t>(128, std::max<int64_t>(128, ceil_div(ceil_div(N, 2048), 32) * 32));
  P.nschunk = (int)ceil_div(N, P.schunk);
  const int R1 = restart + 1;
  // The workspace persists across solves of the same size, so buffer addresses (and the captured
  // graph that bakes them in) stay the same from one solve to the next.
  struct Workspace {
    int64_t key[4];
    KPtr P;
    cplx<TV> *Y, *W0, *W1, *V;
    PSync* sync;          // persistent solve: barrier state and partial sums over its CTAs
    c128 *pp1, *pp2;
    double* ppn;
  };
  const int64_t key[4] = {R, N, restart, (int64_t)sizeof(TV)};
  Workspace* ws = reinterpret_cast<Workspace*>(ctx->kry_ws);
  if (!ws || std::memcmp(ws->key, key, sizeof(key)) != 0 || ctx->kry_ws_bytes != sizeof(Workspace)) {
    dfree_group(ctx, ctx->kry_bufs);
    std::free(ctx->kry_ws);
    ctx->kry_ws = nullptr;
    ws = reinterpret_cast<Workspace*>(std::calloc(1, sizeof(Workspace)));
    if (!ws) return ctx->fail(SWM_ENOMEM, "host allocation failed");
    ctx->kry_ws = ws;
    ctx->kry_ws_bytes = sizeof(Workspace);
    std::memcpy(ws->key, key, sizeof(key));
    auto& K = ctx->kry_bufs;
    SWM_TRY(dalloc(ctx, K, (void**)&P.st, sizeof(KState)));
    SWM_TRY(dalloc(ctx, K, (void**)&P.counter, sizeof(unsigned) * (R + 1)));
    SWM_TRY(dalloc(ctx, K, (void**)&P.active, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.jlast, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.inv_h, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.bnorm, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.resid, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.H, sizeof(c128) * R * R1 * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.cs, sizeof(double) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.sn, sizeof(c128) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.g, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.hc, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.hc2, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.coef, sizeof(c128) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.part, sizeof(c128) * (size_t)R * std::max(P.nchunk, P.nschunk) * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.partn, sizeof(double) * (size_t)R * P.nchunk));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->Y, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->W0, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->W1, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->V, sizeof(cplx<TV>) * (size_t)R1 * R * N));
    if (R <= kPersistMaxR && ctx->nsm > 0) {
      SWM_TRY(dalloc(ctx, K, (void**)&ws->sync, sizeof(PSync)));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->pp1, sizeof(c128) * (size_t)R * R1 * ctx->nsm));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->pp2, sizeof(c128) * (size_t)R * R1 * ctx->nsm));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->ppn, sizeof(double) * (size_t)R * ctx->nsm));
    }
    ws->P = P;
  } else {
    const double tol_now = P.tol;
    P = ws->P;
    P.tol = tol_now;
  }
  cplx<TV> *Y = ws->Y, *W0 = ws->W0, *W1 = ws->W1, *V = ws->V;
  SWM_CK(cudaMemsetAsync(P.st, 0, sizeof(KState), st));
  SWM_CK(cudaMemsetAsync(P.counter, 0, sizeof(unsigned) * (R + 1), st));
  SWM_CK(cudaMemsetAsync(Y, 0, sizeof(cplx<TV>) * R * N, st));
  (void)S;

  const cplx<TV>* E = (const cplx<TV>*)ctx->Zp;
  const cplx<TV>* Bv = (const cplx<TV>*)ctx->Bv;
  KState hs{};
  int cycles = 0;
  // small systems: the whole solve as one persistent cooperative kernel
  bool persisted = false;
  const int prows = (int)(ceil_div(ceil_div(std::max<int64_t>(N, 1), ctx->nsm > 0 ? ctx->nsm : 1), 32) * 32);
  if (ctx->persist && ctx->coop && ws->sync && N > 0 && N < ctx->split_rows &&
      prows <= kPersistMaxRowsPerThread * kPT) {
    const int G = (int)ceil_div(N, prows);
    const int RB = R == 1 ? 1 : kPersistMaxR;
    const void* fn = R == 1 ? (const void*)k_gmres_persist<TV, 1> : (const void*)k_gmres_persist<TV, kPersistMaxR>;
    cudaFuncAttributes fa{};
    SWM_CK(cudaFuncGetAttributes(&fa, fn));
    const size_t limit = (size_t)std::max(0, ctx->smem_optin - (int)fa.sharedSizeBytes - 1024);
    const size_t cb = sizeof(cplx<TV>);
    // V in shared memory when it fits (it is read four times a step); then as large an E slice as
    // the rest holds (column map + gathered vector about a third of the E entries: the rows of a
    // wire share their column map).  A CTA whose slice is larger reads E from global memory.
    int vsm = persist_layout(RB, R, restart, prows, cb, 1, 0, 0, 0).total <= limit ? 1 : 0;
    const size_t base = persist_layout(RB, R, restart, prows, cb, vsm, 1, 0, 0).total + 64;
    const int64_t mean_e = ceil_div(ctx->offd.nval, G);
    int64_t emax = 0, cmax = 0;
    if (base < limit) {
      emax = (int64_t)((limit - base) / (cb + (4 + cb * R) / 3.0));
      cmax = emax / 3;
    }
    const int esm = emax >= mean_e && emax > 0 ? 1 : 0;
    if (!esm) emax = cmax = 0;
    const size_t smem = persist_layout(RB, R, restart, prows, cb, vsm, esm, emax, cmax).total;
    const bool fits = smem <= limit;
    int occ = 0;
    if (fits) {
      SWM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      SWM_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPT, smem));
    }
    if (occ >= 1 && G <= occ * ctx->nsm) {
      PArgs pa{};
      pa.P = P;
      pa.sync = ws->sync;
      pa.rinfo = (const RowInfo*)ctx->rowinfo;
      pa.colmap = ctx->offd.colmap;
      pa.E = E;
      pa.B = Bv;
      pa.Y = Y;
      pa.W = W0;
      pa.V = V;
      pa.part1 = ws->pp1;
      pa.part2 = ws->pp2;
      pa.partn = ws->ppn;
      pa.G = G;
      pa.rows = prows;
      pa.max_iter = max_iter;
      pa.vsm = vsm;
      pa.esm = esm;
      pa.emax = emax;
      pa.cmax = cmax;
      SWM_CK(cudaMemsetAsync(ws->sync, 0, sizeof(PSync), st));
      void* args[] = {&pa};
      ctx->prof_begin(SWM_K_GMRES);
      SWM_CK(cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kPT), args, smem, st));
      ctx->prof_end(SWM_K_GMRES);
      SWM_LAUNCHED();
      PSync hsync{};
      SWM_CK(cudaMemcpyAsync(&hs, P.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaMemcpyAsync(&hsync, ws->sync, sizeof(PSync), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaStreamSynchronize(st));
      if (hsync.abort) return ctx->fail(SWM_ETIMEOUT, "GMRES: a grid barrier of the persistent solve timed out");
      cycles = hs.cycles;
      persisted = true;
    }
  }
  const dim3 g_rows((unsigned)ceil_div(N * kG, kRows), R);
  const dim3 g_chunk((unsigned)P.nchunk, R);
  constexpr int kRB = 8;
  const bool multi = R > 1;
  // large systems: streaming product and separate dots (bandwidth); small: one fused kernel (latency)
  const bool split = N >= ctx->split_rows;
  const dim3 g_schunk((unsigned)P.nschunk, multi ? (unsigned)ceil_div(R, kRB) : 1u);
  const size_t sm = sizeof(cplx<TV>) * P.chunk;
  const size_t ssm = sizeof(cplx<TV>) * P.schunk * (multi ? kRB : 1);
  if (sm > 48 * 1024) {
    SWM_CK(cudaFuncSetAttribute(k_update<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SWM_CK(cudaFuncSetAttribute(k_dots_big<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SWM_CK(cudaFuncSetAttribute(k_finish<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  }
  // back substitution stages the triangle in shared memory when it fits
  size_t bs_smem = sizeof(c128) * (size_t)restart * restart;
  if (bs_smem > 160 * 1024) bs_smem = 0;
  if (bs_smem > 0)
    SWM_CK(cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs_smem));
  bool first = true;
  SWM_TRY(ensure_poll_slots(ctx));
  static_assert(2 * sizeof(KState) <= kPollSlotBytes, "poll slots");
  KState* slot = reinterpret_cast<KState*>(ctx->pinned_state);
  constexpr int kChunkSteps = 4;
  auto launch_steps = [&](cudaStream_t s, int n) -> int {
    for (int i = 0; i < n; ++i) {
      ctx->prof_begin(SWM_K_APPLY);
      if (split) {
        const dim3 gsp((unsigned)ceil_div(N * kG, kRows), multi ? (unsigned)ceil_div(R, kRB) : 1u);
        if (multi)
          k_spmv<TV, kRB><<<gsp, kRows, 0, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        else
          k_spmv<TV, 1><<<gsp, kRows, 0, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        ctx->prof_end(SWM_K_APPLY);
        SWM_LAUNCHED();
        ctx->prof_begin(SWM_K_DOTS);
        k_dots_big<TV><<<g_chunk, kRows, sm, s>>>(P, W0, W1, V);
        ctx->prof_end(SWM_K_DOTS);
      } else if (multi) {
        k_step<TV, kRB><<<g_schunk, kRows, ssm, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        ctx->prof_end(SWM_K_APPLY);
      } else {
        k_step<TV, 1><<<g_schunk, kRows, ssm, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        ctx->prof_end(SWM_K_APPLY);
      }
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
  const bool use_graph = !persisted && ctx->prof_cls != SWM_K_APPLY && ctx->prof_cls != SWM_K_DOTS &&
                         ctx->prof_cls != SWM_K_UPDATE && ctx->prof_cls != SWM_K_FINISH;
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
    const void* ptrs[6] = {ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V};
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
  while (!persisted) {
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
    k_backsolve<<<(unsigned)R, kRows, bs_smem, st>>>(P, bs_smem > 0 ? 1 : 0);
    SWM_LAUNCHED();
    k_update_y<TV><<<dim3((unsigned)ceil_div(N, 256), R), 256, 0, st>>>(P, V, Y);
    SWM_LAUNCHED();
    ++cycles;
  }
  // x = M^-1 y
  SWM_TRY(apply_minv(ctx, Y));
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

int ensure_poll_slots(swm_ctx* ctx) {
  if (ctx->pinned_state) return SWM_OK;
  SWM_CK(cudaMallocHost(&ctx->pinned_state, kPollSlotBytes));
  SWM_CK(cudaEventCreateWithFlags(&ctx->poll_ev[0], cudaEventDisableTiming));
  SWM_CK(cudaEventCreateWithFlags(&ctx->poll_ev[1], cudaEventDisableTiming));
  return SWM_OK;
}

int ensure_rowinfo(swm_ctx* ctx) {
  if (ctx->rowwire) return SWM_OK;
  const int64_t N = ctx->N;
  if (ctx->offd.ncm > INT32_MAX) return ctx->fail(SWM_EINVAL, "column map too large for 32-bit offsets");
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, (void**)&ctx->rowwire, sizeof(int32_t) * std::max<int64_t>(1, N)));
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, &ctx->rowinfo, sizeof(RowInfo) * std::max<int64_t>(1, N)));
  k_rowwire<<<(unsigned)ceil_div(ctx->nw, 256), 256, 0, ctx->stream>>>(ctx->nw, ctx->off, ctx->offd, ctx->rowwire,
                                                                      (RowInfo*)ctx->rowinfo);
  SWM_LAUNCHED();
  return SWM_OK;
}

int apply_minv(swm_ctx* ctx, const void* Y) {
  const int64_t N = ctx->N;
  const int R = ctx->n_rhs;
  const dim3 grid((unsigned)ceil_div(N, 256), R);
  if (ctx->prec == SWM_C128)
    k_apply_minv<double><<<grid, 256, 0, ctx->stream>>>(N, R, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off,
                                                         (const c128*)ctx->Minv, (const c128*)Y, (c128*)ctx->Xv);
  else
    k_apply_minv<float><<<grid, 256, 0, ctx->stream>>>(N, R, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off,
                                                        (const c64*)ctx->Minv, (const c64*)Y, (c64*)ctx->Xv);
  SWM_LAUNCHED();
  return SWM_OK;
}

int gmres_solve(swm_ctx* ctx, double tol, int restart, int max_iter) {
  if (ctx->prec == SWM_C128) return gmres_impl<double>(ctx, tol, restart, max_iter);
  return gmres_impl<float>(ctx, tol, restart, max_iter);
}

}  // namespace swm
