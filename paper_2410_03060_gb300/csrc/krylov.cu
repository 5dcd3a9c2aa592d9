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
#include "krylov_common.cuh"

namespace swm {

namespace {

constexpr int kRows = 256;  // CTA width of the vector kernels
constexpr int kMinorR = 12;  // right-hand sides from which the large-system product reads them
                             // right-hand-side minor (one lane each)
constexpr int kG = 8;       // lanes per scalar row in the block-sparse product

template <typename T>
__device__ __forceinline__ bool finite_c(cplx<T> z) {
  return isfinite((double)z.re) && isfinite((double)z.im);
}

// mode 0 (Arnoldi): x = W_src * inv_h; V[j] = x (row owners); W_dst = x + E x.
// mode 1 (residual): W_dst = B - (Y + E Y).
template <typename TV, typename TE>
__global__ void __launch_bounds__(kRows) k_apply(int mode, KPtr P, const int32_t* __restrict__ rowwire,
                                                 const int64_t* __restrict__ off, Layout lay,
                                                 const TE* __restrict__ E, const cplx<TV>* __restrict__ B,
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
    for (int c = sub; c < K; c += kG) cfma(acc, ELoad<TV, TE>::ld(E + vb + c), src[cm[c]]);
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
    for (; t + 224 < cnt; t += 256) {  // eight loads in flight per lane
      cplx<TV> v[8], w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[u] = vi[t + 32 * u];
        w[u] = w_sm[t + 32 * u];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
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
template <typename TV, typename TE, int RB>
__global__ void __launch_bounds__(kRows) k_step(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const TE* __restrict__ E,
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
  for (int tb = 0; tb < cnt; tb += 32 * kMaxRowsPerGroup) {  // same trip count in every lane
  RowInfo ri[kMaxRowsPerGroup];
#pragma unroll
  for (int t = 0; t < kMaxRowsPerGroup; ++t) {
    const int row = tb + g + 32 * t;
    ri[t] = (row < cnt) ? rinfo[n0 + row] : RowInfo{0, 0, 0};
  }
#pragma unroll
  for (int t = 0; t < kMaxRowsPerGroup; ++t) {
    const int row = tb + g + 32 * t;
    if (tb + 32 * t >= cnt) break;  // uniform across the CTA
    cplx<TV> acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
    if (any) {
      const int32_t* cm = colmap + ri[t].cmb;
      for (int c = sub; c < ri[t].K; c += kG) {
        const cplx<TV> e = ELoad<TV, TE>::ld(E + ri[t].vb + c);
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
template <typename TV, typename TE, int RB>
__global__ void __launch_bounds__(kRows) k_spmv(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const TE* __restrict__ E,
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
      const cplx<TV> e0 = ELoad<TV, TE>::ld(E + ri.vb + c), e1 = ELoad<TV, TE>::ld(E + ri.vb + c + kG);
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
      const cplx<TV> e0 = ELoad<TV, TE>::ld(E + ri.vb + c);
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

// Large-N form of the step with many right-hand sides, part 0: the current Krylov vectors
// (right-hand-side major, [R][N]) copied to right-hand-side minor order Xt[N][R], through
// shared-memory tiles of 32 rows x 32 right-hand sides, so that the product below reads the values
// of all right-hand sides at a column as one contiguous run.
template <typename TV>
__global__ void __launch_bounds__(256) k_rhs_minor(KPtr P, const cplx<TV>* __restrict__ W0,
                                                   const cplx<TV>* __restrict__ W1, cplx<TV>* __restrict__ Xt) {
  if (P.st->cycle_done) return;
  const cplx<TV>* src = (P.st->j & 1) ? W1 : W0;
  __shared__ cplx<TV> tile[32][33];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k;
    const int64_t n = n0 + tx;
    if (r < P.R && n < P.N) tile[k][tx] = src[(int64_t)r * P.N + n];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t n = n0 + k;
    const int r = r0 + tx;
    if (r < P.R && n < P.N) Xt[n * P.R + r] = tile[tx][k];
  }
}

// Large-N form of the step with many right-hand sides, part 1: normalise and multiply by
// A = I + E with one lane per right-hand side: the RB lanes of a row group read each entry of E
// once (the same address: one transaction) and the RB values of the gathered column as one
// contiguous run of Xt.  E is read once per block of RB right-hand sides.  A CTA covers 32 rows;
// its results go through shared memory so that V_j and w are written right-hand-side major as
// runs of 32 consecutive rows.
constexpr int kTileRows = 32;
template <typename TV, typename TE, int RB>
__global__ void __launch_bounds__(256) k_spmv_t(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const TE* __restrict__ E,
                                                const cplx<TV>* __restrict__ Xt, cplx<TV>* __restrict__ W0,
                                                cplx<TV>* __restrict__ W1, cplx<TV>* __restrict__ V) {
  if (P.st->cycle_done) return;
  __shared__ cplx<TV> xs[kTileRows][RB + 1], ys[kTileRows][RB + 1];
  const int j = P.st->j;
  const int64_t N = P.N;
  const int R = P.R;
  const int64_t n0 = (int64_t)blockIdx.x * kTileRows;
  const int lr = (int)(threadIdx.x % RB);          // right-hand side within the block
  const int r = blockIdx.y * RB + lr;
  const bool on = r < R && P.active[r];
  const TV sc = r < R ? (TV)P.inv_h[r] : TV(0);
  constexpr int kGroups = 256 / RB;                 // rows per pass
  for (int t = (int)(threadIdx.x / RB); t < kTileRows; t += kGroups) {
    const int64_t n = n0 + t;
    cplx<TV> x = mkc<TV>(0, 0), y = mkc<TV>(0, 0);
    if (n < N && on) {
      const RowInfo ri = rinfo[n];
      const int32_t* cm = colmap + ri.cmb;
      cplx<TV> acc = mkc<TV>(0, 0);
      int c = 0;
      for (; c + 3 < ri.K; c += 4) {
        cplx<TV> e[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          e[u] = ELoad<TV, TE>::ld(E + ri.vb + c + u);
          xv[u] = Xt[(int64_t)cm[c + u] * R + r];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) cfma(acc, e[u], xv[u]);
      }
      for (; c < ri.K; ++c) cfma(acc, ELoad<TV, TE>::ld(E + ri.vb + c), Xt[(int64_t)cm[c] * R + r]);
      x = sc * Xt[n * R + r];
      y = x + sc * acc;
    }
    xs[t][lr] = x;
    ys[t][lr] = y;
  }
  __syncthreads();
  // write: warp w takes right-hand sides w, w + 8, ...; its lanes take the 32 rows
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = n0 + lane;
  for (int b = w; b < RB; b += 8) {
    const int rr = blockIdx.y * RB + b;
    if (rr >= R || n >= N) continue;
    V[((int64_t)j * R + rr) * N + n] = xs[lane][b];
    ((j & 1) ? W0 : W1)[(int64_t)rr * N + n] = ys[lane][b];
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

// Restarted GMRES on A = I + E with E stored as TE.  With y_out the result stays in y-space
// (*y_out = the workspace's y, no M^-1 and no statistics); otherwise x = M^-1 y goes to ctx->Xv.
template <typename TV, typename TE>
int gmres_impl(swm_ctx* ctx, const TE* E, double tol, int restart, int max_iter, void** y_out, KState* hs_out) {
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
  // rows per CTA of the Gram-Schmidt kernels: about 512 chunks per right-hand side, or 2048 for a
  // single one (smaller chunks, less shared memory each, more CTAs and loads in flight per SM)
  P.chunk = (int)std::max<int64_t>(kRows, ceil_div(ceil_div(N, R == 1 ? 2048 : 512), kRows) * kRows);
  P.nchunk = (int)ceil_div(N, P.chunk);
  // the fused step kernel: 128 rows per CTA for one right-hand side; with several, chunks as large as
  // keep about four CTAs per SM busy over the blocks of 8 right-hand sides (at most 1024 rows), so
  // the partial dot products the last CTA sums stay few
  {
    const int64_t nrb = ceil_div(R, 8);
    const int64_t want = std::max<int64_t>(1, 4 * std::max(ctx->nsm, 1) / std::max<int64_t>(1, nrb));
    P.schunk = R > 1 ? (int)std::min<int64_t>(1024, std::max<int64_t>(128, ceil_div(ceil_div(N, want), 32) * 32))
                     : 128;
  }
  P.nschunk = (int)ceil_div(N, P.schunk);
  const int R1 = restart + 1;
  // The workspace persists across solves of the same size, so buffer addresses (and the captured
  // graph that bakes them in) stay the same from one solve to the next.
  struct Workspace {
    int64_t key[4];
    KPtr P;
    cplx<TV> *Y, *W0, *W1, *V;
    cplx<TV>* Xt;         // many right-hand sides, large systems: the current vectors, [N][R]
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
    if (R >= kMinorR && N >= ctx->split_rows)
      SWM_TRY(dalloc(ctx, K, (void**)&ws->Xt, sizeof(cplx<TV>) * (size_t)R * N));
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
  // with an initial guess the tolerance stays relative to |b|, so |b| is measured first
  const bool given_b = ctx->guess && !y_out;
  if (y_out)  // inner solve of the refinement: the correction starts from zero
    SWM_CK(cudaMemsetAsync(Y, 0, sizeof(cplx<TV>) * R * N, st));
  else
    SWM_TRY(init_y(ctx, Y, sizeof(TV) == sizeof(double)));
  if (given_b) SWM_TRY(norms_of_b(ctx, ctx->Bv, sizeof(TV) == sizeof(double), P.bnorm));
  (void)S;

  const cplx<TV>* Bv = (const cplx<TV>*)ctx->Bv;
  KState hs{};
  int cycles = 0;
  // small systems: the whole solve as one persistent cooperative kernel
  bool persisted = false;
  {
    PBuffers pb{ws->sync, ws->pp1, ws->pp2, ws->ppn, E, Bv, Y, W0, V, given_b ? 1 : 0};
    SWM_TRY((gmres_persistent<TV, TE>(ctx, P, pb, max_iter, &hs, &persisted)));
    if (persisted) cycles = hs.cycles;
  }
  const dim3 g_rows((unsigned)ceil_div(N * kG, kRows), R);
  const dim3 g_chunk((unsigned)P.nchunk, R);
  constexpr int kRB = 8;  // right-hand sides sharing each read of E in the streaming product
  const bool multi = R > 1;
  // large systems: streaming product and separate dots (bandwidth); small: one fused kernel (latency)
  const bool split = N >= ctx->split_rows;
  const size_t sm = sizeof(cplx<TV>) * P.chunk;
  // Fused step with several right-hand sides: how many share each read of E (4, 8 or 16) is
  // measured on this system the first time its shape is seen, and kept.
  int rb = multi ? 8 : 1;
  auto ssm_of = [&](int b) { return sizeof(cplx<TV>) * (size_t)P.schunk * b; };
  auto step_fn = [&](int b) -> const void* {
    switch (b) {
      case 1: return (const void*)k_step<TV, TE, 1>;
      case 4: return (const void*)k_step<TV, TE, 4>;
      case 16: return (const void*)k_step<TV, TE, 16>;
      default: return (const void*)k_step<TV, TE, 8>;
    }
  };
  auto launch_step = [&](cudaStream_t s, int b) {
    const dim3 gs((unsigned)P.nschunk, (unsigned)ceil_div(R, b));
    const size_t sz = ssm_of(b);
    const RowInfo* ri = (const RowInfo*)ctx->rowinfo;
    switch (b) {
      case 1: k_step<TV, TE, 1><<<gs, kRows, sz, s>>>(P, ri, ctx->offd.colmap, E, W0, W1, V); break;
      case 4: k_step<TV, TE, 4><<<gs, kRows, sz, s>>>(P, ri, ctx->offd.colmap, E, W0, W1, V); break;
      case 16: k_step<TV, TE, 16><<<gs, kRows, sz, s>>>(P, ri, ctx->offd.colmap, E, W0, W1, V); break;
      default: k_step<TV, TE, 8><<<gs, kRows, sz, s>>>(P, ri, ctx->offd.colmap, E, W0, W1, V); break;
    }
  };
  for (int b : {1, 4, 8, 16})
    if (ssm_of(b) > 48 * 1024 && ssm_of(b) <= 200 * 1024)
      SWM_CK(allow_max_dyn_smem(step_fn(b), ctx->smem_optin));
  if (sm > 48 * 1024) {
    SWM_CK(allow_max_dyn_smem((const void*)k_update<TV>, ctx->smem_optin));
    SWM_CK(allow_max_dyn_smem((const void*)k_dots_big<TV>, ctx->smem_optin));
    SWM_CK(allow_max_dyn_smem((const void*)k_finish<TV>, ctx->smem_optin));
  }
  // back substitution stages the triangle in shared memory when it fits
  size_t bs_smem = sizeof(c128) * (size_t)restart * restart;
  if (bs_smem > 160 * 1024) bs_smem = 0;
  if (bs_smem > 0)
    SWM_CK(allow_max_dyn_smem((const void*)k_backsolve, ctx->smem_optin));
  bool first = !given_b;
  SWM_TRY(ensure_poll_slots(ctx));
  static_assert(2 * sizeof(KState) <= kPollSlotBytes, "poll slots");
  KState* slot = reinterpret_cast<KState*>(ctx->pinned_state);
  constexpr int kChunkSteps = 4;
  auto launch_steps = [&](cudaStream_t s, int n) -> int {
    for (int i = 0; i < n; ++i) {
      ctx->prof_begin(SWM_K_APPLY);
      if (split) {
        const dim3 gsp((unsigned)ceil_div(N * kG, kRows), multi ? (unsigned)ceil_div(R, kRB) : 1u);
        if (ws->Xt) {
          const RowInfo* ri = (const RowInfo*)ctx->rowinfo;
          k_rhs_minor<TV><<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, W0, W1, ws->Xt);
          SWM_LAUNCHED();
          const unsigned gx = (unsigned)ceil_div(N, kTileRows);
          if (R >= 24)
            k_spmv_t<TV, TE, 32><<<dim3(gx, (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, ri, ctx->offd.colmap, E,
                                                                                   ws->Xt, W0, W1, V);
          else
            k_spmv_t<TV, TE, 16><<<dim3(gx, (unsigned)ceil_div(R, 16)), 256, 0, s>>>(P, ri, ctx->offd.colmap, E,
                                                                                   ws->Xt, W0, W1, V);
        } else if (multi)
          k_spmv<TV, TE, kRB><<<gsp, kRows, 0, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        else
          k_spmv<TV, TE, 1><<<gsp, kRows, 0, s>>>(P, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, E, W0, W1, V);
        ctx->prof_end(SWM_K_APPLY);
        SWM_LAUNCHED();
        ctx->prof_begin(SWM_K_DOTS);
        k_dots_big<TV><<<g_chunk, kRows, sm, s>>>(P, W0, W1, V);
        ctx->prof_end(SWM_K_DOTS);
      } else {
        launch_step(s, rb);
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
  if (!persisted && multi && !split) {
    const int64_t shape[6] = {N, R, (int64_t)sizeof(TV), (int64_t)sizeof(TE), P.schunk, restart};
    int found = 0;
    for (const auto& t : ctx->tuned)
      if (std::memcmp(t.shape, shape, sizeof(shape)) == 0) found = t.rb;
    if (found) {
      rb = found;
    } else {
      // first cycle's residual and start (the loop below repeats them; both are idempotent), then
      // each candidate step once untimed and once timed; the step is idempotent at a fixed j
      k_apply<TV, TE><<<g_rows, kRows, 0, st>>>(1, P, ctx->rowwire, ctx->off, ctx->offd, E, Bv, Y, W0, W1, V);
      SWM_LAUNCHED();
      k_cycle_start<TV><<<g_chunk, kRows, 0, st>>>(P, W0, first ? 1 : 0);
      SWM_LAUNCHED();
      cudaEvent_t e0, e1;
      SWM_CK(cudaEventCreate(&e0));
      SWM_CK(cudaEventCreate(&e1));
      float best = 0.f;
      for (int b : {4, 8, 16}) {
        if (ssm_of(b) > 200 * 1024) continue;
        if (b == 16 && ceil_div(R, 16) == ceil_div(R, 8)) continue;  // no fewer reads of E than with 8
        launch_step(st, b);
        SWM_CK(cudaEventRecord(e0, st));
        launch_step(st, b);
        SWM_CK(cudaEventRecord(e1, st));
        ctx->launches += 2;
        SWM_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        SWM_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best == 0.f || ms < best) {
          best = ms;
          rb = b;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      SWM_CK(cudaGetLastError());
      swm_ctx::Tuned t{};
      std::memcpy(t.shape, shape, sizeof(shape));
      t.rb = rb;
      ctx->tuned.push_back(t);
    }
  }
  ctx->stats.step_rhs_block = rb;
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
    key.bits = (unsigned)(sizeof(TV) * 64 + sizeof(TE) + 4096 * rb);
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
    k_apply<TV, TE><<<g_rows, kRows, 0, st>>>(1, P, ctx->rowwire, ctx->off, ctx->offd, E, Bv, Y, W0, W1, V);
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
        ctx->launches += (split ? (ws->Xt ? 5 : 4) : 3) * kChunkSteps;
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
  if (hs_out) *hs_out = hs;
  if (y_out) {  // inner solve of the refinement: the result stays in y-space
    *y_out = Y;
    dfree_group(ctx, tmp);
    if (hs.numeric) return ctx->fail(SWM_ECUDA, "GMRES produced a non-finite value");
    return hs.all_conv ? SWM_OK : SWM_ENOTCONV;
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

template <typename TV>
__global__ void k_init_y(int64_t n, const c128* __restrict__ g, cplx<TV>* __restrict__ Y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) Y[i] = ccast<TV>(g[i]);
}

// |b_r| per right-hand side (one CTA each, float64), 1 for a zero right-hand side.
template <typename TV>
__global__ void __launch_bounds__(256) k_bnorm(int64_t N, const cplx<TV>* __restrict__ B, double* __restrict__ out) {
  const int r = blockIdx.x;
  double s = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += 256) {
    const cplx<TV> v = B[(int64_t)r * N + n];
    s += (double)v.re * v.re + (double)v.im * v.im;
  }
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    out[r] = t > 0.0 ? sqrt(t) : 1.0;
  }
}

int norms_of_b(swm_ctx* ctx, const void* B, bool f64, double* bnorm_dev) {
  if (f64)
    k_bnorm<double><<<(unsigned)ctx->n_rhs, 256, 0, ctx->stream>>>(ctx->N, (const c128*)B, bnorm_dev);
  else
    k_bnorm<float><<<(unsigned)ctx->n_rhs, 256, 0, ctx->stream>>>(ctx->N, (const c64*)B, bnorm_dev);
  SWM_LAUNCHED();
  return SWM_OK;
}

int init_y(swm_ctx* ctx, void* Y, bool f64) {
  const int64_t n = (int64_t)ctx->n_rhs * ctx->N;
  if (!ctx->guess) {
    SWM_CK(cudaMemsetAsync(Y, 0, (f64 ? sizeof(c128) : sizeof(c64)) * n, ctx->stream));
    return SWM_OK;
  }
  if (f64)
    k_init_y<double><<<(unsigned)ceil_div(n, 256), 256, 0, ctx->stream>>>(n, (const c128*)ctx->guess, (c128*)Y);
  else
    k_init_y<float><<<(unsigned)ceil_div(n, 256), 256, 0, ctx->stream>>>(n, (const c128*)ctx->guess, (c64*)Y);
  SWM_LAUNCHED();
  return SWM_OK;
}

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
  if (ctx->prec == SWM_C128)
    return gmres_impl<double, c128>(ctx, (const c128*)ctx->Zp, tol, restart, max_iter, nullptr, nullptr);
  return gmres_impl<float, c64>(ctx, (const c64*)ctx->Zp, tol, restart, max_iter, nullptr, nullptr);
}

int gmres_inner_bf16(swm_ctx* ctx, double tol, int restart, int max_iter, void** y_out, int* iters) {
  KState hs{};
  const int rc = gmres_impl<float, __nv_bfloat162>(ctx, (const __nv_bfloat162*)ctx->E16, tol, restart, max_iter,
                                                   y_out, &hs);
  *iters = hs.iters;
  return rc;
}

}  // namespace swm
