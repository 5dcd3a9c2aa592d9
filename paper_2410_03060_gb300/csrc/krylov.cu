// Restarted GMRES on the block-Jacobi right-preconditioned S-NFC system (Sec. II-B, after
// Eq. neardef: iterative solve with block-diagonal preconditioning; the cost per iteration is
// the block-sparse product, O(b_mean N_dof)).
//
// The operator is A = Z M^-1 = I + E (E stored, see precond.cu); GMRES finds y with A y = b and
// the currents are x = M^-1 y.  Several right-hand sides (incidences) run as independent GMRES
// instances that share every pass over E.  The basis is orthogonalised by classical Gram-Schmidt
// with one reorthogonalisation, the reorthogonalisation delayed by one step so that a step reads
// the basis twice instead of four times: with Q = q_0..q_{j-1} final and u_j the pending vector
// (one Gram-Schmidt pass done, not yet normalised), step j is
//   product  : w = A u_j
//   k_dots   : s = Q^H u_j, t = Q^H w, |u_j|^2, u_j^H w; the last CTA completes Hessenberg column
//              j-1 (subdiagonal rho = |u_j - Q s|), its Givens rotation and residual estimate, and
//              the first-pass coefficients of column j from these inner products
//   k_update : q_j = (u_j - Q s) / rho, u_{j+1} = (w - Q t) / rho - (q_j^H w / rho) q_j
// and a closing dots pass without product completes the last column of the cycle.  Reductions end
// in the last CTA to arrive (no spin-waits).  Every kernel reads the step index and the activity
// flags from device memory, so the host issues identical launches every step; it keeps one chunk
// of steps queued ahead of the convergence flag it is reading, so the GPU does not wait for the
// host inside a restart cycle.  Vectors are stored right-hand-side major: V[j][r][n].  Dot
// products, norms, the Hessenberg matrix and the rotations are float64.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "ctx.h"
#include "krylov_common.cuh"

namespace swm {

namespace {

constexpr int kRows = 256;  // CTA width of the vector kernels
constexpr int kMinorR = 12;  // right-hand sides from which the large-system product reads them
                             // right-hand-side minor (one lane each)
constexpr int kG = 8;       // lanes per scalar row in the block-sparse product
constexpr int kMaxChunk = 2048;  // rows per CTA of the Gram-Schmidt kernels, at most

template <typename T>
__device__ __forceinline__ bool finite_c(cplx<T> z) {
  return isfinite((double)z.re) && isfinite((double)z.im);
}

// Last CTA of right-hand side r to arrive at the end of a pass.
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

// Product w = u + E u for the active right-hand sides, streaming: one scalar row per group of eight
// lanes, RB right-hand sides sharing every read of E, no shared memory and no barrier, so many
// rows' loads are in flight.
// With RES (the residual at the start of a cycle) every right-hand side takes part, the source
// is Y and the result W = B - (y + E y).
template <typename TV, typename TE, int RB, bool RES = false>
__global__ void __launch_bounds__(kRows) k_spmv(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const TE* __restrict__ E,
                                                const cplx<TV>* __restrict__ U, cplx<TV>* __restrict__ Wv,
                                                const cplx<TV>* __restrict__ B = nullptr) {
  if (!RES && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  const int r0 = blockIdx.y * RB;
  const int nr = min(RB, P.R - r0);
  const int64_t N = P.N;
  const int64_t n = (blockIdx.x * (int64_t)kRows + threadIdx.x) / kG;
  const int sub = threadIdx.x % kG;
  bool act[RB];
  bool any = false;
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    act[b] = b < nr && (RES || P.active[r0 + b]);
    any |= act[b];
  }
  if (!any) return;  // the same for the whole CTA
  cplx<TV> acc[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
  if (n < N) {
    const RowInfo ri = rinfo[n];
    const int32_t* cm = colmap + ri.cmb;
    int c = sub;
    for (; c + kG < ri.K; c += 2 * kG) {
      const cplx<TV> e0 = ELoad<TV, TE>::ld(E + ri.vb + c), e1 = ELoad<TV, TE>::ld(E + ri.vb + c + kG);
      const int64_t c0 = cm[c], c1 = cm[c + kG];
#pragma unroll
      for (int b = 0; b < RB; ++b)
        if (act[b]) {
          const cplx<TV>* x = U + (int64_t)(r0 + b) * N;
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
        if (act[b]) cfma(acc[b], e0, U[(int64_t)(r0 + b) * N + c0]);
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
      const int64_t o = (int64_t)(r0 + b) * N + n;
      if (act[b]) Wv[o] = RES ? B[o] - (U[o] + acc[b]) : U[o] + acc[b];
    }
  }
}

// Product with many right-hand sides, part 0: the pending vectors U (right-hand-side major,
// [R][N]) copied to right-hand-side minor order Xt[N][R] through shared-memory tiles of 32 rows x
// 32 right-hand sides, so that the product below reads the values of all right-hand sides at a
// column as one contiguous run.
// The same copy for all right-hand sides at once, T rows per CTA: each warp loads whole runs of T
// consecutive entries of one right-hand side, and the CTA's output Xt[n0 .. n0 + T)[0 .. xst) is one
// contiguous block written in order (the padding column of an odd R is written as zero).
template <typename TV, bool RES = false>
__global__ void __launch_bounds__(256) k_rhs_minor_all(KPtr P, const cplx<TV>* __restrict__ U,
                                                       cplx<TV>* __restrict__ Xt, int xst, int T) {
  if (!RES && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  extern __shared__ __align__(16) unsigned char sm_tr[];
  cplx<TV>* tile = reinterpret_cast<cplx<TV>*>(sm_tr);  // [T][xst + 1]
  const int ts = xst + 1;
  const int64_t n0 = (int64_t)blockIdx.x * T;
  const int cnt = (int)min((int64_t)T, P.N - n0);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nwp = blockDim.x >> 5;
  for (int r = wp; r < P.R; r += nwp) {
    const cplx<TV>* u = U + (int64_t)r * P.N + n0;
    for (int t = lane; t < cnt; t += 32) tile[t * ts + r] = u[t];
  }
  __syncthreads();
  cplx<TV>* out = Xt + n0 * xst;
  for (int t = wp; t < cnt; t += nwp)
    for (int r = lane; r < xst; r += 32) out[(int64_t)t * xst + r] = r < P.R ? tile[t * ts + r] : mkc<TV>(0, 0);
}

template <typename TV, bool RES = false>
__global__ void __launch_bounds__(256) k_rhs_minor(KPtr P, const cplx<TV>* __restrict__ U, cplx<TV>* __restrict__ Xt,
                                                   int xst = 0) {
  if (!RES && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  __shared__ cplx<TV> tile[32][33];
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
  for (int k = ty; k < 32; k += 8) {
    const int r = r0 + k;
    const int64_t n = n0 + tx;
    if (r < P.R && n < P.N) tile[k][tx] = U[(int64_t)r * P.N + n];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t n = n0 + k;
    const int r = r0 + tx;
    if (r < P.R && n < P.N) Xt[n * (xst > 0 ? xst : P.R) + r] = tile[tx][k];
  }
}

// Product with many right-hand sides, part 1: w = u + E u with one lane per right-hand side: the RB
// lanes of a row group read each entry of E once (the same address: one transaction) and the RB
// values of the gathered column as one contiguous run of Xt.  A CTA covers 32 rows; its results go
// through shared memory so that w is written right-hand-side major as runs of 32 consecutive rows.
constexpr int kTileRows = 32;
template <typename TV, typename TE, int RB, bool RES = false>
__global__ void __launch_bounds__(256) k_spmv_t(KPtr P, const RowInfo* __restrict__ rinfo,
                                                const int32_t* __restrict__ colmap, const TE* __restrict__ E,
                                                const cplx<TV>* __restrict__ Xt, cplx<TV>* __restrict__ Wv,
                                                const cplx<TV>* __restrict__ B = nullptr) {
  if (!RES && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  __shared__ cplx<TV> ys[kTileRows][RB + 1];
  const int64_t N = P.N;
  const int R = P.R;
  const int64_t n0 = (int64_t)blockIdx.x * kTileRows;
  const int lr = (int)(threadIdx.x % RB);  // right-hand side within the block
  const int r = blockIdx.y * RB + lr;
  const bool on = r < R && (RES || P.active[r]);
  constexpr int kGroups = 256 / RB;  // rows per pass
  for (int t = (int)(threadIdx.x / RB); t < kTileRows; t += kGroups) {
    const int64_t n = n0 + t;
    cplx<TV> y = mkc<TV>(0, 0);
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
      y = Xt[n * R + r] + acc;
    }
    ys[t][lr] = y;
  }
  __syncthreads();
  // write: warp w takes right-hand sides w, w + 8, ...; its lanes take the 32 rows
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = n0 + lane;
  for (int b = w; b < RB; b += 8) {
    const int rr = blockIdx.y * RB + b;
    if (rr >= R || n >= N || (!RES && !P.active[rr])) continue;
    const int64_t o = (int64_t)rr * N + n;
    Wv[o] = RES ? B[o] - ys[lane][b] : ys[lane][b];
  }
}

// Product with many right-hand sides, wire-tiled: w = u + E u.  A CTA takes WB consecutive wires
// (block-rows of E) and RG right-hand sides, one thread per (wire, right-hand side): it
// accumulates all m_p rows of its wire over the wire's K_p columns, so each gathered value of u
// serves every row of the wire from a register, and writes its rows itself (a short run per
// thread; no shared memory and no barrier, so nothing waits for the slowest wire of the CTA).  The
// gathers read Xt, u right-hand-side minor ([N][R], XT), where the threads of a wire (consecutive
// right-hand sides) read consecutive addresses, or, without XT, u itself (right-hand-side major).
// The column map is loaded one group of four ahead of its gathers.  The entries of E are the same
// address for every thread of a wire (one transaction per warp).  Rows are taken eight at a time
// (a wire has at most SWM_MAX_SEG - 1 rows).
// MODE kStepW: a GMRES step (active right-hand sides only); kResW: the residual at the start of a
// cycle, every right-hand side, source Y, result W = B - (y + E y); kPlainW: every right-hand side,
// W = u + E u (the product on its own, for callers outside GMRES).
constexpr int kStepW = 0, kResW = 1, kPlainW = 2;
template <typename TV, typename TE, int MODE = kStepW, bool XT = false, int MINB = sizeof(TV) == 4 ? 4 : 2>
__global__ void __launch_bounds__(256, MINB) k_spmv_w(KPtr P, const int64_t* __restrict__ off, Layout lay, int64_t nw,
                                                   const TE* __restrict__ E, const cplx<TV>* __restrict__ U,
                                                   const cplx<TV>* __restrict__ Xt, cplx<TV>* __restrict__ Wv,
                                                   const cplx<TV>* __restrict__ B, int RG, int WB) {
  constexpr bool RES = MODE == kResW, ALL = MODE != kStepW;
  if (!ALL && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  const int64_t N = P.N;
  const int64_t p0 = (int64_t)blockIdx.x * WB;
  const int r0 = blockIdx.y * RG;
  const int pl = (int)threadIdx.x / RG, rl = (int)threadIdx.x % RG;
  const int64_t p = p0 + pl;
  const int r = r0 + rl;
  if (pl >= WB || p >= nw || r >= P.R || !(ALL || P.active[r])) return;
  const int64_t op = off[p];
  const int m = (int)(off[p + 1] - op);
  const int K = lay.K[p];
  const TE* Ep = E + lay.rowbase[p];
  const int32_t* cm = lay.colmap + lay.cmbase[p];
  // gathered value of column c for this right-hand side
  const cplx<TV>* xs = XT ? Xt + r : U + (int64_t)r * N;
  const int64_t xstride = XT ? P.R : 1;
  const int64_t orow = (int64_t)r * N + op;
  for (int i0 = 0; i0 < m; i0 += 8) {
    const int mm = min(8, m - i0);
    const TE* Ei = Ep + (int64_t)i0 * K;
    cplx<TV> acc[8];
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) acc[ii] = mkc<TV>(0, 0);
    const int K4 = K & ~3;
    int32_t c[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) c[u] = u < K4 ? cm[u] : 0;
    for (int k = 0; k < K4; k += 4) {
      cplx<TV> x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = xs[(int64_t)c[u] * xstride];
      // the next group's columns while these gathers are in flight
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] = k + 4 + u < K4 ? cm[k + 4 + u] : 0;
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
        if (ii < mm) {
          cplx<TV> e[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) e[u] = ELoad<TV, TE>::ld(Ei + (int64_t)ii * K + k + u);
#pragma unroll
          for (int u = 0; u < 4; ++u) cfma(acc[ii], e[u], x[u]);
        }
    }
    for (int k = K4; k < K; ++k) {
      const cplx<TV> x = xs[(int64_t)cm[k] * xstride];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
        if (ii < mm) cfma(acc[ii], ELoad<TV, TE>::ld(Ei + (int64_t)ii * K + k), x);
    }
#pragma unroll
    for (int ii = 0; ii < 8; ++ii)
      if (ii < mm) {
        const int64_t o = orow + i0 + ii;
        const cplx<TV> v = U[o] + acc[ii];
        Wv[o] = RES ? B[o] - v : v;
      }
  }
}

// The product with two right-hand sides per thread and the tile's E in shared memory.  Thread
// (wire, pair q) takes right-hand sides 2q and 2q + 1 of its group: each entry of E it reads serves
// both, and their gathered values are one 16-byte load from Xt, whose rows are padded to an even
// length xst.  The CTA first copies the E rows of its wires into shared memory (coalesced, each row
// padded to an even length so that two consecutive entries are one 16-byte load), then every thread
// multiplies; tiles whose E exceeds the shared-memory budget read E from global memory instead.
constexpr int kWpSmemBytes = 40 * 1024;
template <typename TE, bool SM>
__device__ __forceinline__ void e_pair(const TE* Eg, const c64* Es, int64_t idx, c64& e0, c64& e1) {
  if constexpr (SM) {
    const float4 v = *reinterpret_cast<const float4*>(Es + idx);
    e0 = mkc<float>(v.x, v.y);
    e1 = mkc<float>(v.z, v.w);
  } else {
    e0 = ELoad<float, TE>::ld(Eg + idx);
    e1 = ELoad<float, TE>::ld(Eg + idx + 1);
  }
}
template <typename TE, int MODE, bool SM>
__device__ __forceinline__ void wp_rows(const KPtr& P, int64_t N, int m, int K, int estr, const TE* Eg, const c64* Es,
                                        const int32_t* __restrict__ cm, const c64* __restrict__ xs, int xst,
                                        const c64* __restrict__ U, c64* __restrict__ Wv, const c64* __restrict__ B,
                                        int64_t orow, bool wa, bool wb) {
  constexpr bool RES = MODE == kResW;
  for (int i0 = 0; i0 < m; i0 += 8) {
    const int mm = min(8, m - i0);
    c64 a0[8], a1[8];
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) a0[ii] = a1[ii] = mkc<float>(0, 0);
    const int K2 = K & ~1;
    for (int k = 0; k < K2; k += 2) {
      const int32_t c0 = cm[k], c1 = cm[k + 1];
      const float4 x0 = *reinterpret_cast<const float4*>(xs + (int64_t)c0 * xst);
      const float4 x1 = *reinterpret_cast<const float4*>(xs + (int64_t)c1 * xst);
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
        if (ii < mm) {
          c64 e0, e1;
          e_pair<TE, SM>(Eg, Es, (int64_t)(i0 + ii) * estr + k, e0, e1);
          cfma(a0[ii], e0, mkc<float>(x0.x, x0.y));
          cfma(a1[ii], e0, mkc<float>(x0.z, x0.w));
          cfma(a0[ii], e1, mkc<float>(x1.x, x1.y));
          cfma(a1[ii], e1, mkc<float>(x1.z, x1.w));
        }
    }
    if (K2 < K) {
      const float4 x0 = *reinterpret_cast<const float4*>(xs + (int64_t)cm[K2] * xst);
#pragma unroll
      for (int ii = 0; ii < 8; ++ii)
        if (ii < mm) {
          const c64 e0 = SM ? Es[(int64_t)(i0 + ii) * estr + K2] : ELoad<float, TE>::ld(Eg + (int64_t)(i0 + ii) * estr + K2);
          cfma(a0[ii], e0, mkc<float>(x0.x, x0.y));
          cfma(a1[ii], e0, mkc<float>(x0.z, x0.w));
        }
    }
#pragma unroll
    for (int ii = 0; ii < 8; ++ii)
      if (ii < mm) {
        if (wa) {
          const int64_t o = orow + i0 + ii;
          const c64 v = U[o] + a0[ii];
          Wv[o] = RES ? B[o] - v : v;
        }
        if (wb) {
          const int64_t o = orow + N + i0 + ii;
          const c64 v = U[o] + a1[ii];
          Wv[o] = RES ? B[o] - v : v;
        }
      }
  }
}
constexpr int kWpMaxWires = 32;  // wires per CTA of k_spmv_wp, at most
template <typename TE, int MODE = kStepW>
__global__ void __launch_bounds__(256, 3) k_spmv_wp(KPtr P, const int64_t* __restrict__ off, Layout lay, int64_t nw,
                                                    const TE* __restrict__ E, const c64* __restrict__ U,
                                                    const c64* __restrict__ Xt, int xst, c64* __restrict__ Wv,
                                                    const c64* __restrict__ B, int RQ, int WB) {
  constexpr bool ALL = MODE != kStepW;
  if (!ALL && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  extern __shared__ __align__(16) unsigned char sm_wp[];
  c64* Es = reinterpret_cast<c64*>(sm_wp);
  __shared__ int soff[kWpMaxWires + 1], sK[kWpMaxWires], sm_m[kWpMaxWires];
  __shared__ int64_t sbase[kWpMaxWires];
  __shared__ bool fits;
  const int64_t N = P.N;
  const int64_t p0 = (int64_t)blockIdx.x * WB;
  const int nwt = (int)min((int64_t)min(WB, kWpMaxWires), nw - p0);
  if (threadIdx.x < nwt) {
    const int64_t p = p0 + threadIdx.x;
    sK[threadIdx.x] = lay.K[p];
    sm_m[threadIdx.x] = (int)(off[p + 1] - off[p]);
    sbase[threadIdx.x] = lay.rowbase[p];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int o = 0;
    for (int w = 0; w < nwt; ++w) {
      soff[w] = o;
      o += sm_m[w] * (sK[w] + (sK[w] & 1));
    }
    soff[nwt] = o;
    fits = (size_t)o * sizeof(c64) <= kWpSmemBytes;
  }
  __syncthreads();
  if (fits) {
    // E rows of the tile, each padded to an even length (the pad entry is zero)
    for (int w = 0; w < nwt; ++w) {
      const int K = sK[w], K2 = K + (K & 1), cnt = sm_m[w] * K2;
      const TE* src = E + sbase[w];
      c64* dst = Es + soff[w];
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const int i = e / K2, k = e - i * K2;
        dst[e] = k < K ? ELoad<float, TE>::ld(src + (int64_t)i * K + k) : mkc<float>(0, 0);
      }
    }
    __syncthreads();
  }
  const int pl = (int)threadIdx.x / RQ, q = (int)threadIdx.x % RQ;
  if (pl >= nwt) return;
  const int ra = blockIdx.y * 2 * RQ + 2 * q, rb = ra + 1;
  if (ra >= P.R) return;
  const bool wa = ALL || P.active[ra];
  const bool wb = rb < P.R && (ALL || P.active[rb]);
  if (!wa && !wb) return;
  const int64_t p = p0 + pl;
  const int K = sK[pl], m = sm_m[pl];
  const int32_t* cm = lay.colmap + lay.cmbase[p];
  const c64* xs = Xt + ra;
  const int64_t orow = (int64_t)ra * N + off[p];
  if (fits)
    wp_rows<TE, MODE, true>(P, N, m, K, K + (K & 1), nullptr, Es + soff[pl], cm, xs, xst, U, Wv, B, orow, wa, wb);
  else
    wp_rows<TE, MODE, false>(P, N, m, K, K, E + sbase[pl], nullptr, cm, xs, xst, U, Wv, B, orow, wa, wb);
}

// The product with packed FP32x2 arithmetic.  As k_spmv_wp, thread (wire, pair q) accumulates
// right-hand sides 2q and 2q + 1 of every row of its wire, but the two right-hand sides sit in the
// two halves of each packed operation: the real parts of both in one register pair, the imaginary
// parts in another, so one complex multiply-add of an E entry into both right-hand sides is four
// FFMA2.  The CTA copies its tile's E (one contiguous range, the wires being consecutive) into
// shared memory with each entry expanded to (re, re, im, im), so one 16-byte load gives the two
// packed operands; it copies the tile's column map too.  The row loop is unrolled to the largest
// row count of the warp's wires (warp-uniform, rows beyond a wire's own are predicated off), and
// the gathered values of the next column pair are loaded while the current pair is multiplied
// (their column indices one pair earlier still).
constexpr int kWmSmemC = 4 * 1024;  // column-map entries of a tile
// E budgets (expanded entries, 16 bytes each) of the two launch shapes: three CTAs per SM with
// 48 KB (measured faster than 64 KB although more tiles of dense regions fall back to global
// memory), two with 96 KB (nearly every tile fits, fewer warps)
constexpr int kWmSmemE3 = 48 * 1024, kWmSmemE2 = 96 * 1024;
__device__ __forceinline__ void wm_xsplit(const float4 v, float2& xr, float2& xi, float2& nxi) {
  xr = make_float2(v.x, v.z);
  xi = make_float2(v.y, v.w);
  nxi = make_float2(-v.y, -v.w);
}
__device__ __forceinline__ void wm_fma(float2& ar, float2& ai, const float4 e, const float2 xr, const float2 xi,
                                       const float2 nxi) {
  const float2 er = make_float2(e.x, e.y), ei = make_float2(e.z, e.w);
  ar = __ffma2_rn(er, xr, ar);
  ar = __ffma2_rn(ei, nxi, ar);
  ai = __ffma2_rn(er, xi, ai);
  ai = __ffma2_rn(ei, xr, ai);
}
// Entries of E as the packed operands (re, re, im, im): from the expanded copy in shared memory,
// or read from global memory in the storage type and expanded in registers.
struct EStaged {
  const float4* p;
  __device__ __forceinline__ float4 operator[](int64_t i) const { return p[i]; }
};
template <typename TE>
struct EGlobal {
  const TE* p;
  __device__ __forceinline__ float4 operator[](int64_t i) const {
    const c64 v = ELoad<float, TE>::ld(p + i);
    return make_float4(v.re, v.re, v.im, v.im);
  }
};
// MINOR: the vectors are incidence-minor like the gathered copy ([N][xst]; U, Wv and B point at
// incidence ra, orow is the wire's first row) and the thread reads and writes its two incidences
// of a row as one 16-byte access; otherwise incidence-major ([R][N]; orow = ra N + first row).
template <int MODE, int MW, typename EA, bool MINOR = false>
__device__ __forceinline__ void wm_rows(int64_t N, int i0, int mm, int K, EA Es, const int32_t* __restrict__ cms,
                                        const c64* __restrict__ xs, int xst, const c64* __restrict__ U,
                                        c64* __restrict__ Wv, const c64* __restrict__ B, int64_t orow, bool wa,
                                        bool wb) {
  constexpr bool RES = MODE == kResW;
  float2 ar[MW], ai[MW];
#pragma unroll
  for (int ii = 0; ii < MW; ++ii) ar[ii] = ai[ii] = make_float2(0.f, 0.f);
  float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
  if (K > 0) {
    x0 = __ldg(reinterpret_cast<const float4*>(xs + (int64_t)cms[0] * xst));
    x1 = __ldg(reinterpret_cast<const float4*>(xs + (int64_t)cms[K > 1 ? 1 : 0] * xst));
  }
  // column indices one pair further ahead than the gathered values, so that a gather's address
  // never waits on its column-map load
  int d0 = 0, d1 = 0;
  if (K > 2) {
    d0 = cms[2];
    d1 = cms[K > 3 ? 3 : 2];
  }
  EA er = Es;
  er.p += (int64_t)i0 * K;
  for (int k = 0; k < K; k += 2) {
    float4 n0 = x0, n1 = x1;
    if (k + 2 < K) {
      n0 = __ldg(reinterpret_cast<const float4*>(xs + (int64_t)d0 * xst));
      n1 = __ldg(reinterpret_cast<const float4*>(xs + (int64_t)d1 * xst));
      if (k + 4 < K) {
        d0 = cms[k + 4];
        d1 = cms[k + 5 < K ? k + 5 : k + 4];
      }
    }
    const bool two = k + 1 < K;
    float2 xr0, xi0, nxi0, xr1, xi1, nxi1;
    wm_xsplit(x0, xr0, xi0, nxi0);
    wm_xsplit(x1, xr1, xi1, nxi1);
#pragma unroll
    for (int ii = 0; ii < MW; ++ii)
      if (ii < mm) {
        wm_fma(ar[ii], ai[ii], er[ii * K + k], xr0, xi0, nxi0);
        if (two) wm_fma(ar[ii], ai[ii], er[ii * K + k + 1], xr1, xi1, nxi1);
      }
    x0 = n0;
    x1 = n1;
  }
  if constexpr (MINOR) {
    // both incidences of a row at once (the second may be the padding column or inactive: its
    // value is written too and never read as a result)
#pragma unroll
    for (int ii = 0; ii < MW; ++ii)
      if (ii < mm) {
        const int64_t o = (orow + i0 + ii) * xst;
        const float4 u = *reinterpret_cast<const float4*>(U + o);
        float4 v = make_float4(u.x + ar[ii].x, u.y + ai[ii].x, u.z + ar[ii].y, u.w + ai[ii].y);
        if (RES) {
          const float4 b = *reinterpret_cast<const float4*>(B + o);
          v = make_float4(b.x - v.x, b.y - v.y, b.z - v.z, b.w - v.w);
        }
        *reinterpret_cast<float4*>(Wv + o) = v;
      }
  } else {
#pragma unroll
    for (int ii = 0; ii < MW; ++ii)
      if (ii < mm) {
        if (wa) {
          const int64_t o = orow + i0 + ii;
          const c64 v = U[o] + mkc<float>(ar[ii].x, ai[ii].x);
          Wv[o] = RES ? B[o] - v : v;
        }
        if (wb) {
          const int64_t o = orow + N + i0 + ii;
          const c64 v = U[o] + mkc<float>(ar[ii].y, ai[ii].y);
          Wv[o] = RES ? B[o] - v : v;
        }
      }
  }
}
template <typename TE, int MODE = kStepW, int MINB = 3, int EB = kWmSmemE3, bool MINOR = false>
__global__ void __launch_bounds__(256, MINB) k_spmv_wm(KPtr P, const int64_t* __restrict__ off, Layout lay, int64_t nw,
                                                    const TE* __restrict__ E, const c64* __restrict__ U,
                                                    const c64* __restrict__ Xt, int xst, c64* __restrict__ Wv,
                                                    const c64* __restrict__ B, int RQ, int WB) {
  constexpr bool ALL = MODE != kStepW;
  if (!ALL && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  extern __shared__ __align__(16) unsigned char sm_wm[];
  float4* Es = reinterpret_cast<float4*>(sm_wm);
  int32_t* Cs = reinterpret_cast<int32_t*>(sm_wm + EB);
  __shared__ int sK[kWpMaxWires], sm_m[kWpMaxWires], seo[kWpMaxWires], sco[kWpMaxWires];
  const int64_t N = P.N;
  const int64_t p0 = (int64_t)blockIdx.x * WB;
  const int nwt = (int)min((int64_t)min(WB, kWpMaxWires), nw - p0);
  // the tile's E entries and column-map entries are contiguous ranges
  const int64_t e0 = lay.rowbase[p0], c0 = lay.cmbase[p0];
  const int64_t ne = lay.rowbase[p0 + nwt] - e0, nc = lay.cmbase[p0 + nwt] - c0;
  const bool fits = ne * (int64_t)sizeof(float4) <= EB && nc * (int64_t)sizeof(int32_t) <= kWmSmemC;
  if (threadIdx.x < nwt) {
    const int64_t p = p0 + threadIdx.x;
    sK[threadIdx.x] = lay.K[p];
    sm_m[threadIdx.x] = (int)(off[p + 1] - off[p]);
    seo[threadIdx.x] = (int)(lay.rowbase[p] - e0);
    sco[threadIdx.x] = (int)(lay.cmbase[p] - c0);
  }
  if (fits) {
    const int ne4 = (int)ne, nc4 = (int)nc;
#pragma unroll 4
    for (int e = threadIdx.x; e < ne4; e += blockDim.x) {
      const c64 v = ELoad<float, TE>::ld(E + e0 + e);
      Es[e] = make_float4(v.re, v.re, v.im, v.im);
    }
    for (int c = threadIdx.x; c < nc4; c += blockDim.x) Cs[c] = lay.colmap[c0 + c];
  }
  __syncthreads();
  const int pl = (int)threadIdx.x / RQ, q = (int)threadIdx.x % RQ;
  const int ra = blockIdx.y * 2 * RQ + 2 * q, rb = ra + 1;
  const bool valid = pl < nwt && ra < P.R;
  // warp-uniform row bound: the largest row count among the warp's wires
  const int mw = __reduce_max_sync(0xffffffffu, valid ? sm_m[pl] : 0);
  if (!valid) return;
  const bool wa = ALL || P.active[ra];
  const bool wb = rb < P.R && (ALL || P.active[rb]);
  if (!wa && !wb) return;
  const int64_t p = p0 + pl;
  const int K = sK[pl], m = sm_m[pl];
  const c64* xs = Xt + ra;
  const int64_t orow = MINOR ? off[p] : (int64_t)ra * N + off[p];
  if constexpr (MINOR) {
    U += ra;
    Wv += ra;
    if (B) B += ra;
  }
  if (!fits) {
    // the tile's E or column map exceed the budgets: read them from global memory
    const EGlobal<TE> eg{E + lay.rowbase[p]};
    const int32_t* cmg = lay.colmap + lay.cmbase[p];
    for (int i0 = 0; i0 < m; i0 += 8)
      wm_rows<MODE, 8, EGlobal<TE>, MINOR>(N, i0, min(8, m - i0), K, eg, cmg, xs, xst, U, Wv, B, orow, wa, wb);
    return;
  }
  const EStaged er{Es + seo[pl]};
  const int32_t* cms = Cs + sco[pl];
  switch (mw) {
    case 1: wm_rows<MODE, 1, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 2: wm_rows<MODE, 2, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 3: wm_rows<MODE, 3, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 4: wm_rows<MODE, 4, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 5: wm_rows<MODE, 5, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 6: wm_rows<MODE, 6, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 7: wm_rows<MODE, 7, EStaged, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    default:
      for (int i0 = 0; i0 < m; i0 += 8)
        wm_rows<MODE, 8, EStaged, MINOR>(N, i0, min(8, m - i0), K, er, cms, xs, xst, U, Wv, B, orow, wa, wb);
      break;
  }
}

// The packed product without shared memory: each thread reads its wire's E (broadcast in L1 to
// the wire's other threads) and column map from global memory, no staging and no barrier.
template <typename TE, int MODE = kStepW, int MINB = 3, bool MINOR = false>
__global__ void __launch_bounds__(256, MINB) k_spmv_wg(KPtr P, const int64_t* __restrict__ off, Layout lay, int64_t nw,
                                                    const TE* __restrict__ E, const c64* __restrict__ U,
                                                    const c64* __restrict__ Xt, int xst, c64* __restrict__ Wv,
                                                    const c64* __restrict__ B, int RQ, int WB) {
  constexpr bool ALL = MODE != kStepW;
  if (!ALL && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  const int64_t N = P.N;
  const int64_t p0 = (int64_t)blockIdx.x * WB;
  const int pl = (int)threadIdx.x / RQ, q = (int)threadIdx.x % RQ;
  const int64_t p = p0 + pl;
  const int ra = blockIdx.y * 2 * RQ + 2 * q, rb = ra + 1;
  const bool valid = pl < WB && p < nw && ra < P.R;
  const int64_t op = valid ? off[p] : 0;
  const int m = valid ? (int)(off[p + 1] - op) : 0;
  // warp-uniform row bound: the largest row count among the warp's wires
  const int mw = __reduce_max_sync(0xffffffffu, m);
  if (!valid) return;
  const bool wa = ALL || P.active[ra];
  const bool wb = rb < P.R && (ALL || P.active[rb]);
  if (!wa && !wb) return;
  const int K = lay.K[p];
  const EGlobal<TE> er{E + lay.rowbase[p]};
  const int32_t* cms = lay.colmap + lay.cmbase[p];
  const c64* xs = Xt + ra;
  const int64_t orow = MINOR ? op : (int64_t)ra * N + op;
  if constexpr (MINOR) {
    U += ra;
    Wv += ra;
    if (B) B += ra;
  }
  switch (mw) {
    case 1: wm_rows<MODE, 1, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 2: wm_rows<MODE, 2, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 3: wm_rows<MODE, 3, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 4: wm_rows<MODE, 4, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 5: wm_rows<MODE, 5, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 6: wm_rows<MODE, 6, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 7: wm_rows<MODE, 7, EGlobal<TE>, MINOR>(N, 0, m, K, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    default:
      for (int i0 = 0; i0 < m; i0 += 8)
        wm_rows<MODE, 8, EGlobal<TE>, MINOR>(N, i0, min(8, m - i0), K, er, cms, xs, xst, U, Wv, B, orow, wa, wb);
      break;
  }
}

// The packed product in small CTAs with each wire's E rows and column map staged in shared memory
// as stored (not expanded) by cp.async: every thread issues 16-byte copies of the 16-byte-aligned
// spans around the tile's ranges (a partial last chunk reads only its own bytes and zero-fills the
// rest), so the whole tile is in flight at once and the row loop reads E and the column map at
// shared-memory latency.  A tile whose spans exceed the budgets reads them from global memory.
// E and the column map must start on 16-byte boundaries (the launch checks), so that no span
// reaches before either buffer.  With records (rec, nullable) the CTA takes the wires of
// rec[p0 + i], in the order the records were written, instead of wires p0 + i; every warp reads
// the CTA's few records itself and issues its share of the copies, so the only barrier is the one
// after the copies.
// The E budget, 22 KB, holds all but about 0.5 % of the work's tiles at three CTAs' register
// budget (eight CTAs per SM, as many as its registers allow).
constexpr int kWaSmemE3 = 22 * 1024, kWaSmemC = 4 * 1024;
constexpr int kWaMaxWires = 8;  // wires per small CTA, at most
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gsrc), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
// A wire of the small-CTA product as its prologue needs it: its index, first E entry and first
// column-map entry, K and rows (the order build writes one per position, in the product's order).
struct WaRec {
  int64_t ebeg, cbeg;
  int32_t p, K, m, pad;
};
template <typename TE, int MODE = kStepW, int MINB = 3, bool MINOR = false, int EB = kWaSmemE3>
__global__ void __launch_bounds__(256, MINB) k_spmv_wa(KPtr P, const int64_t* __restrict__ off, Layout lay, int64_t nw,
                                                    const TE* __restrict__ E, const c64* __restrict__ U,
                                                    const c64* __restrict__ Xt, int xst, c64* __restrict__ Wv,
                                                    const c64* __restrict__ B, int RQ, int WB,
                                                    const WaRec* __restrict__ rec) {
  constexpr bool ALL = MODE != kStepW;
  if (!ALL && (P.st->cycle_done || P.st->j >= P.st->jmax)) return;
  extern __shared__ __align__(16) unsigned char sm_wa[];
  // per wire (written by warp 0, read after the barrier): its index, K, rows, and the offsets of
  // its E rows and column map in shared memory
  __shared__ int64_t sp[kWaMaxWires];
  __shared__ int sK[kWaMaxWires], sm_m[kWaMaxWires], sE[kWaMaxWires], sC[kWaMaxWires];
  const int64_t N = P.N;
  const int64_t p0 = (int64_t)blockIdx.x * WB;
  const int nwt = (int)min((int64_t)min(WB, kWaMaxWires), nw - p0);
  // every warp: lane i < nwt takes wire i (its record, or the layout in the cell order), the spans
  // and their offsets in shared memory (inclusive scans of the 16-byte-rounded sizes), so that each
  // warp issues its share of the copies without waiting for another
  const int lane = threadIdx.x & 31;
  int64_t p = 0, eoff = 0, coff = 0;
  int K = 0, m = 0, en = 0, cn = 0, he = 0, hc = 0;
  const unsigned char *ea = nullptr, *ca = nullptr;
  if (lane < nwt) {
    if (rec) {
      const WaRec r = rec[p0 + lane];
      p = r.p;
      eoff = r.ebeg;
      coff = r.cbeg;
      K = r.K;
      m = r.m;
    } else {
      p = p0 + lane;
      eoff = lay.rowbase[p];
      coff = lay.cmbase[p];
      K = lay.K[p];
      m = (int)(off[p + 1] - off[p]);
    }
    const unsigned char* eb = reinterpret_cast<const unsigned char*>(E + eoff);
    const unsigned char* cb = reinterpret_cast<const unsigned char*>(lay.colmap + coff);
    ea = reinterpret_cast<const unsigned char*>(reinterpret_cast<uintptr_t>(eb) & ~(uintptr_t)15);
    ca = reinterpret_cast<const unsigned char*>(reinterpret_cast<uintptr_t>(cb) & ~(uintptr_t)15);
    en = (int)(reinterpret_cast<const unsigned char*>(E + eoff + (int64_t)m * K) - ea);
    cn = (int)(reinterpret_cast<const unsigned char*>(lay.colmap + coff + K) - ca);
    he = (int)(eb - ea);
    hc = (int)(cb - ca);
  }
  int oe = (en + 15) & ~15, oc = (cn + 15) & ~15;
#pragma unroll
  for (int o = 1; o < kWaMaxWires; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, oe, o), b = __shfl_up_sync(0xffffffffu, oc, o);
    if (lane >= o) {
      oe += a;
      oc += b;
    }
  }
  const int soe = oe - ((en + 15) & ~15), soc = EB + oc - ((cn + 15) & ~15);
  const bool fits = __shfl_sync(0xffffffffu, oe, kWaMaxWires - 1) <= EB &&
                    __shfl_sync(0xffffffffu, oc, kWaMaxWires - 1) <= kWaSmemC;
  if (threadIdx.x < 32 && lane < nwt) {
    sp[lane] = p;
    sK[lane] = K;
    sm_m[lane] = m;
    sE[lane] = fits ? soe + he : 0;
    sC[lane] = fits ? soc + hc : 0;
  }
  if (fits) {
    for (int w = 0; w < nwt; ++w) {
      const int ne = __shfl_sync(0xffffffffu, en, w), nc = __shfl_sync(0xffffffffu, cn, w);
      const int de = __shfl_sync(0xffffffffu, soe, w), dc = __shfl_sync(0xffffffffu, soc, w);
      const unsigned char* a = reinterpret_cast<const unsigned char*>(
          __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(ea), w));
      const unsigned char* c = reinterpret_cast<const unsigned char*>(
          __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(ca), w));
      for (int x = 16 * (int)threadIdx.x; x < ne; x += 16 * (int)blockDim.x) cp_async16(sm_wa + de + x, a + x, min(16, ne - x));
      for (int x = 16 * (int)threadIdx.x; x < nc; x += 16 * (int)blockDim.x) cp_async16(sm_wa + dc + x, c + x, min(16, nc - x));
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const int pl = (int)threadIdx.x / RQ, q = (int)threadIdx.x % RQ;
  const int ra = blockIdx.y * 2 * RQ + 2 * q, rb = ra + 1;
  const bool valid = pl < nwt && ra < P.R;
  const int mw = __reduce_max_sync(0xffffffffu, valid ? sm_m[pl] : 0);
  if (!valid) return;
  const bool wa = ALL || P.active[ra];
  const bool wb = rb < P.R && (ALL || P.active[rb]);
  if (!wa && !wb) return;
  const int64_t pw = sp[pl];
  const int Kw = sK[pl], mwr = sm_m[pl];
  // E and the column map of the wire: in shared memory, else in global memory
  const TE* ep = fits ? reinterpret_cast<const TE*>(sm_wa + sE[pl]) : E + lay.rowbase[pw];
  const int32_t* cms = fits ? reinterpret_cast<const int32_t*>(sm_wa + sC[pl]) : lay.colmap + lay.cmbase[pw];
  const EGlobal<TE> er{ep};
  const c64* xs = Xt + ra;
  const int64_t orow = MINOR ? off[pw] : (int64_t)ra * N + off[pw];
  if constexpr (MINOR) {
    U += ra;
    Wv += ra;
    if (B) B += ra;
  }
  switch (mw) {
    case 1: wm_rows<MODE, 1, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 2: wm_rows<MODE, 2, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 3: wm_rows<MODE, 3, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 4: wm_rows<MODE, 4, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 5: wm_rows<MODE, 5, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 6: wm_rows<MODE, 6, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    case 7: wm_rows<MODE, 7, EGlobal<TE>, MINOR>(N, 0, mwr, Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb); break;
    default:
      for (int i0 = 0; i0 < mwr; i0 += 8)
        wm_rows<MODE, 8, EGlobal<TE>, MINOR>(N, i0, min(8, mwr - i0), Kw, er, cms, xs, xst, U, Wv, B, orow, wa, wb);
      break;
  }
}

// Wire order of the small-CTA product: within each window of kOrderWin consecutive wires (wires
// near one another in space), the wires sorted by (column pairs, rows), so that the two or three
// wires sharing a warp run row loops of about the same length.  One CTA per window, a bitonic
// sort of (key, position) in shared memory; positions past the last wire sort last.
constexpr int kOrderWin = 4096;
__global__ void __launch_bounds__(1024) k_wire_order(int64_t nw, Layout lay, const int64_t* __restrict__ off,
                                                     WaRec* __restrict__ rec) {
  const int32_t* __restrict__ K = lay.K;
  __shared__ unsigned long long key[kOrderWin];
  const int64_t base = (int64_t)blockIdx.x * kOrderWin;
  for (int t = threadIdx.x; t < kOrderWin; t += blockDim.x) {
    const int64_t p = base + t;
    unsigned hi = 0xffffffffu;
    if (p < nw) {
      const unsigned kp = (unsigned)min((K[p] + 1) / 2, 32767);
      const unsigned mp = (unsigned)min((int64_t)65535, off[p + 1] - off[p]);
      hi = (kp << 16) | mp;
    }
    key[t] = ((unsigned long long)hi << 32) | (unsigned)t;
  }
  __syncthreads();
  for (int k = 2; k <= kOrderWin; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < kOrderWin; t += blockDim.x) {
        const int o = t ^ j;
        if (o > t) {
          const unsigned long long a = key[t], b = key[o];
          if ((a > b) == ((t & k) == 0)) {
            key[t] = b;
            key[o] = a;
          }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < kOrderWin; t += blockDim.x) {
    const int64_t i = base + t;
    if (i < nw) {
      const int64_t p = base + (int64_t)(key[t] & 0xffffffffu);
      WaRec r;
      r.ebeg = lay.rowbase[p];
      r.cbeg = lay.cmbase[p];
      r.p = (int32_t)p;
      r.K = K[p];
      r.m = (int32_t)(off[p + 1] - off[p]);
      r.pad = 0;
      rec[i] = r;
    }
  }
}
}  // namespace
int build_wire_order(swm_ctx* ctx) {
  if (ctx->wrec || ctx->nw <= 0 || ctx->nw > INT32_MAX) return SWM_OK;  // built for this pattern
  SWM_TRY(dalloc(ctx, ctx->pattern_bufs, &ctx->wrec, sizeof(WaRec) * ctx->nw));
  k_wire_order<<<(unsigned)ceil_div(ctx->nw, kOrderWin), 1024, 0, ctx->stream>>>(
      ctx->nw, ctx->offd, ctx->off, reinterpret_cast<WaRec*>(ctx->wrec));
  SWM_LAUNCHED();
  return SWM_OK;
}
namespace {

// Launch of k_spmv_wm in one of its two shapes (three CTAs per SM with the 64 KB E budget, or two
// with 96 KB), and the shared-memory opt-in of its instances.
template <typename TE, bool RS, bool MINOR = false>
int launch_wm(cudaStream_t s, int form, const KPtr& P, swm_ctx* ctx, const TE* E, const c64* src, const c64* Xt,
              int xst, c64* dst, const c64* Bv, int RQ, int WBp) {
  const dim3 g((unsigned)ceil_div(ctx->nw, WBp), (unsigned)ceil_div(P.R, 2 * RQ));
  constexpr int MODE = RS ? kResW : kStepW;
  switch (form) {
    case 68:
      k_spmv_wm<TE, MODE, 3, kWmSmemE3, MINOR><<<g, 256, kWmSmemE3 + kWmSmemC, s>>>(
          P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ, WBp);
      break;
    case 69:
      k_spmv_wm<TE, MODE, 2, kWmSmemE2, MINOR><<<g, 256, kWmSmemE2 + kWmSmemC, s>>>(
          P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ, WBp);
      break;
    case 70:
      k_spmv_wg<TE, MODE, 3, MINOR><<<g, 256, 0, s>>>(P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ,
                                                      WBp);
      break;
    case 72:
    case 73:
    case 74:
    case 75: {
      // small CTAs (a few whole warps) so that a CTA's registers come free as soon as its few
      // wires are done: w wires of RQ threads in 32 ceil(w RQ / 32) threads, w chosen for the
      // fewest idle lanes
      int bw = 1, bt = 32;
      double be = 0.0;
      for (int w = 1; w <= 8; ++w) {
        const int t = 32 * (int)ceil_div(w * RQ, 32);
        if (t > 256) break;
        const double e = (double)(w * RQ) / t;
        if (e > be + 1e-9) {
          be = e;
          bw = w;
          bt = t;
        }
      }
      const dim3 gs((unsigned)ceil_div(ctx->nw, bw), g.y);
      // E and the column map staged by cp.async: the 16-byte spans around the tiles' ranges stay
      // inside the buffers only if both start on 16-byte boundaries (else form 73)
      const bool al16 =
          !(reinterpret_cast<uintptr_t>(E) & 15) && !(reinterpret_cast<uintptr_t>(ctx->offd.colmap) & 15);
      if ((form == 74 || (form == 75 && ctx->wrec)) && al16) {
        if (form == 74)
          k_spmv_wa<TE, MODE, 3, MINOR, kWaSmemE3><<<gs, bt, kWaSmemE3 + kWaSmemC, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ, bw, nullptr);
        else
          k_spmv_wa<TE, MODE, 3, MINOR, kWaSmemE3><<<gs, bt, kWaSmemE3 + kWaSmemC, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ, bw,
              reinterpret_cast<const WaRec*>(ctx->wrec));
      } else if (form == 72)
        k_spmv_wg<TE, MODE, 3, MINOR><<<gs, bt, 0, s>>>(P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ,
                                                        bw);
      else
        k_spmv_wg<TE, MODE, 4, MINOR><<<gs, bt, 0, s>>>(P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ,
                                                        bw);
      break;
    }
    default:
      k_spmv_wg<TE, MODE, 4, MINOR><<<g, 256, 0, s>>>(P, ctx->off, ctx->offd, ctx->nw, E, src, Xt, xst, dst, Bv, RQ,
                                                      WBp);
      break;
  }
  return SWM_OK;  // the caller checks and counts the launch
}
template <typename TE>
int allow_wm(swm_ctx* ctx) {
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kStepW, 3, kWmSmemE3>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kResW, 3, kWmSmemE3>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kStepW, 2, kWmSmemE2>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kResW, 2, kWmSmemE2>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kStepW, 3, kWmSmemE3, true>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kResW, 3, kWmSmemE3, true>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kStepW, 2, kWmSmemE2, true>, ctx->smem_optin));
  SWM_CK(allow_max_dyn_smem((const void*)k_spmv_wm<TE, kResW, 2, kWmSmemE2, true>, ctx->smem_optin));
  return SWM_OK;
}

// Tile shape of k_spmv_w for R right-hand sides: RG right-hand sides per CTA (all of them up to
// 64, else balanced groups of at most 64) and WB = 256 / RG wires per CTA.
struct WireTile {
  int RG, WB;
  unsigned gx, gy;
};
inline WireTile wire_tile(int R, int64_t nw) {
  WireTile t{};
  const int groups = (int)ceil_div(R, 64);
  t.RG = (int)ceil_div(R, groups);
  t.WB = std::max(1, 256 / t.RG);
  t.gx = (unsigned)ceil_div(nw, t.WB);
  t.gy = (unsigned)ceil_div(R, t.RG);
  return t;
}

// Arrival of one right-hand side at the end of the dots pass of step j; the last one advances the
// step (and counts the Hessenberg column it completed) and ends the cycle when nothing is active
// or the closing pass is done.
__device__ void step_arrive(const KPtr& P, int j, bool closing) {
  __threadfence();
  const unsigned done = atomicAdd(&P.counter[P.R], 1u);
  if (done == (unsigned)P.R - 1) {
    P.counter[P.R] = 0;
    int any = 0;
    for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
    P.st->j = j + 1;
    if (j >= 1) P.st->iters += 1;
    if (!any || closing) P.st->cycle_done = 1;
  }
}

// Last CTA of right-hand side r after the dots of step j (sums s_i = q_i^H u, t_i = q_i^H w for
// i < j, alpha = |u|^2 and beta = u^H w in sv/tv[j]): completes Hessenberg column j-1 (first-pass
// coefficients + reorthogonalisation s, subdiagonal rho = |u - Q s|), applies its Givens rotations
// and the residual test, and, unless this is the closing pass or r stopped, forms the first-pass
// coefficients of column j and the coefficients of the update pass.
template <typename TV>
__device__ void dots_tail(const KPtr& P, int j, int r, bool closing) {
  const int R1 = P.restart + 1, RS = P.restart;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  __shared__ c128 sv[SWM_MAX_RESTART + 1], tv[SWM_MAX_RESTART + 1], col[SWM_MAX_RESTART + 1];
  __shared__ double scs[SWM_MAX_RESTART];
  __shared__ c128 ssn[SWM_MAX_RESTART];
  __shared__ double rho_s;
  __shared__ int go_on;
  const c128* part = P.part + (int64_t)r * 2 * R1 * P.nchunk;
  for (int i = wp; i < 2 * (j + 1); i += kRows / 32) {
    if (closing && (i & 1)) continue;
    const c128 v = sum_partials_c(part + (int64_t)i * P.nchunk, 1, P.nchunk, lane);
    if (lane == 0) {
      if (i & 1)
        tv[i >> 1] = v;
      else
        sv[i >> 1] = v;
    }
  }
  for (int i = threadIdx.x; i < j; i += kRows) col[i] = P.hc[(int64_t)r * R1 + i];
  for (int i = threadIdx.x; i + 1 < j; i += kRows) {
    scs[i] = P.cs[(int64_t)r * RS + i];
    ssn[i] = P.sn[(int64_t)r * RS + i];
  }
  __syncthreads();
  if (wp == 0) {
    double ss = 0.0;
    for (int i = lane; i < j; i += 32) ss += sv[i].re * sv[i].re + sv[i].im * sv[i].im;
    ss = warp_sum(ss);
    if (lane == 0) {
      const double a = sv[j].re - ss;  // |u - Q s|^2 = |u|^2 - |s|^2 (Q orthonormal)
      rho_s = !isfinite(a) ? a : (a > 0.0 ? sqrt(a) : 0.0);
      P.counter[r] = 0;
    }
  }
  __syncthreads();
  const double rho = rho_s;
  c128* Hraw = P.Hraw + (int64_t)r * R1 * RS;  // unrotated Hessenberg, [i][l] at i * restart + l
  if (j >= 1)
    for (int i = threadIdx.x; i <= j; i += kRows) {
      const c128 v = i < j ? col[i] + sv[i] : mkc(rho, 0.0);
      col[i] = v;
      Hraw[i * RS + j - 1] = v;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    int act = 1;
    if (j >= 1) {
      const int l = j - 1;  // the column being completed
      for (int i = 0; i < l; ++i) {  // previous rotations
        const c128 a = col[i], b = col[i + 1];
        const c128 sc = ssn[i];
        col[i] = scs[i] * a + sc * b;
        col[i + 1] = mkc(-sc.re, sc.im) * a + scs[i] * b;  // -conj(s) a + c b
      }
      // new rotation zeroing the subdiagonal rho (real, >= 0)
      const c128 a = col[l];
      const double aa = sqrt(a.re * a.re + a.im * a.im);
      const double nu = sqrt(aa * aa + rho * rho);
      double c;
      c128 sg;
      if (aa == 0.0) {
        c = 0.0;
        sg = mkc(1.0, 0.0);
      } else {
        c = aa / nu;
        sg = mkc(a.re / aa * rho / nu, a.im / aa * rho / nu);
      }
      P.cs[(int64_t)r * RS + l] = c;
      P.sn[(int64_t)r * RS + l] = sg;
      col[l] = c * a + rho * sg;
      c128* g = P.g + (int64_t)r * R1;
      const c128 gl = g[l];
      const c128 gn = mkc(-sg.re, sg.im) * gl;
      g[l + 1] = gn;
      g[l] = c * gl;
      const double res = sqrt(gn.re * gn.re + gn.im * gn.im) / P.bnorm[r];
      P.resid[r] = res;
      P.jlast[r] = j;
      if (!isfinite(rho) || !isfinite(res)) {
        P.st->numeric = 1;
        act = 0;
      } else if (res <= P.tol || rho == 0.0) {
        act = 0;
      }
    } else {
      P.g[(int64_t)r * R1] = mkc(rho, 0.0);
      if (!isfinite(rho)) P.st->numeric = 1;
      if (!(rho > 0.0) || !isfinite(rho)) act = 0;
    }
    P.active[r] = act;
    go_on = act && !closing;
  }
  __syncthreads();
  c128* Hr = P.H + (int64_t)r * R1 * RS;
  if (j >= 1)
    for (int i = threadIdx.x; i < j; i += kRows) Hr[i * RS + j - 1] = col[i];
  if (go_on) {
    // A q_j = (w - A Q s) / rho and A Q s = Q (Hraw s) + q_j rho s_{j-1}; with Q orthonormal the
    // first-pass coefficients of column j are (t - Hraw s) / rho and q_j^H w / rho - s_{j-1}, where
    // q_j^H w = (beta - s^H t) / rho.
    const double ir = 1.0 / rho;
    for (int k = threadIdx.x; k < j; k += kRows) {
      c128 c = mkc(0.0, 0.0);
      for (int i = k > 0 ? k - 1 : 0; i < j; ++i) cfma(c, Hraw[k * RS + i], sv[i]);
      P.hc[(int64_t)r * R1 + k] = ir * (tv[k] - c);
      P.hc2[(int64_t)r * R1 + k] = sv[k];
      P.ht[(int64_t)r * R1 + k] = tv[k];
    }
    if (wp == 0) {
      double re = 0.0, im = 0.0;
      for (int i = lane; i < j; i += 32) {
        const c128 p = cmulc(sv[i], tv[i]);
        re += p.re;
        im += p.im;
      }
      re = warp_sum(re);
      im = warp_sum(im);
      if (lane == 0) {
        const c128 gam = (ir * ir) * (tv[j] - mkc(re, im));  // q_j^H w / rho
        P.gam[r] = gam;
        P.hc[(int64_t)r * R1 + j] = j >= 1 ? gam - sv[j - 1] : gam;
        P.inv_h[r] = ir;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) step_arrive(P, j, closing);
}

// Dots of step j, one CTA per chunk of rows and right-hand side: for i < j the pairs
// (q_i^H u, q_i^H w), and (|u|^2, u^H w), where u is the pending vector and w = A u; the closing
// pass of a cycle (j = jmax, no product) takes only the first of each pair.  The chunk's rows of u
// and w are staged in shared memory; the warps take (i, row slice) items, q_j standing for u itself,
// with the rows split into S slices while j + 1 < 8 so that every warp streams, and eight loads in
// flight per lane.  Slice sums are added in a fixed order (results do not depend on timing).
template <typename TV, typename TQ = cplx<TV>>
__global__ void __launch_bounds__(kRows) k_dots(KPtr P, const cplx<TV>* __restrict__ U,
                                                const cplx<TV>* __restrict__ Wv, const TQ* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j, r = blockIdx.y;
  const bool closing = j >= P.st->jmax;
  if (!P.active[r]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) step_arrive(P, j, closing);
    return;
  }
  const int R1 = P.restart + 1;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* u_sm = reinterpret_cast<cplx<TV>*>(sm_raw);  // [chunk]
  cplx<TV>* w_sm = u_sm + P.chunk;                       // [chunk]
  __shared__ c128 slot[2 * (SWM_MAX_RESTART + 1)];
  const cplx<TV>* u = U + (int64_t)r * P.N + n0;
  const cplx<TV>* w = Wv + (int64_t)r * P.N + n0;
  for (int t = threadIdx.x; t < cnt; t += kRows) {
    u_sm[t] = u[t];
    if (!closing) w_sm[t] = w[t];
  }
  __syncthreads();
  constexpr int kWarps = kRows / 32;
  const int S = j + 1 >= kWarps ? 1 : kWarps / (j + 1);  // row slices per i
  const int len = ((cnt + S - 1) / S + 31) / 32 * 32;
  for (int item = wp; item < (j + 1) * S; item += kWarps) {
    const int i = item / S, sl = item % S;
    const int lo = sl * len, hi = min(cnt, lo + len);
    // q_i from the basis, or (i == j) the pending vector u itself from shared memory; a basis in
    // the vector type is read through one pointer, a half-precision one converted on load
    constexpr bool full = std::is_same<TQ, cplx<TV>>::value;
    const TQ* vq = V + ((int64_t)i * P.R + r) * P.N + n0;  // i <= j <= restart: inside the basis
    const cplx<TV>* vi = full ? (i < j ? reinterpret_cast<const cplx<TV>*>(vq) : u_sm) : u_sm;
    const bool own = i >= j;
    const float qsi = P.qsi;
    auto ldv = [&](int t) -> cplx<TV> {
      if constexpr (full) return vi[t];
      else return own ? u_sm[t] : QStore<TV, TQ>::ld(vq + t, qsi);
    };
    cplx<TV> a = mkc<TV>(0, 0), b = mkc<TV>(0, 0);
    int t = lo + lane;
    for (; t + 224 < hi; t += 256) {
      cplx<TV> v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = ldv(t + 32 * k);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const cplx<TV> x = u_sm[t + 32 * k];
        a.re = fma(v[k].re, x.re, fma(v[k].im, x.im, a.re));
        a.im = fma(v[k].re, x.im, fma(-v[k].im, x.re, a.im));
        if (!closing) {
          const cplx<TV> y = w_sm[t + 32 * k];
          b.re = fma(v[k].re, y.re, fma(v[k].im, y.im, b.re));
          b.im = fma(v[k].re, y.im, fma(-v[k].im, y.re, b.im));
        }
      }
    }
    for (; t < hi; t += 32) {
      const cplx<TV> v = ldv(t), x = u_sm[t];
      a.re = fma(v.re, x.re, fma(v.im, x.im, a.re));
      a.im = fma(v.re, x.im, fma(-v.im, x.re, a.im));
      if (!closing) {
        const cplx<TV> y = w_sm[t];
        b.re = fma(v.re, y.re, fma(v.im, y.im, b.re));
        b.im = fma(v.re, y.im, fma(-v.im, y.re, b.im));
      }
    }
    const double ar = warp_sum((double)a.re), ai = warp_sum((double)a.im);
    const double br = warp_sum((double)b.re), bi = warp_sum((double)b.im);
    if (lane == 0) {
      slot[2 * item] = mkc(ar, ai);
      slot[2 * item + 1] = mkc(br, bi);
    }
  }
  __syncthreads();
  // partials laid out [r][2 i + k][chunk]: the last CTA reads each as one contiguous run
  c128* part = P.part + (int64_t)r * 2 * R1 * P.nchunk;
  for (int e = threadIdx.x; e < 2 * (j + 1); e += kRows) {
    const int i = e >> 1, k = e & 1;
    c128 v = slot[2 * (i * S) + k];
    for (int sl = 1; sl < S; ++sl) v = v + slot[2 * (i * S + sl) + k];
    part[(int64_t)e * P.nchunk + blockIdx.x] = v;
  }
  if (!last_cta(P, r)) return;
  dots_tail<TV>(P, j, r, closing);
}

// Update of step j (after its dots): q_j = (u - Q s) / rho goes to V_j and the next pending vector
// u' = (w - Q t) / rho - gamma q_j (the first Gram-Schmidt pass of A q_j) replaces u, in one read of
// Q_{<j}.  A thread takes KQ rows (kRows apart, so every load is coalesced) and reads BI basis
// vectors per pass: KQ * BI independent loads issued before their multiply-adds.  Two rows and
// four vectors measured fastest on the 1M-wire, 37-incidence workload (339 ms per step against
// 355 ms for four rows and two vectors, 398 ms for 4 x 4 and 634 ms for 8 x 2).
template <typename TV, typename TQ = cplx<TV>, int KQ = 2, int BI = 4>
__global__ void __launch_bounds__(kRows) k_update(KPtr P, cplx<TV>* __restrict__ U, const cplx<TV>* __restrict__ Wv,
                                                  TQ* __restrict__ V) {
  if (P.st->cycle_done) return;
  const int j = P.st->j - 1, r = blockIdx.y;
  if (!P.active[r]) return;
  const int R1 = P.restart + 1;
  __shared__ cplx<TV> ss[SWM_MAX_RESTART], ts[SWM_MAX_RESTART];
  for (int i = threadIdx.x; i < j; i += kRows) {
    ss[i] = ccast<TV>(P.hc2[(int64_t)r * R1 + i]);
    ts[i] = ccast<TV>(P.ht[(int64_t)r * R1 + i]);
  }
  const TV ih = (TV)P.inv_h[r];
  const cplx<TV> gm = ccast<TV>(P.gam[r]);
  __syncthreads();
  const int64_t N = P.N;
  const int64_t n0 = (int64_t)blockIdx.x * P.uchunk;
  const int cnt = (int)min((int64_t)P.uchunk, N - n0);
  cplx<TV>* u = U + (int64_t)r * N + n0;
  const cplx<TV>* w = Wv + (int64_t)r * N + n0;
  TQ* vj = V + ((int64_t)j * P.R + r) * N + n0;
  const float qs = P.qs, qsi = P.qsi;
  const int64_t vstride = (int64_t)P.R * N;
  for (int t0 = threadIdx.x; t0 < cnt; t0 += KQ * kRows) {
    cplx<TV> x[KQ], y[KQ];
    bool ok[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const int t = t0 + q * kRows;
      ok[q] = t < cnt;
      x[q] = ok[q] ? u[t] : mkc<TV>(0, 0);
      y[q] = ok[q] ? w[t] : mkc<TV>(0, 0);
    }
    const TQ* vb = V + (int64_t)r * N + n0 + t0;
    int i = 0;
    for (; i + BI <= j; i += BI) {
      cplx<TV> v[BI][KQ];
#pragma unroll
      for (int b = 0; b < BI; ++b)
#pragma unroll
        for (int q = 0; q < KQ; ++q)
          v[b][q] = ok[q] ? QStore<TV, TQ>::ld(vb + (int64_t)(i + b) * vstride + q * kRows, qsi) : mkc<TV>(0, 0);
#pragma unroll
      for (int b = 0; b < BI; ++b) {
        const cplx<TV> a = ss[i + b], c = ts[i + b];
#pragma unroll
        for (int q = 0; q < KQ; ++q) {
          x[q].re = fma(-v[b][q].re, a.re, fma(v[b][q].im, a.im, x[q].re));
          x[q].im = fma(-v[b][q].re, a.im, fma(-v[b][q].im, a.re, x[q].im));
          y[q].re = fma(-v[b][q].re, c.re, fma(v[b][q].im, c.im, y[q].re));
          y[q].im = fma(-v[b][q].re, c.im, fma(-v[b][q].im, c.re, y[q].im));
        }
      }
    }
    for (; i < j; ++i) {
      const cplx<TV> a = ss[i], c = ts[i];
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const cplx<TV> v = ok[q] ? QStore<TV, TQ>::ld(vb + (int64_t)i * vstride + q * kRows, qsi) : mkc<TV>(0, 0);
        x[q].re = fma(-v.re, a.re, fma(v.im, a.im, x[q].re));
        x[q].im = fma(-v.re, a.im, fma(-v.im, a.re, x[q].im));
        y[q].re = fma(-v.re, c.re, fma(v.im, c.im, y[q].re));
        y[q].im = fma(-v.re, c.im, fma(-v.im, c.re, y[q].im));
      }
    }
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
      const int t = t0 + q * kRows;
      if (ok[q]) {
        const cplx<TV> qv = ih * x[q];
        QStore<TV, TQ>::st(vj + t, qv, qs);
        u[t] = ih * y[q] - qv * gm;
      }
    }
  }
}

// Start of a cycle: norms of the residuals in U, activity, and the number of columns this cycle
// may take (restart, or what max_iter leaves).
template <typename TV>
__global__ void __launch_bounds__(kRows) k_cycle_start(KPtr P, const cplx<TV>* __restrict__ U, int first) {
  const int r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  const cplx<TV>* w = U + (int64_t)r * P.N + n0;
  double s = 0.0;
#pragma unroll 4
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
    P.g[(int64_t)r * (P.restart + 1)] = mkc(beta, 0.0);
    __threadfence();
    const unsigned done = atomicAdd(&P.counter[P.R], 1u);
    if (done == (unsigned)P.R - 1) {
      P.counter[P.R] = 0;
      int any = 0;
      for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
      P.st->j = 0;
      P.st->jmax = min(P.restart, P.max_iter - P.st->iters);
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

// Y += V coef, in the precision of the vectors (float64 arithmetic issues far slower than float32
// on GB300, and the complex64 path stores y in complex64 anyway).
template <typename TV, typename TQ = cplx<TV>>
__global__ void __launch_bounds__(256) k_update_y(KPtr P, const TQ* __restrict__ V, cplx<TV>* __restrict__ Y) {
  const int r = blockIdx.y;
  const int jl = P.jlast[r];
  if (jl == 0) return;
  __shared__ cplx<TV> cf[SWM_MAX_RESTART];
  for (int i = threadIdx.x; i < jl; i += blockDim.x) cf[i] = ccast<TV>(P.coef[(int64_t)r * P.restart + i]);
  __syncthreads();
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= P.N) return;
  cplx<TV> acc = mkc<TV>(0, 0);
#pragma unroll 4
  for (int i = 0; i < jl; ++i) cfma(acc, QStore<TV, TQ>::ld(V + ((int64_t)i * P.R + r) * P.N + n, P.qsi), cf[i]);
  Y[(int64_t)r * P.N + n] = Y[(int64_t)r * P.N + n] + acc;
}

// x = M^-1 y, block by block, in the precision of the vectors.
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
  cplx<TV> acc = mkc<TV>(0, 0);
  for (int l = 0; l < mp; ++l) cfma(acc, Mi[l], y[l]);
  X[(int64_t)r * N + n] = acc;
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
template <typename TV, typename TE, typename TQ = cplx<TV>>
int gmres_impl(swm_ctx* ctx, const TE* E, double tol, int restart, int max_iter, void** y_out, KState* hs_out) {
  constexpr bool kFullBasis = std::is_same<TQ, cplx<TV>>::value;
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
  P.max_iter = max_iter;
  P.qs = kFullBasis ? 1.f : (float)std::sqrt((double)std::max<int64_t>(1, N));
  P.qsi = 1.f / P.qs;
  // rows per CTA of the Gram-Schmidt kernels, at least kRows and at most kMaxChunk (the dots stage
  // a chunk of u and w in shared memory): the update about 16 CTAs per SM over all right-hand
  // sides; the dots about 4, so that the last CTA of each right-hand side adds fewer partial sums
  const int64_t nsm = std::max(ctx->nsm, 1);
  P.uchunk = (int)std::min<int64_t>(kMaxChunk, std::max<int64_t>(kRows, ceil_div(ceil_div(N * R, 16 * nsm), kRows) * kRows));
  P.nuchunk = (int)ceil_div(N, P.uchunk);
  P.chunk = (int)std::min<int64_t>(kMaxChunk, std::max<int64_t>(kRows, ceil_div(ceil_div(N * R, 4 * nsm), kRows) * kRows));
  P.nchunk = (int)ceil_div(N, P.chunk);
  const int R1 = restart + 1;
  // The workspace persists across solves of the same size, so buffer addresses (and the captured
  // graph that bakes them in) stay the same from one solve to the next.
  struct Workspace {
    int64_t key[4];
    KPtr P;
    cplx<TV> *Y, *W0, *W1;
    TQ* V;                // the basis, in the vector type or half precision
    cplx<TV>* Xt;         // many right-hand sides: the pending vectors right-hand-side minor, [N][R]
    PSync* sync;          // persistent solve: barrier state and partial sums over its CTAs
    c128 *pp1, *pp2;
    double* ppn;
    bool sync_clean;      // the barrier state is zero
  };
  const int64_t key[4] = {R, N, restart, (int64_t)(sizeof(TV) + 64 * sizeof(TQ))};
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
    SWM_TRY(dalloc(ctx, K, (void**)&P.Hraw, sizeof(c128) * R * R1 * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.cs, sizeof(double) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.sn, sizeof(c128) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.g, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.hc, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.hc2, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.ht, sizeof(c128) * R * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.gam, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&P.coef, sizeof(c128) * R * restart));
    SWM_TRY(dalloc(ctx, K, (void**)&P.part, sizeof(c128) * (size_t)R * P.nchunk * 2 * R1));
    SWM_TRY(dalloc(ctx, K, (void**)&P.partn, sizeof(double) * (size_t)R * P.nchunk));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->Y, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->W0, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->W1, sizeof(cplx<TV>) * R * N));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->V, sizeof(TQ) * (size_t)R1 * R * N));
    // rows padded to an even length (16-byte aligned pairs of right-hand sides)
    if (R >= kMinorR) SWM_TRY(dalloc(ctx, K, (void**)&ws->Xt, sizeof(cplx<TV>) * (size_t)(R + (R & 1)) * N));
    if (R <= kPersistMaxR && ctx->nsm > 0) {
      SWM_TRY(dalloc(ctx, K, (void**)&ws->sync, sizeof(PSync)));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->pp1, sizeof(c128) * (size_t)R * R1 * ctx->nsm));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->pp2, sizeof(c128) * (size_t)R * R1 * ctx->nsm));
      SWM_TRY(dalloc(ctx, K, (void**)&ws->ppn, sizeof(double) * (size_t)R * ctx->nsm));
    }
    ws->P = P;
  } else {
    const double tol_now = P.tol;
    const int max_iter_now = P.max_iter;
    P = ws->P;
    P.tol = tol_now;
    P.max_iter = max_iter_now;
  }
  cplx<TV> *Y = ws->Y, *W0 = ws->W0, *W1 = ws->W1;
  TQ* V = ws->V;
  // per-kernel path: W0 holds the pending vector u, W1 the product w = A u
  cplx<TV> *U = W0, *Wv = W1;
  // with an initial guess y0 = M x0 is copied in and, the tolerance staying relative to |b|, |b|
  // is measured first; otherwise (and for the refinement's correction) y starts at zero
  const bool given_b = ctx->guess && !y_out;
  if (given_b) {
    SWM_TRY(init_y(ctx, Y, sizeof(TV) == sizeof(double)));
    SWM_TRY(norms_of_b(ctx, ctx->Bv, sizeof(TV) == sizeof(double), P.bnorm));
  }
  (void)S;

  const cplx<TV>* Bv = (const cplx<TV>*)ctx->Bv;
  KState hs{};
  int cycles = 0;
  // small systems: the whole solve as one persistent cooperative kernel, which clears y itself
  bool persisted = false;
  SWM_TRY(ensure_poll_slots(ctx));
  {
    PBuffers pb{ws->sync, ws->pp1, ws->pp2, ws->ppn, E, Bv, Y, W0, V, given_b ? 1 : 0, given_b ? 0 : 1,
                &ws->sync_clean, y_out ? nullptr : ctx->Xv, y_out ? nullptr : ctx->rhs_frames};
    // the persistent solve keeps its basis in the vector type
    if (kFullBasis) SWM_TRY((gmres_persistent<TV, TE>(ctx, P, pb, max_iter, &hs, &persisted)));
  }
  if (!persisted && !y_out && ctx->rhs_frames) SWM_TRY(compute_rhs(ctx, R, ctx->rhs_frames));
  if (!y_out) ctx->rhs_frames = nullptr;
  if (!persisted) {
    SWM_CK(cudaMemsetAsync(P.st, 0, sizeof(KState), st));
    SWM_CK(cudaMemsetAsync(P.counter, 0, sizeof(unsigned) * (R + 1), st));
    if (!given_b) SWM_CK(cudaMemsetAsync(Y, 0, sizeof(cplx<TV>) * R * N, st));
  }
  const dim3 g_chunk((unsigned)P.nchunk, R), g_uchunk((unsigned)P.nuchunk, R);
  const bool multi = R > 1;
  const RowInfo* ri = (const RowInfo*)ctx->rowinfo;
  // The product: k_spmv with 1, 4, 8 or 16 right-hand sides sharing each read of E, or (kMinor)
  // the right-hand-side-minor form; with several right-hand sides the form is timed on this system
  // the first time its shape is solved, and kept.
  constexpr int kMinor = 32;
  constexpr int kWire = 64;  // k_spmv_w: wire-tiled, right-hand-side major, no transposed copy
  int rb = multi ? 8 : 1;
  const WireTile wt = wire_tile(R, ctx->nw);

  // res: the residual U = B - A Y of a cycle's start in the same form (every right-hand side)
  auto product = [&](cudaStream_t s, int b, auto res_tag) -> int {
    constexpr bool RS = decltype(res_tag)::value;
    const cplx<TV>* src = RS ? Y : U;
    cplx<TV>* dst = RS ? U : Wv;
    const dim3 gsp((unsigned)ceil_div(N * kG, kRows), (unsigned)ceil_div(R, std::min(b, 16)));
    switch (b) {
      case 1: k_spmv<TV, TE, 1, RS><<<gsp, kRows, 0, s>>>(P, ri, ctx->offd.colmap, E, src, dst, Bv); break;
      case 4: k_spmv<TV, TE, 4, RS><<<gsp, kRows, 0, s>>>(P, ri, ctx->offd.colmap, E, src, dst, Bv); break;
      case 16: k_spmv<TV, TE, 16, RS><<<gsp, kRows, 0, s>>>(P, ri, ctx->offd.colmap, E, src, dst, Bv); break;
      case kMinor: {
        k_rhs_minor<TV, RS><<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, src, ws->Xt);
        SWM_LAUNCHED();
        const unsigned gx = (unsigned)ceil_div(N, kTileRows);
        if (R >= 24)
          k_spmv_t<TV, TE, 32, RS><<<dim3(gx, (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, ri, ctx->offd.colmap, E,
                                                                                       ws->Xt, dst, Bv);
        else
          k_spmv_t<TV, TE, 16, RS><<<dim3(gx, (unsigned)ceil_div(R, 16)), 256, 0, s>>>(P, ri, ctx->offd.colmap, E,
                                                                                       ws->Xt, dst, Bv);
        break;
      }
      case kWire + 3:  // two right-hand sides per thread, E of the tile in shared memory
        if constexpr (std::is_same<TV, float>::value) {
          if (ws->Xt && R <= 256) {  // the transposing copy keeps T rows x (R + 1) in <= 48 KB
            const int xst = R + (R & 1);
            const int RQ = std::min(32, (int)ceil_div(R, 2));
            // at most 32 wires: the kernel's per-wire tables in shared memory hold 32
            const int WBp = std::max(1, std::min(kWpMaxWires, 256 / RQ));
            // all right-hand sides of T rows per CTA (T x (xst + 1) entries in shared memory, <= 48 KB)
            const int T = std::max(8, std::min(64, (int)((48 * 1024 / sizeof(cplx<TV>)) / (xst + 1)) / 8 * 8));
            ctx->prof_end(SWM_K_APPLY);
            ctx->prof_begin(SWM_K_TRANSPOSE);
            k_rhs_minor_all<TV, RS><<<(unsigned)ceil_div(N, T), 256, sizeof(cplx<TV>) * T * (xst + 1), s>>>(
                P, src, ws->Xt, xst, T);
            ctx->prof_end(SWM_K_TRANSPOSE);
            ctx->prof_begin(SWM_K_APPLY);
            SWM_LAUNCHED();
            k_spmv_wp<TE, RS ? kResW : kStepW>
                <<<dim3((unsigned)ceil_div(ctx->nw, WBp), (unsigned)ceil_div(R, 2 * RQ)), 256, kWpSmemBytes, s>>>(
                    P, ctx->off, ctx->offd, ctx->nw, E, src, ws->Xt, xst, dst, Bv, RQ, WBp);
            break;
          }
        }
        k_spmv_w<TV, TE, RS ? kResW : kStepW, false><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
            P, ctx->off, ctx->offd, ctx->nw, E, src, nullptr, dst, Bv, wt.RG, wt.WB);
        break;
      case kWire + 4:  // packed FP32x2 arithmetic, E expanded and the column map in shared memory
      case kWire + 5:  // the same with two CTAs per SM and a larger E budget
      case kWire + 6:  // packed, E and the column map read from global memory (three CTAs per SM)
      case kWire + 7:  // the same with four CTAs per SM
      case kWire + 8:  // the same in small CTAs of a few whole warps (register budget of 70)
      case kWire + 9:  // the same in small CTAs (register budget of 71)
      case kWire + 10:  // small CTAs, E and the column map staged by cp.async (budget of 70)
      case kWire + 11:  // the same over the wires sorted by loop length within windows
        if constexpr (std::is_same<TV, float>::value) {
          if (ws->Xt && R <= 256) {
            const int xst = R + (R & 1);
            const int RQ = std::min(32, (int)ceil_div(R, 2));
            const int WBp = std::max(1, std::min(kWpMaxWires, 256 / RQ));
            const int T = std::max(8, std::min(64, (int)((48 * 1024 / sizeof(cplx<TV>)) / (xst + 1)) / 8 * 8));
            ctx->prof_end(SWM_K_APPLY);
            ctx->prof_begin(SWM_K_TRANSPOSE);
            k_rhs_minor_all<TV, RS><<<(unsigned)ceil_div(N, T), 256, sizeof(cplx<TV>) * T * (xst + 1), s>>>(
                P, src, ws->Xt, xst, T);
            ctx->prof_end(SWM_K_TRANSPOSE);
            ctx->prof_begin(SWM_K_APPLY);
            SWM_LAUNCHED();
            SWM_TRY((launch_wm<TE, RS>(s, b, P, ctx, E, src, ws->Xt, xst, dst, Bv, RQ, WBp)));
            break;
          }
        }
        k_spmv_w<TV, TE, RS ? kResW : kStepW, false><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
            P, ctx->off, ctx->offd, ctx->nw, E, src, nullptr, dst, Bv, wt.RG, wt.WB);
        break;
      case kWire + 1:  // the same with five CTAs per SM (fewer registers)
        if (ws->Xt) {
          k_rhs_minor<TV, RS><<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, src,
                                                                                                        ws->Xt);
          SWM_LAUNCHED();
          k_spmv_w<TV, TE, RS ? kResW : kStepW, true, 5><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, ws->Xt, dst, Bv, wt.RG, wt.WB);
        } else {
          k_spmv_w<TV, TE, RS ? kResW : kStepW, false, 5><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, nullptr, dst, Bv, wt.RG, wt.WB);
        }
        break;
      case kWire:
        if (ws->Xt) {
          // the gathers read u right-hand-side minor: transposed first
          k_rhs_minor<TV, RS><<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(R, 32)), 256, 0, s>>>(P, src,
                                                                                                        ws->Xt);
          SWM_LAUNCHED();
          k_spmv_w<TV, TE, RS ? kResW : kStepW, true><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, ws->Xt, dst, Bv, wt.RG, wt.WB);
        } else {
          k_spmv_w<TV, TE, RS ? kResW : kStepW, false><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
              P, ctx->off, ctx->offd, ctx->nw, E, src, nullptr, dst, Bv, wt.RG, wt.WB);
        }
        break;
      default: k_spmv<TV, TE, 8, RS><<<gsp, kRows, 0, s>>>(P, ri, ctx->offd.colmap, E, src, dst, Bv); break;
    }
    SWM_LAUNCHED();
    return SWM_OK;
  };
  auto launch_product = [&](cudaStream_t s, int b) { return product(s, b, std::false_type{}); };
  auto launch_residual = [&](cudaStream_t s, int b) { return product(s, b, std::true_type{}); };
  if constexpr (std::is_same<TV, float>::value) {
    if (multi && ws->Xt) {
      SWM_TRY(allow_wm<TE>(ctx));
    }
  }
  const size_t dots_smem = 2 * sizeof(cplx<TV>) * (size_t)P.chunk;
  if (dots_smem > 48 * 1024) SWM_CK(allow_max_dyn_smem((const void*)k_dots<TV, TQ>, ctx->smem_optin));
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
      SWM_TRY(launch_product(s, rb));
      ctx->prof_end(SWM_K_APPLY);
      ctx->prof_begin(SWM_K_DOTS);
      k_dots<TV, TQ><<<g_chunk, kRows, dots_smem, s>>>(P, U, Wv, V);
      ctx->prof_end(SWM_K_DOTS);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_UPDATE);
      k_update<TV, TQ><<<g_uchunk, kRows, 0, s>>>(P, U, Wv, V);
      ctx->prof_end(SWM_K_UPDATE);
      SWM_LAUNCHED();
    }
    return SWM_OK;
  };
  if (!persisted && multi) {
    SWM_TRY(build_wire_order(ctx));  // form 75 (tuned or forced) takes the wires in this order
    const int64_t shape[6] = {N, R, (int64_t)sizeof(TV), (int64_t)sizeof(TE), P.chunk, restart};
    int found = 0;
    for (const auto& t : ctx->tuned)
      if (std::memcmp(t.shape, shape, sizeof(shape)) == 0) found = t.rb;
    const int forced = ctx->product_form;
    if (forced == 4 || forced == 8 || forced == 16 || forced == kWire || forced == kWire + 1 ||
        (forced >= kWire + 3 && forced <= kWire + 11) || (forced == kMinor && ws->Xt)) {
      rb = forced;
    } else if (found) {
      rb = found;
    } else {
      // first cycle's residual and start (the loop below repeats them; both are idempotent), then
      // each candidate product once untimed and once timed; the product is idempotent
      SWM_TRY(launch_residual(st, rb));
      k_cycle_start<TV><<<g_chunk, kRows, 0, st>>>(P, U, first ? 1 : 0);
      SWM_LAUNCHED();
      cudaEvent_t e0, e1;
      SWM_CK(cudaEventCreate(&e0));
      SWM_CK(cudaEventCreate(&e1));
      float best = 0.f;
      for (int b : {4, 8, 16, kMinor, kWire, kWire + 1, kWire + 3, kWire + 4, kWire + 5, kWire + 6, kWire + 7,
                    kWire + 8, kWire + 9, kWire + 10, kWire + 11}) {
        if (b == 16 && ceil_div(R, 16) == ceil_div(R, 8)) continue;  // no fewer reads of E than with 8
        if (b == kMinor && !ws->Xt) continue;
        SWM_TRY(launch_product(st, b));
        SWM_CK(cudaEventRecord(e0, st));
        SWM_TRY(launch_product(st, b));
        SWM_CK(cudaEventRecord(e1, st));
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
                         ctx->prof_cls != SWM_K_UPDATE && ctx->prof_cls != SWM_K_TRANSPOSE;
  if (use_graph) {
    struct Key {
      KPtr P;
      const void* ptr[8];
      Layout lay;
      unsigned gx, gy, bits;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.P = P;
    const void* ptrs[8] = {ctx->rowinfo, ctx->offd.colmap, E, U, Wv, V, ws->Xt, ctx->off};
    for (int i = 0; i < 8; ++i) key.ptr[i] = ptrs[i];
    key.lay = ctx->offd;
    key.gx = g_chunk.x;
    key.gy = g_chunk.y;
    key.bits = (unsigned)(sizeof(TV) * 64 + sizeof(TE) + 4096 * rb + (kFullBasis ? 0 : 1u << 24));
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
  const int launches_per_step = (rb == kMinor || (rb >= kWire && ws->Xt) ? 2 : 1) + 2;
  while (!persisted) {
    // residual of the current y and the start of a cycle
    ctx->prof_begin(SWM_K_APPLY);
    SWM_TRY(launch_residual(st, rb));
    ctx->prof_end(SWM_K_APPLY);
    k_cycle_start<TV><<<g_chunk, kRows, 0, st>>>(P, U, first ? 1 : 0);
    SWM_LAUNCHED();
    first = false;
    KState* hpin = reinterpret_cast<KState*>(static_cast<char*>(ctx->pinned_state) + kPersistStateOffset);
    SWM_CK(cudaMemcpyAsync(hpin, P.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    hs = *hpin;
    if (hs.all_conv || hs.numeric || hs.iters >= max_iter) break;
    // the cycle's Arnoldi steps and its closing pass
    const int steps = std::min(restart, max_iter - hs.iters) + 1;
    // chunks of steps; the host reads the flag of chunk c - 1 while chunk c is queued
    int c = 0;
    for (int s0 = 0; s0 < steps; s0 += kChunkSteps, ++c) {
      const int n = std::min(steps - s0, kChunkSteps);
      if (use_graph && n == kChunkSteps) {
        SWM_CK(cudaGraphLaunch(ctx->gm_exec, st));
        ctx->launches += launches_per_step * kChunkSteps;
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
    k_update_y<TV, TQ><<<dim3((unsigned)ceil_div(N, 256), R), 256, 0, st>>>(P, V, Y);
    SWM_LAUNCHED();
    ++cycles;
  }
  if (y_out) {  // inner solve of the refinement: the result stays in y-space
    if (persisted) {
      SWM_CK(cudaStreamSynchronize(st));
      SWM_TRY(persist_result(ctx, &hs, &ws->sync_clean));
    }
    if (hs_out) *hs_out = hs;
    *y_out = Y;
    dfree_group(ctx, tmp);
    if (hs.numeric) return ctx->fail(SWM_ECUDA, "GMRES produced a non-finite value");
    return hs.all_conv ? SWM_OK : SWM_ENOTCONV;
  }
  // x = M^-1 y (the persistent solve forms it itself), then one synchronisation for the residuals
  // (and the persistent solve's state)
  if (!persisted) SWM_TRY(apply_minv(ctx, Y));
  std::vector<double> res(R);
  double* rpin = reinterpret_cast<double*>(static_cast<char*>(ctx->pinned_state) + kPinnedResidOffset);
  const bool rp = R <= kPinnedResidMax;
  if (persisted && rp && ctx->fused && !hs_out) {
    // inside swm_run: the residuals and the solver state are read after the run's last
    // synchronisation (finish_solve)
    SWM_CK(cudaMemcpyAsync(rpin, P.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
    ctx->pend.active = true;
    ctx->pend.R = R;
    ctx->pend.sync_clean = &ws->sync_clean;
    dfree_group(ctx, tmp);
    return SWM_OK;
  }
  SWM_CK(cudaMemcpyAsync(rp ? rpin : res.data(), P.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaStreamSynchronize(st));
  if (rp) std::memcpy(res.data(), rpin, sizeof(double) * R);
  if (persisted) {
    SWM_TRY(persist_result(ctx, &hs, &ws->sync_clean));
    cycles = hs.cycles;
  }
  if (hs_out) *hs_out = hs;
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


// ---------------------------------------------------------------------------------------------
// BiCGSTAB on the same right-preconditioned system A y = b (A = I + E, x = M^-1 y): a
// short-recurrence Krylov method (van der Vorst 1992) whose step is two products and a fixed
// number of vector passes, so its cost per step does not grow with the step index as the
// Gram-Schmidt passes of GMRES do.  Each right-hand side is an independent instance; all share
// every pass over E.  Per step, with the shadow residual rh:
//   k_bi_dir (p) : p = r + beta (p - omega v)   (p = r and rh = r after a (re)start)
//   product      : v = A p
//   k_bi_rv      : alpha = rho / (rh^H v)
//   k_bi_dir (s) : s = r - alpha v
//   product      : t = A s
//   k_bi_ts      : omega = (t^H s) / (t^H t)
//   k_bi_xr      : y += alpha p + omega s,  r = s - omega t,  rho' = rh^H r,  |r|;
//                  beta = (rho' / rho)(alpha / omega)
// The two direction kernels also write their result right-hand-side minor (Xt) for the product's
// gathers.  Inner products: each thread sums its run of rows in the vector type (as the GMRES dots
// do), the CTA's threads and then the CTAs are added in float64, the CTAs in a fixed order by the
// last CTA of each right-hand side to arrive, which also updates that right-hand side's scalars.  A
// right-hand side stops when its recursive residual meets tol (or on a breakdown); when none is
// left the true residual b - A y is formed and those above tol restart from it.
struct BState {
  int nactive;  // right-hand sides still iterating
  int numeric;  // a NaN/Inf appeared
  int pad[6];
};
static_assert(sizeof(BState) == sizeof(KState), "poll slot layout");
struct BPtr {
  BState* st;
  int* active;        // [R] 1 while iterating
  int* fresh;         // [R] the next direction starts from r (and rh = r)
  int* its;           // [R] steps taken
  unsigned* counter;  // [R] CTAs of the current pass that have arrived
  double* bnorm;      // [R]
  double* resid;      // [R] relative residual: recursive while iterating, true after a check
  c128 *rho, *alpha, *omega, *beta;  // [R]
  c128* part;         // [R][nchunk][2]
  int64_t N;
  int R, nchunk, chunk, max_iter;
  double tol;
};

__device__ bool bi_last_cta(const BPtr& B, int r) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&B.counter[r], 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// Sums of a CTA (kRows threads) of two complex values, on thread 0.
__device__ void bi_block_sum2(c128& a, c128& b) {
  __shared__ double sh[4][kRows / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double v[4] = {warp_sum(a.re), warp_sum(a.im), warp_sum(b.re), warp_sum(b.im)};
  if (lane == 0)
    for (int k = 0; k < 4; ++k) sh[k][w] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      double s = 0.0;
      for (int i = 0; i < kRows / 32; ++i) s += sh[k][i];
      v[k] = s;
    }
    a = mkc(v[0], v[1]);
    b = mkc(v[2], v[3]);
  }
}

// The CTA's two partial sums to part[r][chunk]; the last CTA of r returns true with the totals
// (summed over the chunks in order) on thread 0 and resets the arrival counter.
__device__ bool bi_reduce2(const BPtr& B, int r, c128 a, c128 b, c128& ta, c128& tb) {
  bi_block_sum2(a, b);
  c128* part = B.part + ((int64_t)r * B.nchunk) * 2;
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
  if (!bi_last_cta(B, r)) return false;
  if (threadIdx.x < 32) {
    ta = sum_partials_c(part, 2, B.nchunk, threadIdx.x);
    tb = sum_partials_c(part + 1, 2, B.nchunk, threadIdx.x);
  }
  if (threadIdx.x == 0) B.counter[r] = 0;
  return threadIdx.x == 0;
}

__device__ __forceinline__ bool finite_z(c128 z) { return isfinite(z.re) && isfinite(z.im); }
// acc += conj(a) b and n += |b|^2 in the vector type (a thread's run of rows); the sums over
// threads and CTAs are float64
template <typename T>
__device__ __forceinline__ void bi_acc(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename T>
__device__ __forceinline__ void bi_nrm(T& acc, cplx<T> b) {
  acc = fma(b.re, b.re, fma(b.im, b.im, acc));
}
__device__ __forceinline__ c128 bi_cdiv(c128 a, c128 b) {
  const double s = 1.0 / (b.re * b.re + b.im * b.im);
  return s * cmulc(b, a);
}

// the product kernels' step state (never done: step 0 of 1) and every right-hand side active for
// the residual
__global__ void k_bi_init(KState* k, int* pact, int R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    KState z{};
    z.jmax = 1;
    *k = z;
  }
  if (i < R) pact[i] = 1;
}

__device__ void bi_stop(const BPtr& B, int r, bool numeric) {
  B.active[r] = 0;
  atomicSub(&B.st->nactive, 1);
  if (numeric) B.st->numeric = 1;
}

// p = r + beta (p - omega v), or p = r and rh = r after a (re)start (SMODE false); s = r - alpha v
// (SMODE true).  T rows x all right-hand sides per CTA; with XT the result is also written
// right-hand-side minor, Xt[n][0 .. xst), through a shared-memory tile (inactive right-hand sides
// and the padding column as zero).
template <typename TV, bool SMODE, bool XT>
__global__ void __launch_bounds__(256) k_bi_dir(BPtr B, const cplx<TV>* __restrict__ Rv, cplx<TV>* __restrict__ Rh,
                                                cplx<TV>* __restrict__ Pv, const cplx<TV>* __restrict__ Vv,
                                                cplx<TV>* __restrict__ Out, cplx<TV>* __restrict__ Xt, int xst,
                                                int T) {
  extern __shared__ __align__(16) unsigned char sm_bi[];
  cplx<TV>* tile = reinterpret_cast<cplx<TV>*>(sm_bi);  // [T][xst + 1]
  const int ts = xst + 1;
  const int64_t N = B.N;
  const int64_t n0 = (int64_t)blockIdx.x * T;
  const int cnt = (int)min((int64_t)T, N - n0);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nwp = blockDim.x >> 5;
  for (int r = wp; r < B.R; r += nwp) {
    const bool act = B.active[r] != 0;
    const int64_t base = (int64_t)r * N + n0;
    if (act) {
      if (SMODE) {
        const cplx<TV> a = ccast<TV>(B.alpha[r]);
        for (int t = lane; t < cnt; t += 32) {
          const cplx<TV> o = Rv[base + t] - a * Vv[base + t];
          Out[base + t] = o;
          if (XT) tile[t * ts + r] = o;
        }
      } else if (B.fresh[r]) {
        for (int t = lane; t < cnt; t += 32) {
          const cplx<TV> o = Rv[base + t];
          Rh[base + t] = o;
          Out[base + t] = o;
          if (XT) tile[t * ts + r] = o;
        }
      } else {
        const cplx<TV> be = ccast<TV>(B.beta[r]), om = ccast<TV>(B.omega[r]);
        for (int t = lane; t < cnt; t += 32) {
          const cplx<TV> o = Rv[base + t] + be * (Pv[base + t] - om * Vv[base + t]);
          Out[base + t] = o;
          if (XT) tile[t * ts + r] = o;
        }
      }
    } else if (XT) {
      for (int t = lane; t < cnt; t += 32) tile[t * ts + r] = mkc<TV>(0, 0);
    }
  }
  if (!XT) return;
  __syncthreads();
  cplx<TV>* out = Xt + n0 * xst;
  for (int t = wp; t < cnt; t += nwp)
    for (int r = lane; r < xst; r += 32) out[(int64_t)t * xst + r] = r < B.R ? tile[t * ts + r] : mkc<TV>(0, 0);
}

// alpha = rho / (rh^H v)
template <typename TV>
__global__ void __launch_bounds__(kRows) k_bi_rv(BPtr B, const cplx<TV>* __restrict__ Rh,
                                                 const cplx<TV>* __restrict__ Vv) {
  const int r = blockIdx.y;
  if (!B.active[r]) return;
  const int64_t N = B.N, n0 = (int64_t)blockIdx.x * B.chunk, n1 = min(N, n0 + B.chunk);
  const cplx<TV>* h = Rh + (int64_t)r * N;
  const cplx<TV>* v = Vv + (int64_t)r * N;
  cplx<TV> a = mkc<TV>(0, 0);
#pragma unroll 4
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kRows) bi_acc(a, h[n], v[n]);
  c128 rv, dummy;
  if (!bi_reduce2(B, r, ccast<double>(a), mkc(0.0, 0.0), rv, dummy)) return;
  B.fresh[r] = 0;
  const double mag = sqrt(rv.re * rv.re + rv.im * rv.im);
  if (!finite_z(rv)) {
    bi_stop(B, r, true);
  } else if (mag == 0.0) {
    bi_stop(B, r, false);  // breakdown: the true-residual check restarts it
  } else {
    B.alpha[r] = bi_cdiv(B.rho[r], rv);
  }
}

// omega = (t^H s) / (t^H t)
template <typename TV>
__global__ void __launch_bounds__(kRows) k_bi_ts(BPtr B, const cplx<TV>* __restrict__ Tv,
                                                 const cplx<TV>* __restrict__ Sv) {
  const int r = blockIdx.y;
  if (!B.active[r]) return;
  const int64_t N = B.N, n0 = (int64_t)blockIdx.x * B.chunk, n1 = min(N, n0 + B.chunk);
  const cplx<TV>* t = Tv + (int64_t)r * N;
  const cplx<TV>* s = Sv + (int64_t)r * N;
  cplx<TV> ts = mkc<TV>(0, 0);
  TV tt = 0;
#pragma unroll 4
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kRows) {
    const cplx<TV> tv = t[n];
    bi_acc(ts, tv, s[n]);
    bi_nrm(tt, tv);
  }
  c128 sts, stt;
  if (!bi_reduce2(B, r, ccast<double>(ts), mkc((double)tt, 0.0), sts, stt)) return;
  if (!finite_z(sts) || !isfinite(stt.re)) {
    bi_stop(B, r, true);
    return;
  }
  B.omega[r] = stt.re > 0.0 ? (1.0 / stt.re) * sts : mkc(0.0, 0.0);
}

// y += alpha p + omega s, r = s - omega t; rho' = rh^H r and |r| decide the next step
template <typename TV>
__global__ void __launch_bounds__(kRows) k_bi_xr(BPtr B, cplx<TV>* __restrict__ Y, cplx<TV>* __restrict__ Rv,
                                                 const cplx<TV>* __restrict__ Rh, const cplx<TV>* __restrict__ Pv,
                                                 const cplx<TV>* __restrict__ Sv, const cplx<TV>* __restrict__ Tv) {
  const int r = blockIdx.y;
  if (!B.active[r]) return;
  const int64_t N = B.N, n0 = (int64_t)blockIdx.x * B.chunk, n1 = min(N, n0 + B.chunk);
  const int64_t o = (int64_t)r * N;
  const cplx<TV> a = ccast<TV>(B.alpha[r]), om = ccast<TV>(B.omega[r]);
  cplx<TV> hr = mkc<TV>(0, 0);
  TV rr = 0;
#pragma unroll 4
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kRows) {
    const cplx<TV> sv = Sv[o + n];
    Y[o + n] = Y[o + n] + a * Pv[o + n] + om * sv;
    const cplx<TV> rn = sv - om * Tv[o + n];
    Rv[o + n] = rn;
    bi_acc(hr, Rh[o + n], rn);
    bi_nrm(rr, rn);
  }
  c128 shr, srr;
  if (!bi_reduce2(B, r, ccast<double>(hr), mkc((double)rr, 0.0), shr, srr)) return;
  const int it = ++B.its[r];
  const double rel = B.bnorm[r] > 0.0 ? sqrt(srr.re) / B.bnorm[r] : 0.0;
  B.resid[r] = rel;
  const c128 om64 = B.omega[r];
  if (!finite_z(shr) || !isfinite(rel)) {
    bi_stop(B, r, true);
  } else if (rel <= B.tol || it >= B.max_iter || (om64.re == 0.0 && om64.im == 0.0) ||
             (shr.re == 0.0 && shr.im == 0.0)) {
    bi_stop(B, r, false);  // converged by the recursion, out of steps, or a breakdown
  } else {
    B.beta[r] = bi_cdiv(shr, B.rho[r]) * bi_cdiv(B.alpha[r], om64);
    B.rho[r] = shr;
  }
}

// True residual check: r holds b - A y; right-hand sides above tol with steps left restart from it
// (rho = |r|^2, the next direction p = r and rh = r).
template <typename TV>
__global__ void __launch_bounds__(kRows) k_bi_check(BPtr B, const cplx<TV>* __restrict__ Rv) {
  const int r = blockIdx.y;
  const int64_t N = B.N, n0 = (int64_t)blockIdx.x * B.chunk, n1 = min(N, n0 + B.chunk);
  const cplx<TV>* v = Rv + (int64_t)r * N;
  TV rr = 0;
#pragma unroll 4
  for (int64_t n = n0 + threadIdx.x; n < n1; n += kRows) bi_nrm(rr, v[n]);
  c128 srr, dummy;
  if (!bi_reduce2(B, r, mkc((double)rr, 0.0), mkc(0.0, 0.0), srr, dummy)) return;
  const double rel = B.bnorm[r] > 0.0 ? sqrt(srr.re) / B.bnorm[r] : 0.0;
  B.resid[r] = rel;
  if (!isfinite(rel)) {
    B.active[r] = 0;
    B.st->numeric = 1;
  } else if (rel > B.tol && B.its[r] < B.max_iter) {
    B.active[r] = 1;
    B.fresh[r] = 1;
    B.rho[r] = mkc(srr.re, 0.0);
    atomicAdd(&B.st->nactive, 1);
  } else {
    B.active[r] = 0;
  }
}

template <typename TV, typename TE>
int bicgstab_impl(swm_ctx* ctx, const TE* E, double tol, int max_iter) {
  SWM_TRY(build_wire_order(ctx));  // the order of product form 75, once per pattern
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  const int64_t nsm = std::max(ctx->nsm, 1);
  // the right-hand-side-minor copy for the wire-tiled product with two right-hand sides per thread
  const bool xt = std::is_same<TV, float>::value && R >= 2 && R <= 256;
  const int xst = R + (R & 1);
  struct Workspace {
    int64_t key[4];
    BPtr B;
    KState* kst;  // the product kernels' step state: never done
    int* pact;    // the product kernels' activity flags (all right-hand sides: the residual)
    cplx<TV> *Y, *Rv, *Rh, *Pv, *Vv, *Sv, *Tv, *Xt;
  };
  const int64_t key[4] = {R, N, (int64_t)sizeof(TV), -2};
  Workspace* ws = reinterpret_cast<Workspace*>(ctx->kry_ws);
  if (!ws || ctx->kry_ws_bytes != sizeof(Workspace) || std::memcmp(ws->key, key, sizeof(key)) != 0) {
    dfree_group(ctx, ctx->kry_bufs);
    std::free(ctx->kry_ws);
    ctx->kry_ws = nullptr;
    ws = reinterpret_cast<Workspace*>(std::calloc(1, sizeof(Workspace)));
    if (!ws) return ctx->fail(SWM_ENOMEM, "host allocation failed");
    ctx->kry_ws = ws;
    ctx->kry_ws_bytes = sizeof(Workspace);
    std::memcpy(ws->key, key, sizeof(key));
    auto& K = ctx->kry_bufs;
    BPtr B{};
    B.N = N;
    B.R = R;
    B.chunk = (int)std::min<int64_t>(kMaxChunk, std::max<int64_t>(kRows, ceil_div(ceil_div(N * R, 4 * nsm), kRows) * kRows));
    B.nchunk = (int)ceil_div(N, B.chunk);
    SWM_TRY(dalloc(ctx, K, (void**)&B.st, sizeof(BState)));
    SWM_TRY(dalloc(ctx, K, (void**)&B.active, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.fresh, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.its, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.counter, sizeof(unsigned) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.bnorm, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.resid, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.rho, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.alpha, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.omega, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.beta, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.part, sizeof(c128) * 2 * (size_t)R * B.nchunk));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->kst, sizeof(KState)));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->pact, sizeof(int) * R));
    cplx<TV>** vecs[7] = {&ws->Y, &ws->Rv, &ws->Rh, &ws->Pv, &ws->Vv, &ws->Sv, &ws->Tv};
    for (auto v : vecs) SWM_TRY(dalloc(ctx, K, (void**)v, sizeof(cplx<TV>) * R * N));
    if (xt) SWM_TRY(dalloc(ctx, K, (void**)&ws->Xt, sizeof(cplx<TV>) * (size_t)xst * N));
    ws->B = B;
  }
  BPtr B = ws->B;
  B.tol = tol;
  B.max_iter = max_iter;
  cplx<TV> *Y = ws->Y, *Rv = ws->Rv, *Rh = ws->Rh, *Pv = ws->Pv, *Vv = ws->Vv, *Sv = ws->Sv, *Tv = ws->Tv;
  const cplx<TV>* Bv = (const cplx<TV>*)ctx->Bv;
  SWM_TRY(ensure_poll_slots(ctx));
  // product kernels' view: N, R, their step state (never done) and activity flags
  KPtr P{};
  P.N = N;
  P.R = R;
  P.st = ws->kst;
  P.active = B.active;
  KPtr Pall = P;  // residual: every right-hand side
  Pall.active = ws->pact;
  k_bi_init<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(ws->kst, ws->pact, R);
  SWM_LAUNCHED();
  SWM_CK(cudaMemsetAsync(B.st, 0, sizeof(BState), st));
  SWM_CK(cudaMemsetAsync(B.its, 0, sizeof(int) * R, st));
  SWM_CK(cudaMemsetAsync(B.counter, 0, sizeof(unsigned) * R, st));
  SWM_CK(cudaMemsetAsync(B.active, 0, sizeof(int) * R, st));
  SWM_TRY(norms_of_b(ctx, ctx->Bv, sizeof(TV) == sizeof(double), B.bnorm));
  SWM_TRY(init_y(ctx, Y, sizeof(TV) == sizeof(double)));
  const WireTile wt = wire_tile(R, ctx->nw);
  const int RQ = std::min(32, (int)ceil_div(R, 2));
  const int WBp = std::max(1, std::min(kWpMaxWires, 256 / RQ));
  const int T = std::max(8, std::min(64, (int)((48 * 1024 / sizeof(cplx<TV>)) / (xst + 1)) / 8 * 8));
  const size_t dir_smem = xt ? sizeof(cplx<TV>) * T * (xst + 1) : 0;
  if constexpr (std::is_same<TV, float>::value) {
    if (xt) SWM_TRY(allow_wm<TE>(ctx));
  }
  // product form: the packed wire-tiled product in one of its two shapes, or (no copy) the
  // wire-tiled product reading u in place; with the copy the shape is timed on this system the
  // first time its size is solved (the product is idempotent) and kept
  int form = xt ? 68 : 64;
  // w = u + E u (active right-hand sides), or with RES w = b - (u + E u) for all of them; with the
  // right-hand-side-minor copy the source's copy is in Xt already
  auto product = [&](cudaStream_t s, const cplx<TV>* src, cplx<TV>* dst, auto res_tag) -> int {
    constexpr bool RS = decltype(res_tag)::value;
    const KPtr& PP = RS ? Pall : P;
    if constexpr (std::is_same<TV, float>::value) {
      if (xt) {
        SWM_TRY((launch_wm<TE, RS>(s, form, PP, ctx, E, src, ws->Xt, xst, dst, Bv, RQ, WBp)));
        SWM_LAUNCHED();
        return SWM_OK;
      }
    }
    k_spmv_w<TV, TE, RS ? kResW : kStepW, false><<<dim3(wt.gx, wt.gy), 256, 0, s>>>(
        PP, ctx->off, ctx->offd, ctx->nw, E, src, nullptr, dst, Bv, wt.RG, wt.WB);
    SWM_LAUNCHED();
    return SWM_OK;
  };
  const unsigned gT = (unsigned)ceil_div(N, T);
  const dim3 gC((unsigned)B.nchunk, R);
  auto launch_steps = [&](cudaStream_t s, int n) -> int {
    for (int i = 0; i < n; ++i) {
      ctx->prof_begin(SWM_K_TRANSPOSE);
      if (xt)
        k_bi_dir<TV, false, true><<<gT, 256, dir_smem, s>>>(B, Rv, Rh, Pv, Vv, Pv, ws->Xt, xst, T);
      else
        k_bi_dir<TV, false, false><<<gT, 256, 0, s>>>(B, Rv, Rh, Pv, Vv, Pv, nullptr, xst, T);
      ctx->prof_end(SWM_K_TRANSPOSE);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_APPLY);
      SWM_TRY(product(s, Pv, Vv, std::false_type{}));
      ctx->prof_end(SWM_K_APPLY);
      ctx->prof_begin(SWM_K_DOTS);
      k_bi_rv<TV><<<gC, kRows, 0, s>>>(B, Rh, Vv);
      ctx->prof_end(SWM_K_DOTS);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_TRANSPOSE);
      if (xt)
        k_bi_dir<TV, true, true><<<gT, 256, dir_smem, s>>>(B, Rv, Rh, Pv, Vv, Sv, ws->Xt, xst, T);
      else
        k_bi_dir<TV, true, false><<<gT, 256, 0, s>>>(B, Rv, Rh, Pv, Vv, Sv, nullptr, xst, T);
      ctx->prof_end(SWM_K_TRANSPOSE);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_APPLY);
      SWM_TRY(product(s, Sv, Tv, std::false_type{}));
      ctx->prof_end(SWM_K_APPLY);
      ctx->prof_begin(SWM_K_DOTS);
      k_bi_ts<TV><<<gC, kRows, 0, s>>>(B, Tv, Sv);
      ctx->prof_end(SWM_K_DOTS);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_UPDATE);
      k_bi_xr<TV><<<gC, kRows, 0, s>>>(B, Y, Rv, Rh, Pv, Sv, Tv);
      ctx->prof_end(SWM_K_UPDATE);
      SWM_LAUNCHED();
    }
    return SWM_OK;
  };
  // the true residual r = b - A y of every right-hand side and the restart decision
  auto check = [&]() -> int {
    if (xt) {
      k_rhs_minor_all<TV, true><<<gT, 256, dir_smem, st>>>(Pall, Y, ws->Xt, xst, T);
      SWM_LAUNCHED();
    }
    ctx->prof_begin(SWM_K_APPLY);
    SWM_TRY(product(st, Y, Rv, std::true_type{}));
    ctx->prof_end(SWM_K_APPLY);
    k_bi_check<TV><<<gC, kRows, 0, st>>>(B, Rv);
    SWM_LAUNCHED();
    return SWM_OK;
  };
  if (xt) {
    const int64_t shape[6] = {N, R, (int64_t)sizeof(TV), (int64_t)sizeof(TE), -3, 0};
    int found = 0;
    for (const auto& t : ctx->tuned)
      if (std::memcmp(t.shape, shape, sizeof(shape)) == 0) found = t.rb;
    if (ctx->product_form >= 68 && ctx->product_form <= 75) {
      form = ctx->product_form;
    } else if (found) {
      form = found;
    } else {
      // p = b transposed, then each shape once untimed and once timed on it
      k_rhs_minor_all<TV, true><<<gT, 256, dir_smem, st>>>(Pall, Bv, ws->Xt, xst, T);
      SWM_LAUNCHED();
      cudaEvent_t e0, e1;
      SWM_CK(cudaEventCreate(&e0));
      SWM_CK(cudaEventCreate(&e1));
      float best = 0.f;
      for (int f : {68, 69, 70, 71, 72, 73, 74, 75}) {
        form = f;
        SWM_TRY(product(st, Bv, Vv, std::true_type{}));
        SWM_CK(cudaEventRecord(e0, st));
        SWM_TRY(product(st, Bv, Vv, std::true_type{}));
        SWM_CK(cudaEventRecord(e1, st));
        SWM_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        SWM_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best == 0.f || ms < best) {
          best = ms;
          found = f;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      form = found;
      swm_ctx::Tuned t{};
      std::memcpy(t.shape, shape, sizeof(shape));
      t.rb = form;
      ctx->tuned.push_back(t);
    }
  }
  constexpr int kChunk = 4;
  ctx->stats.step_rhs_block = form;
  const bool use_graph = ctx->prof_cls != SWM_K_APPLY && ctx->prof_cls != SWM_K_DOTS &&
                         ctx->prof_cls != SWM_K_UPDATE && ctx->prof_cls != SWM_K_TRANSPOSE;
  if (use_graph) {
    struct Key {
      BPtr B;
      const void* ptr[12];
      Layout lay;
      int64_t bits;
    } gk;
    std::memset(&gk, 0, sizeof(gk));
    gk.B = B;
    const void* ptrs[12] = {E, Y, Rv, Rh, Pv, Vv, Sv, Tv, ws->Xt, ctx->off, ws->kst, Bv};
    for (int i = 0; i < 12; ++i) gk.ptr[i] = ptrs[i];
    gk.lay = ctx->offd;
    gk.bits = -(int64_t)(sizeof(TV) * 64 + sizeof(TE));
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&gk);
    std::vector<unsigned char> kv(kb, kb + sizeof(gk));
    if (!ctx->gm_exec || kv != ctx->gm_key) {
      if (!ctx->cap_stream) SWM_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      const int64_t launches0 = ctx->launches;
      SWM_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_steps(ctx->cap_stream, kChunk);
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
  const int launches_per_step = 7;
  KState* slot = reinterpret_cast<KState*>(ctx->pinned_state);
  BState hs{};
  int restarts = 0;
  for (;;) {
    SWM_TRY(check());
    BState* hpin = reinterpret_cast<BState*>(static_cast<char*>(ctx->pinned_state) + kPersistStateOffset);
    SWM_CK(cudaMemcpyAsync(hpin, B.st, sizeof(BState), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    hs = *hpin;
    if (hs.nactive <= 0 || hs.numeric) break;
    ++restarts;
    // chunks of steps; the host reads the count of chunk c - 1 while chunk c is queued.  Each
    // right-hand side stops by itself after at most max_iter steps, so the loop ends.
    for (int c = 0;; ++c) {
      if (use_graph) {
        SWM_CK(cudaGraphLaunch(ctx->gm_exec, st));
        ctx->launches += launches_per_step * kChunk;
      } else {
        SWM_TRY(launch_steps(st, kChunk));
      }
      SWM_CK(cudaMemcpyAsync(&slot[c & 1], B.st, sizeof(BState), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaEventRecord(ctx->poll_ev[c & 1], st));
      if (c >= 1) {
        SWM_CK(cudaEventSynchronize(ctx->poll_ev[(c - 1) & 1]));
        const BState* b = reinterpret_cast<const BState*>(&slot[(c - 1) & 1]);
        if (b->nactive <= 0 || b->numeric) break;
      }
    }
  }
  SWM_TRY(apply_minv(ctx, Y));
  std::vector<double> res(R);
  std::vector<int> its(R);
  SWM_CK(cudaMemcpyAsync(res.data(), B.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaMemcpyAsync(its.data(), B.its, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaStreamSynchronize(st));
  double mx = 0.0;
  int itmax = 0;
  for (int r = 0; r < R; ++r) {
    mx = std::max(mx, res[r]);
    itmax = std::max(itmax, its[r]);
  }
  ctx->stats.iterations = itmax;
  ctx->stats.restarts = std::max(0, restarts - 1);
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = (!hs.numeric && mx <= tol) ? 1 : 0;
  if (hs.numeric) return ctx->fail(SWM_ECUDA, "BiCGSTAB produced a non-finite value");
  return ctx->stats.converged ? SWM_OK : SWM_ENOTCONV;
}


// ---------------------------------------------------------------------------------------------
// BiCGSTAB on incidence-minor vectors (complex64, two to 256 incidences): every vector is stored
// [N][xst] (xst = R rounded up to even, the padding column zero) like the product's gathered
// copy, so the product reads its source in place, writes its image with 16-byte accesses at its
// own rows, and the direction updates need no transposed copy.  Each vector kernel takes a chunk
// of rows with all incidences (thread (row lane, incidence)); the per-incidence partial sums of a
// CTA are added over its row lanes in order, written per chunk, and the last CTA of the pass adds
// the chunks in order for every incidence and updates that incidence's scalars (float64).
struct BmPtr {
  BState* st;
  int* active;        // [R] 1 while iterating
  int* fresh;         // [R] the next direction starts from r (and rh = r)
  int* its;           // [R] steps taken
  unsigned* counter;  // [1] CTAs of the current pass that have arrived
  double* bnorm;      // [R]
  double* resid;      // [R]
  c128 *rho, *alpha, *omega, *beta;  // [R]
  c128* part;         // [R][nchunk][2]
  int64_t N;
  int R, xst, nchunk, chunk, max_iter;
  double tol;
};

// The last CTA: warp w takes incidences w, w + 8, ...; lane 0 gets the totals.
template <typename F>
__device__ void bm_finish(const BmPtr& B, F&& f) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw8 = blockDim.x >> 5;
  for (int c = w; c < B.R; c += nw8) {
    const c128* base = B.part + (int64_t)c * B.nchunk * 2;
    const c128 ta = sum_partials_c(base, 2, B.nchunk, lane);
    const c128 tb = sum_partials_c(base + 1, 2, B.nchunk, lane);
    if (lane == 0) f(c, ta, tb);
  }
  if (threadIdx.x == 0) *B.counter = 0;
}

__device__ void bm_stop(const BmPtr& B, int r, bool numeric) {
  B.active[r] = 0;
  atomicSub(&B.st->nactive, 1);
  if (numeric) B.st->numeric = 1;
}

// Pair-granular forms of the incidence-minor BiCGSTAB passes: thread (row lane, pair q) takes
// incidences 2q and 2q + 1 (the second may be the padding column) of its rows as one 16-byte
// access; scalars of inactive or padding halves are zero, so those halves stay finite.
struct BpRow {
  int q, rl, nrl;
  bool valid;
  int64_t n0, n1;
};
__device__ __forceinline__ BpRow bp_row(const BmPtr& B) {
  BpRow t;
  const int pq = B.xst >> 1;
  t.nrl = blockDim.x / pq;
  t.q = threadIdx.x % pq;
  t.rl = threadIdx.x / pq;
  t.valid = t.rl < t.nrl;
  t.n0 = (int64_t)blockIdx.x * B.chunk;
  t.n1 = min(B.N, t.n0 + B.chunk);
  return t;
}
__device__ __forceinline__ float4 ld4(const c64* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(c64* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ c64 lo(float4 v) { return mkc(v.x, v.y); }
__device__ __forceinline__ c64 hi(float4 v) { return mkc(v.z, v.w); }
__device__ __forceinline__ float4 f4(c64 a, c64 b) { return make_float4(a.re, a.im, b.re, b.im); }
// Per-incidence sums of the pair passes: a (complex) and b (real) for both halves, the row lanes
// added in order, one partial per chunk; true on every thread of the last CTA to arrive.
__device__ bool bp_reduce(const BmPtr& B, const BpRow& t, c128 a0, c128 b0, c128 a1, c128 b1) {
  __shared__ c128 red[4][256];
  __shared__ bool last;
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = b0;
  red[2][threadIdx.x] = a1;
  red[3][threadIdx.x] = b1;
  __syncthreads();
  const int pq = B.xst >> 1;
  if (t.valid && t.rl == 0) {
    c128 s[4] = {mkc(0.0, 0.0), mkc(0.0, 0.0), mkc(0.0, 0.0), mkc(0.0, 0.0)};
    for (int l = 0; l < t.nrl; ++l)
      for (int k = 0; k < 4; ++k) s[k] = s[k] + red[k][l * pq + t.q];
    const int c0 = 2 * t.q, c1 = c0 + 1;
    c128* p0 = B.part + ((int64_t)c0 * B.nchunk + blockIdx.x) * 2;
    p0[0] = s[0];
    p0[1] = s[1];
    if (c1 < B.R) {
      c128* p1 = B.part + ((int64_t)c1 * B.nchunk + blockIdx.x) * 2;
      p1[0] = s[2];
      p1[1] = s[3];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(B.counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}
__device__ __forceinline__ bool bp_act(const BmPtr& B, int c) { return c < B.R && B.active[c]; }
__device__ __forceinline__ c64 bp_sc(const BmPtr& B, const c128* v, int c) {
  return bp_act(B, c) ? ccast<float>(v[c]) : mkc(0.f, 0.f);
}

// p = r + beta (p - omega v), or p = r and rh = r for a (re)started incidence (SMODE false);
// s = r - alpha v (SMODE true).
template <bool SMODE>
__global__ void __launch_bounds__(256) k_bp_dir(BmPtr B, const c64* __restrict__ Rv, c64* __restrict__ Rh,
                                                const c64* __restrict__ Pv, const c64* __restrict__ Vv,
                                                c64* __restrict__ Out) {
  const BpRow t = bp_row(B);
  const int c0 = 2 * t.q, c1 = c0 + 1;
  const bool a0 = bp_act(B, c0), a1 = bp_act(B, c1);
  if (!t.valid || (!a0 && !a1)) return;
  const int xst = B.xst;
  if (SMODE) {
    const c64 al0 = bp_sc(B, B.alpha, c0), al1 = bp_sc(B, B.alpha, c1);
#pragma unroll 4
    for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
      const int64_t o = n * xst + c0;
      const float4 r = ld4(Rv + o), v = ld4(Vv + o);
      st4(Out + o, f4(lo(r) - al0 * lo(v), hi(r) - al1 * hi(v)));
    }
    return;
  }
  const bool f0 = a0 && B.fresh[c0], f1 = a1 && B.fresh[c1];
  // a fresh half takes beta = 0 (p = r); its rh is set to r
  const c64 be0 = f0 ? mkc(0.f, 0.f) : bp_sc(B, B.beta, c0), be1 = f1 ? mkc(0.f, 0.f) : bp_sc(B, B.beta, c1);
  const c64 om0 = bp_sc(B, B.omega, c0), om1 = bp_sc(B, B.omega, c1);
#pragma unroll 4
  for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
    const int64_t o = n * xst + c0;
    const float4 r = ld4(Rv + o), p = ld4(Pv + o), v = ld4(Vv + o);
    st4(Out + o, f4(lo(r) + be0 * (lo(p) - om0 * lo(v)), hi(r) + be1 * (hi(p) - om1 * hi(v))));
    if (f0 && f1) {
      st4(Rh + o, r);
    } else if (f0) {
      Rh[o] = lo(r);
    } else if (f1) {
      Rh[o + 1] = hi(r);
    }
  }
}

// alpha = rho / (rh^H v)
__global__ void __launch_bounds__(256) k_bp_rv(BmPtr B, const c64* __restrict__ Rh, const c64* __restrict__ Vv) {
  const BpRow t = bp_row(B);
  const int c0 = 2 * t.q, c1 = c0 + 1;
  const bool on = t.valid && (bp_act(B, c0) || bp_act(B, c1));
  c64 x0 = mkc(0.f, 0.f), x1 = x0;
  if (on)
#pragma unroll 4
    for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
      const int64_t o = n * B.xst + c0;
      const float4 h = ld4(Rh + o), v = ld4(Vv + o);
      bi_acc(x0, lo(h), lo(v));
      bi_acc(x1, hi(h), hi(v));
    }
  const c128 z = mkc(0.0, 0.0);
  if (!bp_reduce(B, t, ccast<double>(x0), z, ccast<double>(x1), z)) return;
  bm_finish(B, [&](int r, c128 rv, c128) {
    if (!B.active[r]) return;
    B.fresh[r] = 0;
    if (!finite_z(rv)) {
      bm_stop(B, r, true);
    } else if (rv.re == 0.0 && rv.im == 0.0) {
      bm_stop(B, r, false);  // breakdown: the true-residual check restarts it
    } else {
      B.alpha[r] = bi_cdiv(B.rho[r], rv);
    }
  });
}

// omega = (t^H s) / (t^H t)
__global__ void __launch_bounds__(256) k_bp_ts(BmPtr B, const c64* __restrict__ Tv, const c64* __restrict__ Sv) {
  const BpRow t = bp_row(B);
  const int c0 = 2 * t.q, c1 = c0 + 1;
  const bool on = t.valid && (bp_act(B, c0) || bp_act(B, c1));
  c64 x0 = mkc(0.f, 0.f), x1 = x0;
  float y0 = 0.f, y1 = 0.f;
  if (on)
#pragma unroll 4
    for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
      const int64_t o = n * B.xst + c0;
      const float4 tv = ld4(Tv + o), sv = ld4(Sv + o);
      bi_acc(x0, lo(tv), lo(sv));
      bi_acc(x1, hi(tv), hi(sv));
      bi_nrm(y0, lo(tv));
      bi_nrm(y1, hi(tv));
    }
  if (!bp_reduce(B, t, ccast<double>(x0), mkc((double)y0, 0.0), ccast<double>(x1), mkc((double)y1, 0.0))) return;
  bm_finish(B, [&](int r, c128 sts, c128 stt) {
    if (!B.active[r]) return;
    if (!finite_z(sts) || !isfinite(stt.re)) {
      bm_stop(B, r, true);
      return;
    }
    B.omega[r] = stt.re > 0.0 ? (1.0 / stt.re) * sts : mkc(0.0, 0.0);
  });
}

// y += alpha p + omega s, r = s - omega t for the active halves (an inactive half keeps y, whose
// scalars are zero, and r, which is not written); rho' = rh^H r and |r| decide the next step
__global__ void __launch_bounds__(256) k_bp_xr(BmPtr B, c64* __restrict__ Y, c64* __restrict__ Rv,
                                               const c64* __restrict__ Rh, const c64* __restrict__ Pv,
                                               const c64* __restrict__ Sv, const c64* __restrict__ Tv) {
  const BpRow t = bp_row(B);
  const int c0 = 2 * t.q, c1 = c0 + 1;
  const bool a0 = bp_act(B, c0), a1 = bp_act(B, c1);
  const bool on = t.valid && (a0 || a1);
  c64 x0 = mkc(0.f, 0.f), x1 = x0;
  float y0 = 0.f, y1 = 0.f;
  if (on) {
    const c64 al0 = bp_sc(B, B.alpha, c0), al1 = bp_sc(B, B.alpha, c1);
    const c64 om0 = bp_sc(B, B.omega, c0), om1 = bp_sc(B, B.omega, c1);
#pragma unroll 4
    for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
      const int64_t o = n * B.xst + c0;
      const float4 y = ld4(Y + o), p = ld4(Pv + o), s = ld4(Sv + o), tv = ld4(Tv + o), h = ld4(Rh + o);
      st4(Y + o, f4(lo(y) + al0 * lo(p) + om0 * lo(s), hi(y) + al1 * hi(p) + om1 * hi(s)));
      const c64 r0 = lo(s) - om0 * lo(tv), r1 = hi(s) - om1 * hi(tv);
      if (a0 && a1) {
        st4(Rv + o, f4(r0, r1));
      } else if (a0) {
        Rv[o] = r0;
      } else {
        Rv[o + 1] = r1;
      }
      bi_acc(x0, lo(h), r0);
      bi_acc(x1, hi(h), r1);
      bi_nrm(y0, r0);
      bi_nrm(y1, r1);
    }
  }
  if (!bp_reduce(B, t, ccast<double>(x0), mkc((double)y0, 0.0), ccast<double>(x1), mkc((double)y1, 0.0))) return;
  bm_finish(B, [&](int r, c128 shr, c128 srr) {
    if (!B.active[r]) return;
    const int it = ++B.its[r];
    const double rel = B.bnorm[r] > 0.0 ? sqrt(srr.re) / B.bnorm[r] : 0.0;
    B.resid[r] = rel;
    const c128 om64 = B.omega[r];
    if (!finite_z(shr) || !isfinite(rel)) {
      bm_stop(B, r, true);
    } else if (rel <= B.tol || it >= B.max_iter || (om64.re == 0.0 && om64.im == 0.0) ||
               (shr.re == 0.0 && shr.im == 0.0)) {
      bm_stop(B, r, false);  // converged by the recursion, out of steps, or a breakdown
    } else {
      B.beta[r] = bi_cdiv(shr, B.rho[r]) * bi_cdiv(B.alpha[r], om64);
      B.rho[r] = shr;
    }
  });
}

// True residual check: r holds b - A y; incidences above tol with steps left restart from it.
__global__ void __launch_bounds__(256) k_bp_check(BmPtr B, const c64* __restrict__ Rv) {
  const BpRow t = bp_row(B);
  const int c0 = 2 * t.q;
  float y0 = 0.f, y1 = 0.f;
  if (t.valid)
#pragma unroll 4
    for (int64_t n = t.n0 + t.rl; n < t.n1; n += t.nrl) {
      const float4 r = ld4(Rv + n * B.xst + c0);
      bi_nrm(y0, lo(r));
      bi_nrm(y1, hi(r));
    }
  const c128 z = mkc(0.0, 0.0);
  if (!bp_reduce(B, t, mkc((double)y0, 0.0), z, mkc((double)y1, 0.0), z)) return;
  bm_finish(B, [&](int r, c128 srr, c128) {
    const double rel = B.bnorm[r] > 0.0 ? sqrt(srr.re) / B.bnorm[r] : 0.0;
    B.resid[r] = rel;
    if (!isfinite(rel)) {
      B.active[r] = 0;
      B.st->numeric = 1;
    } else if (rel > B.tol && B.its[r] < B.max_iter) {
      B.active[r] = 1;
      B.fresh[r] = 1;
      B.rho[r] = mkc(srr.re, 0.0);
      atomicAdd(&B.st->nactive, 1);
    } else {
      B.active[r] = 0;
    }
  });
}

// Incidence-minor [N][xst] to incidence-major [R][N] through shared-memory tiles of T rows.
__global__ void __launch_bounds__(256) k_minor_to_major(int64_t N, int R, int xst, int T, const c64* __restrict__ X,
                                                        c64* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char sm_mm[];
  c64* tile = reinterpret_cast<c64*>(sm_mm);  // [T][xst + 1]
  const int ts = xst + 1;
  const int64_t n0 = (int64_t)blockIdx.x * T;
  const int cnt = (int)min((int64_t)T, N - n0);
  const c64* in = X + n0 * xst;
  for (int e = threadIdx.x; e < cnt * xst; e += blockDim.x) tile[(e / xst) * ts + e % xst] = in[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nwp = blockDim.x >> 5;
  for (int r = wp; r < R; r += nwp)
    for (int t = lane; t < cnt; t += 32) Y[(int64_t)r * N + n0 + t] = tile[t * ts + r];
}

int bicgstab_minor(swm_ctx* ctx, const c64* E, double tol, int max_iter) {
  SWM_TRY(build_wire_order(ctx));  // the order of product form 75, once per pattern
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  const int64_t nsm = std::max(ctx->nsm, 1);
  const int xst = R + (R & 1);
  struct Workspace {
    int64_t key[4];
    BmPtr B;
    KState* kst;
    int* pact;
    c64 *Y, *Rv, *Rh, *Pv, *Vv, *Sv, *Tv, *Bt;
  };
  const int64_t key[4] = {R, N, (int64_t)sizeof(float), -4};
  Workspace* ws = reinterpret_cast<Workspace*>(ctx->kry_ws);
  const size_t vbytes = sizeof(c64) * (size_t)xst * N;
  if (!ws || ctx->kry_ws_bytes != sizeof(Workspace) || std::memcmp(ws->key, key, sizeof(key)) != 0) {
    dfree_group(ctx, ctx->kry_bufs);
    std::free(ctx->kry_ws);
    ctx->kry_ws = nullptr;
    ws = reinterpret_cast<Workspace*>(std::calloc(1, sizeof(Workspace)));
    if (!ws) return ctx->fail(SWM_ENOMEM, "host allocation failed");
    ctx->kry_ws = ws;
    ctx->kry_ws_bytes = sizeof(Workspace);
    std::memcpy(ws->key, key, sizeof(key));
    auto& K = ctx->kry_bufs;
    BmPtr B{};
    B.N = N;
    B.R = R;
    B.xst = xst;
    // chunks of rows: about bicg_ctas (4) CTAs per SM, at least 2048 rows each
    B.chunk = (int)std::max<int64_t>(2048, ceil_div(N, (int64_t)ctx->bicg_ctas * nsm));
    B.nchunk = (int)ceil_div(N, B.chunk);
    SWM_TRY(dalloc(ctx, K, (void**)&B.st, sizeof(BState)));
    SWM_TRY(dalloc(ctx, K, (void**)&B.active, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.fresh, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.its, sizeof(int) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.counter, sizeof(unsigned)));
    SWM_TRY(dalloc(ctx, K, (void**)&B.bnorm, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.resid, sizeof(double) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.rho, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.alpha, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.omega, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.beta, sizeof(c128) * R));
    SWM_TRY(dalloc(ctx, K, (void**)&B.part, sizeof(c128) * 2 * (size_t)R * B.nchunk));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->kst, sizeof(KState)));
    SWM_TRY(dalloc(ctx, K, (void**)&ws->pact, sizeof(int) * R));
    c64** vecs[8] = {&ws->Y, &ws->Rv, &ws->Rh, &ws->Pv, &ws->Vv, &ws->Sv, &ws->Tv, &ws->Bt};
    for (auto v : vecs) {
      SWM_TRY(dalloc(ctx, K, (void**)v, vbytes));
      // the padding column (odd R) is read by the product as a second incidence: zero, and never
      // written with anything but the product of zeros
      SWM_CK(cudaMemsetAsync(*v, 0, vbytes, st));
    }
    ws->B = B;
  }
  BmPtr B = ws->B;
  B.tol = tol;
  B.max_iter = max_iter;
  c64 *Y = ws->Y, *Rv = ws->Rv, *Rh = ws->Rh, *Pv = ws->Pv, *Vv = ws->Vv, *Sv = ws->Sv, *Tv = ws->Tv, *Bt = ws->Bt;
  SWM_TRY(ensure_poll_slots(ctx));
  KPtr P{};
  P.N = N;
  P.R = R;
  P.st = ws->kst;
  P.active = B.active;
  KPtr Pall = P;
  Pall.active = ws->pact;
  k_bi_init<<<(unsigned)ceil_div(R, 256), 256, 0, st>>>(ws->kst, ws->pact, R);
  SWM_LAUNCHED();
  SWM_CK(cudaMemsetAsync(B.st, 0, sizeof(BState), st));
  SWM_CK(cudaMemsetAsync(B.its, 0, sizeof(int) * R, st));
  SWM_CK(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), st));
  SWM_CK(cudaMemsetAsync(B.active, 0, sizeof(int) * R, st));
  SWM_TRY(norms_of_b(ctx, ctx->Bv, false, B.bnorm));
  // b and the start y0 (zero, or M x0 for a guess) to incidence-minor order
  const int T = std::max(8, std::min(64, (int)((48 * 1024 / sizeof(c64)) / (xst + 1)) / 8 * 8));
  const size_t tsm = sizeof(c64) * T * (xst + 1);
  const unsigned gT = (unsigned)ceil_div(N, T);
  k_rhs_minor_all<float, true><<<gT, 256, tsm, st>>>(Pall, (const c64*)ctx->Bv, Bt, xst, T);
  SWM_LAUNCHED();
  if (ctx->guess) {
    // y0 in incidence-major order in Vv's storage first
    SWM_TRY(init_y(ctx, Vv, false));
    k_rhs_minor_all<float, true><<<gT, 256, tsm, st>>>(Pall, Vv, Y, xst, T);
    SWM_LAUNCHED();
  } else {
    SWM_CK(cudaMemsetAsync(Y, 0, vbytes, st));
  }
  SWM_TRY(allow_wm<c64>(ctx));
  const int RQ = std::min(32, (int)ceil_div(R, 2));
  const int WBp = std::max(1, std::min(kWpMaxWires, 256 / RQ));
  int form = 71;
  // v = A u (active incidences) or, RS, v = b - A u (every incidence): u is its own gathered copy
  auto product = [&](cudaStream_t s, const c64* src, c64* dst, auto res_tag) -> int {
    constexpr bool RS = decltype(res_tag)::value;
    SWM_TRY((launch_wm<c64, RS, true>(s, form, RS ? Pall : P, ctx, E, src, src, xst, dst, Bt, RQ, WBp)));
    SWM_LAUNCHED();
    return SWM_OK;
  };
  {
    const int64_t shape[6] = {N, R, (int64_t)sizeof(float), (int64_t)sizeof(c64), -4, 0};
    int found = 0;
    for (const auto& t : ctx->tuned)
      if (std::memcmp(t.shape, shape, sizeof(shape)) == 0) found = t.rb;
    if (ctx->product_form >= 68 && ctx->product_form <= 75) {
      form = ctx->product_form;
    } else if (found) {
      form = found;
    } else {
      // each shape once untimed and once timed on b (the product is idempotent)
      cudaEvent_t e0, e1;
      SWM_CK(cudaEventCreate(&e0));
      SWM_CK(cudaEventCreate(&e1));
      float best = 0.f;
      for (int f : {68, 69, 70, 71, 72, 73, 74, 75}) {
        form = f;
        SWM_TRY(product(st, Bt, Vv, std::true_type{}));
        SWM_CK(cudaEventRecord(e0, st));
        SWM_TRY(product(st, Bt, Vv, std::true_type{}));
        SWM_CK(cudaEventRecord(e1, st));
        SWM_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        SWM_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (best == 0.f || ms < best) {
          best = ms;
          found = f;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      form = found;
      swm_ctx::Tuned t{};
      std::memcpy(t.shape, shape, sizeof(shape));
      t.rb = form;
      ctx->tuned.push_back(t);
    }
  }
  ctx->stats.step_rhs_block = form;
  const unsigned gC = (unsigned)B.nchunk;
  auto launch_steps = [&](cudaStream_t s, int n) -> int {
    for (int i = 0; i < n; ++i) {
      ctx->prof_begin(SWM_K_TRANSPOSE);
      k_bp_dir<false><<<gC, 256, 0, s>>>(B, Rv, Rh, Pv, Vv, Pv);
      ctx->prof_end(SWM_K_TRANSPOSE);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_APPLY);
      SWM_TRY(product(s, Pv, Vv, std::false_type{}));
      ctx->prof_end(SWM_K_APPLY);
      ctx->prof_begin(SWM_K_DOTS);
      k_bp_rv<<<gC, 256, 0, s>>>(B, Rh, Vv);
      ctx->prof_end(SWM_K_DOTS);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_TRANSPOSE);
      k_bp_dir<true><<<gC, 256, 0, s>>>(B, Rv, Rh, Pv, Vv, Sv);
      ctx->prof_end(SWM_K_TRANSPOSE);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_APPLY);
      SWM_TRY(product(s, Sv, Tv, std::false_type{}));
      ctx->prof_end(SWM_K_APPLY);
      ctx->prof_begin(SWM_K_DOTS);
      k_bp_ts<<<gC, 256, 0, s>>>(B, Tv, Sv);
      ctx->prof_end(SWM_K_DOTS);
      SWM_LAUNCHED();
      ctx->prof_begin(SWM_K_UPDATE);
      k_bp_xr<<<gC, 256, 0, s>>>(B, Y, Rv, Rh, Pv, Sv, Tv);
      ctx->prof_end(SWM_K_UPDATE);
      SWM_LAUNCHED();
    }
    return SWM_OK;
  };
  auto check = [&]() -> int {
    ctx->prof_begin(SWM_K_APPLY);
    SWM_TRY(product(st, Y, Rv, std::true_type{}));
    ctx->prof_end(SWM_K_APPLY);
    k_bp_check<<<gC, 256, 0, st>>>(B, Rv);
    SWM_LAUNCHED();
    return SWM_OK;
  };
  constexpr int kChunk = 4;
  const bool use_graph = ctx->prof_cls != SWM_K_APPLY && ctx->prof_cls != SWM_K_DOTS &&
                         ctx->prof_cls != SWM_K_UPDATE && ctx->prof_cls != SWM_K_TRANSPOSE;
  if (use_graph) {
    struct Key {
      BmPtr B;
      const void* ptr[11];
      Layout lay;
      int64_t bits;
    } gk;
    std::memset(&gk, 0, sizeof(gk));
    gk.B = B;
    const void* ptrs[11] = {E, Y, Rv, Rh, Pv, Vv, Sv, Tv, Bt, ctx->off, ws->kst};
    for (int i = 0; i < 11; ++i) gk.ptr[i] = ptrs[i];
    gk.lay = ctx->offd;
    gk.bits = -(int64_t)(1000 + form);
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&gk);
    std::vector<unsigned char> kv(kb, kb + sizeof(gk));
    if (!ctx->gm_exec || kv != ctx->gm_key) {
      if (!ctx->cap_stream) SWM_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
      const int64_t launches0 = ctx->launches;
      SWM_CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = launch_steps(ctx->cap_stream, kChunk);
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
  const int launches_per_step = 7;
  KState* slot = reinterpret_cast<KState*>(ctx->pinned_state);
  BState hs{};
  int restarts = 0;
  for (;;) {
    SWM_TRY(check());
    BState* hpin = reinterpret_cast<BState*>(static_cast<char*>(ctx->pinned_state) + kPersistStateOffset);
    SWM_CK(cudaMemcpyAsync(hpin, B.st, sizeof(BState), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    hs = *hpin;
    if (hs.nactive <= 0 || hs.numeric) break;
    ++restarts;
    // chunks of steps; the host reads the count of chunk c - 1 while chunk c is queued.  Each
    // incidence stops by itself after at most max_iter steps, so the loop ends.
    for (int c = 0;; ++c) {
      if (use_graph) {
        SWM_CK(cudaGraphLaunch(ctx->gm_exec, st));
        ctx->launches += launches_per_step * kChunk;
      } else {
        SWM_TRY(launch_steps(st, kChunk));
      }
      SWM_CK(cudaMemcpyAsync(&slot[c & 1], B.st, sizeof(BState), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaEventRecord(ctx->poll_ev[c & 1], st));
      if (c >= 1) {
        SWM_CK(cudaEventSynchronize(ctx->poll_ev[(c - 1) & 1]));
        const BState* b = reinterpret_cast<const BState*>(&slot[(c - 1) & 1]);
        if (b->nactive <= 0 || b->numeric) break;
      }
    }
  }
  // y back to incidence-major order (in Vv's storage), then x = M^-1 y
  k_minor_to_major<<<gT, 256, tsm, st>>>(N, R, xst, T, Y, Vv);
  SWM_LAUNCHED();
  SWM_TRY(apply_minv(ctx, Vv));
  std::vector<double> res(R);
  std::vector<int> its(R);
  SWM_CK(cudaMemcpyAsync(res.data(), B.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaMemcpyAsync(its.data(), B.its, sizeof(int) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaStreamSynchronize(st));
  double mx = 0.0;
  int itmax = 0;
  for (int r = 0; r < R; ++r) {
    mx = std::max(mx, res[r]);
    itmax = std::max(itmax, its[r]);
  }
  ctx->stats.iterations = itmax;
  ctx->stats.restarts = std::max(0, restarts - 1);
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = (!hs.numeric && mx <= tol) ? 1 : 0;
  if (hs.numeric) return ctx->fail(SWM_ECUDA, "BiCGSTAB produced a non-finite value");
  return ctx->stats.converged ? SWM_OK : SWM_ENOTCONV;
}

}  // namespace

template <typename TV>
__global__ void k_init_y(int64_t n, const c128* __restrict__ g, cplx<TV>* __restrict__ Y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) Y[i] = ccast<TV>(g[i]);
}

// |b_r| per right-hand side (one CTA each, float64), 1 for a zero right-hand side.
// |b| per right-hand side in two deterministic passes: partial sums of kBnormRows rows per CTA,
// then the partials of each right-hand side added in order (|b| = 0 is stored as 1).
constexpr int kBnormRows = 65536;
template <typename TV>
__global__ void __launch_bounds__(256) k_bnorm_part(int64_t N, const cplx<TV>* __restrict__ B, double* __restrict__ part) {
  const int r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * kBnormRows, n1 = min(N, n0 + kBnormRows);
  const cplx<TV>* b = B + (int64_t)r * N;
  double s = 0.0;
  for (int64_t n = n0 + threadIdx.x; n < n1; n += 256) {
    const cplx<TV> v = b[n];
    s += (double)v.re * v.re + (double)v.im * v.im;
  }
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[(int64_t)r * gridDim.x + blockIdx.x] = t;
  }
}
__global__ void k_bnorm_fin(int nchunk, const double* __restrict__ part, double* __restrict__ out) {
  const int r = blockIdx.x;
  const double t = sum_partials_d(part + (int64_t)r * nchunk, nchunk, threadIdx.x);
  if (threadIdx.x == 0) out[r] = t > 0.0 ? sqrt(t) : 1.0;
}

int norms_of_b(swm_ctx* ctx, const void* B, bool f64, double* bnorm_dev) {
  const int64_t N = ctx->N;
  const int R = ctx->n_rhs;
  const int nchunk = (int)std::max<int64_t>(1, ceil_div(N, kBnormRows));
  std::vector<Buf> tmp;
  double* part = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&part, sizeof(double) * (size_t)nchunk * R));
  const dim3 g((unsigned)nchunk, (unsigned)R);
  if (f64)
    k_bnorm_part<double><<<g, 256, 0, ctx->stream>>>(N, (const c128*)B, part);
  else
    k_bnorm_part<float><<<g, 256, 0, ctx->stream>>>(N, (const c64*)B, part);
  SWM_LAUNCHED();
  k_bnorm_fin<<<(unsigned)R, 32, 0, ctx->stream>>>(nchunk, part, bnorm_dev);
  SWM_LAUNCHED();
  dfree_group(ctx, tmp);  // stream order makes the reuse of the scratch safe
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

int finish_solve(swm_ctx* ctx) {
  ctx->pend.active = false;
  KState hs{};
  SWM_TRY(persist_result(ctx, &hs, ctx->pend.sync_clean));
  const double* rpin = reinterpret_cast<const double*>(static_cast<const char*>(ctx->pinned_state) +
                                                       kPinnedResidOffset);
  double mx = 0.0;
  for (int r = 0; r < ctx->pend.R; ++r) mx = std::max(mx, rpin[r]);
  ctx->stats.iterations = hs.iters;
  ctx->stats.restarts = hs.cycles;
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = hs.all_conv ? 1 : 0;
  if (hs.numeric) return ctx->fail(SWM_ECUDA, "GMRES produced a non-finite value");
  return hs.all_conv ? SWM_OK : SWM_ENOTCONV;
}

int gmres_solve(swm_ctx* ctx, double tol, int restart, int max_iter) {
  if (ctx->prec == SWM_C128)
    return gmres_impl<double, c128>(ctx, (const c128*)ctx->Zp, tol, restart, max_iter, nullptr, nullptr);
  return gmres_impl<float, c64>(ctx, (const c64*)ctx->Zp, tol, restart, max_iter, nullptr, nullptr);
}

int bicgstab_solve(swm_ctx* ctx, double tol, int max_iter) {
  if (ctx->prec == SWM_C128) return bicgstab_impl<double, c128>(ctx, (const c128*)ctx->Zp, tol, max_iter);
  // complex64 with 2 to 256 incidences: the vectors incidence-minor (the headline's form)
  if (ctx->n_rhs >= 2 && ctx->n_rhs <= 256 && !ctx->bicg_major)
    return bicgstab_minor(ctx, (const c64*)ctx->Zp, tol, max_iter);
  return bicgstab_impl<float, c64>(ctx, (const c64*)ctx->Zp, tol, max_iter);
}

int residual_f64_wire(swm_ctx* ctx, const c128* B, const c128* Y, c128* Rr, c128* Yt) {
  KPtr P{};
  P.R = ctx->n_rhs;
  P.N = ctx->N;
  const WireTile wt = wire_tile(P.R, ctx->nw);
  if (Yt) {
    // y right-hand-side minor first, so that the gathers of a wire's threads are contiguous
    k_rhs_minor<double, true><<<dim3((unsigned)ceil_div(P.N, 32), (unsigned)ceil_div(P.R, 32)), 256, 0,
                                ctx->stream>>>(P, Y, Yt);
    SWM_LAUNCHED();
    k_spmv_w<double, c64, kResW, true><<<dim3(wt.gx, wt.gy), 256, 0, ctx->stream>>>(
        P, ctx->off, ctx->offd, ctx->nw, (const c64*)ctx->Zp, Y, Yt, Rr, B, wt.RG, wt.WB);
  } else {
    k_spmv_w<double, c64, kResW, false><<<dim3(wt.gx, wt.gy), 256, 0, ctx->stream>>>(
        P, ctx->off, ctx->offd, ctx->nw, (const c64*)ctx->Zp, Y, nullptr, Rr, B, wt.RG, wt.WB);
  }
  SWM_LAUNCHED();
  return SWM_OK;
}

int product_f64(swm_ctx* ctx, int R, const c128* X, c128* Y) {
  KPtr P{};
  P.R = R;
  P.N = ctx->N;
  const WireTile wt = wire_tile(R, ctx->nw);
  if (ctx->prec == SWM_C128)
    k_spmv_w<double, c128, kPlainW, false><<<dim3(wt.gx, wt.gy), 256, 0, ctx->stream>>>(
        P, ctx->off, ctx->offd, ctx->nw, (const c128*)ctx->Zp, X, nullptr, Y, nullptr, wt.RG, wt.WB);
  else
    k_spmv_w<double, c64, kPlainW, false><<<dim3(wt.gx, wt.gy), 256, 0, ctx->stream>>>(
        P, ctx->off, ctx->offd, ctx->nw, (const c64*)ctx->Zp, X, nullptr, Y, nullptr, wt.RG, wt.WB);
  SWM_LAUNCHED();
  return SWM_OK;
}

int gmres_inner_bf16(swm_ctx* ctx, double tol, int restart, int max_iter, void** y_out, int* iters) {
  KState hs{};
  // the inner solve only needs a few digits: its basis is stored in half precision
  const int rc = gmres_impl<float, __nv_bfloat162, __half2>(ctx, (const __nv_bfloat162*)ctx->E16, tol, restart,
                                                            max_iter, y_out, &hs);
  *iters = hs.iters;
  return rc;
}

}  // namespace swm
