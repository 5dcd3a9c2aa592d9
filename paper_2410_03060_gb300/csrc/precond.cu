// Block-diagonal (block-Jacobi) preconditioner named with the solver after Eq. (neardef):
// M = blockdiag(Z_pp).  GMRES runs on the right-preconditioned operator Z M^-1 = I + E, where
// E_pq = Z_pq Z_qq^-1 for the kept off-diagonal blocks; E is stored (layout `offd`) so that each
// Krylov step is one block-sparse product plus the identity, and x = M^-1 y at the end.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {


// Gauss-Jordan inversion with partial pivoting of Z_pp in precision R, one warp per wire, the
// lanes spread over the (row, column) entries of each elimination step: the float64 form (a
// lane-per-column sweep would chain m float64 operations per lane, slow on GB300's float64 pipe).
template <typename R, typename TV>
__global__ void __launch_bounds__(128) k_invert_self_entries(int64_t nw, const int32_t* __restrict__ m,
                                                    const int64_t* __restrict__ diag_b, Layout lay,
                                                    const cplx<TV>* __restrict__ Z, const int64_t* __restrict__ moff,
                                                    cplx<TV>* __restrict__ Minv, int* __restrict__ singular) {
  __shared__ cplx<R> A[4][kMaxM][2 * kMaxM];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + wl;
  if (p >= nw) return;
  const int n = m[p];
  const int K = lay.K[p];
  const int64_t base = lay.rowbase[p] + lay.colpos[diag_b[p]];
  cplx<R>(*a)[2 * kMaxM] = A[wl];
  for (int e = lane; e < n * 2 * n; e += 32) {
    const int i = e / (2 * n), j = e % (2 * n);
    a[i][j] = j < n ? ccast<R>(Z[base + (int64_t)i * K + j]) : mkc<R>(j - n == i ? R(1) : R(0), R(0));
  }
  __syncwarp();
  for (int c = 0; c < n; ++c) {
    // pivot: largest |a[r][c]|, r >= c (ties: smallest r)
    R best = -1;
    int br = c;
    for (int r = c; r < n; ++r) {
      const R v = a[r][c].re * a[r][c].re + a[r][c].im * a[r][c].im;
      if (v > best) {
        best = v;
        br = r;
      }
    }
    if (best == R(0)) {
      if (lane == 0) atomicExch(singular, 1);
      return;
    }
    if (br != c) {
      for (int j = lane; j < 2 * n; j += 32) {
        const cplx<R> t = a[c][j];
        a[c][j] = a[br][j];
        a[br][j] = t;
      }
      __syncwarp();
    }
    const cplx<R> piv = a[c][c];
    const R den = piv.re * piv.re + piv.im * piv.im;
    const cplx<R> inv = mkc<R>(piv.re / den, -piv.im / den);
    __syncwarp();
    for (int j = lane; j < 2 * n; j += 32) a[c][j] = a[c][j] * inv;
    __syncwarp();
    for (int e = lane; e < n * 2 * n; e += 32) {
      const int r = e / (2 * n), j = e % (2 * n);
      if (r != c && j != c) a[r][j] = a[r][j] - a[r][c] * a[c][j];
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32)
      if (r != c) a[r][c] = mkc<R>(0, 0);
    __syncwarp();
  }
  const int64_t mo = moff[p];
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, j = e % n;
    Minv[mo + e] = ccast<TV>(a[i][n + j]);
  }
}

// The same inversion, float32 form: lane j owns column j of the augmented matrix [Z_pp | I]
// (2 m_p <= 30 columns) and sweeps the rows, so no lane divides indices; the pivot row is the
// warp's arg-max of |a[r][c]| (ties: smallest r).
template <typename R, typename TV>
__global__ void __launch_bounds__(128) k_invert_self(int64_t nw, const int32_t* __restrict__ m,
                                                    const int64_t* __restrict__ diag_b, Layout lay,
                                                    const cplx<TV>* __restrict__ Z, const int64_t* __restrict__ moff,
                                                    cplx<TV>* __restrict__ Minv, int* __restrict__ singular) {
  __shared__ cplx<R> A[4][kMaxM][2 * kMaxM];
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * 4 + wl;
  if (p >= nw) return;
  const int n = m[p];
  const int K = lay.K[p];
  const int64_t base = lay.rowbase[p] + lay.colpos[diag_b[p]];
  cplx<R>(*a)[2 * kMaxM] = A[wl];
  const int j = lane;
  const bool col = j < 2 * n;
  if (col)
    for (int i = 0; i < n; ++i)
      a[i][j] = j < n ? ccast<R>(Z[base + (int64_t)i * K + j]) : mkc<R>(j - n == i ? R(1) : R(0), R(0));
  __syncwarp();
  for (int c = 0; c < n; ++c) {
    // pivot: lane r (c <= r < n) offers |a[r][c]|^2; warp arg-max, smallest r on ties
    R v = R(-1);
    int br = lane;
    if (lane >= c && lane < n) v = a[lane][c].re * a[lane][c].re + a[lane][c].im * a[lane][c].im;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int b2 = __shfl_xor_sync(0xffffffffu, br, o);
      if (v2 > v || (v2 == v && b2 < br)) {
        v = v2;
        br = b2;
      }
    }
    if (!(v > R(0))) {
      if (lane == 0) atomicExch(singular, 1);
      return;
    }
    if (br != c && col) {
      const cplx<R> t = a[c][j];
      a[c][j] = a[br][j];
      a[br][j] = t;
    }
    __syncwarp();
    const cplx<R> piv = a[c][c];
    const R den = piv.re * piv.re + piv.im * piv.im;
    const cplx<R> inv = mkc<R>(piv.re / den, -piv.im / den);
    cplx<R> f[kMaxM];
#pragma unroll
    for (int r = 0; r < kMaxM; ++r) f[r] = r < n ? a[r][c] : mkc<R>(0, 0);  // column c before the sweep
    __syncwarp();
    if (col) {
      const cplx<R> pc = a[c][j] * inv;
      a[c][j] = pc;
#pragma unroll
      for (int r = 0; r < kMaxM; ++r)
        if (r < n && r != c) a[r][j] = a[r][j] - f[r] * pc;
    }
    __syncwarp();
  }
  const int64_t mo = moff[p];
  for (int e = lane; e < n * n; e += 32) {
    const int i = e / n, jj = e % n;
    Minv[mo + e] = ccast<TV>(a[i][n + jj]);
  }
}

// E_pq = Z_pq Minv_q for every kept block with q != p; one warp per block.
template <typename TV>
__global__ void k_form_E(int64_t nb, const int32_t* __restrict__ col, const int64_t* __restrict__ bt,
                         const int32_t* __restrict__ m, Layout full, Layout offd, const cplx<TV>* __restrict__ Z,
                         const int64_t* __restrict__ moff, const cplx<TV>* __restrict__ Minv, cplx<TV>* __restrict__ E) {
  const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;
  const int q = col[b];
  const int p = col[bt[b]];
  if (p == q) return;
  const int mp = m[p], mq = m[q];
  const int Kf = full.K[p], Ko = offd.K[p];
  const int64_t zb = full.rowbase[p] + full.colpos[b];
  const int64_t eb = offd.rowbase[p] + offd.colpos[b];
  const cplx<TV>* Mi = Minv + moff[q];
  for (int e = lane; e < mp * mq; e += 32) {
    const int i = e / mq, j = e % mq;
    cplx<TV> acc = mkc<TV>(0, 0);
    for (int l = 0; l < mq; ++l) cfma(acc, Z[zb + (int64_t)i * Kf + l], Mi[l * mq + j]);
    E[eb + (int64_t)i * Ko + j] = acc;
  }
}

}  // namespace

// M^-1, E and the singularity flag, allocated and cleared on the context's stream.
int precond_alloc(swm_ctx* ctx) {
  const size_t esz = ctx->prec == SWM_C128 ? sizeof(c128) : sizeof(c64);
  SWM_TRY(dalloc(ctx, ctx->build_bufs, &ctx->Minv, esz * std::max<int64_t>(1, ctx->nminv)));
  SWM_TRY(dalloc(ctx, ctx->build_bufs, &ctx->Zp, esz * std::max<int64_t>(1, ctx->offd.nval)));
  SWM_TRY(dalloc(ctx, ctx->build_bufs, (void**)&ctx->d_sing, sizeof(int)));
  SWM_CK(cudaMemsetAsync(ctx->d_sing, 0, sizeof(int), ctx->stream));
  return SWM_OK;
}

// M^-1 = blockdiag(Z_pp)^-1 from the self blocks, on stream s.
int precond_invert(swm_ctx* ctx, cudaStream_t s) {
  const int64_t nw = ctx->nw;
  const unsigned g1 = (unsigned)ceil_div(nw, 4);
  ctx->prof_begin(SWM_K_INVERT);
  if (ctx->prec == SWM_C128)
    k_invert_self_entries<double, double><<<g1, 128, 0, s>>>(nw, ctx->m, ctx->diag_b, ctx->full, (const c128*)ctx->Z,
                                                             ctx->minv_off, (c128*)ctx->Minv, ctx->d_sing);
  else
    k_invert_self<float, float><<<g1, 128, 0, s>>>(nw, ctx->m, ctx->diag_b, ctx->full, (const c64*)ctx->Z,
                                                   ctx->minv_off, (c64*)ctx->Minv, ctx->d_sing);
  ctx->prof_end(SWM_K_INVERT);
  SWM_LAUNCHED();
  return SWM_OK;
}

// E = Z M^-1 off the diagonal, on the context's stream (after the fill and the inversion).
int precond_form_E(swm_ctx* ctx) {
  const unsigned g2 = (unsigned)std::max<int64_t>(1, ceil_div(ctx->nb * 32, 256));
  ctx->prof_begin(SWM_K_FORM_E);
  if (ctx->prec == SWM_C128)
    k_form_E<double><<<g2, 256, 0, ctx->stream>>>(ctx->nb, ctx->col, ctx->bt, ctx->m, ctx->full, ctx->offd,
                                                  (const c128*)ctx->Z, ctx->minv_off, (const c128*)ctx->Minv,
                                                  (c128*)ctx->Zp);
  else
    k_form_E<float><<<g2, 256, 0, ctx->stream>>>(ctx->nb, ctx->col, ctx->bt, ctx->m, ctx->full, ctx->offd,
                                                 (const c64*)ctx->Z, ctx->minv_off, (const c64*)ctx->Minv,
                                                 (c64*)ctx->Zp);
  ctx->prof_end(SWM_K_FORM_E);
  SWM_LAUNCHED();
  return SWM_OK;
}

// E rounded to complex bfloat16 (round to nearest even), one __nv_bfloat162 per entry.
__global__ void k_to_bf16(int64_t n, const c64* __restrict__ src, __nv_bfloat162* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float22bfloat162_rn(make_float2(src[i].re, src[i].im));
}

int make_e16(swm_ctx* ctx) {
  const int64_t n = std::max<int64_t>(1, ctx->offd.nval);
  SWM_TRY(dalloc(ctx, ctx->build_bufs, &ctx->E16, sizeof(__nv_bfloat162) * n));
  if (ctx->offd.nval > 0) {
    k_to_bf16<<<(unsigned)ceil_div(ctx->offd.nval, 256), 256, 0, ctx->stream>>>(ctx->offd.nval, (const c64*)ctx->Zp,
                                                                                 (__nv_bfloat162*)ctx->E16);
    SWM_LAUNCHED();
  }
  return SWM_OK;
}

// The build's counters (fill evaluations, singular self block) to pinned memory; checked here, or
// inside swm_run after its last synchronisation.
int finish_build(swm_ctx* ctx) {
  SWM_TRY(ensure_poll_slots(ctx));
  char* pin = static_cast<char*>(ctx->pinned_state) + kBuildCountersOffset;
  SWM_CK(cudaMemcpyAsync(pin, ctx->d_evals, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(pin + 8, ctx->d_sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->fused) {
    ctx->build_check_pending = true;
    return SWM_OK;
  }
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  return finish_build_check(ctx);
}

int finish_build_check(swm_ctx* ctx) {
  const char* pin = static_cast<const char*>(ctx->pinned_state) + kBuildCountersOffset;
  unsigned long long evals = 0;
  int sing = 0;
  std::memcpy(&evals, pin, sizeof(evals));
  std::memcpy(&sing, pin + 8, sizeof(sing));
  ctx->stats.fill_evals = (int64_t)evals;
  if (sing) return ctx->fail(SWM_EINVAL, "a self block is singular (degenerate wire geometry?)");
  return SWM_OK;
}

}  // namespace swm
