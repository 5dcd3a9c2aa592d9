// Mixed-precision solve (precision SWM_BF16): float64 iterative refinement around GMRES whose
// products read E stored as complex bfloat16.
//
// The values are filled in float32 (complex64 Z, M^-1 and E = Z M^-1, as on the SWM_C64 path) and
// E is also kept rounded to complex bfloat16, which halves the bytes each inner product moves.
// Outer loop, in float64 vectors and arithmetic, on A = I + E with the complex64 E:
//   r = b - A y;  stop when |r| / |b| <= tol for every right-hand side;
//   solve A_bf16 d = r / |r| by GMRES (complex64 vectors) to a loose tolerance;  y += |r| d.
// The rounding of E to bfloat16 (relative 2^-9) only slows the contraction of the outer loop; the
// limit is the solution of the complex64-valued system, reached with float64 residuals.  Finally
// x = M^-1 y in float64 arithmetic, stored as complex64 for the RCS calls.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {

constexpr int kT = 256;
constexpr int kL = 8;              // lanes per scalar row in the product
constexpr double kInnerTol = 2e-3;  // about the bfloat16 rounding of E: a tighter inner solve gains nothing
constexpr double kInnerTolMax = 0.5;
constexpr int kMaxOuter = 40;

// r = b - (y + E y) in float64 (E complex64), partial sums of |r|^2 per chunk of rows.
__global__ void __launch_bounds__(kT) k_ir_residual(int64_t N, int chunk, const RowInfo* __restrict__ rinfo,
                                                    const int32_t* __restrict__ colmap, const c64* __restrict__ E,
                                                    const c128* __restrict__ B, const c128* __restrict__ Y,
                                                    c128* __restrict__ Rr, double* __restrict__ part) {
  const int r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * chunk;
  const int cnt = (int)min((int64_t)chunk, N - n0);
  const c128* y = Y + (int64_t)r * N;
  const int g = threadIdx.x / kL, sub = threadIdx.x % kL;
  double s = 0.0;
  for (int t0 = 0; t0 < cnt; t0 += kT / kL) {
    const int t = t0 + g;
    c128 acc = mkc(0.0, 0.0);
    if (t < cnt) {
      const RowInfo ri = rinfo[n0 + t];
      const int32_t* cm = colmap + ri.cmb;
      for (int c = sub; c < ri.K; c += kL) cfma(acc, ccast<double>(E[ri.vb + c]), y[cm[c]]);
    }
#pragma unroll
    for (int o = kL / 2; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (t < cnt && sub == 0) {
      const int64_t n = n0 + t;
      const c128 v = B[(int64_t)r * N + n] - (y[n] + acc);
      Rr[(int64_t)r * N + n] = v;
      s += v.re * v.re + v.im * v.im;
    }
  }
  __shared__ double red[kT / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kT / 32; ++i) t += red[i];
    part[(int64_t)r * gridDim.x + blockIdx.x] = t;
  }
}

// Partial sums of |r|^2 per chunk of rows (the residual formed by the wire-tiled product).
__global__ void __launch_bounds__(kT) k_ir_norms(int64_t N, int chunk, const c128* __restrict__ Rr,
                                                 double* __restrict__ part) {
  const int r = blockIdx.y;
  const int64_t n0 = (int64_t)blockIdx.x * chunk;
  const int cnt = (int)min((int64_t)chunk, N - n0);
  const c128* v = Rr + (int64_t)r * N + n0;
  double s = 0.0;
  for (int t = threadIdx.x; t < cnt; t += kT) {
    const c128 a = v[t];
    s += a.re * a.re + a.im * a.im;
  }
  __shared__ double red[kT / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kT / 32; ++i) t += red[i];
    part[(int64_t)r * gridDim.x + blockIdx.x] = t;
  }
}

// Right-hand side of the inner solve: complex64 r / |r| (0 for converged right-hand sides).
__global__ void k_ir_scale(int64_t N, const c128* __restrict__ Rr, const double* __restrict__ scale,
                           c64* __restrict__ Bv) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n < N) Bv[(int64_t)r * N + n] = ccast<float>(scale[r] * Rr[(int64_t)r * N + n]);
}

// y += |r| d (float64).
__global__ void k_ir_accumulate(int64_t N, const c64* __restrict__ D, const double* __restrict__ gain,
                                c128* __restrict__ Y) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n < N) Y[(int64_t)r * N + n] = Y[(int64_t)r * N + n] + gain[r] * ccast<double>(D[(int64_t)r * N + n]);
}

// x = M^-1 y in float64 arithmetic (M^-1 complex64), stored complex64.
__global__ void k_ir_minv(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                          const int32_t* __restrict__ m, const int64_t* __restrict__ moff, const c64* __restrict__ Minv,
                          const c128* __restrict__ Y, c64* __restrict__ X) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t o = off[p];
  const int i = (int)(n - o), mp = m[p];
  const c64* Mi = Minv + moff[p] + (int64_t)i * mp;
  const c128* y = Y + (int64_t)r * N + o;
  c128 acc = mkc(0.0, 0.0);
  for (int l = 0; l < mp; ++l) cfma(acc, ccast<double>(Mi[l]), y[l]);
  X[(int64_t)r * N + n] = ccast<float>(acc);
}

}  // namespace

int refine_solve(swm_ctx* ctx, const double* frames_dev, double tol, int restart, int max_iter) {
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  SWM_TRY(ensure_rowinfo(ctx));
  std::vector<Buf>& S = ctx->solve_bufs;
  c128 *B64 = nullptr, *Y64 = nullptr, *Rr = nullptr;
  double *part = nullptr, *dscale = nullptr, *dgain = nullptr;
  const int chunk = (int)std::max<int64_t>(kT, ceil_div(ceil_div(N, 512), kT) * kT);
  const int nchunk = (int)ceil_div(N, chunk);
  SWM_TRY(dalloc(ctx, S, (void**)&B64, sizeof(c128) * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&Y64, sizeof(c128) * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&Rr, sizeof(c128) * R * N));
  c128* Yt = nullptr;  // y right-hand-side minor for the residual's gathers (several right-hand sides)
  if (R > 1) SWM_TRY(dalloc(ctx, S, (void**)&Yt, sizeof(c128) * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&part, sizeof(double) * (size_t)R * nchunk));
  SWM_TRY(dalloc(ctx, S, (void**)&dscale, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&dgain, sizeof(double) * R));
  SWM_TRY(compute_rhs_f64(ctx, R, frames_dev, B64));
  SWM_TRY(init_y(ctx, Y64, true));
  const dim3 gres((unsigned)nchunk, (unsigned)R), gvec((unsigned)ceil_div(N, 256), (unsigned)R);
  std::vector<double> hp((size_t)R * nchunk), bn(R, 1.0), rn(R), rel(R), scale(R), gain(R);
  {
    // |b| per right-hand side: the residual of y = 0
    c128* y0 = nullptr;
    SWM_TRY(dalloc(ctx, S, (void**)&y0, sizeof(c128) * R * N));
    SWM_CK(cudaMemsetAsync(y0, 0, sizeof(c128) * R * N, st));
    k_ir_residual<<<gres, kT, 0, st>>>(N, chunk, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap, (const c64*)ctx->Zp,
                                       B64, y0, Rr, part);
    SWM_LAUNCHED();
    SWM_CK(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) {
      double t = 0.0;
      for (int c = 0; c < nchunk; ++c) t += hp[(size_t)r * nchunk + c];
      bn[r] = t > 0.0 ? std::sqrt(t) : 1.0;
    }
  }
  int total = 0, outer = 0, rc_inner = SWM_OK;
  bool conv = false;
  while (true) {
    ctx->prof_begin(SWM_K_APPLY);
    if (R > 1) {
      // several right-hand sides share each read of E (wire-tiled product), then the norms
      SWM_TRY(residual_f64_wire(ctx, B64, Y64, Rr, Yt));
      k_ir_norms<<<gres, kT, 0, st>>>(N, chunk, Rr, part);
    } else {
      k_ir_residual<<<gres, kT, 0, st>>>(N, chunk, (const RowInfo*)ctx->rowinfo, ctx->offd.colmap,
                                         (const c64*)ctx->Zp, B64, Y64, Rr, part);
    }
    ctx->prof_end(SWM_K_APPLY);
    SWM_LAUNCHED();
    SWM_CK(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    conv = true;
    for (int r = 0; r < R; ++r) {
      double t = 0.0;
      for (int c = 0; c < nchunk; ++c) t += hp[(size_t)r * nchunk + c];
      rn[r] = std::sqrt(t);
      rel[r] = rn[r] / bn[r];
      if (!std::isfinite(rel[r])) return ctx->fail(SWM_ECUDA, "refinement produced a non-finite residual");
      conv = conv && rel[r] <= tol;
    }
    if (conv || outer >= kMaxOuter || total >= max_iter) break;
    for (int r = 0; r < R; ++r) {
      const bool act = rel[r] > tol && rn[r] > 0.0;
      scale[r] = act ? 1.0 / rn[r] : 0.0;
      gain[r] = act ? rn[r] : 0.0;
    }
    SWM_CK(cudaMemcpyAsync(dscale, scale.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
    SWM_CK(cudaMemcpyAsync(dgain, gain.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
    k_ir_scale<<<gvec, 256, 0, st>>>(N, Rr, dscale, (c64*)ctx->Bv);
    SWM_LAUNCHED();
    void* d = nullptr;
    int its = 0;
    // the inner solve only has to bring the worst residual just below tol: no tighter than the
    // bfloat16 rounding allows, no looser than halving it
    double worst = 0.0;
    for (int r = 0; r < R; ++r) worst = std::max(worst, rel[r]);
    const double inner_tol = std::min(kInnerTolMax, std::max(kInnerTol, 0.5 * tol / worst));
    rc_inner = gmres_inner_bf16(ctx, inner_tol, restart, max_iter - total, &d, &its);
    if (rc_inner < 0) return rc_inner;
    total += its;
    k_ir_accumulate<<<gvec, 256, 0, st>>>(N, (const c64*)d, dgain, Y64);
    SWM_LAUNCHED();
    ++outer;
  }
  k_ir_minv<<<gvec, 256, 0, st>>>(N, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off, (const c64*)ctx->Minv, Y64,
                                  (c64*)ctx->Xv);
  SWM_LAUNCHED();
  SWM_CK(cudaStreamSynchronize(st));
  double mx = 0.0;
  for (double v : rel) mx = std::max(mx, v);
  ctx->stats.iterations = total;
  ctx->stats.restarts = outer;
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = conv ? 1 : 0;
  return conv ? SWM_OK : SWM_ENOTCONV;
}

}  // namespace swm
