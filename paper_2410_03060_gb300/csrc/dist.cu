// Building blocks of a Krylov solve driven from outside the library, one cloud split over ranks
// (each rank a context holding its own wires and a read-only halo of the neighbours' wires within
// r_c).  The S-NFC system couples only wires within r_c (Sec. II-B, Eq. neardef), so a rank's rows
// of the right-preconditioned operator A = Z M^-1 = I + E need the current vector on its own wires
// and on the halo only; the driver exchanges the halo values between products and sums the inner
// products and the far-field components over the ranks.  These entry points give it the product,
// the preconditioner, the right-hand side, the vector algebra of Gram-Schmidt and the far-field
// components, each on the context's device and stream, in float64 arithmetic and complex128
// vectors in the caller's unknown order.
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace swm {
namespace {

constexpr int kT = 256;

int dev_of(swm_ctx* ctx) {
  SWM_CK(cudaSetDevice(ctx->device));
  return SWM_OK;
}

// Caller [R][N] -> internal order (float64).
__global__ void k_user_to_internal(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                                   const int64_t* __restrict__ uoff, const c128* __restrict__ in,
                                   c128* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  out[(int64_t)r * N + n] = in[(int64_t)r * N + uoff[p] + (n - off[p])];
}

// Internal [R][N] -> caller order (float64).
__global__ void k_internal_to_user(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                                   const int64_t* __restrict__ uoff, const c128* __restrict__ in,
                                   c128* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  out[(int64_t)r * N + uoff[p] + (n - off[p])] = in[(int64_t)r * N + n];
}

// x = M^-1 y, the inverses of the self blocks applied wire by wire (internal order, float64
// arithmetic on the stored inverses).
template <typename TM>
__global__ void k_minv_f64(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ m, const int64_t* __restrict__ moff,
                           const cplx<TM>* __restrict__ Minv, const c128* __restrict__ Y, c128* __restrict__ X) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t o = off[p];
  const int i = (int)(n - o), mp = m[p];
  const cplx<TM>* Mi = Minv + moff[p] + (int64_t)i * mp;
  const c128* y = Y + (int64_t)r * N + o;
  c128 acc = mkc(0.0, 0.0);
  for (int l = 0; l < mp; ++l) cfma(acc, ccast<double>(Mi[l]), y[l]);
  X[(int64_t)r * N + n] = acc;
}

// Partial inner products out[c][i][r] = sum over the rows of chunk c of conj(Q[i][r][n]) v[r][n],
// chunks of kT * 8 rows; summed over the chunks in a fixed order by the host.
constexpr int kDotRows = kT * 8;
__global__ void __launch_bounds__(kT) k_vec_dots(int64_t n, int k, int R, const c128* __restrict__ Q,
                                                 const c128* __restrict__ v, c128* __restrict__ part) {
  const int ir = blockIdx.y;  // i * R + r
  const int r = ir % R;
  const int64_t n0 = (int64_t)blockIdx.x * kDotRows;
  const c128* q = Q + (int64_t)ir * n;
  const c128* w = v + (int64_t)r * n;
  double re = 0.0, im = 0.0;
  for (int64_t t = n0 + threadIdx.x; t < min(n, n0 + kDotRows); t += kT) {
    const c128 a = q[t], b = w[t];
    re += a.re * b.re + a.im * b.im;
    im += a.re * b.im - a.im * b.re;
  }
  __shared__ double sr[kT / 32], si[kT / 32];
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kT / 32; ++i) {
      a += sr[i];
      b += si[i];
    }
    part[(int64_t)blockIdx.x * k * R + ir] = mkc(a, b);
  }
}

// v[r] -= sum over i < k of coef[i][r] Q[i][r]  (coef on the device, k x R).
__global__ void k_vec_axpy(int64_t n, int k, int R, const c128* __restrict__ Q, const c128* __restrict__ coef,
                           c128* __restrict__ v) {
  const int r = blockIdx.y;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  c128 acc = v[(int64_t)r * n + t];
  for (int i = 0; i < k; ++i) {
    const c128 c = coef[(int64_t)i * R + r];
    const c128 q = Q[((int64_t)i * R + r) * n + t];
    acc.re -= c.re * q.re - c.im * q.im;
    acc.im -= c.re * q.im + c.im * q.re;
  }
  v[(int64_t)r * n + t] = acc;
}

// out[r] = a[r] v[r] (a real, on the device).
__global__ void k_vec_scale(int64_t n, const double* __restrict__ a, const c128* __restrict__ v,
                            c128* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const c128 x = v[(int64_t)r * n + t];
  out[(int64_t)r * n + t] = mkc(a[r] * x.re, a[r] * x.im);
}

// Block Gram matrix partials: part[c][a][b] = sum over the rows of chunk c of conj(Q[a][n]) W[b][n]
// for a < K, b < S, by 16 x 16 tiles (a CTA per chunk and tile); the chunk's rows are staged in
// shared memory 64 at a time and each thread accumulates one (a, b) entry.
constexpr int kGT = 16, kGRows = 64, kGChunk = 2048;
__global__ void __launch_bounds__(kGT* kGT) k_vec_gram(int64_t n, int K, int S, const c128* __restrict__ Q,
                                                       const c128* __restrict__ W, c128* __restrict__ part) {
  __shared__ c128 qs[kGT][kGRows + 1], ws[kGT][kGRows + 1];
  const int ta = blockIdx.y, tb = blockIdx.z;
  const int a = threadIdx.x / kGT, b = threadIdx.x % kGT;
  const int64_t n0 = (int64_t)blockIdx.x * kGChunk, n1 = min(n, n0 + kGChunk);
  double re = 0.0, im = 0.0;
  for (int64_t m0 = n0; m0 < n1; m0 += kGRows) {
    for (int e = threadIdx.x; e < kGT * kGRows; e += kGT * kGT) {
      const int row = e / kGRows, t = e % kGRows;
      const int64_t nn = m0 + t;
      const int ga = ta * kGT + row, gb = tb * kGT + row;
      qs[row][t] = (ga < K && nn < n1) ? Q[(int64_t)ga * n + nn] : mkc(0.0, 0.0);
      ws[row][t] = (gb < S && nn < n1) ? W[(int64_t)gb * n + nn] : mkc(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int t = 0; t < kGRows; ++t) {
      const c128 x = qs[a][t], y = ws[b][t];
      re += x.re * y.re + x.im * y.im;
      im += x.re * y.im - x.im * y.re;
    }
    __syncthreads();
  }
  const int ga = ta * kGT + a, gb = tb * kGT + b;
  if (ga < K && gb < S) part[((int64_t)blockIdx.x * K + ga) * S + gb] = mkc(re, im);
}

// W[b][n] -= sum over a < K of Q[a][n] C[a][b] (C on the device, K x S), 16 outputs per thread.
__global__ void k_vec_gemm(int64_t n, int K, int S, const c128* __restrict__ Q, const c128* __restrict__ C,
                           c128* __restrict__ W) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int b0 = blockIdx.y * kGT;
  if (t >= n) return;
  c128 acc[kGT];
#pragma unroll
  for (int b = 0; b < kGT; ++b) acc[b] = mkc(0.0, 0.0);
  for (int a = 0; a < K; ++a) {
    const c128 q = Q[(int64_t)a * n + t];
#pragma unroll
    for (int b = 0; b < kGT; ++b)
      if (b0 + b < S) cfma(acc[b], q, C[(int64_t)a * S + b0 + b]);
  }
#pragma unroll
  for (int b = 0; b < kGT; ++b)
    if (b0 + b < S) {
      c128& w = W[(int64_t)(b0 + b) * n + t];
      w = w - acc[b];
    }
}

bool is_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// In and out of the internal order through device scratch; host buffers are copied.
int to_internal(swm_ctx* ctx, std::vector<Buf>& tmp, int R, const double* in, int kind, c128** out) {
  const int64_t N = ctx->N;
  const c128* src = (const c128*)in;
  if (kind == SWM_HOST) {
    c128* d = nullptr;
    SWM_TRY(dalloc(ctx, tmp, (void**)&d, sizeof(c128) * R * N));
    SWM_CK(cudaMemcpyAsync(d, in, sizeof(c128) * R * N, cudaMemcpyHostToDevice, ctx->stream));
    src = d;
  }
  SWM_TRY(dalloc(ctx, tmp, (void**)out, sizeof(c128) * R * N));
  k_user_to_internal<<<dim3((unsigned)ceil_div(N, kT), R), kT, 0, ctx->stream>>>(N, ctx->rowwire, ctx->off,
                                                                                 ctx->uoff, src, *out);
  SWM_LAUNCHED();
  return SWM_OK;
}

int from_internal(swm_ctx* ctx, std::vector<Buf>& tmp, int R, const c128* in, double* out, int kind) {
  const int64_t N = ctx->N;
  c128* dst = (c128*)out;
  if (kind == SWM_HOST) SWM_TRY(dalloc(ctx, tmp, (void**)&dst, sizeof(c128) * R * N));
  k_internal_to_user<<<dim3((unsigned)ceil_div(N, kT), R), kT, 0, ctx->stream>>>(N, ctx->rowwire, ctx->off,
                                                                                 ctx->uoff, in, dst);
  SWM_LAUNCHED();
  if (kind == SWM_HOST)
    SWM_CK(cudaMemcpyAsync(out, dst, sizeof(c128) * R * N, cudaMemcpyDeviceToHost, ctx->stream));
  return SWM_OK;
}

int check_built(swm_ctx* ctx, int R, const void* a, const void* b, int ka, int kb, const char* who) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (!ctx->built) return ctx->fail(SWM_ESTATE, std::string(who) + " before swm_build");
  if (R < 1 || R > 65535 || !a || !b) return ctx->fail(SWM_EINVAL, std::string(who) + ": bad argument");
  if ((ka != SWM_HOST && ka != SWM_DEVICE) || (kb != SWM_HOST && kb != SWM_DEVICE))
    return ctx->fail(SWM_EINVAL, std::string(who) + ": bad memory kind");
  return SWM_OK;
}

}  // namespace
}  // namespace swm

using namespace swm;

extern "C" {

int swm_apply(swm_ctx* ctx, int n_rhs, const double* x, int x_kind, double* y, int y_kind) {
  SWM_TRY(check_built(ctx, n_rhs, x, y, x_kind, y_kind, "swm_apply"));
  SWM_TRY(dev_of(ctx));
  SWM_TRY(ensure_rowinfo(ctx));
  SWM_TRY(ensure_user_offsets(ctx));
  std::vector<Buf> tmp;
  c128 *xi = nullptr, *yi = nullptr;
  SWM_TRY(to_internal(ctx, tmp, n_rhs, x, x_kind, &xi));
  SWM_TRY(dalloc(ctx, tmp, (void**)&yi, sizeof(c128) * n_rhs * ctx->N));
  SWM_TRY(product_f64(ctx, n_rhs, xi, yi));
  SWM_TRY(from_internal(ctx, tmp, n_rhs, yi, y, y_kind));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int swm_precond_apply(swm_ctx* ctx, int n_rhs, const double* y, int y_kind, double* x, int x_kind) {
  SWM_TRY(check_built(ctx, n_rhs, y, x, y_kind, x_kind, "swm_precond_apply"));
  SWM_TRY(dev_of(ctx));
  SWM_TRY(ensure_rowinfo(ctx));
  SWM_TRY(ensure_user_offsets(ctx));
  std::vector<Buf> tmp;
  c128 *yi = nullptr, *xi = nullptr;
  SWM_TRY(to_internal(ctx, tmp, n_rhs, y, y_kind, &yi));
  SWM_TRY(dalloc(ctx, tmp, (void**)&xi, sizeof(c128) * n_rhs * ctx->N));
  const dim3 g((unsigned)ceil_div(ctx->N, kT), n_rhs);
  if (ctx->prec == SWM_C128)
    k_minv_f64<double><<<g, kT, 0, ctx->stream>>>(ctx->N, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off,
                                                  (const c128*)ctx->Minv, yi, xi);
  else
    k_minv_f64<float><<<g, kT, 0, ctx->stream>>>(ctx->N, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off,
                                                 (const c64*)ctx->Minv, yi, xi);
  SWM_LAUNCHED();
  SWM_TRY(from_internal(ctx, tmp, n_rhs, xi, x, x_kind));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int swm_rhs(swm_ctx* ctx, int n_inc, const double* inc, double* b_out, int out_kind) {
  SWM_TRY(check_built(ctx, n_inc, inc, b_out, SWM_HOST, out_kind, "swm_rhs"));
  for (int i = 0; i < 3 * n_inc; ++i)
    if (!std::isfinite(inc[i])) return ctx->fail(SWM_EINVAL, "swm_rhs: non-finite incidence angle");
  SWM_TRY(dev_of(ctx));
  SWM_TRY(ensure_rowinfo(ctx));
  SWM_TRY(ensure_user_offsets(ctx));
  std::vector<Buf> tmp;
  std::vector<double> fh;
  frames_host(inc, n_inc, fh);
  double* frames = nullptr;
  c128* bi = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&frames, sizeof(double) * fh.size()));
  SWM_CK(cudaMemcpyAsync(frames, fh.data(), sizeof(double) * fh.size(), cudaMemcpyHostToDevice, ctx->stream));
  SWM_TRY(dalloc(ctx, tmp, (void**)&bi, sizeof(c128) * n_inc * ctx->N));
  SWM_TRY(compute_rhs_f64(ctx, n_inc, frames, bi));
  SWM_TRY(from_internal(ctx, tmp, n_inc, bi, b_out, out_kind));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int swm_vec_dots(swm_ctx* ctx, int64_t n, int k, int n_rhs, const double* Q, const double* v, double* out) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (n < 0 || k < 1 || n_rhs < 1 || n_rhs > 65535 || (int64_t)k * n_rhs > 65535 || !Q || !v || !out)
    return ctx->fail(SWM_EINVAL, "swm_vec_dots: bad argument");
  if (!is_device(Q) || !is_device(v)) return ctx->fail(SWM_EINVAL, "swm_vec_dots: vectors must be device memory");
  SWM_TRY(dev_of(ctx));
  const int64_t nch = std::max<int64_t>(1, ceil_div(n, kDotRows));
  std::vector<Buf> tmp;
  c128* part = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&part, sizeof(c128) * nch * k * n_rhs));
  if (n > 0) {
    k_vec_dots<<<dim3((unsigned)nch, k * n_rhs), kT, 0, ctx->stream>>>(n, k, n_rhs, (const c128*)Q, (const c128*)v,
                                                                       part);
    SWM_LAUNCHED();
  } else {
    SWM_CK(cudaMemsetAsync(part, 0, sizeof(c128) * k * n_rhs, ctx->stream));
  }
  std::vector<c128> hp((size_t)nch * k * n_rhs);
  SWM_CK(cudaMemcpyAsync(hp.data(), part, sizeof(c128) * hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  for (int e = 0; e < k * n_rhs; ++e) {
    double re = 0.0, im = 0.0;
    for (int64_t c = 0; c < nch; ++c) {
      re += hp[(size_t)c * k * n_rhs + e].re;
      im += hp[(size_t)c * k * n_rhs + e].im;
    }
    out[2 * e] = re;
    out[2 * e + 1] = im;
  }
  return SWM_OK;
}

int swm_vec_axpy(swm_ctx* ctx, int64_t n, int k, int n_rhs, const double* Q, const double* coef, double* v) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (n < 0 || k < 1 || n_rhs < 1 || n_rhs > 65535 || !Q || !coef || !v)
    return ctx->fail(SWM_EINVAL, "swm_vec_axpy: bad argument");
  if (!is_device(Q) || !is_device(v)) return ctx->fail(SWM_EINVAL, "swm_vec_axpy: vectors must be device memory");
  if (n == 0) return SWM_OK;
  SWM_TRY(dev_of(ctx));
  std::vector<Buf> tmp;
  c128* cd = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&cd, sizeof(c128) * k * n_rhs));
  SWM_CK(cudaMemcpyAsync(cd, coef, sizeof(c128) * k * n_rhs, cudaMemcpyHostToDevice, ctx->stream));
  k_vec_axpy<<<dim3((unsigned)ceil_div(n, kT), n_rhs), kT, 0, ctx->stream>>>(n, k, n_rhs, (const c128*)Q, cd,
                                                                             (c128*)v);
  SWM_LAUNCHED();
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int swm_vec_scale(swm_ctx* ctx, int64_t n, int n_rhs, const double* a, const double* v, double* out) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (n < 0 || n_rhs < 1 || n_rhs > 65535 || !a || !v || !out)
    return ctx->fail(SWM_EINVAL, "swm_vec_scale: bad argument");
  if (!is_device(v) || !is_device(out)) return ctx->fail(SWM_EINVAL, "swm_vec_scale: vectors must be device memory");
  if (n == 0) return SWM_OK;
  SWM_TRY(dev_of(ctx));
  std::vector<Buf> tmp;
  double* ad = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&ad, sizeof(double) * n_rhs));
  SWM_CK(cudaMemcpyAsync(ad, a, sizeof(double) * n_rhs, cudaMemcpyHostToDevice, ctx->stream));
  k_vec_scale<<<dim3((unsigned)ceil_div(n, kT), n_rhs), kT, 0, ctx->stream>>>(n, ad, (const c128*)v, (c128*)out);
  SWM_LAUNCHED();
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

int swm_vec_gram(swm_ctx* ctx, int64_t n, int K, int S, const double* Q, const double* W, double* out) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (n < 0 || K < 1 || S < 1 || K > 65535 * kGT || S > 65535 * kGT || !Q || !W || !out)
    return ctx->fail(SWM_EINVAL, "swm_vec_gram: bad argument");
  if (!is_device(Q) || !is_device(W)) return ctx->fail(SWM_EINVAL, "swm_vec_gram: vectors must be device memory");
  SWM_TRY(dev_of(ctx));
  const int64_t nch = std::max<int64_t>(1, ceil_div(n, kGChunk));
  std::vector<Buf> tmp;
  c128* part = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&part, sizeof(c128) * nch * K * S));
  if (n > 0) {
    k_vec_gram<<<dim3((unsigned)nch, (unsigned)ceil_div(K, kGT), (unsigned)ceil_div(S, kGT)), kGT * kGT, 0,
                 ctx->stream>>>(n, K, S, (const c128*)Q, (const c128*)W, part);
    SWM_LAUNCHED();
  } else {
    SWM_CK(cudaMemsetAsync(part, 0, sizeof(c128) * K * S, ctx->stream));
  }
  std::vector<c128> hp((size_t)nch * K * S);
  SWM_CK(cudaMemcpyAsync(hp.data(), part, sizeof(c128) * hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  const int64_t KS = (int64_t)K * S;
  for (int64_t e = 0; e < KS; ++e) {
    double re = 0.0, im = 0.0;
    for (int64_t c = 0; c < nch; ++c) {
      re += hp[(size_t)(c * KS + e)].re;
      im += hp[(size_t)(c * KS + e)].im;
    }
    out[2 * e] = re;
    out[2 * e + 1] = im;
  }
  return SWM_OK;
}

int swm_vec_gemm(swm_ctx* ctx, int64_t n, int K, int S, const double* Q, const double* C, double* W) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (n < 0 || K < 1 || S < 1 || S > 65535 * kGT || !Q || !C || !W)
    return ctx->fail(SWM_EINVAL, "swm_vec_gemm: bad argument");
  if (!is_device(Q) || !is_device(W)) return ctx->fail(SWM_EINVAL, "swm_vec_gemm: vectors must be device memory");
  if (n == 0) return SWM_OK;
  SWM_TRY(dev_of(ctx));
  std::vector<Buf> tmp;
  c128* cd = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&cd, sizeof(c128) * K * S));
  SWM_CK(cudaMemcpyAsync(cd, C, sizeof(c128) * K * S, cudaMemcpyHostToDevice, ctx->stream));
  k_vec_gemm<<<dim3((unsigned)ceil_div(n, kT), (unsigned)ceil_div(S, kGT)), kT, 0, ctx->stream>>>(
      n, K, S, (const c128*)Q, cd, (c128*)W);
  SWM_LAUNCHED();
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

}  // extern "C"
