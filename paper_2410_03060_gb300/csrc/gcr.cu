// Restarted GCR (generalized conjugate residual) on the block-Jacobi right-preconditioned S-NFC
// system: the Krylov solver the paper names (Sec. II-B, after Eq. neardef: GCR with a
// block-diagonal preconditioner).  It works on A = Z M^-1 = I + E like the GMRES of krylov.cu and
// finds y with A y = b, x = M^-1 y.  One GCR step k, per right-hand side:
//   q = A r,  p = r                                    (search direction and its image)
//   q -= Q beta, p -= P beta, beta = Q^H q             (twice: classical Gram-Schmidt, two passes)
//   alpha = q^H r / q^H q;  y += alpha p;  r -= alpha q;  Q_k = q / |q|,  P_k = p / |q|
// so the residual is minimised over the Krylov space, as in GMRES, and |r| is known exactly after
// every step.  Four kernels per step over chunks of rows, each reduction finishing in the last
// CTA to arrive; every kernel reads the step index from device memory, so the host queues
// identical launches and polls a flag one chunk behind, as krylov.cu does.  Vectors are
// right-hand-side major; dot products and norms are float64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {

constexpr int kT = 256;  // CTA width
constexpr int kL = 8;    // lanes per scalar row in the product

struct GState {
  int j;           // step inside the cycle
  int cycle_done;  // no active right-hand side left in this cycle, or the cycle is full
  int all_conv;    // every right-hand side met tol at the start of this cycle
  int iters;       // total steps
  int numeric;     // a NaN/Inf appeared
  int pad[3];
};

struct GPtr {
  GState* st;
  unsigned* counter;  // [R + 1]: per right-hand side, and for all of them
  int* active;        // [R]
  double* bnorm;      // [R]
  double* resid;      // [R]
  c128* beta1;        // [R][m]
  c128* beta2;        // [R][m]
  c128* alpha;        // [R]
  double* scal;       // [R] 1 / |q|
  c128* part;         // [R][nchunk][m + 1]
  double* partn;      // [R][nchunk]
  int R, m, nchunk, chunk;
  int64_t N;
  double tol;
};

__device__ bool last_block(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// Block sum of one double per thread (result valid in thread 0).
__device__ double block_sum(double v) {
  __shared__ double red[kT / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kT / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Sum of n partials with stride `stride` by one warp, in a fixed order, eight loads per lane in
// flight (the last batch predicated).
__device__ c128 warp_sum_partials(const c128* __restrict__ base, int stride, int n) {
  const int lane = threadIdx.x & 31;
  double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
  for (int c = lane; c < n; c += 8 * 32) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = c + u * 32;
      v[u] = i < n ? __ldcg(reinterpret_cast<const double2*>(base + (int64_t)i * stride)) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      re[u & 3] += v[u].x;
      im[u & 3] += v[u].y;
    }
  }
  return mkc(warp_sum((re[0] + re[1]) + (re[2] + re[3])), warp_sum((im[0] + im[1]) + (im[2] + im[3])));
}
__device__ double warp_sum_partials_d(const double* __restrict__ base, int n) {
  const int lane = threadIdx.x & 31;
  double a[4] = {0, 0, 0, 0};
  for (int c = lane; c < n; c += 8 * 32) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = c + u * 32 < n ? __ldcg(base + c + u * 32) : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u & 3] += v[u];
  }
  return warp_sum((a[0] + a[1]) + (a[2] + a[3]));
}

// Partial dots conj(Q_i) . w over the CTA's rows for i < j (one warp per i), to part.
template <typename TV>
__device__ void dots_prev(const GPtr& P, int j, int r, const cplx<TV>* __restrict__ Q, const cplx<TV>* w_sm, int64_t n0,
                          int cnt) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  c128* out = P.part + ((int64_t)r * P.nchunk + blockIdx.x) * (P.m + 1);
  for (int i = wp; i < j; i += kT / 32) {
    const cplx<TV>* qi = Q + ((int64_t)i * P.R + r) * P.N + n0;
    double re = 0.0, im = 0.0;
    for (int t = lane; t < cnt; t += 32) {
      const cplx<TV> a = qi[t], b = w_sm[t];
      re += (double)a.re * b.re + (double)a.im * b.im;
      im += (double)a.re * b.im - (double)a.im * b.re;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) out[i] = mkc(re, im);
  }
}

// The last CTA of right-hand side r sums the dot partials of i < j into dst[r][i].
__device__ void reduce_prev(const GPtr& P, int j, int r, c128* __restrict__ dst) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const c128* base = P.part + (int64_t)r * P.nchunk * (P.m + 1);
  for (int i = wp; i < j; i += kT / 32) {
    const c128 v = warp_sum_partials(base + i, P.m + 1, P.nchunk);
    if (lane == 0) dst[(int64_t)r * P.m + i] = v;
  }
}

// K1: q = A r (eight lanes per row, gathering r), p = r; first dots Q_i^H q.
template <typename TV>
__global__ void __launch_bounds__(kT) k_gcr_product(GPtr P, const RowInfo* __restrict__ rinfo,
                                                    const int32_t* __restrict__ colmap, const cplx<TV>* __restrict__ E,
                                                    const cplx<TV>* __restrict__ Rv, cplx<TV>* __restrict__ Q,
                                                    cplx<TV>* __restrict__ Pb) {
  const int r = blockIdx.y;
  if (P.st->cycle_done || !P.active[r]) return;
  const int j = P.st->j;
  const int64_t N = P.N, n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, N - n0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  const cplx<TV>* src = Rv + (int64_t)r * N;
  const int g = threadIdx.x / kL, sub = threadIdx.x % kL;
  for (int t0 = 0; t0 < cnt; t0 += kT / kL) {
    const int t = t0 + g;
    cplx<TV> acc = mkc<TV>(0, 0);
    if (t < cnt) {
      const RowInfo ri = rinfo[n0 + t];
      const int32_t* cm = colmap + ri.cmb;
      for (int c = sub; c < ri.K; c += kL) cfma(acc, E[ri.vb + c], src[cm[c]]);
    }
#pragma unroll
    for (int o = kL / 2; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (t < cnt && sub == 0) {
      const int64_t n = n0 + t;
      const cplx<TV> x = src[n];
      const cplx<TV> q = x + acc;
      Q[((int64_t)j * P.R + r) * N + n] = q;
      Pb[((int64_t)j * P.R + r) * N + n] = x;
      w_sm[t] = q;
    }
  }
  __syncthreads();
  dots_prev<TV>(P, j, r, Q, w_sm, n0, cnt);
  if (last_block(&P.counter[r])) {
    reduce_prev(P, j, r, P.beta1);
    if (threadIdx.x == 0) P.counter[r] = 0;
  }
}

// q -= sum_{i<j} Q_i beta_i and p -= sum_{i<j} P_i beta_i on the CTA's rows; q kept in w_sm.
template <typename TV>
__device__ void update_pair(const GPtr& P, int j, int r, const c128* __restrict__ beta, cplx<TV>* __restrict__ Q,
                            cplx<TV>* __restrict__ Pb, cplx<TV>* w_sm, int64_t n0, int cnt) {
  __shared__ cplx<TV> bs[SWM_MAX_RESTART];
  for (int i = threadIdx.x; i < j; i += kT) bs[i] = ccast<TV>(beta[(int64_t)r * P.m + i]);
  __syncthreads();
  const int64_t N = P.N;
  for (int t = threadIdx.x; t < cnt; t += kT) {
    const int64_t n = n0 + t;
    cplx<TV> q = Q[((int64_t)j * P.R + r) * N + n], p = Pb[((int64_t)j * P.R + r) * N + n];
    for (int i = 0; i < j; ++i) {
      const cplx<TV> b = bs[i];
      const cplx<TV> qi = Q[((int64_t)i * P.R + r) * N + n], pi = Pb[((int64_t)i * P.R + r) * N + n];
      q = q - qi * b;
      p = p - pi * b;
    }
    Q[((int64_t)j * P.R + r) * N + n] = q;
    Pb[((int64_t)j * P.R + r) * N + n] = p;
    w_sm[t] = q;
  }
  __syncthreads();
}

// K2: first update, second dots.
template <typename TV>
__global__ void __launch_bounds__(kT) k_gcr_pass2(GPtr P, cplx<TV>* __restrict__ Q, cplx<TV>* __restrict__ Pb) {
  const int r = blockIdx.y;
  if (P.st->cycle_done || !P.active[r]) return;
  const int j = P.st->j;
  const int64_t n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, P.N - n0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  update_pair<TV>(P, j, r, P.beta1, Q, Pb, w_sm, n0, cnt);
  dots_prev<TV>(P, j, r, Q, w_sm, n0, cnt);
  if (last_block(&P.counter[r])) {
    reduce_prev(P, j, r, P.beta2);
    if (threadIdx.x == 0) P.counter[r] = 0;
  }
}

// K3: second update, then |q|^2 and q^H r; the last CTA forms alpha and 1/|q|.
template <typename TV>
__global__ void __launch_bounds__(kT) k_gcr_coef(GPtr P, cplx<TV>* __restrict__ Q, cplx<TV>* __restrict__ Pb,
                                                 const cplx<TV>* __restrict__ Rv) {
  const int r = blockIdx.y;
  if (P.st->cycle_done || !P.active[r]) return;
  const int j = P.st->j;
  const int64_t N = P.N, n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, N - n0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cplx<TV>* w_sm = reinterpret_cast<cplx<TV>*>(sm_raw);
  update_pair<TV>(P, j, r, P.beta2, Q, Pb, w_sm, n0, cnt);
  double qq = 0.0, qre = 0.0, qim = 0.0;
  for (int t = threadIdx.x; t < cnt; t += kT) {
    const cplx<TV> q = w_sm[t], x = Rv[(int64_t)r * N + n0 + t];
    qq += (double)q.re * q.re + (double)q.im * q.im;
    qre += (double)q.re * x.re + (double)q.im * x.im;
    qim += (double)q.re * x.im - (double)q.im * x.re;
  }
  qq = block_sum(qq);
  qre = block_sum(qre);
  qim = block_sum(qim);
  if (threadIdx.x == 0) {
    P.partn[(int64_t)r * P.nchunk + blockIdx.x] = qq;
    P.part[((int64_t)r * P.nchunk + blockIdx.x) * (P.m + 1)] = mkc(qre, qim);
  }
  if (!last_block(&P.counter[r])) return;
  if (threadIdx.x < 32) {
    const double nq2 = warp_sum_partials_d(P.partn + (int64_t)r * P.nchunk, P.nchunk);
    const c128 qr = warp_sum_partials(P.part + (int64_t)r * P.nchunk * (P.m + 1), P.m + 1, P.nchunk);
    if (threadIdx.x == 0) {
      P.counter[r] = 0;
      if (nq2 > 0.0 && isfinite(nq2)) {
        P.alpha[r] = mkc(qr.re / nq2, qr.im / nq2);
        P.scal[r] = 1.0 / sqrt(nq2);
      } else {  // breakdown: the direction adds nothing
        P.alpha[r] = mkc(0.0, 0.0);
        P.scal[r] = 0.0;
        if (!isfinite(nq2)) P.st->numeric = 1;
      }
    }
  }
}

// K4: y += alpha p, r -= alpha q, normalise Q_j and P_j; |r|^2, residual, activity, next step.
template <typename TV>
__global__ void __launch_bounds__(kT) k_gcr_axpy(GPtr P, cplx<TV>* __restrict__ Q, cplx<TV>* __restrict__ Pb,
                                                 cplx<TV>* __restrict__ Rv, cplx<TV>* __restrict__ Y) {
  const int r = blockIdx.y;
  if (P.st->cycle_done) return;
  const bool act = P.active[r];
  const int j = P.st->j;
  const int64_t N = P.N, n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, N - n0);
  double rr = 0.0;
  if (act) {
    const cplx<TV> al = ccast<TV>(P.alpha[r]);
    const TV sc = (TV)P.scal[r];
    for (int t = threadIdx.x; t < cnt; t += kT) {
      const int64_t n = n0 + t, row = (int64_t)r * N + n, v = ((int64_t)j * P.R + r) * N + n;
      const cplx<TV> q = Q[v], p = Pb[v];
      Y[row] = Y[row] + al * p;
      const cplx<TV> x = Rv[row] - al * q;
      Rv[row] = x;
      Q[v] = sc * q;
      Pb[v] = sc * p;
      rr += (double)x.re * x.re + (double)x.im * x.im;
    }
    rr = block_sum(rr);
    if (threadIdx.x == 0) P.partn[(int64_t)r * P.nchunk + blockIdx.x] = rr;
  }
  // every CTA of every right-hand side arrives once, so the last one advances the step
  __shared__ bool last_r;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_r = act && atomicAdd(&P.counter[r], 1u) == gridDim.x - 1;
  __syncthreads();
  if (last_r && threadIdx.x < 32) {
    const double t = warp_sum_partials_d(P.partn + (int64_t)r * P.nchunk, P.nchunk);
    if (threadIdx.x == 0) {
      P.counter[r] = 0;
      const double res = sqrt(t) / P.bnorm[r];
      P.resid[r] = res;
      if (!isfinite(res)) {
        P.st->numeric = 1;
        P.active[r] = 0;
      } else if (res <= P.tol || P.scal[r] == 0.0) {
        P.active[r] = 0;
      }
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    if (atomicAdd(&P.counter[P.R], 1u) == total - 1) {
      P.counter[P.R] = 0;
      int any = 0;
      for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
      P.st->j = j + 1;
      P.st->iters += 1;
      if (!any || j + 1 >= P.m) P.st->cycle_done = 1;
    }
  }
}

// Start of a cycle: r = b - A y (true residual), its norm, activity.
template <typename TV>
__global__ void __launch_bounds__(kT) k_gcr_residual(GPtr P, int first, const RowInfo* __restrict__ rinfo,
                                                     const int32_t* __restrict__ colmap,
                                                     const cplx<TV>* __restrict__ E, const cplx<TV>* __restrict__ B,
                                                     const cplx<TV>* __restrict__ Y, cplx<TV>* __restrict__ Rv) {
  const int r = blockIdx.y;
  const int64_t N = P.N, n0 = (int64_t)blockIdx.x * P.chunk;
  const int cnt = (int)min((int64_t)P.chunk, N - n0);
  const cplx<TV>* src = Y + (int64_t)r * N;
  const int g = threadIdx.x / kL, sub = threadIdx.x % kL;
  double rr = 0.0;
  for (int t0 = 0; t0 < cnt; t0 += kT / kL) {
    const int t = t0 + g;
    cplx<TV> acc = mkc<TV>(0, 0);
    if (t < cnt) {
      const RowInfo ri = rinfo[n0 + t];
      const int32_t* cm = colmap + ri.cmb;
      for (int c = sub; c < ri.K; c += kL) cfma(acc, E[ri.vb + c], src[cm[c]]);
    }
#pragma unroll
    for (int o = kL / 2; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (t < cnt && sub == 0) {
      const int64_t n = n0 + t;
      const cplx<TV> x = B[(int64_t)r * N + n] - (src[n] + acc);
      Rv[(int64_t)r * N + n] = x;
      rr += (double)x.re * x.re + (double)x.im * x.im;
    }
  }
  rr = block_sum(rr);
  if (threadIdx.x == 0) P.partn[(int64_t)r * P.nchunk + blockIdx.x] = rr;
  if (!last_block(&P.counter[r])) return;
  if (threadIdx.x < 32) {
    const double t = warp_sum_partials_d(P.partn + (int64_t)r * P.nchunk, P.nchunk);
    if (threadIdx.x == 0) {
      P.counter[r] = 0;
      const double beta = sqrt(t);
      if (first) P.bnorm[r] = beta > 0.0 ? beta : 1.0;
      const double res = beta / P.bnorm[r];
      P.resid[r] = res;
      if (!isfinite(res)) P.st->numeric = 1;
      P.active[r] = (isfinite(res) && res > P.tol) ? 1 : 0;
      __threadfence();
      if (atomicAdd(&P.counter[P.R], 1u) == (unsigned)P.R - 1) {
        P.counter[P.R] = 0;
        int any = 0;
        for (int q = 0; q < P.R; ++q) any |= __ldcg(P.active + q);
        P.st->j = 0;
        P.st->cycle_done = any ? 0 : 1;
        P.st->all_conv = any ? 0 : 1;
      }
    }
  }
}

template <typename TV>
int gcr_impl(swm_ctx* ctx, double tol, int m, int max_iter) {
  cudaStream_t st = ctx->stream;
  const int R = ctx->n_rhs;
  const int64_t N = ctx->N;
  using C = cplx<TV>;
  SWM_TRY(ensure_rowinfo(ctx));
  std::vector<Buf>& S = ctx->solve_bufs;
  GPtr P{};
  P.R = R;
  P.m = m;
  P.N = N;
  P.tol = tol;
  P.chunk = (int)std::max<int64_t>(kT, ceil_div(ceil_div(N, 512), kT) * kT);
  P.nchunk = (int)ceil_div(N, P.chunk);
  C *Y = nullptr, *Rv = nullptr, *Q = nullptr, *Pb = nullptr;
  SWM_TRY(dalloc(ctx, S, (void**)&P.st, sizeof(GState)));
  SWM_TRY(dalloc(ctx, S, (void**)&P.counter, sizeof(unsigned) * (R + 1)));
  SWM_TRY(dalloc(ctx, S, (void**)&P.active, sizeof(int) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&P.bnorm, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&P.resid, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&P.beta1, sizeof(c128) * R * m));
  SWM_TRY(dalloc(ctx, S, (void**)&P.beta2, sizeof(c128) * R * m));
  SWM_TRY(dalloc(ctx, S, (void**)&P.alpha, sizeof(c128) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&P.scal, sizeof(double) * R));
  SWM_TRY(dalloc(ctx, S, (void**)&P.part, sizeof(c128) * (size_t)R * P.nchunk * (m + 1)));
  SWM_TRY(dalloc(ctx, S, (void**)&P.partn, sizeof(double) * (size_t)R * P.nchunk));
  SWM_TRY(dalloc(ctx, S, (void**)&Y, sizeof(C) * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&Rv, sizeof(C) * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&Q, sizeof(C) * (size_t)m * R * N));
  SWM_TRY(dalloc(ctx, S, (void**)&Pb, sizeof(C) * (size_t)m * R * N));
  SWM_CK(cudaMemsetAsync(P.st, 0, sizeof(GState), st));
  SWM_CK(cudaMemsetAsync(P.counter, 0, sizeof(unsigned) * (R + 1), st));
  SWM_TRY(init_y(ctx, Y, sizeof(TV) == sizeof(double)));
  if (ctx->guess) SWM_TRY(norms_of_b(ctx, ctx->Bv, sizeof(TV) == sizeof(double), P.bnorm));
  const C* E = (const C*)ctx->Zp;
  const C* Bv = (const C*)ctx->Bv;
  const RowInfo* ri = (const RowInfo*)ctx->rowinfo;
  const dim3 grid((unsigned)P.nchunk, (unsigned)R);
  const size_t sm = sizeof(C) * P.chunk;
  if (sm > 48 * 1024) {
    SWM_CK(allow_max_dyn_smem((const void*)k_gcr_product<TV>, ctx->smem_optin));
    SWM_CK(allow_max_dyn_smem((const void*)k_gcr_pass2<TV>, ctx->smem_optin));
    SWM_CK(allow_max_dyn_smem((const void*)k_gcr_coef<TV>, ctx->smem_optin));
  }
  SWM_TRY(ensure_poll_slots(ctx));
  static_assert(2 * sizeof(GState) <= kPollSlotBytes, "poll slots");
  auto slot = [&](int c) { return reinterpret_cast<GState*>(ctx->pinned_state) + (c & 1); };
  constexpr int kChunkSteps = 4;
  GState hs{};
  int cycles = 0;
  bool first = !ctx->guess;
  while (true) {
    ctx->prof_begin(SWM_K_APPLY);
    k_gcr_residual<TV><<<grid, kT, 0, st>>>(P, first ? 1 : 0, ri, ctx->offd.colmap, E, Bv, Y, Rv);
    ctx->prof_end(SWM_K_APPLY);
    SWM_LAUNCHED();
    first = false;
    SWM_CK(cudaMemcpyAsync(&hs, P.st, sizeof(GState), cudaMemcpyDeviceToHost, st));
    SWM_CK(cudaStreamSynchronize(st));
    if (hs.all_conv || hs.numeric || hs.iters >= max_iter) break;
    const int steps = std::min(m, max_iter - hs.iters);
    int c = 0;
    for (int s0 = 0; s0 < steps; s0 += kChunkSteps, ++c) {
      const int n = std::min(steps - s0, kChunkSteps);
      for (int i = 0; i < n; ++i) {
        ctx->prof_begin(SWM_K_APPLY);
        k_gcr_product<TV><<<grid, kT, sm, st>>>(P, ri, ctx->offd.colmap, E, Rv, Q, Pb);
        ctx->prof_end(SWM_K_APPLY);
        ctx->prof_begin(SWM_K_UPDATE);
        k_gcr_pass2<TV><<<grid, kT, sm, st>>>(P, Q, Pb);
        ctx->prof_end(SWM_K_UPDATE);
        ctx->prof_begin(SWM_K_FINISH);
        k_gcr_coef<TV><<<grid, kT, sm, st>>>(P, Q, Pb, Rv);
        k_gcr_axpy<TV><<<grid, kT, 0, st>>>(P, Q, Pb, Rv, Y);
        ctx->prof_end(SWM_K_FINISH);
        ctx->launches += 4;
      }
      SWM_CK(cudaGetLastError());
      SWM_CK(cudaMemcpyAsync(slot(c), P.st, sizeof(GState), cudaMemcpyDeviceToHost, st));
      SWM_CK(cudaEventRecord(ctx->poll_ev[c & 1], st));
      if (c >= 1) {
        SWM_CK(cudaEventSynchronize(ctx->poll_ev[(c - 1) & 1]));
        if (slot(c - 1)->cycle_done) break;
      }
    }
    ++cycles;
  }
  SWM_TRY(apply_minv(ctx, Y));
  std::vector<double> res(R);
  SWM_CK(cudaMemcpyAsync(res.data(), P.resid, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaStreamSynchronize(st));
  double mx = 0.0;
  for (double v : res) mx = std::max(mx, v);
  ctx->stats.iterations = hs.iters;
  ctx->stats.restarts = cycles;
  ctx->stats.rel_residual = mx;
  ctx->stats.converged = hs.all_conv ? 1 : 0;
  if (hs.numeric) return ctx->fail(SWM_ECUDA, "GCR produced a non-finite value");
  return hs.all_conv ? SWM_OK : SWM_ENOTCONV;
}

}  // namespace

int gcr_solve(swm_ctx* ctx, double tol, int restart, int max_iter) {
  if (ctx->prec == SWM_C128) return gcr_impl<double>(ctx, tol, restart, max_iter);
  return gcr_impl<float>(ctx, tol, restart, max_iter);
}

}  // namespace swm
