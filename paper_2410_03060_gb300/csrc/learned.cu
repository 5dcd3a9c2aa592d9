// Learned warm start: a small rotation-invariant network predicts, for every wire and incidence, a
// correction of the isolated-wire current Z_pp^-1 b_p from the wire's neighbourhood; the corrected
// currents are the initial guess of the Krylov solve (swm_solve_guess).  The paper has no such
// part; the network is this library's own.  Forward, backward and the Adam update are the kernels
// below, trained on currents the solver produces.
//
// Per wire p and incidence (k_hat, e), in the wire's frame (t_p):
//   modes phi_k(i) = sin(k pi (i+1) / n_s), k = 1..3; isolated amplitudes
//       a_p,k = (2 / n_s) sum_i x_iso_{p,i} phi_k(i) exp(+j k k_hat.c_p), x_iso = Z_pp^-1 b_p;
//   neighbours: up to 16 wires q != p of the S-NFC pattern, nearest first (ties: lower caller index);
//   neighbour features (16): z/r_c, rho/r_c, t_p.t_q, t_q.d/r_c, L_q/lambda, L_p/lambda, e.t_p,
//       k_hat.t_p, e.t_q, k_hat.t_q, cos(k k_hat.d), sin(k k_hat.d), cos(kR), sin(kR), 1/(1+kR), 1
//       (d = c_q - c_p, R = |d|, z = d.t_p, rho^2 = R^2 - z^2; empty slots all zero);
//   self features (8): e.t_p, k_hat.t_p, L_p/lambda, neighbours/16, (e.t_p)(k_hat.t_p), (k_hat.t_p)^2, 0, 0;
//   coupling C_pq = W3 s(W2 s(W1 f_q + b1) + b2) + b3 (s = SiLU): a complex 3 x 3 matrix (18 values,
//       real parts row-major, then imaginary parts);
//   h = sum over present q of C_pq a_q exp(-j k k_hat.d) (the neighbours' amplitudes in p's phase);
//   o = W6 s(W5 s(W4 [Re h, Im h, self, Re a_p, Im a_p] + b4) + b5) + b6;  c_k = h_k + o_k;
//   x0_{p,i} = x_iso_{p,i} + exp(-j k k_hat.c_p) sum_k c_k phi_k(i).
// The correction is linear in the neighbours' isolated currents, as the first-order coupling
// -Z_pp^-1 sum_q Z_pq x_iso_q is; the network learns the coupling matrices from the geometry.
// Loss: sum |x0 - x_true|^2 / sum |x_true|^2.  Weights are float32; the dense layers run as tiled
// float32 GEMMs on the CUDA cores (64 x 64 tiles, 16-deep, 4 x 4 outputs per thread), the weight
// gradients as split sums over the rows reduced in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"

struct swm_net {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* params = nullptr;  // device
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int64_t step = 0;
  std::string err;
  // workspace sized for the largest batch so far
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
};

namespace swm {

namespace {

constexpr int kNbr = 16, kFe = 16, kFs = 8, kHm = 18, kModes = 3;
constexpr int kUin = 2 * kModes + kFs + 2 * kModes;  // [Re h, Im h, self, Re a_p, Im a_p]
constexpr int kLayers = 6;
constexpr int kIn[kLayers] = {16, 128, 128, kUin, 256, 256};
constexpr int kOut[kLayers] = {128, 128, kHm, 256, 256, 6};

int64_t param_offset(int l) {  // start of W_l; b_l follows W_l
  int64_t o = 0;
  for (int i = 0; i < l; ++i) o += (int64_t)kIn[i] * kOut[i] + kOut[i];
  return o;
}
constexpr int64_t kNumParams = 93720;

// ---- neighbour lists: the nearest kNbr pattern partners of each wire (internal indices)
__global__ void k_nbr_select(int64_t nw, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
                             const int32_t* __restrict__ perm, int32_t* __restrict__ nbr) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nw) return;
  double bd[kNbr];
  int32_t bq[kNbr], bu[kNbr];
  int n = 0;
  for (int64_t b = row_ptr[p]; b < row_ptr[p + 1]; ++b) {
    const int32_t q = col[b];
    if (q == (int32_t)p) continue;
    const double dx = cx[q] - cx[p], dy = cy[q] - cy[p], dz = cz[q] - cz[p];
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const int32_t u = perm[q];
    // insertion into the sorted list (d2, caller index)
    int pos = n;
    while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bu[pos - 1] > u))) --pos;
    if (pos >= kNbr) continue;
    const int last = n < kNbr ? n : kNbr - 1;
    for (int s = last; s > pos; --s) {
      bd[s] = bd[s - 1];
      bq[s] = bq[s - 1];
      bu[s] = bu[s - 1];
    }
    bd[pos] = d2;
    bq[pos] = q;
    bu[pos] = u;
    if (n < kNbr) ++n;
  }
  for (int s = 0; s < kNbr; ++s) nbr[p * kNbr + s] = s < n ? bq[s] : -1;
}

// ---- features of sample (r, p) = r * nw + p: Xe [S * 16][16], Xs [S][8]
__global__ void k_features(int64_t nw, int R, const int32_t* __restrict__ nbr, const double* __restrict__ cx,
                           const double* __restrict__ cy, const double* __restrict__ cz, const double* __restrict__ tx,
                           const double* __restrict__ ty, const double* __restrict__ tz, const double* __restrict__ Ls,
                           const double* __restrict__ frames, double k, double r_c, float* __restrict__ Xe,
                           float* __restrict__ Xs) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // (sample, slot)
  if (e >= (int64_t)R * nw * kNbr) return;
  const int slot = (int)(e % kNbr);
  const int64_t s = e / kNbr;
  const int64_t p = s % nw;
  const int r = (int)(s / nw);
  const double* f = frames + 6 * r;
  const double kh[3] = {f[0], f[1], f[2]}, ev[3] = {f[3], f[4], f[5]};
  const double lam = 2.0 * kPi / k;
  const double tp[3] = {tx[p], ty[p], tz[p]};
  const double et_p = ev[0] * tp[0] + ev[1] * tp[1] + ev[2] * tp[2];
  const double kt_p = kh[0] * tp[0] + kh[1] * tp[1] + kh[2] * tp[2];
  float* out = Xe + e * kFe;
  const int q = nbr[p * kNbr + slot];
  if (q < 0) {
    for (int i = 0; i < kFe; ++i) out[i] = 0.f;
  } else {
    const double d[3] = {cx[q] - cx[p], cy[q] - cy[p], cz[q] - cz[p]};
    const double tq[3] = {tx[q], ty[q], tz[q]};
    const double R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double Rd = sqrt(R2);
    const double z = d[0] * tp[0] + d[1] * tp[1] + d[2] * tp[2];
    const double rho = sqrt(fmax(R2 - z * z, 0.0));
    const double ph = k * (kh[0] * d[0] + kh[1] * d[1] + kh[2] * d[2]);
    double sph, cph, skr, ckr;
    sincos(ph, &sph, &cph);
    sincos(k * Rd, &skr, &ckr);
    out[0] = (float)(z / r_c);
    out[1] = (float)(rho / r_c);
    out[2] = (float)(tp[0] * tq[0] + tp[1] * tq[1] + tp[2] * tq[2]);
    out[3] = (float)((tq[0] * d[0] + tq[1] * d[1] + tq[2] * d[2]) / r_c);
    out[4] = (float)(Ls[q] / lam);
    out[5] = (float)(Ls[p] / lam);
    out[6] = (float)et_p;
    out[7] = (float)kt_p;
    out[8] = (float)(ev[0] * tq[0] + ev[1] * tq[1] + ev[2] * tq[2]);
    out[9] = (float)(kh[0] * tq[0] + kh[1] * tq[1] + kh[2] * tq[2]);
    out[10] = (float)cph;
    out[11] = (float)sph;
    out[12] = (float)ckr;
    out[13] = (float)skr;
    out[14] = (float)(1.0 / (1.0 + k * Rd));
    out[15] = 1.f;
  }
  if (slot == 0) {
    int cnt = 0;
    for (int i = 0; i < kNbr; ++i) cnt += nbr[p * kNbr + i] >= 0 ? 1 : 0;
    float* xs = Xs + s * kFs;
    xs[0] = (float)et_p;
    xs[1] = (float)kt_p;
    xs[2] = (float)(Ls[p] / lam);
    xs[3] = (float)cnt / kNbr;
    xs[4] = (float)(et_p * kt_p);
    xs[5] = (float)(kt_p * kt_p);
    xs[6] = 0.f;
    xs[7] = 0.f;
  }
}

// ---- tiled float32 GEMM C[M][N] = op(A)[M][K] op(B)[K][N] with an epilogue.
//   TA: A stored [K][M] (op = transpose); TB: B stored [N][K].
//   EPI 0: C = acc;  1: C = acc + bias;  2: Z = acc + bias, C = silu(Z) (Z to Z2);
//   3: C = acc * silu'(Zs) (Zs = Z2, read);  4: split-K partial (blockIdx.z = split, rows
//   [z * mchunk, (z + 1) * mchunk) of the reduction dimension) written to C + z * M * N.
constexpr int kTM = 64, kTN = 64, kTK = 16;
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_SILU = 2, EPI_DSILU = 3, EPI_SPLIT = 4 };

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.f / (1.f + expf(-z));
  return s * (1.f + z * (1.f - s));
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int N, int64_t K, const float* __restrict__ A,
                                              const float* __restrict__ B, const float* __restrict__ bias,
                                              float* __restrict__ C, float* __restrict__ Z2, int64_t kchunk) {
  __shared__ float As[kTK][kTM + 4];
  __shared__ float Bs[kTK][kTN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int n0 = blockIdx.x * kTN;
  const int64_t mtiles = ceil_div(M, kTM);
  for (int64_t mt = blockIdx.y; mt < mtiles; mt += gridDim.y) {  // row tiles beyond the grid's 65,535
  const int64_t m0 = mt * kTM;
  int64_t k_begin = 0, k_end = K;
  if (EPI == EPI_SPLIT) {
    k_begin = (int64_t)blockIdx.z * kchunk;
    k_end = min(K, k_begin + kchunk);
  }
  float acc[4][4] = {};
  for (int64_t kb = k_begin; kb < k_end; kb += kTK) {
    // A tile: kTM x kTK, 1024 values, 4 per thread
    for (int t = threadIdx.x; t < kTM * kTK; t += 256) {
      int mm, kk;
      if (TA) {  // coalesced along m
        mm = t % kTM;
        kk = t / kTM;
      } else {   // coalesced along k
        kk = t % kTK;
        mm = t / kTK;
      }
      const int64_t gm = m0 + mm, gk = kb + kk;
      float v = 0.f;
      if (gm < M && gk < k_end) v = TA ? A[gk * M + gm] : A[gm * K + gk];
      As[kk][mm] = v;
    }
    for (int t = threadIdx.x; t < kTK * kTN; t += 256) {
      int nn, kk;
      if (TB) {
        kk = t % kTK;
        nn = t / kTK;
      } else {
        nn = t % kTN;
        kk = t / kTN;
      }
      const int gn = n0 + nn;
      const int64_t gk = kb + kk;
      float v = 0.f;
      if (gn < N && gk < k_end) v = TB ? B[(int64_t)gn * K + gk] : B[gk * N + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      const int64_t o = gm * N + gn;
      float v = acc[i][j];
      if (EPI == EPI_NONE) C[o] = v;
      if (EPI == EPI_BIAS) C[o] = v + bias[gn];
      if (EPI == EPI_BIAS_SILU) {
        v += bias[gn];
        Z2[o] = v;
        C[o] = silu_f(v);
      }
      if (EPI == EPI_DSILU) C[o] = v * dsilu_f(Z2[o]);
      if (EPI == EPI_SPLIT) C[(int64_t)blockIdx.z * M * N + o] = v;
    }
  }
  }
}

// dst[i] (+)= sum over z of part[z][i], in order (deterministic).
__global__ void k_split_sum(int64_t n, int nz, const float* __restrict__ part, float* __restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int z = 0; z < nz; ++z) s += part[(int64_t)z * n + i];
  dst[i] = s;
}

// Partial column sums of X[M][N]: CTA (column block of 32, row chunk z) writes part[z][N]; rows
// in a fixed order.
__global__ void k_colsum(int64_t M, int N, int64_t rchunk, const float* __restrict__ X, float* __restrict__ part) {
  __shared__ float red[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.y * rchunk, r1 = min(M, r0 + rchunk);
  float s = 0.f;
  if (c < N)
    for (int64_t m = r0 + w; m < r1; m += 8) s += X[m * N + c];
  red[w][threadIdx.x & 31] = s;
  __syncthreads();
  if (w == 0 && c < N) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
    part[(int64_t)blockIdx.y * N + c] = t;
  }
}

// Isolated amplitudes of sample (r, p): AMP[s] = (re, im) of a_p,k, k = 1..3.
__global__ void k_amplitudes(int64_t nw, int R, int64_t N, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ ns, const double* __restrict__ cx,
                             const double* __restrict__ cy, const double* __restrict__ cz,
                             const double* __restrict__ frames, double k, const c128* __restrict__ xiso,
                             float* __restrict__ AMP) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= (int64_t)R * nw) return;
  const int64_t p = s % nw;
  const int r = (int)(s / nw);
  const double* f = frames + 6 * r;
  double sp, cp;
  sincos(k * (f[0] * cx[p] + f[1] * cy[p] + f[2] * cz[p]), &sp, &cp);
  const c128 ph = mkc(cp, sp);
  const int nsp = ns[p];
  c128 a[kModes] = {};
  for (int i = 0; i < nsp - 1; ++i) {
    const c128 x = xiso[(int64_t)r * N + off[p] + i];
    for (int q = 0; q < kModes; ++q) a[q] = a[q] + sin((q + 1) * kPi * (i + 1) / nsp) * x;
  }
  for (int q = 0; q < kModes; ++q) {
    const c128 v = (2.0 / nsp) * (ph * a[q]);
    AMP[s * 2 * kModes + 2 * q] = (float)v.re;
    AMP[s * 2 * kModes + 2 * q + 1] = (float)v.im;
  }
}

// Neighbour amplitude of slot `slot` of sample s in p's phase: a_q exp(-j phi), phi = k k_hat.d.
__device__ __forceinline__ void rel_amp(int64_t s, int slot, int64_t nw, const int32_t* __restrict__ nbr,
                                        const float* __restrict__ Xe, const float* __restrict__ AMP, float* re,
                                        float* im) {
  const int64_t p = s % nw, r = s / nw;
  const int q = nbr[p * kNbr + slot];
  const float* fe = Xe + (s * kNbr + slot) * kFe;
  const float c = fe[10], sn = fe[11];
  for (int l = 0; l < kModes; ++l) {
    if (q < 0) {
      re[l] = im[l] = 0.f;
      continue;
    }
    const float ar = AMP[(r * nw + q) * 2 * kModes + 2 * l], ai = AMP[(r * nw + q) * 2 * kModes + 2 * l + 1];
    re[l] = ar * c + ai * sn;  // (ar + j ai)(c - j sn)
    im[l] = ai * c - ar * sn;
  }
}

// U0[s] = [Re h, Im h, self features, Re a_p, Im a_p], h = sum over present slots of C a_rel.
__global__ void k_aggregate(int64_t S, int64_t nw, const int32_t* __restrict__ nbr, const float* __restrict__ Cm,
                            const float* __restrict__ Xe, const float* __restrict__ Xs, const float* __restrict__ AMP,
                            float* __restrict__ U0) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= S) return;
  float hr[kModes] = {}, hi[kModes] = {};
  for (int slot = 0; slot < kNbr; ++slot) {
    const int64_t row = s * kNbr + slot;
    const float pres = Xe[row * kFe + kFe - 1];
    if (pres == 0.f) continue;
    float ar[kModes], ai[kModes];
    rel_amp(s, slot, nw, nbr, Xe, AMP, ar, ai);
    const float* c = Cm + row * kHm;
    for (int k = 0; k < kModes; ++k)
      for (int l = 0; l < kModes; ++l) {
        const float cr = c[k * 3 + l], ci = c[9 + k * 3 + l];
        hr[k] += pres * (cr * ar[l] - ci * ai[l]);
        hi[k] += pres * (cr * ai[l] + ci * ar[l]);
      }
  }
  float* u = U0 + s * kUin;
  for (int k = 0; k < kModes; ++k) {
    u[k] = hr[k];
    u[kModes + k] = hi[k];
  }
  for (int i = 0; i < kFs; ++i) u[2 * kModes + i] = Xs[s * kFs + i];
  for (int k = 0; k < kModes; ++k) {
    u[2 * kModes + kFs + k] = AMP[s * 2 * kModes + 2 * k];
    u[2 * kModes + kFs + kModes + k] = AMP[s * 2 * kModes + 2 * k + 1];
  }
}

// dL/dC of every (sample, slot): with G = dL/dRe h + j dL/dIm h (from c = h + o and from the
// output MLP's input), g_kl = conj(G_k) a_rel_l pres, dRe C_kl = Re g, dIm C_kl = -Im g.
__global__ void k_scatter_dmsg(int64_t S, int64_t nw, const int32_t* __restrict__ nbr, const float* __restrict__ dO,
                               const float* __restrict__ dU0, const float* __restrict__ Xe,
                               const float* __restrict__ AMP, float* __restrict__ dmsg) {
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= S * kNbr) return;
  const int64_t s = row / kNbr;
  const int slot = (int)(row % kNbr);
  const float pres = Xe[row * kFe + kFe - 1];
  float* d = dmsg + row * kHm;
  if (pres == 0.f) {
    for (int i = 0; i < kHm; ++i) d[i] = 0.f;
    return;
  }
  float ar[kModes], ai[kModes];
  rel_amp(s, slot, nw, nbr, Xe, AMP, ar, ai);
  for (int k = 0; k < kModes; ++k) {
    const float gr = dO[s * 2 * kModes + 2 * k] + dU0[s * kUin + k];
    const float gi = dO[s * 2 * kModes + 2 * k + 1] + dU0[s * kUin + kModes + k];
    for (int l = 0; l < kModes; ++l) {
      // conj(G) a = (gr - j gi)(ar + j ai)
      d[k * 3 + l] = pres * (gr * ar[l] + gi * ai[l]);
      d[9 + k * 3 + l] = -pres * (gr * ai[l] - gi * ar[l]);
    }
  }
}

// x_iso[r][n] = sum_l Minv_p[i][l] b[r][off_p + l] (float64 arithmetic)
template <typename TM>
__global__ void k_xiso(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                       const int32_t* __restrict__ m, const int64_t* __restrict__ moff, const cplx<TM>* __restrict__ Minv,
                       const c128* __restrict__ B, c128* __restrict__ X) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t o = off[p];
  const int i = (int)(n - o), mp = m[p];
  const cplx<TM>* Mi = Minv + moff[p] + (int64_t)i * mp;
  const c128* b = B + (int64_t)r * N + o;
  c128 acc = mkc(0.0, 0.0);
  for (int l = 0; l < mp; ++l) cfma(acc, ccast<double>(Mi[l]), b[l]);
  X[(int64_t)r * N + n] = acc;
}

// Per sample (r, p): x0 on the wire's rows; with targets, the loss partial and dL/do.
__global__ void k_assemble(int64_t nw, int R, int64_t N, const int64_t* __restrict__ off, const int32_t* __restrict__ ns,
                           const double* __restrict__ cx, const double* __restrict__ cy, const double* __restrict__ cz,
                           const double* __restrict__ frames, double k, const float* __restrict__ O,
                           const float* __restrict__ U0, const c128* __restrict__ xiso, c128* __restrict__ x0, const c128* __restrict__ xt,
                           double scale, float* __restrict__ dO, double* __restrict__ lpart) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double l = 0.0;
  if (s < (int64_t)R * nw) {
    const int64_t p = s % nw;
    const int r = (int)(s / nw);
    const double* f = frames + 6 * r;
    double sp, cp;
    sincos(-k * (f[0] * cx[p] + f[1] * cy[p] + f[2] * cz[p]), &sp, &cp);
    const c128 ph = mkc(cp, sp);
    const float* o = O + s * (2 * kModes);
    const float* hu = U0 + s * kUin;
    c128 cm[kModes];
    for (int q = 0; q < kModes; ++q)
      cm[q] = mkc((double)o[2 * q] + (double)hu[q], (double)o[2 * q + 1] + (double)hu[kModes + q]);
    const int nsp = ns[p];
    c128 g[kModes] = {};
    for (int i = 0; i < nsp - 1; ++i) {
      c128 dlt = mkc(0.0, 0.0);
      double md[kModes];
      for (int q = 0; q < kModes; ++q) {
        md[q] = sin((q + 1) * kPi * (i + 1) / nsp);
        dlt = dlt + md[q] * cm[q];
      }
      const int64_t n = (int64_t)r * N + off[p] + i;
      const c128 v = xiso[n] + ph * dlt;
      x0[n] = v;
      if (xt) {
        const c128 res = v - xt[n];
        l += res.re * res.re + res.im * res.im;
        for (int q = 0; q < kModes; ++q) g[q] = g[q] + md[q] * res;
      }
    }
    if (xt) {
      // dL/dRe(c) + j dL/dIm(c) = 2 scale conj(phase) sum_i mode(i) res_i
      const c128 cph = mkc(ph.re, -ph.im);
      for (int q = 0; q < kModes; ++q) {
        const c128 gq = (2.0 * scale) * (cph * g[q]);
        dO[s * (2 * kModes) + 2 * q] = (float)gq.re;
        dO[s * (2 * kModes) + 2 * q + 1] = (float)gq.im;
      }
    }
  }
  if (lpart) {
    __shared__ double red[8];
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
      lpart[blockIdx.x] = t;
    }
  }
}

// Sum of |x|^2 of a complex128 vector, per CTA.
__global__ void k_norm2_part(int64_t n, const c128* __restrict__ x, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i].re * x[i].re + x[i].im * x[i].im;
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < 8; ++i) t += red[i];
    part[blockIdx.x] = t;
  }
}

// Internal <-> caller order of [R][N] complex128 vectors.
__global__ void k_order(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                        const int64_t* __restrict__ uoff, const c128* __restrict__ src, c128* __restrict__ dst,
                        int to_caller) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t u = (int64_t)r * N + uoff[p] + (n - off[p]), v = (int64_t)r * N + n;
  if (to_caller)
    dst[u] = src[v];
  else
    dst[v] = src[u];
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned nb(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, ceil_div(n, t)); }

// Workspace carve-out.
struct Net {
  int64_t S, Me;  // samples, message rows
  int32_t* nbr;
  float *Xe, *Xs, *Z1, *A1, *Z2, *A2, *MSG, *U0, *Z4, *U1, *Z5, *U2, *O;
  float *dO, *dU2, *dU1, *dU0, *dMSG, *dA2, *dA1, *part, *AMP;
  double* frames;
  double* lpart;
  c128 *B64, *xiso, *x0, *xt;
  size_t part_floats;
};

size_t carve(Net& w, void* base, int64_t nw, int R, int64_t N, bool grads) {
  const int64_t S = (int64_t)R * nw, Me = S * kNbr;
  w.S = S;
  w.Me = Me;
  w.part_floats = (size_t)64 * 256 * 256;  // split-K partials of the largest weight gradient
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~size_t(255);
    return base ? (void*)((char*)base + at) : nullptr;
  };
  w.nbr = (int32_t*)take(sizeof(int32_t) * nw * kNbr);
  w.Xe = (float*)take(sizeof(float) * Me * kFe);
  w.Xs = (float*)take(sizeof(float) * S * kFs);
  w.Z1 = (float*)take(sizeof(float) * Me * 128);
  w.A1 = (float*)take(sizeof(float) * Me * 128);
  w.Z2 = (float*)take(sizeof(float) * Me * 128);
  w.A2 = (float*)take(sizeof(float) * Me * 128);
  w.MSG = (float*)take(sizeof(float) * Me * kHm);
  w.U0 = (float*)take(sizeof(float) * S * kUin);
  w.AMP = (float*)take(sizeof(float) * S * 2 * kModes);
  w.Z4 = (float*)take(sizeof(float) * S * 256);
  w.U1 = (float*)take(sizeof(float) * S * 256);
  w.Z5 = (float*)take(sizeof(float) * S * 256);
  w.U2 = (float*)take(sizeof(float) * S * 256);
  w.O = (float*)take(sizeof(float) * S * 2 * kModes);
  w.frames = (double*)take(sizeof(double) * 6 * R);
  w.lpart = (double*)take(sizeof(double) * nb(S, 256) + sizeof(double) * 1024);
  w.B64 = (c128*)take(sizeof(c128) * R * N);
  w.xiso = (c128*)take(sizeof(c128) * R * N);
  w.x0 = (c128*)take(sizeof(c128) * R * N);
  w.xt = (c128*)take(sizeof(c128) * R * N);
  if (grads) {
    w.dO = (float*)take(sizeof(float) * S * 2 * kModes);
    w.dU2 = (float*)take(sizeof(float) * S * 256);
    w.dU1 = (float*)take(sizeof(float) * S * 256);
    w.dU0 = (float*)take(sizeof(float) * S * kUin);
    w.dMSG = (float*)take(sizeof(float) * Me * kHm);
    w.dA2 = (float*)take(sizeof(float) * Me * 128);
    w.dA1 = (float*)take(sizeof(float) * Me * 128);
    w.part = (float*)take(sizeof(float) * w.part_floats);
  }
  return o;
}

template <bool TA, bool TB, int EPI>
void gemm(cudaStream_t st, int64_t M, int N, int64_t K, const float* A, const float* B, const float* bias, float* C,
          float* Z2, int splits = 1, int64_t kchunk = 0) {
  const dim3 grid((unsigned)ceil_div(N, kTN), (unsigned)std::min<int64_t>(65535, ceil_div(M, kTM)), (unsigned)splits);
  k_gemm<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, B, bias, C, Z2, kchunk);
}

// dW[K][N] = X^T dZ over M rows (split over the rows, summed in a fixed order), db = colsum(dZ)
void weight_grad(cudaStream_t st, const Net& w, int64_t M, int Kin, int N, const float* X, const float* dZ,
                 float* dW, float* db) {
  const int splits = (int)std::min<int64_t>(64, std::max<int64_t>(1, ceil_div(M, 4096)));
  const int64_t kchunk = ceil_div(ceil_div(M, splits), kTK) * kTK;
  gemm<true, false, EPI_SPLIT>(st, Kin, N, M, X, dZ, nullptr, w.part, nullptr, splits, kchunk);
  k_split_sum<<<nb((int64_t)Kin * N, 256), 256, 0, st>>>((int64_t)Kin * N, splits, w.part, dW);
  const int rz = (int)std::min<int64_t>(256, std::max<int64_t>(1, ceil_div(M, 4096)));
  const int64_t rchunk = ceil_div(M, rz);
  k_colsum<<<dim3(nb(N, 32), (unsigned)rz), 256, 0, st>>>(M, N, rchunk, dZ, w.part);
  k_split_sum<<<nb(N, 256), 256, 0, st>>>(N, rz, w.part, db);
}

int net_run(swm_net* net, swm_ctx* ctx, int R, const double* inc, const double* x_true, int xt_kind, bool train,
            float lr, double* loss_out, float* grad_out, double* x0_out, int x0_kind) {
  if (!ctx->built) return net->fail(SWM_ESTATE, "the context has no built system");
  if (ctx->dense || !(ctx->rc > 0.0)) return net->fail(SWM_EINVAL, "the network needs a finite coupling radius");
  if (R < 1 || R > 65535 || !inc) return net->fail(SWM_EINVAL, "bad incidence list");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return net->fail(SWM_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = ctx->stream;
  const int64_t nw = ctx->nw, N = ctx->N;
  if (ensure_rowinfo(ctx) < 0 || ensure_user_offsets(ctx) < 0) return net->fail(SWM_ECUDA, ctx->err);
  Net w{};
  const bool grads = x_true != nullptr;
  if ((int64_t)R * nw > ((int64_t)1 << 31) / kNbr)
    return net->fail(SWM_EINVAL, "too many wire-incidence samples for one network call");
  const size_t need = carve(w, nullptr, nw, R, N, grads);
  if (need > net->ws_bytes) {
    if (net->ws) cudaFree(net->ws);
    net->ws = nullptr;
    net->ws_bytes = 0;
    if (cudaMalloc(&net->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return net->fail(SWM_ENOMEM, "network workspace allocation failed");
    }
    net->ws_bytes = need;
  }
  carve(w, net->ws, nw, R, N, grads);
  std::vector<double> fh;
  frames_host(inc, R, fh);
  if (cudaMemcpyAsync(w.frames, fh.data(), sizeof(double) * 6 * R, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return net->fail(SWM_ECUDA, "copy failed");
  // neighbours, features, isolated-wire currents
  k_nbr_select<<<nb(nw, 128), 128, 0, st>>>(nw, ctx->row_ptr, ctx->col, ctx->cx, ctx->cy, ctx->cz, ctx->perm, w.nbr);
  k_features<<<nb(w.Me, 256), 256, 0, st>>>(nw, R, w.nbr, ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz,
                                            ctx->L, w.frames, ctx->k, ctx->rc, w.Xe, w.Xs);
  if (compute_rhs_f64(ctx, R, w.frames, w.B64) < 0) return net->fail(SWM_ECUDA, ctx->err);
  const dim3 gv(nb(N, 256), (unsigned)R);
  if (ctx->prec == SWM_C128)
    k_xiso<double><<<gv, 256, 0, st>>>(N, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off, (const c128*)ctx->Minv,
                                       w.B64, w.xiso);
  else
    k_xiso<float><<<gv, 256, 0, st>>>(N, ctx->rowwire, ctx->off, ctx->m, ctx->minv_off, (const c64*)ctx->Minv,
                                      w.B64, w.xiso);
  // forward
  const float* P = net->params;
  auto Wp = [&](int l) { return P + param_offset(l); };
  auto Bp = [&](int l) { return P + param_offset(l) + (int64_t)kIn[l] * kOut[l]; };
  gemm<false, false, EPI_BIAS_SILU>(st, w.Me, 128, kFe, w.Xe, Wp(0), Bp(0), w.A1, w.Z1);
  gemm<false, false, EPI_BIAS_SILU>(st, w.Me, 128, 128, w.A1, Wp(1), Bp(1), w.A2, w.Z2);
  gemm<false, false, EPI_BIAS>(st, w.Me, kHm, 128, w.A2, Wp(2), Bp(2), w.MSG, nullptr);
  k_amplitudes<<<nb(w.S, 256), 256, 0, st>>>(nw, R, N, ctx->off, ctx->ns, ctx->cx, ctx->cy, ctx->cz, w.frames, ctx->k,
                                              w.xiso, w.AMP);
  k_aggregate<<<nb(w.S, 128), 128, 0, st>>>(w.S, nw, w.nbr, w.MSG, w.Xe, w.Xs, w.AMP, w.U0);
  gemm<false, false, EPI_BIAS_SILU>(st, w.S, 256, kUin, w.U0, Wp(3), Bp(3), w.U1, w.Z4);
  gemm<false, false, EPI_BIAS_SILU>(st, w.S, 256, 256, w.U1, Wp(4), Bp(4), w.U2, w.Z5);
  gemm<false, false, EPI_BIAS>(st, w.S, 2 * kModes, 256, w.U2, Wp(5), Bp(5), w.O, nullptr);
  double scale = 0.0;
  if (grads) {
    const c128* src = (const c128*)x_true;
    c128* staged = nullptr;
    if (xt_kind == SWM_HOST) {
      staged = w.x0;  // staging area, overwritten by the assembly below
      if (cudaMemcpyAsync(staged, x_true, sizeof(c128) * R * N, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return net->fail(SWM_ECUDA, "copy failed");
      src = staged;
    }
    k_order<<<gv, 256, 0, st>>>(N, ctx->rowwire, ctx->off, ctx->uoff, src, w.xt, 0);
    const int nbk = 1024;
    k_norm2_part<<<nbk, 256, 0, st>>>((int64_t)R * N, w.xt, w.lpart);
    std::vector<double> hp(nbk);
    if (cudaMemcpyAsync(hp.data(), w.lpart, sizeof(double) * nbk, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return net->fail(SWM_ECUDA, "copy failed");
    double t = 0.0;
    for (double v : hp) t += v;
    if (!(t > 0.0)) return net->fail(SWM_EINVAL, "target currents are zero");
    scale = 1.0 / t;
  }
  const unsigned gs = nb(w.S, 256);
  k_assemble<<<gs, 256, 0, st>>>(nw, R, N, ctx->off, ctx->ns, ctx->cx, ctx->cy, ctx->cz, w.frames, ctx->k, w.O,
                                 w.U0, w.xiso, w.x0, grads ? w.xt : nullptr, scale, grads ? w.dO : nullptr,
                                 grads ? w.lpart : nullptr);
  if (grads) {
    std::vector<double> hp(gs);
    if (cudaMemcpyAsync(hp.data(), w.lpart, sizeof(double) * gs, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return net->fail(SWM_ECUDA, "copy failed");
    // backward
    float* G = net->grad;
    auto GW = [&](int l) { return G + param_offset(l); };
    auto GB = [&](int l) { return G + param_offset(l) + (int64_t)kIn[l] * kOut[l]; };
    weight_grad(st, w, w.S, 256, 2 * kModes, w.U2, w.dO, GW(5), GB(5));
    gemm<false, true, EPI_DSILU>(st, w.S, 256, 2 * kModes, w.dO, Wp(5), nullptr, w.dU2, w.Z5);  // dZ5
    weight_grad(st, w, w.S, 256, 256, w.U1, w.dU2, GW(4), GB(4));
    gemm<false, true, EPI_DSILU>(st, w.S, 256, 256, w.dU2, Wp(4), nullptr, w.dU1, w.Z4);        // dZ4
    weight_grad(st, w, w.S, kUin, 256, w.U0, w.dU1, GW(3), GB(3));
    gemm<false, true, EPI_NONE>(st, w.S, kUin, 256, w.dU1, Wp(3), nullptr, w.dU0, nullptr);  // dU0
    k_scatter_dmsg<<<nb(w.Me, 128), 128, 0, st>>>(w.S, nw, w.nbr, w.dO, w.dU0, w.Xe, w.AMP, w.dMSG);
    weight_grad(st, w, w.Me, 128, kHm, w.A2, w.dMSG, GW(2), GB(2));
    gemm<false, true, EPI_DSILU>(st, w.Me, 128, kHm, w.dMSG, Wp(2), nullptr, w.dA2, w.Z2);       // dZ2
    weight_grad(st, w, w.Me, 128, 128, w.A1, w.dA2, GW(1), GB(1));
    gemm<false, true, EPI_DSILU>(st, w.Me, 128, 128, w.dA2, Wp(1), nullptr, w.dA1, w.Z1);       // dZ1
    weight_grad(st, w, w.Me, kFe, 128, w.Xe, w.dA1, GW(0), GB(0));
    if (train && lr > 0.f) {
      net->step += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
      k_adam<<<nb(kNumParams, 256), 256, 0, st>>>(kNumParams, net->params, net->grad, net->adam_m, net->adam_v, lr,
                                                  b1, b2, 1e-8f, c1, c2);
    }
    if (grad_out &&
        cudaMemcpyAsync(grad_out, net->grad, sizeof(float) * kNumParams, cudaMemcpyDefault, st) != cudaSuccess)
      return net->fail(SWM_ECUDA, "copy failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return net->fail(SWM_ECUDA, "network kernels failed");
    double l = 0.0;
    for (double v : hp) l += v;
    if (loss_out) *loss_out = l * scale;
  }
  if (x0_out) {
    c128* dst = (c128*)x0_out;
    c128* tmp = nullptr;
    if (x0_kind == SWM_HOST) {
      if (cudaMalloc(&tmp, sizeof(c128) * R * N) != cudaSuccess) {
        cudaGetLastError();
        return net->fail(SWM_ENOMEM, "allocation failed");
      }
      dst = tmp;
    }
    k_order<<<gv, 256, 0, st>>>(N, ctx->rowwire, ctx->off, ctx->uoff, w.x0, dst, 1);
    if (tmp) {
      cudaMemcpyAsync(x0_out, tmp, sizeof(c128) * R * N, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      cudaFree(tmp);
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return net->fail(SWM_ECUDA, "network kernels failed");
  return SWM_OK;
}

}  // namespace

}  // namespace swm

using namespace swm;

extern "C" {

int64_t swm_net_num_params(void) { return kNumParams; }

int swm_net_create(swm_net** out, int device, void* cuda_stream) {
  if (!out) return SWM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SWM_EINVAL;
  }
  swm_net* net = new (std::nothrow) swm_net();
  if (!net) return SWM_ENOMEM;
  net->device = device;
  net->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&net->params, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&net->grad, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&net->adam_m, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&net->adam_v, sizeof(float) * kNumParams) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(net->params);
    cudaFree(net->grad);
    cudaFree(net->adam_m);
    cudaFree(net->adam_v);
    delete net;
    return SWM_ENOMEM;
  }
  cudaMemset(net->params, 0, sizeof(float) * kNumParams);
  cudaMemset(net->adam_m, 0, sizeof(float) * kNumParams);
  cudaMemset(net->adam_v, 0, sizeof(float) * kNumParams);
  cudaDeviceSynchronize();
  *out = net;
  return SWM_OK;
}

void swm_net_destroy(swm_net* net) {
  if (!net) return;
  cudaSetDevice(net->device);
  cudaDeviceSynchronize();
  cudaFree(net->params);
  cudaFree(net->grad);
  cudaFree(net->adam_m);
  cudaFree(net->adam_v);
  if (net->ws) cudaFree(net->ws);
  delete net;
}

const char* swm_net_last_error(const swm_net* net) { return net ? net->err.c_str() : "null network"; }

int swm_net_set_params(swm_net* net, const float* params, int mem_kind) {
  if (!net || !params) return SWM_EINVAL;
  if (cudaSetDevice(net->device) != cudaSuccess ||
      cudaMemcpy(net->params, params, sizeof(float) * kNumParams, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemset(net->adam_m, 0, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMemset(net->adam_v, 0, sizeof(float) * kNumParams) != cudaSuccess) {
    cudaGetLastError();
    return net->fail(SWM_ECUDA, "parameter copy failed");
  }
  (void)mem_kind;
  net->step = 0;
  return SWM_OK;
}

int swm_net_get_params(swm_net* net, float* params, int mem_kind) {
  if (!net || !params) return SWM_EINVAL;
  (void)mem_kind;
  if (cudaSetDevice(net->device) != cudaSuccess ||
      cudaMemcpy(params, net->params, sizeof(float) * kNumParams, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return net->fail(SWM_ECUDA, "parameter copy failed");
  }
  return SWM_OK;
}

int swm_net_predict(swm_net* net, swm_ctx* ctx, int n_inc, const double* inc, double* x0_out, int out_kind) {
  if (!net || !ctx || !x0_out) return SWM_EINVAL;
  net->err.clear();
  return net_run(net, ctx, n_inc, inc, nullptr, SWM_HOST, false, 0.f, nullptr, nullptr, x0_out, out_kind);
}

int swm_net_train_step(swm_net* net, swm_ctx* ctx, int n_inc, const double* inc, const double* x_true, int xt_kind,
                       float lr, double* loss_out, float* grad_out) {
  if (!net || !ctx || !x_true) return SWM_EINVAL;
  if (xt_kind != SWM_HOST && xt_kind != SWM_DEVICE) return net->fail(SWM_EINVAL, "bad memory kind");
  net->err.clear();
  return net_run(net, ctx, n_inc, inc, x_true, xt_kind, true, lr, loss_out, grad_out, nullptr, SWM_HOST);
}

}  // extern "C"
