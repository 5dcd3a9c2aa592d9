// Persistent cooperative GMRES (the whole restarted solve in one launch) for small systems.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "krylov_common.cuh"
#include "rhs_entry.cuh"

namespace swm {

namespace {

// ------------------------------------------------------------------------------------------------
// Persistent solve: the whole restarted GMRES in one cooperative launch, for systems of up to a
// few hundred thousand unknowns with at most 8 right-hand sides.  There one Arnoldi step moves
// only a few megabytes, so launch gaps, host polls and dependent latencies (L2 round trips,
// float64 divides and square roots) set its time, not bandwidth.  Every CTA owns a contiguous
// chunk of rows and keeps in shared memory, when they fit: its slice of the current Krylov
// vector, its rows of the basis V, and its rows of E with their column map and row descriptors
// (loaded once).  The product first gathers the vector at the CTA's column-map slice (the rows
// of one wire share their block-row's column map) into shared memory, each thread's loads issued
// together, and then forms each row's sum from shared memory, four lanes per row.  The basis is orthogonalised by
// classical Gram-Schmidt with its second pass delayed by one step (as in the per-kernel solve),
// so one Arnoldi step is two phases separated by two grid barriers:
//   A: w = A u_j for the pending vector u_j (own rows), partial dots s = Q^H u_j, |u_j|^2,
//      t = Q^H w, u_j^H w
//   B: sums of the partials; rho = |u_j - Q s|, Hessenberg column j-1 completed (first-pass
//      coefficients + s, subdiagonal rho), its Givens rotation, residual estimate and activity;
//      the first-pass coefficients of column j (each CTA forms those of the Hessenberg rows it
//      owns, from its rows of the unrotated matrix); q_j = (u_j - Q s) / rho to V_j and the next
//      pending vector (w - Q t) / rho - (q_j^H w / rho) q_j, written for the next gather
// and a closing phase A/B without product completes the last column of a cycle.  Phase B and
// every partial sum are computed by every CTA from the same partials in the same order, so all
// CTAs reach identical decisions and run identical barrier sequences.  The dot
// products, their sums over the CTAs (in a fixed pairwise order), the rotations and the
// triangular solve run in the precision of the vectors: float64 on the complex128 path, float32 on
// the complex64 path, whose vectors carry float32 rounding anyway (on GB300 a float64 warp
// instruction issues about sixteen times slower than a float32 one, which would otherwise set
// the step time).  The initial residual norm and the relative residual estimate are float64.
// A barrier waits at most kBarrierNs; a CTA that gives up raises an abort flag that the other
// CTAs also poll, every CTA then returns, and the host reports SWM_ETIMEOUT.
constexpr int kPT = 512;              // threads of a persistent-solve CTA
constexpr int kPWarps = kPT / 32;
constexpr int kPersistMaxRowsPerThread = 4;
constexpr unsigned long long kBarrierNs = 1000000000ull;  // 1 s
constexpr unsigned kBarrierMaxPolls = 1u << 26;            // second bound on a wait (>= 1.3 s of sleeps)
constexpr int kPLanesPerRow = 4;                         // lanes per row of the persistent product

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
  unsigned arrivals;       // arrivals a grid barrier waits for (G; more only in the timeout test)
  int vsm, esm;            // V / E slices in shared memory
  int64_t emax, cmax;      // largest E and column-map slice of a CTA (entries)
  int bnorm_given;         // P.bnorm holds |b| (else the first residual norm is |b|)
  int y_zero;              // Y starts at zero: each CTA clears its rows and the first residual is B
  int do_minv;             // at the end, X = M^-1 Y on the CTA's rows
  const int32_t* rowwire;  // scalar row -> wire
  const int64_t* off;      // first unknown of each wire
  const int32_t* mw;       // unknowns per wire
  const int64_t* minv_off; // M^-1 block of each wire (row-major m x m)
  const void* Minv;
  void* X;
  const double* frames;    // non-null: the first residual forms B (and stores it) from these frames
  double k;
  RhsGeo geo;
};

// Byte offsets of the shared-memory arrays of the persistent kernel.
struct PLayout {
  size_t h1, h2, yv, gg, sn, col, hr, ri, ys, ws, vs, es, xg, cs, cm, total;
};
__host__ __device__ inline size_t p_align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline PLayout persist_layout(int RB, int R, int restart, int rows, int hown, size_t cb,
                                                  size_t eb, int vsm, int esm, int64_t emax, int64_t cmax) {
  PLayout L;
  const size_t R1 = restart + 1;
  size_t o = 0;
  L.yv = o; o += sizeof(c128) * RB * restart;
  L.h1 = o; o += p_align16(cb * RB * R1);  // coefficients and rotations in the vector precision
  L.h2 = o; o += p_align16(cb * RB * R1);
  L.gg = o; o += p_align16(cb * RB * R1);
  L.sn = o; o += p_align16(cb * RB * restart);
  L.col = o; o += p_align16(cb * RB * R1);
  L.hr = o; o += p_align16(cb * RB * (size_t)hown * restart);
  L.ri = o; o += esm ? 16 * (size_t)rows : 0;
  L.ys = o; o += p_align16(cb * RB * rows);
  L.ws = o; o += p_align16(cb * RB * rows);
  L.vs = o; o += vsm ? p_align16(cb * R1 * R * rows) : 0;
  L.es = o; o += esm ? p_align16(eb * (size_t)emax) : 0;
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
// or saw another CTA give up.  Thread 0 arrives with an acquire-release add on the counter (its
// release covers the CTA's writes before the __syncthreads); the arrival that completes the
// barrier has acquired every earlier one, the others poll the counter with acquire loads.
__device__ bool grid_sync(PSync* s, unsigned G, unsigned* epoch, int* ok_sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (*epoch + 1u) * G;
    *epoch += 1u;
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(&s->count) : "memory");
    int ok = 1;
    if (prev + 1u != target) {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (ld_acquire_u32(&s->count) < target) {
        if (*(volatile int*)&s->abort) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > kBarrierNs || ++polls > kBarrierMaxPolls) {
          atomicExch(&s->abort, 1);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
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

// The sums of both partial arrays in one pass (every warp's loads of one item in flight together):
// d1[b][i] from p1 and, unless closing, d2[b][i] from p2, for active b and i <= j.
template <typename T>
__device__ void p_reduce2(const cplx<T>* __restrict__ p1, const cplx<T>* __restrict__ p2, int G, int R, int R1, int j,
                          const int* act, bool closing, cplx<T>* d1, cplx<T>* d2) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int per = R * (j + 1);
  const int nt = closing ? per : 2 * per;
  for (int k = wp; k < nt; k += kPWarps) {
    const int which = k / per, rest = k % per;
    const int b = rest / (j + 1), i = rest % (j + 1);
    if (!act[b]) continue;
    const cplx<T> v = sum_g_c<T>((which ? p2 : p1) + (int64_t)(b * R1 + i) * G, G, lane);
    if (lane == 0) (which ? d2 : d1)[b * R1 + i] = v;
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

// Partial dots of the delayed Gram-Schmidt over the CTA's rows, for active b: part1[b][i] =
// conj(V_i[b]) . u[b] and part2[b][i] = conj(V_i[b]) . w[b] for i < j, and at i = j the same with
// u[b] in place of V_i[b] (|u|^2, u^H w); the closing pass (no product) fills part1 only.
template <typename TV>
__device__ void p_dots2(const VRows<TV>& V, const cplx<TV>* ys, const cplx<TV>* ws, int rows, int cnt, int R, int R1,
                        int j, int G, const int* act, bool closing, cplx<TV>* __restrict__ part1,
                        cplx<TV>* __restrict__ part2) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int nt = R * (j + 1);
  for (int k = wp; k < nt; k += kPWarps) {
    const int b = k / (j + 1), i = k % (j + 1);
    if (!act[b]) continue;
    const cplx<TV>* u = ys + b * rows;
    const cplx<TV>* w = ws + b * rows;
    const cplx<TV>* vi = i < j ? V.at(i, b) : u;
    cplx<TV> a = mkc<TV>(0, 0), c = mkc<TV>(0, 0);
    int t = lane;
    for (; t + 96 < cnt; t += 128) {
      cplx<TV> v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = vi[t + 32 * q];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const cplx<TV> x = u[t + 32 * q];
        a.re = fma(v[q].re, x.re, fma(v[q].im, x.im, a.re));
        a.im = fma(v[q].re, x.im, fma(-v[q].im, x.re, a.im));
        if (!closing) {
          const cplx<TV> y = w[t + 32 * q];
          c.re = fma(v[q].re, y.re, fma(v[q].im, y.im, c.re));
          c.im = fma(v[q].re, y.im, fma(-v[q].im, y.re, c.im));
        }
      }
    }
    for (; t < cnt; t += 32) {
      const cplx<TV> v = vi[t], x = u[t];
      a.re = fma(v.re, x.re, fma(v.im, x.im, a.re));
      a.im = fma(v.re, x.im, fma(-v.im, x.re, a.im));
      if (!closing) {
        const cplx<TV> y = w[t];
        c.re = fma(v.re, y.re, fma(v.im, y.im, c.re));
        c.im = fma(v.re, y.im, fma(-v.im, y.re, c.im));
      }
    }
    const TV are = warp_sum(a.re), aim = warp_sum(a.im);
    const TV cre = warp_sum(c.re), cim = warp_sum(c.im);
    if (lane == 0) {
      part1[(int64_t)(b * R1 + i) * G + blockIdx.x] = mkc<TV>(are, aim);
      if (!closing) part2[(int64_t)(b * R1 + i) * G + blockIdx.x] = mkc<TV>(cre, cim);
    }
  }
}

// The update of the delayed Gram-Schmidt over the CTA's rows, for active b: q = (u - sum_{i<j}
// V_i s_i) / rho goes to V_j and u' = (w - sum_{i<j} V_i t_i) / rho - gamma q replaces u in ys and
// in the global vector W (for the next gather).
template <typename TV, int RB>
__device__ void p_update2(const VRows<TV>& V, cplx<TV>* ys, const cplx<TV>* ws, int rows, int cnt, int64_t n0,
                          int64_t N, int R, int R1, int j, const int* act, const cplx<TV>* sv, const cplx<TV>* tv,
                          const TV* invr, const cplx<TV>* gam, cplx<TV>* __restrict__ W) {
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    if (b >= R) break;
    if (!act[b]) continue;
    const cplx<TV>* sb = sv + b * R1;
    const cplx<TV>* tb = tv + b * R1;
    const TV ir = invr[b];
    const cplx<TV> gm = gam[b];
    cplx<TV>* vj = V.at(j, b);
    for (int t = threadIdx.x; t < cnt; t += kPT) {
      cplx<TV> x = ys[b * rows + t], y = ws[b * rows + t];
      int i = 0;
      for (; i + 3 < j; i += 4) {
        cplx<TV> v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = V.at(i + q, b)[t];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const cplx<TV> a = sb[i + q], c = tb[i + q];
          x.re = fma(-v[q].re, a.re, fma(v[q].im, a.im, x.re));
          x.im = fma(-v[q].re, a.im, fma(-v[q].im, a.re, x.im));
          y.re = fma(-v[q].re, c.re, fma(v[q].im, c.im, y.re));
          y.im = fma(-v[q].re, c.im, fma(-v[q].im, c.re, y.im));
        }
      }
      for (; i < j; ++i) {
        const cplx<TV> v = V.at(i, b)[t];
        const cplx<TV> a = sb[i], c = tb[i];
        x.re = fma(-v.re, a.re, fma(v.im, a.im, x.re));
        x.im = fma(-v.re, a.im, fma(-v.im, a.re, x.im));
        y.re = fma(-v.re, c.re, fma(v.im, c.im, y.re));
        y.im = fma(-v.re, c.im, fma(-v.im, c.re, y.im));
      }
      const cplx<TV> q = ir * x;
      vj[t] = q;
      const cplx<TV> un = ir * y - q * gm;
      ys[b * rows + t] = un;
      W[(int64_t)b * N + n0 + t] = un;
    }
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

// The CTA's slice of E: values, column map, row descriptors, and the gathered vector entries.
template <typename TV, typename TE>
struct ESlice {
  const TE* e;
  const int32_t* cm;
  const RowInfo* ri;
  int64_t ebase, cbase;  // subtracted from the descriptors' offsets
  cplx<TV>* xg;          // [R][cstride] gathered vector at the column-map slice (shared) or null
  int clen, cstride;
};

// Rows of the CTA times A = I + E for the R right-hand sides of `src`.
// mode 0 (Arnoldi): ws = u + E u for the pending vector u (own rows in ys, all rows in src).
// mode 1 (residual): ys = W = B - (Y + E Y), squared norms to partn.
template <typename TV, typename TE, int RB>
__device__ void p_product(int mode, const PArgs& a, const ESlice<TV, TE>& S, const cplx<TV>* __restrict__ src,
                          cplx<TV>* ys, cplx<TV>* ws, int cnt, int64_t n0, const int* act,
                          const cplx<TV>* __restrict__ B, cplx<TV>* __restrict__ W, TV (*red)[RB]) {
  const int R = a.P.R;
  const int64_t N = a.P.N;
  bool on[RB];
  TV nrm[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) {
    on[b] = b < R && (mode == 1 || act[b]);
    nrm[b] = 0;
  }
  if (S.xg) {
    // gather src at the column-map slice: a thread's GB entries (all right-hand sides) are loaded
    // before any is stored, so they are in flight together
    constexpr int GB = RB >= 8 ? 1 : 8 / RB;
    for (int q0 = threadIdx.x; q0 < S.clen; q0 += GB * kPT) {
      int col[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int q = q0 + u * kPT;
        col[u] = q < S.clen ? S.cm[q] : -1;
      }
      cplx<TV> v[GB][RB];
#pragma unroll
      for (int u = 0; u < GB; ++u)
#pragma unroll
        for (int b = 0; b < RB; ++b)
          v[u][b] = (col[u] >= 0 && on[b]) ? ldcg_c<TV>(src + (int64_t)b * N + col[u]) : mkc<TV>(0, 0);
#pragma unroll
      for (int u = 0; u < GB; ++u)
#pragma unroll
        for (int b = 0; b < RB; ++b)
          if (col[u] >= 0 && on[b]) S.xg[b * S.cstride + q0 + u * kPT] = v[u][b];
    }
    __syncthreads();
  }
  // four lanes per row, each taking every fourth entry, so that the rows of a dense part of the
  // cloud spread over the CTA's threads; passes over the rows are warp-uniform (quad sums below)
  const int lane = threadIdx.x & 31, sub = lane & (kPLanesPerRow - 1);
  constexpr int rows_per_warp = 32 / kPLanesPerRow;
  for (int base = (int)(threadIdx.x >> 5) * rows_per_warp; base < cnt; base += kPWarps * rows_per_warp) {
    const int t = base + lane / kPLanesPerRow;
    const bool live = t < cnt;
    cplx<TV> acc[RB];
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[b] = mkc<TV>(0, 0);
    if (live) {
      const RowInfo ri = S.ri[t];
      const TE* e = S.e + (ri.vb - S.ebase);
      if (S.xg) {
        const cplx<TV>* xq = S.xg + (ri.cmb - S.cbase);
#pragma unroll 2
        for (int c = sub; c < ri.K; c += kPLanesPerRow) {
          const cplx<TV> ev = ELoad<TV, TE>::ld(e + c);
#pragma unroll
          for (int b = 0; b < RB; ++b)
            if (on[b]) cfma(acc[b], ev, xq[b * S.cstride + c]);
        }
      } else {
        const int32_t* cm = S.cm + (ri.cmb - S.cbase);
#pragma unroll 2
        for (int c = sub; c < ri.K; c += kPLanesPerRow) {
          const cplx<TV> ev = ELoad<TV, TE>::ld(e + c);
          const int64_t col = cm[c];
#pragma unroll
          for (int b = 0; b < RB; ++b)
            if (on[b]) cfma(acc[b], ev, ldcg_c<TV>(src + (int64_t)b * N + col));
        }
      }
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (b >= R) break;
#pragma unroll
      for (int o = 1; o < kPLanesPerRow; o <<= 1) {
        acc[b].re += __shfl_xor_sync(0xffffffffu, acc[b].re, o);
        acc[b].im += __shfl_xor_sync(0xffffffffu, acc[b].im, o);
      }
    }
    if (!live || sub != 0) continue;
    const int64_t n = n0 + t;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (!on[b]) continue;
      if (mode == 0) {
        ws[b * a.rows + t] = ys[b * a.rows + t] + acc[b];
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

// The first residual when Y starts at zero: the CTA's rows of Y cleared, ys = W = B on its rows,
// squared norms to partn (no product).  With a.frames the CTA forms its rows of B first.
template <typename TV, int RB>
__device__ void p_residual_zero(const PArgs& a, cplx<TV>* ys, int cnt, int64_t n0, cplx<TV>* B,
                                cplx<TV>* __restrict__ Y, cplx<TV>* __restrict__ W, TV (*red)[RB]) {
  const int R = a.P.R;
  const int64_t N = a.P.N;
  TV nrm[RB];
#pragma unroll
  for (int b = 0; b < RB; ++b) nrm[b] = 0;
  for (int t = threadIdx.x; t < cnt; t += kPT) {
    int64_t p = 0;
    int l = 0;
    if (a.frames) {
      p = a.rowwire[n0 + t];
      l = (int)(n0 + t - a.off[p]);
    }
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      if (b >= R) break;
      const int64_t row = (int64_t)b * N + n0 + t;
      cplx<TV> r;
      if (a.frames) {
        r = rhs_entry<TV>(a.geo, p, l, a.frames + 6 * b, a.k);
        B[row] = r;
      } else {
        r = B[row];
      }
      Y[row] = mkc<TV>(0, 0);
      ys[b * a.rows + t] = r;
      W[row] = r;
      nrm[b] = fma(r.re, r.re, fma(r.im, r.im, nrm[b]));
    }
  }
  p_norm_partials<TV, RB>(nrm, R, a.G, (TV*)a.partn, red);
}

template <typename TV, typename TE, int RB>
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
  const int hown = (R1 + G - 1) / G;  // rows of the unrotated Hessenberg matrix this CTA owns, at most
  const PLayout L = persist_layout(RB, R, RS, a.rows, hown, sizeof(C), sizeof(TE), a.vsm, a.esm, a.emax, a.cmax);
  C* h1 = reinterpret_cast<C*>(sm_raw + L.h1);         // [RB][R1] sums Q^H u, with |u|^2 last
  C* h2 = reinterpret_cast<C*>(sm_raw + L.h2);         // [RB][R1] sums Q^H w, with u^H w last
  c128* yv = reinterpret_cast<c128*>(sm_raw + L.yv);   // [RB][RS] back-solve / coefficients
  C* part1 = (C*)a.part1;
  C* part2 = (C*)a.part2;
  TV* partn = (TV*)a.partn;
  C* gg = reinterpret_cast<C*>(sm_raw + L.gg);         // [RB][R1] rotated residual
  C* sn = reinterpret_cast<C*>(sm_raw + L.sn);         // [RB][RS] rotation sines
  C* colv = reinterpret_cast<C*>(sm_raw + L.col);      // [RB][R1] Hessenberg column
  C* hrs = reinterpret_cast<C*>(sm_raw + L.hr);        // [RB][hown][RS] own rows, unrotated
  TV* cs = reinterpret_cast<TV*>(sm_raw + L.cs);       // [RB][RS] rotation cosines
  C* ys = reinterpret_cast<C*>(sm_raw + L.ys);         // [RB][rows] pending vector u (own rows)
  C* ws = reinterpret_cast<C*>(sm_raw + L.ws);         // [RB][rows] w = A u (own rows)
  VRows<TV> V;
  V.R = R;
  if (a.vsm) {
    V.base = reinterpret_cast<C*>(sm_raw + L.vs);
    V.stride = a.rows;
  } else {
    V.base = (C*)a.V + n0;
    V.stride = N;
  }
  ESlice<TV, TE> S;
  S.e = (const TE*)a.E;
  S.cm = a.colmap;
  S.ri = a.rinfo + n0;
  S.ebase = 0;
  S.cbase = 0;
  S.xg = nullptr;
  S.clen = 0;
  S.cstride = 0;
  if (a.esm && cnt > 0) {
    RowInfo* ri_s = reinterpret_cast<RowInfo*>(sm_raw + L.ri);
    TE* e_s = reinterpret_cast<TE*>(sm_raw + L.es);
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
  __shared__ TV nrm2[RB], rho_s[RB], invr[RB];
  __shared__ C gam[RB];
  __shared__ TV red[kPWarps][RB];
  __shared__ int act[RB], jl[RB];
  __shared__ int s_j, s_jmax, s_iters, s_done, s_conv, s_numeric, s_cycles, s_ok;
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
      if (!(ok = grid_sync(a.sync, a.arrivals, &s_epoch, &s_ok))) break;
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
      if (!(ok = grid_sync(a.sync, a.arrivals, &s_epoch, &s_ok))) break;
    }
    // ---- residual W = B - A Y on the CTA's rows, its squared norms
    if (first && a.y_zero)
      p_residual_zero<TV, RB>(a, ys, cnt, n0, (C*)a.B, Y, W, red);
    else
      p_product<TV, TE, RB>(1, a, S, Y, ys, ws, cnt, n0, act, B, W, red);
    if (!(ok = grid_sync(a.sync, a.arrivals, &s_epoch, &s_ok))) break;
    // ---- start of a cycle (every CTA)
    if (wp < R) {
      const TV t = sum_g_d<TV>(partn + (int64_t)wp * G, G, lane);
      if (lane == 0) nrm2[wp] = t;
    }
    __syncthreads();
    if (threadIdx.x < R) {
      const int b = threadIdx.x;
      const double beta = sqrt((double)nrm2[b]);
      if (first) bnorm[b] = a.bnorm_given ? P.bnorm[b] : (beta > 0.0 ? beta : 1.0);
      const double res = beta / bnorm[b];
      resid[b] = res;
      jl[b] = 0;
      const bool ac = isfinite(res) && res > P.tol;
      if (!isfinite(res)) s_numeric = 1;
      act[b] = ac ? 1 : 0;
      gg[b * R1] = mkc<TV>((TV)beta, TV(0));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int any = 0;
      for (int b = 0; b < R; ++b) any |= act[b];
      s_conv = any ? 0 : 1;
      s_j = 0;
      s_jmax = min(RS, a.max_iter - s_iters);
      s_done = (!any || s_iters >= a.max_iter) ? 1 : 0;
      if (!first) s_cycles += 1;
    }
    __syncthreads();
    first = false;
    if (s_conv || s_numeric || s_iters >= a.max_iter) break;
    // ---- Arnoldi steps (u_0 = the residual, in ys and W), then the closing pass
    while (!s_done) {
      const int j = s_j;
      const bool closing = j >= s_jmax;
      // A: w = A u_j on own rows, partial dots
      if (!closing) p_product<TV, TE, RB>(0, a, S, W, ys, ws, cnt, n0, act, B, W, red);
      __syncthreads();
      p_dots2<TV>(V, ys, ws, a.rows, cnt, R, R1, j, G, act, closing, part1, part2);
      if (!(ok = grid_sync(a.sync, a.arrivals, &s_epoch, &s_ok))) break;
      // B1: sums (s and |u|^2 in h1, t and u^H w in h2) and the first-pass coefficients of
      // column j-1, formed at the previous step by the owners of their rows
      const c128* hc_prev = ((j - 1) & 1) ? P.hc2 : P.hc;
      c128* hc_next = (j & 1) ? P.hc2 : P.hc;
      // a thread's first entry of column j-1 is loaded before the sums, so the two loads share
      // one round trip to L2
      const bool pre = j > 0 && (int)threadIdx.x < R * j && act[threadIdx.x / j];
      const c128 hpre = pre ? ldcg_c<double>(hc_prev + (int64_t)(threadIdx.x / j) * R1 + threadIdx.x % j)
                            : mkc(0.0, 0.0);
      p_reduce2<TV>(part1, part2, G, R, R1, j, act, closing, h1, h2);
      if (pre) colv[(threadIdx.x / j) * R1 + threadIdx.x % j] = ccast<TV>(hpre);
      for (int k = threadIdx.x + kPT; k < R * j; k += kPT) {
        const int b = k / j, i = k % j;
        if (act[b]) colv[b * R1 + i] = ccast<TV>(ldcg_c<double>(hc_prev + (int64_t)b * R1 + i));
      }
      __syncthreads();
      // B2: the unrotated column j-1 (first-pass coefficients + s, subdiagonal rho), with
      // rho = |u - Q s| = sqrt(|u|^2 - |s|^2) and gamma = q_j^H w / rho = (u^H w - s^H t) / rho^2
      for (int k = threadIdx.x; k < R * j; k += kPT) {
        const int b = k / j, i = k % j;
        if (act[b]) colv[b * R1 + i] = colv[b * R1 + i] + h1[b * R1 + i];
      }
      // the activity before this step's rotations, for B3 (which runs beside them)
      unsigned actm = 0;
      for (int b = 0; b < R; ++b) actm |= act[b] ? 1u << b : 0u;
      if (wp < R && act[wp]) {
        const int b = wp;
        TV ss = 0, gr = 0, gi = 0;
        for (int i = lane; i < j; i += 32) {
          const C sv = h1[b * R1 + i];
          ss += sv.re * sv.re + sv.im * sv.im;
          if (!closing) {
            const C p = cmulc(sv, h2[b * R1 + i]);
            gr += p.re;
            gi += p.im;
          }
        }
        ss = warp_sum(ss);
        gr = warp_sum(gr);
        gi = warp_sum(gi);
        if (lane == 0) {
          const TV al = h1[b * R1 + j].re - ss;
          const TV rho = !isfinite(al) ? al : (al > TV(0) ? sqrt(al) : TV(0));
          rho_s[b] = rho;
          const TV ir = rho > TV(0) ? TV(1) / rho : TV(0);
          invr[b] = ir;
          if (!closing) gam[b] = (ir * ir) * (h2[b * R1 + j] - mkc<TV>(gr, gi));
          if (j >= 1) colv[b * R1 + j] = mkc<TV>(rho, TV(0));
        }
      }
      __syncthreads();
      // B3 (all warps but the last): rows k = blockIdx.x + m G (m < hown) of the unrotated matrix
      // belong to this CTA and live in its shared memory: store their entries of column j-1, and
      // form their first-pass coefficients of column j, (t_k - (H s)_k) / rho, and gamma - s_{j-1}
      // for row j.  B3 reads the unrotated column, which B4 leaves in place.
      if ((int)blockIdx.x <= j && wp < kPWarps - 1) {
        const int nown = (j - (int)blockIdx.x) / G + 1;
        for (int pr = wp; pr < nown * R; pr += kPWarps - 1) {
          const int m = pr / R, b = pr % R;
          const int k = (int)blockIdx.x + m * G;
          if (!((actm >> b) & 1u)) continue;
          C* hr = hrs + ((int64_t)b * hown + m) * RS;
          if (j >= 1 && lane == 0) hr[j - 1] = colv[b * R1 + k];
          if (closing) continue;
          if (k < j) {
            TV cr = 0, ci = 0;
            for (int i = (k > 0 ? k - 1 : 0) + lane; i < j; i += 32) {
              const C h = i == j - 1 ? colv[b * R1 + k] : hr[i];
              const C sv = h1[b * R1 + i];
              cr += h.re * sv.re - h.im * sv.im;
              ci += h.re * sv.im + h.im * sv.re;
            }
            cr = warp_sum(cr);
            ci = warp_sum(ci);
            if (lane == 0)
              hc_next[(int64_t)b * R1 + k] = ccast<double>(invr[b] * (h2[b * R1 + k] - mkc<TV>(cr, ci)));
          } else if (lane == 0) {
            hc_next[(int64_t)b * R1 + k] = ccast<double>(j >= 1 ? gam[b] - h1[b * R1 + j - 1] : gam[b]);
          }
        }
      }
      // B4 (lanes of the last warp, beside B3): rotations of column j-1, residual estimate and
      // activity (every CTA, same values); CTA 0 stores the rotated column to H
      if (wp == kPWarps - 1 && lane < R && act[lane]) {
        const int b = lane;
        const TV h = rho_s[b];
        if (j >= 1) {
          const int l = j - 1;
          const C* col = colv + b * R1;
          c128* Hc = P.H + (int64_t)b * R1 * RS + l;
          const bool keep = blockIdx.x == 0;
          C xr = col[0];  // entry i of the column, rotated by the rotations before i
          for (int i = 0; i < l; ++i) {
            const C x0 = xr, x1 = col[i + 1];
            const C sg = sn[b * RS + i];
            const TV c = cs[b * RS + i];
            if (keep) Hc[(int64_t)i * RS] = ccast<double>(c * x0 + sg * x1);
            xr = mkc<TV>(-sg.re, sg.im) * x0 + c * x1;
          }
          const C x = xr;
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
          cs[b * RS + l] = c;
          sn[b * RS + l] = sv;
          if (keep) Hc[(int64_t)l * RS] = ccast<double>(c * x + h * sv);
          const C gl = gg[b * R1 + l];
          gg[b * R1 + l + 1] = mkc<TV>(-sv.re, sv.im) * gl;
          gg[b * R1 + l] = c * gl;
          // |g_{l+1}| = |s_l| |g_l| with |s_l| = h / nu
          const double res = resid[b] * (double)(h * inu);
          resid[b] = res;
          jl[b] = j;
          if (!isfinite(h) || !isfinite(res)) {
            s_numeric = 1;
            act[b] = 0;
          } else if (res <= P.tol || h == TV(0)) {
            act[b] = 0;
          }
        } else {
          gg[b * R1] = mkc<TV>(h, TV(0));
          if (!isfinite(h)) s_numeric = 1;
          if (!(h > TV(0)) || !isfinite(h)) act[b] = 0;
        }
      }
      __syncthreads();
      // every thread reads the new activity (thread 0 keeps the counters)
      int any = 0;
      for (int b = 0; b < R; ++b) any |= act[b];
      const bool done = !any || closing;
      if (threadIdx.x == 0) {
        s_j = j + 1;
        if (j >= 1) s_iters += 1;
        s_done = done ? 1 : 0;
      }
      if (done) break;
      // B5: q_j to V_j and the next pending vector (own rows and W), then the barrier that makes
      // W whole for the next gather
      p_update2<TV, RB>(V, ys, ws, a.rows, cnt, n0, N, R, R1, j, act, h1, h2, invr, gam, W);
      if (!(ok = grid_sync(a.sync, a.arrivals, &s_epoch, &s_ok))) break;
    }
    if (!ok) break;
  }
  // ---- x = M^-1 y on the CTA's rows: the loop left after the grid barrier of a cycle's start, so
  // every row of y is final (read through L2: rows of a wire can belong to the next CTA)
  if (ok && a.do_minv) {
    const C* Mi = (const C*)a.Minv;
    C* X = (C*)a.X;
    for (int k = threadIdx.x; k < R * cnt; k += kPT) {
      const int b = k / cnt, t = k % cnt;
      const int64_t n = n0 + t;
      const int p = a.rowwire[n];
      const int64_t o = a.off[p];
      const int i = (int)(n - o), mp = a.mw[p];
      const C* row = Mi + a.minv_off[p] + (int64_t)i * mp;
      const C* y = Y + (int64_t)b * N + o;
      C acc = mkc<TV>(0, 0);
      for (int l = 0; l < mp; ++l) cfma(acc, row[l], ldcg_c<TV>(y + l));
      X[(int64_t)b * N + n] = acc;
    }
  }
  // ---- the last CTA to leave clears the barrier counter for the next launch (every other CTA has
  // passed its last barrier); after a timeout the host clears the state instead
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.sync->exits, 1u) == gridDim.x - 1) {
      a.sync->count = 0;
      a.sync->exits = 0;
      __threadfence();
    }
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


}  // namespace

template <typename TV, typename TE>
int gmres_persistent(swm_ctx* ctx, const KPtr& P, const PBuffers& Bf, int max_iter, KState* hs, bool* done) {
  *done = false;
  cudaStream_t st = ctx->stream;
  const int R = P.R, restart = P.restart;
  const int64_t N = P.N;
  const int ctas = ctx->persist_ctas > 0 ? std::min(ctx->persist_ctas, std::max(ctx->nsm, 1)) : std::max(ctx->nsm, 1);
  const int prows = (int)(ceil_div(ceil_div(std::max<int64_t>(N, 1), ctas), 32) * 32);
  if (!(ctx->persist && ctx->coop && Bf.sync && R <= kPersistMaxR && N > 0 && N < ctx->split_rows &&
        prows <= kPersistMaxRowsPerThread * kPT))
    return SWM_OK;
  const int G = (int)ceil_div(N, prows);
  const int RB = R == 1 ? 1 : kPersistMaxR;
  const void* fn = R == 1 ? (const void*)k_gmres_persist<TV, TE, 1> : (const void*)k_gmres_persist<TV, TE, kPersistMaxR>;
  size_t static_smem = 0;
  SWM_CK(allow_max_dyn_smem(fn, ctx->smem_optin, &static_smem));
  const size_t limit = (size_t)std::max(0, ctx->smem_optin - (int)static_smem - 1024);
  const size_t cb = sizeof(cplx<TV>), eb = sizeof(TE);
  // V in shared memory when it fits (it is read twice a step); then as large an E slice as
  // the rest holds (column map + gathered vector about a third of the E entries: the rows of a
  // wire share their column map).  A CTA whose slice is larger reads E from global memory.
  const int hown = (int)ceil_div(restart + 1, G);
  const int vsm = persist_layout(RB, R, restart, prows, hown, cb, eb, 1, 0, 0, 0).total <= limit ? 1 : 0;
  const size_t base = persist_layout(RB, R, restart, prows, hown, cb, eb, vsm, 1, 0, 0).total + 64;
  const int64_t mean_e = ceil_div(ctx->offd.nval, G);
  int64_t emax = 0, cmax = 0;
  if (base < limit) {
    emax = (int64_t)((limit - base) / (eb + (4 + cb * R) / 3.0));
    cmax = emax / 3;
  }
  const int esm = emax >= mean_e && emax > 0 ? 1 : 0;
  if (!esm) emax = cmax = 0;
  const size_t smem = persist_layout(RB, R, restart, prows, hown, cb, eb, vsm, esm, emax, cmax).total;
  if (smem > limit) return SWM_OK;
  int occ = 0;
  SWM_CK(occupancy_cached(fn, kPT, smem, &occ));
  if (occ < 1 || G > occ * ctx->nsm) return SWM_OK;
  PArgs pa{};
  pa.P = P;
  pa.sync = Bf.sync;
  pa.rinfo = (const RowInfo*)ctx->rowinfo;
  pa.colmap = ctx->offd.colmap;
  pa.E = Bf.E;
  pa.B = Bf.B;
  pa.Y = Bf.Y;
  pa.W = Bf.W;
  pa.V = Bf.V;
  pa.part1 = Bf.part1;
  pa.part2 = Bf.part2;
  pa.partn = Bf.partn;
  pa.G = G;
  pa.arrivals = (unsigned)(G + ctx->test_barrier_extra);
  pa.rows = prows;
  pa.max_iter = max_iter;
  pa.vsm = vsm;
  pa.esm = esm;
  pa.emax = emax;
  pa.cmax = cmax;
  pa.bnorm_given = Bf.bnorm_given;
  pa.y_zero = Bf.y_zero;
  pa.do_minv = Bf.X ? 1 : 0;
  pa.rowwire = ctx->rowwire;
  pa.off = ctx->off;
  pa.mw = ctx->m;
  pa.minv_off = ctx->minv_off;
  pa.Minv = ctx->Minv;
  pa.X = Bf.X;
  pa.frames = Bf.frames;
  pa.k = ctx->k;
  pa.geo = RhsGeo{ctx->cx, ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->ns};
  if (!*Bf.sync_clean) SWM_CK(cudaMemsetAsync(Bf.sync, 0, sizeof(PSync), st));
  *Bf.sync_clean = false;  // until persist_result has seen the launch end without a timeout
  void* args[] = {&pa};
  ctx->prof_begin(SWM_K_GMRES);
  SWM_CK(cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(kPT), args, smem, st));
  ctx->prof_end(SWM_K_GMRES);
  SWM_LAUNCHED();
  // the final state and the abort flag go to pinned memory; the caller reads them after its next
  // synchronisation (persist_result)
  SWM_TRY(ensure_poll_slots(ctx));
  char* pin = static_cast<char*>(ctx->pinned_state);
  SWM_CK(cudaMemcpyAsync(pin + kPersistStateOffset, P.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
  SWM_CK(cudaMemcpyAsync(pin + kPersistAbortOffset, &Bf.sync->abort, sizeof(int), cudaMemcpyDeviceToHost, st));
  *done = true;
  (void)hs;
  return SWM_OK;
}

int persist_result(swm_ctx* ctx, KState* hs, bool* sync_clean) {
  const char* pin = static_cast<const char*>(ctx->pinned_state);
  std::memcpy(hs, pin + kPersistStateOffset, sizeof(KState));
  int abort = 0;
  std::memcpy(&abort, pin + kPersistAbortOffset, sizeof(int));
  if (abort) return ctx->fail(SWM_ETIMEOUT, "GMRES: a grid barrier of the persistent solve timed out");
  *sync_clean = true;
  return SWM_OK;
}

template int gmres_persistent<double, c128>(swm_ctx*, const KPtr&, const PBuffers&, int, KState*, bool*);
template int gmres_persistent<float, c64>(swm_ctx*, const KPtr&, const PBuffers&, int, KState*, bool*);
template int gmres_persistent<float, __nv_bfloat162>(swm_ctx*, const KPtr&, const PBuffers&, int, KState*, bool*);

}  // namespace swm
