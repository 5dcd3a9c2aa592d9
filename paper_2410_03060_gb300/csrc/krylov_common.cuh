// Device state shared by the GMRES kernels (krylov.cu, persist.cu) and the loaders of the stored
// matrix E in its storage precisions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "ctx.h"

namespace swm {

struct KState {
  int j;          // Arnoldi step inside the cycle
  int cycle_done; // no active right-hand side left in this cycle
  int all_conv;   // every right-hand side met tol at the start of this cycle
  int iters;      // total Arnoldi steps
  int numeric;    // a NaN/Inf appeared
  int cycles;     // restart cycles (persistent solve)
  int jmax;       // Hessenberg columns of this cycle (per-kernel solve)
  int pad;
};

struct KPtr {
  KState* st;
  unsigned* counter;  // [R]
  int* active;        // [R]
  int* jlast;         // [R]
  double* inv_h;      // [R]
  double* bnorm;      // [R]
  double* resid;      // [R]
  c128* H;            // [R][(restart + 1) * restart], Givens-rotated
  c128* Hraw;         // [R][(restart + 1) * restart], as formed (per-kernel solve)
  double* cs;         // [R][restart]
  c128* sn;           // [R][restart]
  c128* g;            // [R][restart + 1]
  c128* hc;           // [R][restart + 1]
  c128* hc2;          // [R][restart + 1]
  c128* ht;           // [R][restart + 1]
  c128* gam;          // [R]
  c128* coef;         // [R][restart]
  c128* part;         // [R][2 (restart + 1)][nchunk]
  double* partn;      // [R][nchunk]
  int R, restart, nchunk, chunk;  // rows per CTA of the dots and cycle-start kernels
  int nuchunk, uchunk;             // rows per CTA of the update
  int max_iter;
  int64_t N;
  double tol;
  float qs, qsi;  // scale of a basis stored in half precision (sqrt(N)) and its inverse, else 1
};

// Storage of the Krylov basis: in the vector type, or as complex half (one __half2 per entry,
// 4 bytes) scaled by qs = sqrt(N), so that the entries of a unit vector are of order one and stay
// in the normal range of half precision.
template <typename TV, typename TQ>
struct QStore;
template <typename TV>
struct QStore<TV, cplx<TV>> {
  static __device__ __forceinline__ cplx<TV> ld(const cplx<TV>* p, float) { return *p; }
  static __device__ __forceinline__ void st(cplx<TV>* p, cplx<TV> v, float) { *p = v; }
};
template <>
struct QStore<float, __half2> {
  static __device__ __forceinline__ cplx<float> ld(const __half2* p, float inv) {
    const float2 f = __half22float2(*p);
    return mkc<float>(f.x * inv, f.y * inv);
  }
  static __device__ __forceinline__ void st(__half2* p, cplx<float> v, float s) {
    *p = __floats2half2_rn(v.re * s, v.im * s);
  }
};

// Entry of E as the vector type: complex128 / complex64 storage as is, complex64 storage widened to
// complex128 (the float64 residual of the refinement), complex bfloat16 storage (one
// __nv_bfloat162 per entry, real part first) widened to complex64.
template <typename TV, typename TE>
struct ELoad;
template <typename TV>
struct ELoad<TV, cplx<TV>> {
  static __device__ __forceinline__ cplx<TV> ld(const cplx<TV>* p) { return *p; }
};
template <>
struct ELoad<double, cplx<float>> {
  static __device__ __forceinline__ cplx<double> ld(const cplx<float>* p) {
    const cplx<float> v = *p;
    return mkc<double>(v.re, v.im);
  }
};
template <>
struct ELoad<float, __nv_bfloat162> {
  static __device__ __forceinline__ cplx<float> ld(const __nv_bfloat162* p) {
    const float2 f = __bfloat1622float2(*p);
    return mkc<float>(f.x, f.y);
  }
};

// Buffers of the persistent solve (persist.cu) handed over by the GMRES driver (krylov.cu).
struct PSync {
  unsigned count;  // arrivals at grid barriers since the launch
  int abort;       // a barrier ran out of time
  unsigned exits;  // CTAs that have left the kernel (the last one clears count and exits)
  int pad[29];
};
struct PBuffers {
  PSync* sync;
  void *part1, *part2, *partn;  // partial sums over the CTAs (at most ctx->nsm of them)
  const void* E;                // E in its storage type
  const void* B;
  void *Y, *W, *V;
  int bnorm_given;              // P.bnorm already holds |b| (solve from an initial guess)
  int y_zero;                   // Y starts at zero (the kernel clears it)
  bool* sync_clean;             // the barrier state is zero (else it is cleared before the launch)
  void* X;                      // non-null: the kernel also forms x = M^-1 y there
  const double* frames;         // non-null: B is not formed yet; the kernel forms it (incidence frames)
};
constexpr int kPersistMaxR = 8;  // right-hand sides of one persistent solve

// Runs the whole restarted GMRES as one cooperative kernel when the system is small enough
// (sets *done); otherwise leaves *done false and launches nothing.  The final state is read back
// asynchronously: after the stream's next synchronisation persist_result() gives it (and
// SWM_ETIMEOUT if a grid barrier ran out of time).
template <typename TV, typename TE>
int gmres_persistent(swm_ctx* ctx, const KPtr& P, const PBuffers& B, int max_iter, KState* hs, bool* done);
int persist_result(swm_ctx* ctx, KState* hs, bool* sync_clean);

}  // namespace swm
