// Exclusive prefix sums on the device (tile sums, then a tile rescan that forms its prefix of the
// tile sums itself, or with many tiles a one-CTA scan of the tile sums between the two).
#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kTile = kScanThreads * kScanItems;

// Inclusive block scan of one value per thread; returns the block total in *total.
__device__ int64_t block_incl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t n = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += n;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  if (w > 0) v += warp_tot[w - 1];
  *total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return v;
}

template <typename TIn>
__global__ void k_tile_sums(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile + threadIdx.x;
  int64_t v[kScanItems];
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) {  // all of a thread's loads in flight together
    const int64_t i = base + (int64_t)u * kScanThreads;
    v[u] = i < n ? (int64_t)in[i] : 0;
  }
  int64_t s = 0;
#pragma unroll
  for (int u = 0; u < kScanItems; ++u) s += v[u];
  int64_t tot;
  block_incl_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One CTA: exclusive scan of nt tile sums in place; grand total to sums[nt].
__global__ void k_scan_sums(int64_t* sums, int64_t nt) {
  const int64_t per = ceil_div(nt, kScanThreads);
  const int64_t b = threadIdx.x * per, e = min(nt, b + per);
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += sums[i];
  int64_t tot;
  int64_t incl = block_incl_scan(s, &tot);
  int64_t run = incl - s;
  for (int64_t i = b; i < e; ++i) {
    int64_t v = sums[i];
    sums[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) sums[nt] = tot;
}

template <typename TIn>
__global__ void k_tile_rescan(const TIn* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                              int64_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    int64_t i = base + t;
    v[t] = i < n ? (int64_t)in[i] : 0;
    s += v[t];
  }
  int64_t tot;
  int64_t run = block_incl_scan(s, &tot) - s + sums[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    int64_t i = base + t;
    if (i < n) out[i] = run;
    run += v[t];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = sums[gridDim.x];
}

// Tile rescan for at most kPrefixMaxTiles tiles: each CTA sums the tile sums before its own (loads
// in flight together) instead of a separate scan of the tile sums; the last CTA writes the total.
constexpr int64_t kPrefixMaxTiles = 4 * kScanThreads;
template <typename TIn>
__global__ void k_tile_rescan_prefix(const TIn* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                                     int64_t* __restrict__ out) {
  int64_t pv[kPrefixMaxTiles / kScanThreads];
#pragma unroll
  for (int u = 0; u < (int)(kPrefixMaxTiles / kScanThreads); ++u) {
    const int64_t i = threadIdx.x + (int64_t)u * kScanThreads;
    pv[u] = i < (int64_t)blockIdx.x ? sums[i] : 0;
  }
  int64_t ps = 0;
#pragma unroll
  for (int u = 0; u < (int)(kPrefixMaxTiles / kScanThreads); ++u) ps += pv[u];
  int64_t pre;
  block_incl_scan(ps, &pre);
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    int64_t i = base + t;
    v[t] = i < n ? (int64_t)in[i] : 0;
    s += v[t];
  }
  int64_t tot;
  int64_t run = block_incl_scan(s, &tot) - s + pre;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    int64_t i = base + t;
    if (i < n) out[i] = run;
    run += v[t];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = pre + tot;
}

// Whole scan in one CTA of kSingleThreads for short arrays (one launch instead of three).  Each
// thread owns up to kSingleItems consecutive entries, loaded together before they are summed, so
// the scan costs one memory round trip instead of one per entry.
constexpr int kSingleThreads = 1024;
constexpr int kSingleItems = 16;
constexpr int64_t kSingleMax = (int64_t)kSingleThreads * kSingleItems;

__device__ int64_t block_incl_scan_1024(int64_t v, int64_t* total) {
  __shared__ int64_t warp_tot[kSingleThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t n = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += n;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (w > 0) v += warp_tot[w - 1];
  *total = warp_tot[kSingleThreads / 32 - 1];
  __syncthreads();
  return v;
}

template <typename TIn>
__device__ void cta_scan_short(const TIn* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
  const int64_t per = ceil_div(n, kSingleThreads);  // <= kSingleItems
  const int64_t b = threadIdx.x * per;
  int64_t v[kSingleItems];
  int64_t s = 0;
#pragma unroll
  for (int t = 0; t < kSingleItems; ++t) {
    const int64_t i = b + t;
    v[t] = (t < per && i < n) ? (int64_t)in[i] : 0;
  }
#pragma unroll
  for (int t = 0; t < kSingleItems; ++t) s += v[t];
  int64_t tot;
  int64_t run = block_incl_scan_1024(s, &tot) - s;
#pragma unroll
  for (int t = 0; t < kSingleItems; ++t) {
    const int64_t i = b + t;
    if (t < per && i < n) out[i] = run;
    run += v[t];
  }
  if (threadIdx.x == 0) out[n] = tot;
}

template <typename TIn>
__global__ void __launch_bounds__(kSingleThreads) k_scan_single(const TIn* __restrict__ in, int64_t n,
                                                                int64_t* __restrict__ out) {
  cta_scan_short<TIn>(in, n, out);
}

template <typename TIn>
int scan_impl(swm_ctx* ctx, const TIn* in, int64_t* out, int64_t n, int64_t* total_host) {
  // out has n + 1 entries; out[n] = total.
  if (n == 0) {
    SWM_CK(cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream));
    if (total_host) *total_host = 0;
    return SWM_OK;
  }
  if (n <= kSingleMax) {
    k_scan_single<TIn><<<1, kSingleThreads, 0, ctx->stream>>>(in, n, out);
    SWM_LAUNCHED();
    if (total_host) {
      SWM_CK(cudaMemcpyAsync(total_host, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
      SWM_CK(cudaStreamSynchronize(ctx->stream));
    }
    return SWM_OK;
  }
  const int64_t nt = ceil_div(n, kTile);
  std::vector<Buf> tmp;
  int64_t* sums = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&sums, sizeof(int64_t) * (nt + 1)));
  k_tile_sums<TIn><<<(unsigned)nt, kScanThreads, 0, ctx->stream>>>(in, n, sums);
  SWM_LAUNCHED();
  if (nt <= kPrefixMaxTiles) {
    k_tile_rescan_prefix<TIn><<<(unsigned)nt, kScanThreads, 0, ctx->stream>>>(in, n, sums, out);
  } else {
    k_scan_sums<<<1, kScanThreads, 0, ctx->stream>>>(sums, nt);
    SWM_LAUNCHED();
    k_tile_rescan<TIn><<<(unsigned)nt, kScanThreads, 0, ctx->stream>>>(in, n, sums, out);
  }
  SWM_LAUNCHED();
  if (total_host) {
    SWM_CK(cudaMemcpyAsync(total_host, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SWM_CK(cudaStreamSynchronize(ctx->stream));
  }
  dfree_group(ctx, tmp);
  return SWM_OK;
}

constexpr int kMaxMultiScan = 8;
struct MultiScanArgs {
  const void* in[kMaxMultiScan];
  int is64[kMaxMultiScan];
  int64_t* out[kMaxMultiScan];
  int narr;
  int64_t* totals;  // optional: the totals side by side, totals[k] = out[k][n]
};

// Several exclusive scans of the same short length, one CTA per array.
__global__ void __launch_bounds__(kSingleThreads) k_scan_multi(MultiScanArgs a, int64_t n) {
  const int k = blockIdx.x;
  if (a.is64[k])
    cta_scan_short<int64_t>((const int64_t*)a.in[k], n, a.out[k]);
  else
    cta_scan_short<int32_t>((const int32_t*)a.in[k], n, a.out[k]);
  if (a.totals && threadIdx.x == 0) a.totals[k] = a.out[k][n];  // written by this thread
}

// The totals of long scans side by side.
__global__ void k_scan_totals(MultiScanArgs a, int64_t n) {
  if ((int)threadIdx.x < a.narr) a.totals[threadIdx.x] = a.out[threadIdx.x][n];
}

}  // namespace

int exclusive_scan_multi(swm_ctx* ctx, int narr, const void* const* in, const int* is64, int64_t* const* out,
                         int64_t n, int64_t* totals) {
  if (narr > kMaxMultiScan) return ctx->fail(SWM_EINVAL, "exclusive_scan_multi: too many arrays");
  MultiScanArgs a{};
  a.narr = narr;
  a.totals = totals;
  for (int k = 0; k < narr; ++k) {
    a.in[k] = in[k];
    a.is64[k] = is64[k];
    a.out[k] = out[k];
  }
  if (n <= kSingleMax && n > 0) {
    k_scan_multi<<<narr, kSingleThreads, 0, ctx->stream>>>(a, n);
    SWM_LAUNCHED();
    return SWM_OK;
  }
  for (int k = 0; k < narr; ++k) {
    if (is64[k])
      SWM_TRY(scan_impl<int64_t>(ctx, (const int64_t*)in[k], out[k], n, nullptr));
    else
      SWM_TRY(scan_impl<int32_t>(ctx, (const int32_t*)in[k], out[k], n, nullptr));
  }
  if (totals) {
    k_scan_totals<<<1, 32, 0, ctx->stream>>>(a, n);
    SWM_LAUNCHED();
  }
  return SWM_OK;
}

int exclusive_scan_i64(swm_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host) {
  return scan_impl<int64_t>(ctx, in, out, n, total_host);
}
int exclusive_scan_i32_to_i64(swm_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* total_host) {
  return scan_impl<int32_t>(ctx, in, out, n, total_host);
}

}  // namespace swm
