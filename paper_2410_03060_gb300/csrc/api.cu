// C-ABI entry points of the swm library (declared and documented in include/swm.h).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "ctx.h"

namespace swm {

namespace {
std::mutex g_fn_mutex;
std::map<std::pair<const void*, int>, size_t> g_fn_static;              // (kernel, device) -> static smem
std::map<std::tuple<const void*, int, int, size_t>, int> g_fn_occupancy;  // (kernel, device, threads, smem)
}  // namespace

cudaError_t allow_max_dyn_smem(const void* fn, int smem_optin, size_t* static_bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_fn_mutex);
  auto it = g_fn_static.find({fn, dev});
  if (it == g_fn_static.end()) {
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    it = g_fn_static.emplace(std::make_pair(fn, dev), (size_t)fa.sharedSizeBytes).first;
  }
  if (static_bytes) *static_bytes = it->second;
  return cudaSuccess;
}

cudaError_t occupancy_cached(const void* fn, int threads, size_t smem, int* blocks) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_fn_mutex);
  const auto key = std::make_tuple(fn, dev, threads, smem);
  auto it = g_fn_occupancy.find(key);
  if (it == g_fn_occupancy.end()) {
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem);
    if (e != cudaSuccess) return e;
    it = g_fn_occupancy.emplace(key, b).first;
  }
  *blocks = it->second;
  return cudaSuccess;
}

int dalloc(swm_ctx* ctx, std::vector<Buf>& group, void** out, size_t bytes) {
  bytes = std::max<size_t>((bytes + 255) / 256 * 256, 256);
  // reuse the smallest released buffer that fits without wasting more than half of it
  int best = -1;
  for (int i = 0; i < (int)ctx->free_list.size(); ++i) {
    const size_t b = ctx->free_list[i].bytes;
    if (b >= bytes && b <= 2 * bytes + (size_t(1) << 20) && (best < 0 || b < ctx->free_list[best].bytes)) best = i;
  }
  if (best >= 0) {
    group.push_back(ctx->free_list[best]);
    ctx->free_list.erase(ctx->free_list.begin() + best);
    *out = group.back().p;
    return SWM_OK;
  }
  void* p = nullptr;
  if (ctx->user_alloc) {
    p = ctx->user_alloc(bytes, (void*)ctx->stream, ctx->user_arg);
    if (!p) return ctx->fail(SWM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return ctx->fail(SWM_ENOMEM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  group.push_back(Buf{p, bytes});
  *out = p;
  return SWM_OK;
}

void dfree_group(swm_ctx* ctx, std::vector<Buf>& group) {
  for (auto& b : group) ctx->free_list.push_back(b);
  group.clear();
}

static void release_all(swm_ctx* ctx) {
  dfree_group(ctx, ctx->kry_bufs);
  std::free(ctx->kry_ws);
  ctx->kry_ws = nullptr;
  dfree_group(ctx, ctx->solve_bufs);
  dfree_group(ctx, ctx->build_bufs);
  dfree_group(ctx, ctx->pattern_bufs);
  dfree_group(ctx, ctx->cloud_bufs);
  for (auto& b : ctx->free_list) {
    if (ctx->user_free)
      ctx->user_free(b.p, b.bytes, (void*)ctx->stream, ctx->user_arg);
    else
      cudaFreeAsync(b.p, ctx->stream);
  }
  ctx->free_list.clear();
}

namespace {

// One pass over the caller's wires: copy them into the context's buffers (when the caller's are
// device buffers; host inputs were copied before), check them, and per CTA the bounding box of the
// centres, the check flags (1 NaN/Inf, 2 non-unit direction, 4 length, 8 radius, 16 segments) and
// the largest segment count, part[blk][8] = {min xyz, max xyz, flags, max ns}.  The last CTA to
// arrive combines the partials into res[8] (warp d for field d) and clears the arrival counter.
constexpr int kIngestThreads = 256;
__device__ __forceinline__ double ingest_comb(int d, double v, double x) {
  return d < 3 ? fmin(v, x) : d < 6 ? fmax(v, x) : d == 6 ? (double)((int)v | (int)x) : fmax(v, x);
}
__global__ void __launch_bounds__(kIngestThreads) k_ingest(int64_t nw, const double* __restrict__ sc,
                                                           const double* __restrict__ st,
                                                           const double* __restrict__ sL,
                                                           const double* __restrict__ sa,
                                                           const int32_t* __restrict__ sns, int copy, double* c,
                                                           double* t, double* L, double* a, int32_t* ns,
                                                           double* __restrict__ part, unsigned* __restrict__ arrivals,
                                                           double* __restrict__ res) {
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  int f = 0, mns = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x) {
    double cc[3], tt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cc[d] = sc[3 * i + d];
      tt[d] = st[3 * i + d];
    }
    const double Li = sL[i], ai = sa[i];
    const int ni = sns[i];
    if (copy) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        c[3 * i + d] = cc[d];
        t[3 * i + d] = tt[d];
      }
      L[i] = Li;
      a[i] = ai;
      ns[i] = ni;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!isfinite(cc[d]) || !isfinite(tt[d])) f |= 1;
      mn[d] = fmin(mn[d], cc[d]);
      mx[d] = fmax(mx[d], cc[d]);
    }
    if (!isfinite(Li) || !isfinite(ai)) f |= 1;
    const double tn = tt[0] * tt[0] + tt[1] * tt[1] + tt[2] * tt[2];
    if (!(fabs(tn - 1.0) <= 2e-9)) f |= 2;
    if (!(Li > 0.0)) f |= 4;
    if (!(ai > 0.0)) f |= 8;
    if (ni < 2 || ni > kMaxSeg) f |= 16;
    mns = max(mns, ni);
  }
  __shared__ double s[8][kIngestThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
    f |= __shfl_xor_sync(0xffffffffu, f, o);
    mns = max(mns, __shfl_xor_sync(0xffffffffu, mns, o));
  }
  if (lane == 0) {
    for (int d = 0; d < 3; ++d) {
      s[d][w] = mn[d];
      s[3 + d][w] = mx[d];
    }
    s[6][w] = (double)f;
    s[7][w] = (double)mns;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int d = threadIdx.x;
    double v = s[d][0];
    for (int k = 1; k < kIngestThreads / 32; ++k) v = ingest_comb(d, v, s[d][k]);
    part[blockIdx.x * 8 + d] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(arrivals, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // last CTA: warp d combines field d over all CTAs' partials
  const int d = w;
  double v = __ldcg(part + d);
  for (int k = lane; k < (int)gridDim.x; k += 32) v = ingest_comb(d, v, __ldcg(part + k * 8 + d));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ingest_comb(d, v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) res[d] = v;
  if (threadIdx.x == 0) *arrivals = 0;
}

// Internal [R][N] currents (any precision) -> caller [R][N] complex128 in caller unknown order.
template <typename TV>
__global__ void k_to_user(int64_t N, int R, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                          const int64_t* __restrict__ uoff, const cplx<TV>* __restrict__ X, c128* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  out[(int64_t)r * N + uoff[p] + (n - off[p])] = ccast<double>(X[(int64_t)r * N + n]);
}



// The device address of host memory the GPU can read and write in place (page-locked, registered
// or allocated by CUDA), else null.
void* device_view(const void* host) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int copy_in(swm_ctx* ctx, void* dst, const void* src, size_t bytes, int kind) {
  SWM_CK(cudaMemcpyAsync(dst, src, bytes, kind == SWM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         ctx->stream));
  return SWM_OK;
}

// A small host input copied to the device through the context's pinned staging area (no staged
// pageable copy); inputs that do not fit are copied directly.  ctx->up_used is the part of the area
// whose copies may still be pending: every entry point that ends with a synchronisation clears it
// when it starts, and swm_run (which synchronises only at its end) clears it once for all its steps.
int upload(swm_ctx* ctx, void* dst, const void* src, size_t bytes) {
  SWM_TRY(ensure_poll_slots(ctx));
  if (ctx->up_used + bytes <= kPinnedUpBytes) {
    char* stage = static_cast<char*>(ctx->pinned_state) + kPinnedUpOffset + ctx->up_used;
    std::memcpy(stage, src, bytes);
    SWM_CK(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->up_used += (bytes + 15) & ~size_t(15);
    return SWM_OK;
  }
  SWM_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  return SWM_OK;
}

int set_device(swm_ctx* ctx) {
  SWM_CK(cudaSetDevice(ctx->device));
  return SWM_OK;
}

thread_local std::string g_stateless_err;

}  // namespace

// Caller-order [R][N] complex128 -> internal order.
__global__ void k_from_user(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                            const int64_t* __restrict__ uoff, const c128* __restrict__ in, c128* __restrict__ out) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  out[(int64_t)r * N + n] = in[(int64_t)r * N + uoff[p] + (n - off[p])];
}

// y = blockdiag(Z_pp) x (the right preconditioner applied forward), float64 arithmetic.
template <typename TZ>
__global__ void k_mult_diag(int64_t N, const int32_t* __restrict__ rowwire, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ m, const int64_t* __restrict__ diag_b, Layout full,
                            const cplx<TZ>* __restrict__ Z, const c128* __restrict__ x, c128* __restrict__ y) {
  const int r = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int p = rowwire[n];
  const int64_t o = off[p];
  const int i = (int)(n - o), mp = m[p];
  const cplx<TZ>* zr = Z + full.rowbase[p] + (int64_t)i * full.K[p] + full.colpos[diag_b[p]];
  c128 acc = mkc(0.0, 0.0);
  for (int l = 0; l < mp; ++l) cfma(acc, ccast<double>(zr[l]), x[(int64_t)r * N + o + l]);
  y[(int64_t)r * N + n] = acc;
}

// Incidence frames: k_hat (propagation, = -arrival) and polarisation e, 6 doubles each.
void frames_host(const double* inc, int n, std::vector<double>& out) {
  out.resize(6 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const double th = inc[3 * i], ph = inc[3 * i + 1], ps = inc[3 * i + 2];
    const double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
    const double u[3] = {st * cp, st * sp, ct};
    const double tht[3] = {ct * cp, ct * sp, -st};
    const double pht[3] = {-sp, cp, 0.0};
    for (int d = 0; d < 3; ++d) {
      out[6 * i + d] = -u[d];
      out[6 * i + 3 + d] = std::cos(ps) * tht[d] + std::sin(ps) * pht[d];
    }
  }
}

void set_stateless_error(const std::string& msg) { g_stateless_err = msg; }

// True if every pointer is device (or managed) memory that the current device can address; the
// stateless far-field entry points take device pointers only.
bool all_device_memory(const void* const* ptrs, int n) {
  for (int i = 0; i < n; ++i) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  }
  return true;
}

}  // namespace swm

using namespace swm;

extern "C" {

const char* swm_version(void) { return "swm 0.1 (sm_103a)"; }

int swm_create(swm_ctx** out, int device, void* cuda_stream) {
  if (!out) return SWM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SWM_EINVAL;
  }
  swm_ctx* ctx = new (std::nothrow) swm_ctx();
  if (!ctx) return SWM_ENOMEM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (const char* e = std::getenv("SWM_SPLIT_ROWS")) ctx->split_rows = std::max<long long>(0, std::atoll(e));
  if (const char* e = std::getenv("SWM_PERSIST")) ctx->persist = std::atoi(e) != 0;
  if (const char* e = std::getenv("SWM_PERSIST_CTAS")) ctx->persist_ctas = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("SWM_TEST_BARRIER_EXTRA")) ctx->test_barrier_extra = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("SWM_PRODUCT_FORM")) ctx->product_form = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("SWM_BICGSTAB_MAJOR")) ctx->bicg_major = std::atoi(e) != 0;
  if (const char* e = std::getenv("SWM_BICGSTAB_CTAS")) ctx->bicg_ctas = std::min(64, std::max(1, std::atoi(e)));
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return SWM_ECUDA;
  }
  *out = ctx;
  return SWM_OK;
}

void swm_destroy(swm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& e : ctx->prof_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& e : ctx->ph_ev)
    for (auto ev : e)
      if (ev) cudaEventDestroy(ev);
  for (auto ev : ctx->poll_ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->pinned_state) cudaFreeHost(ctx->pinned_state);
  if (ctx->d_arrive) cudaFree(ctx->d_arrive);
  if (ctx->gm_exec) cudaGraphExecDestroy(ctx->gm_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  for (auto ev : ctx->side_ev)
    if (ev) cudaEventDestroy(ev);
  release_all(ctx);
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

const char* swm_last_error(const swm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int swm_set_allocator(swm_ctx* ctx, swm_alloc_fn alloc, swm_free_fn free_fn, void* user) {
  if (!ctx) return SWM_EINVAL;
  if (!ctx->cloud_bufs.empty() || !ctx->pattern_bufs.empty() || !ctx->build_bufs.empty() ||
      !ctx->solve_bufs.empty() || !ctx->free_list.empty())
    return ctx->fail(SWM_ESTATE, "swm_set_allocator must precede swm_set_cloud");
  if ((alloc == nullptr) != (free_fn == nullptr)) return ctx->fail(SWM_EINVAL, "alloc and free must both be set");
  ctx->user_alloc = alloc;
  ctx->user_free = free_fn;
  ctx->user_arg = user;
  return SWM_OK;
}

int swm_set_cloud(swm_ctx* ctx, int64_t nw, const double* centres, const double* dirs, const double* lengths,
                  const double* radii, const int32_t* nseg, int mem_kind) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (nw < 1 || nw > (int64_t)INT32_MAX / 2) return ctx->fail(SWM_EINVAL, "nw out of range");
  if (!centres || !dirs || !lengths || !radii || !nseg) return ctx->fail(SWM_EINVAL, "null input pointer");
  if (mem_kind != SWM_HOST && mem_kind != SWM_DEVICE) return ctx->fail(SWM_EINVAL, "bad mem_kind");
  SWM_TRY(set_device(ctx));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->side) SWM_CK(cudaStreamSynchronize(ctx->side));
  dfree_group(ctx, ctx->solve_bufs);
  dfree_group(ctx, ctx->build_bufs);
  dfree_group(ctx, ctx->pattern_bufs);
  dfree_group(ctx, ctx->cloud_bufs);
  ctx->built = ctx->solved = false;
  ctx->pattern_ok = false;
  ctx->rowwire = nullptr;
  ctx->wrec = nullptr;
  ctx->nw = nw;
  auto& G = ctx->cloud_bufs;
  SWM_TRY(dalloc(ctx, G, (void**)&ctx->u_c, sizeof(double) * 3 * nw));
  SWM_TRY(dalloc(ctx, G, (void**)&ctx->u_t, sizeof(double) * 3 * nw));
  SWM_TRY(dalloc(ctx, G, (void**)&ctx->u_L, sizeof(double) * nw));
  SWM_TRY(dalloc(ctx, G, (void**)&ctx->u_a, sizeof(double) * nw));
  SWM_TRY(dalloc(ctx, G, (void**)&ctx->u_ns, sizeof(int32_t) * nw));
  // Device inputs are copied by k_ingest itself; host inputs are copied in first by the copy
  // engines (page-locked ones at the host link's full rate; measured faster than the kernel
  // reading them in place) and checked where they land.
  const void* src[5] = {centres, dirs, lengths, radii, nseg};
  const bool dev = mem_kind == SWM_DEVICE;
  if (!dev) {
    SWM_TRY(copy_in(ctx, ctx->u_c, centres, sizeof(double) * 3 * nw, mem_kind));
    SWM_TRY(copy_in(ctx, ctx->u_t, dirs, sizeof(double) * 3 * nw, mem_kind));
    SWM_TRY(copy_in(ctx, ctx->u_L, lengths, sizeof(double) * nw, mem_kind));
    SWM_TRY(copy_in(ctx, ctx->u_a, radii, sizeof(double) * nw, mem_kind));
    SWM_TRY(copy_in(ctx, ctx->u_ns, nseg, sizeof(int32_t) * nw, mem_kind));
  }
  std::vector<Buf> tmp;
  const int np = (int)std::min<int64_t>(ceil_div(nw, kIngestThreads), 2 * std::max(ctx->nsm, 1));
  if (!ctx->d_arrive) {  // the arrival counter of k_ingest: zero, and left zero by every launch
    SWM_CK(cudaMalloc((void**)&ctx->d_arrive, sizeof(unsigned)));
    SWM_CK(cudaMemsetAsync(ctx->d_arrive, 0, sizeof(unsigned), ctx->stream));
  }
  double* part = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&part, sizeof(double) * 8 * (np + 1)));
  double* res = part + 8 * np;
  k_ingest<<<(unsigned)np, kIngestThreads, 0, ctx->stream>>>(
      nw, dev ? (const double*)src[0] : ctx->u_c, dev ? (const double*)src[1] : ctx->u_t,
      dev ? (const double*)src[2] : ctx->u_L, dev ? (const double*)src[3] : ctx->u_a,
      dev ? (const int32_t*)src[4] : ctx->u_ns, dev ? 1 : 0, ctx->u_c, ctx->u_t, ctx->u_L, ctx->u_a, ctx->u_ns, part,
      ctx->d_arrive, res);
  SWM_LAUNCHED();
  SWM_TRY(ensure_poll_slots(ctx));
  double* hres = reinterpret_cast<double*>(static_cast<char*>(ctx->pinned_state) + kIngestSlotOffset);
  SWM_CK(cudaMemcpyAsync(hres, res, sizeof(double) * 8, cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  for (int d = 0; d < 6; ++d) ctx->bbox[d] = hres[d];
  const int hf[2] = {(int)hres[6], (int)hres[7]};
  if (hf[0]) {
    std::string m = "invalid cloud:";
    if (hf[0] & 1) m += " non-finite value;";
    if (hf[0] & 2) m += " direction not of unit length;";
    if (hf[0] & 4) m += " length <= 0;";
    if (hf[0] & 8) m += " radius <= 0;";
    if (hf[0] & 16) m += " segment count outside [2, " + std::to_string(kMaxSeg) + "];";
    dfree_group(ctx, ctx->cloud_bufs);
    ctx->nw = 0;
    return ctx->fail(SWM_EINVAL, m);
  }
  ctx->max_ns = hf[1];
  ctx->stats = swm_stats{};
  ctx->stats.nw = nw;
  return SWM_OK;
}

int swm_build(swm_ctx* ctx, double k, double r_c, int precision) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (ctx->nw < 1) return ctx->fail(SWM_ESTATE, "swm_build before swm_set_cloud");
  if (!(k > 0.0) || !std::isfinite(k)) return ctx->fail(SWM_EINVAL, "k must be positive and finite");
  if (std::isnan(r_c)) return ctx->fail(SWM_EINVAL, "r_c is NaN");
  if (precision != SWM_C128 && precision != SWM_C64 && precision != SWM_BF16)
    return ctx->fail(SWM_EINVAL, "bad precision");
  SWM_TRY(set_device(ctx));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->side) SWM_CK(cudaStreamSynchronize(ctx->side));  // idle unless an earlier build failed midway
  dfree_group(ctx, ctx->solve_bufs);
  dfree_group(ctx, ctx->build_bufs);
  ctx->built = ctx->solved = false;
  const bool dense = !(r_c > 0.0) || std::isinf(r_c);
  // the pattern depends on the cloud and r_c only (Eq. neardef), not on k: a build at a new
  // frequency with the same r_c refills the values on the kept pattern
  const bool reuse = ctx->pattern_ok && ctx->pattern_dense == dense && (dense || ctx->pattern_rc == r_c);
  ctx->k = k;
  ctx->rc = r_c;
  ctx->dense = dense;
  // SWM_BF16 fills and preconditions as SWM_C64 and then adds the bfloat16 copy of E
  ctx->prec = precision == SWM_BF16 ? SWM_C64 : precision;
  ctx->bf16 = precision == SWM_BF16;
  ctx->E16 = nullptr;
  if (!ctx->side) {  // the build's second stream (pattern column maps, self blocks, far-field data)
    SWM_CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    SWM_CK(cudaEventCreateWithFlags(&ctx->side_ev[0], cudaEventDisableTiming));
    SWM_CK(cudaEventCreateWithFlags(&ctx->side_ev[1], cudaEventDisableTiming));
  }
  ctx->phase_begin(swm_ctx::PH_NEIGHBOUR);
  if (!reuse) {
    dfree_group(ctx, ctx->pattern_bufs);
    ctx->pattern_ok = false;
    ctx->rowwire = nullptr;
    ctx->wrec = nullptr;
    ctx->uoff = nullptr;
    ctx->uoff_user = nullptr;
    SWM_TRY(build_pattern(ctx));
    ctx->pattern_ok = true;
    ctx->pattern_rc = r_c;
    ctx->pattern_dense = dense;
  }
  ctx->stats.pattern_reused = reuse ? 1 : 0;
  ctx->phase_end(swm_ctx::PH_NEIGHBOUR);
  // The self blocks and their inverses run on a second stream beside the mutual blocks (they
  // touch disjoint parts of Z); E is formed once both are done.  A profiled self-block or inverse
  // class stays on the context's stream so that its events time it.
  SWM_TRY(fill_alloc(ctx));
  SWM_TRY(precond_alloc(ctx));
  SWM_TRY(far_field_alloc(ctx));  // every buffer the second stream writes exists before the fork
  const bool side = ctx->prof_cls != SWM_K_FILL_SELF && ctx->prof_cls != SWM_K_INVERT;
  cudaStream_t s2 = side ? ctx->side : ctx->stream;
  ctx->phase_begin(swm_ctx::PH_FILL);
  if (side) {
    SWM_CK(cudaEventRecord(ctx->side_ev[0], ctx->stream));
    SWM_CK(cudaStreamWaitEvent(s2, ctx->side_ev[0], 0));
  }
  SWM_TRY(fill_self(ctx, s2));
  SWM_TRY(precond_invert(ctx, s2));
  SWM_TRY(prepare_far_field(ctx, s2));
  SWM_TRY(fill_mutual(ctx));
  ctx->phase_end(swm_ctx::PH_FILL);
  ctx->phase_begin(swm_ctx::PH_PRECOND);
  if (side) {
    SWM_CK(cudaEventRecord(ctx->side_ev[1], s2));
    SWM_CK(cudaStreamWaitEvent(ctx->stream, ctx->side_ev[1], 0));
  }
  SWM_TRY(precond_form_E(ctx));
  if (ctx->bf16) SWM_TRY(make_e16(ctx));
  ctx->phase_end(swm_ctx::PH_PRECOND);
  SWM_TRY(finish_build(ctx));
  if (!ctx->fused) {
    SWM_CK(cudaStreamSynchronize(ctx->stream));
    ctx->phase_collect();
  }
  SWM_CK(cudaGetLastError());
  ctx->stats.n = ctx->N;
  ctx->stats.nb = ctx->nb;
  ctx->stats.nnz = ctx->full.nval;
  ctx->stats.nnz_offd = ctx->offd.nval;
  ctx->stats.ncm_offd = ctx->offd.ncm;
  ctx->stats.nminv = ctx->nminv;
  ctx->built = true;
  if (!ctx->fused) ctx->prof_flush();
  return SWM_OK;
}

int swm_set_solver(swm_ctx* ctx, int method) {
  if (!ctx) return SWM_EINVAL;
  if (method != SWM_SOLVER_GMRES && method != SWM_SOLVER_GCR && method != SWM_SOLVER_BICGSTAB)
    return ctx->fail(SWM_EINVAL, "bad solver");
  ctx->solver = method;
  return SWM_OK;
}

static int solve_impl(swm_ctx* ctx, int n_inc, const double* inc, double tol, int restart, int max_iter,
                      double* currents_out, int out_kind, const double* x0, int x0_kind);

int swm_solve(swm_ctx* ctx, int n_inc, const double* inc, double tol, int restart, int max_iter,
              double* currents_out, int out_kind) {
  return solve_impl(ctx, n_inc, inc, tol, restart, max_iter, currents_out, out_kind, nullptr, SWM_HOST);
}

int swm_solve_guess(swm_ctx* ctx, int n_inc, const double* inc, const double* x0, int x0_kind, double tol,
                    int restart, int max_iter, double* currents_out, int out_kind) {
  if (!ctx) return SWM_EINVAL;
  if (!x0 || (x0_kind != SWM_HOST && x0_kind != SWM_DEVICE)) return ctx->fail(SWM_EINVAL, "bad initial guess");
  return solve_impl(ctx, n_inc, inc, tol, restart, max_iter, currents_out, out_kind, x0, x0_kind);
}

static int solve_impl(swm_ctx* ctx, int n_inc, const double* inc, double tol, int restart, int max_iter,
                      double* currents_out, int out_kind, const double* x0, int x0_kind) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (!ctx->built) return ctx->fail(SWM_ESTATE, "swm_solve before swm_build");
  if (n_inc < 1 || n_inc > 65535 || !inc) return ctx->fail(SWM_EINVAL, "bad incidence list");
  if (!(tol > 0.0) || restart < 1 || restart > SWM_MAX_RESTART || max_iter < 0)
    return ctx->fail(SWM_EINVAL, "bad solver parameters");
  if (currents_out && out_kind != SWM_HOST && out_kind != SWM_DEVICE) return ctx->fail(SWM_EINVAL, "bad out_kind");
  for (int i = 0; i < 3 * n_inc; ++i)
    if (!std::isfinite(inc[i])) return ctx->fail(SWM_EINVAL, "non-finite incidence angle");
  SWM_TRY(set_device(ctx));
  if (!ctx->fused) SWM_CK(cudaStreamSynchronize(ctx->stream));  // inside swm_run the stream orders it
  dfree_group(ctx, ctx->solve_bufs);
  ctx->solved = false;
  ctx->n_rhs = n_inc;
  const size_t esz = ctx->prec == SWM_C128 ? sizeof(c128) : sizeof(c64);
  auto& S = ctx->solve_bufs;
  SWM_TRY(dalloc(ctx, S, &ctx->Bv, esz * n_inc * ctx->N));
  SWM_TRY(dalloc(ctx, S, &ctx->Xv, esz * n_inc * ctx->N));
  SWM_TRY(dalloc(ctx, S, (void**)&ctx->inc_dev, sizeof(double) * 3 * n_inc));
  double* frames = nullptr;
  SWM_TRY(dalloc(ctx, S, (void**)&frames, sizeof(double) * 6 * n_inc));
  std::vector<double> fh;
  frames_host(inc, n_inc, fh);
  if (!ctx->fused) ctx->up_used = 0;  // the stream was synchronised above
  SWM_TRY(upload(ctx, ctx->inc_dev, inc, sizeof(double) * 3 * n_inc));
  SWM_TRY(upload(ctx, frames, fh.data(), sizeof(double) * 6 * n_inc));
  // GMRES from zero forms b itself when it runs as the persistent solve (each CTA its rows, in its
  // first residual); every other path gets it from the RHS kernel here or in the solver
  const bool defer_rhs = !ctx->bf16 && ctx->solver == SWM_SOLVER_GMRES && !x0;
  ctx->phase_begin(swm_ctx::PH_RHS);
  if (defer_rhs)
    ctx->rhs_frames = frames;
  else
    SWM_TRY(compute_rhs(ctx, n_inc, frames));
  ctx->phase_end(swm_ctx::PH_RHS);
  ctx->guess = nullptr;
  if (x0) {
    // y0 = M x0 in internal order: the solvers start from it instead of zero
    SWM_TRY(ensure_rowinfo(ctx));
    SWM_TRY(ensure_user_offsets(ctx));
    const int64_t N = ctx->N;
    c128 *xin = nullptr, *y0 = nullptr;
    SWM_TRY(dalloc(ctx, S, (void**)&xin, sizeof(c128) * n_inc * N));
    SWM_TRY(dalloc(ctx, S, (void**)&y0, sizeof(c128) * n_inc * N));
    const c128* src = (const c128*)x0;
    if (x0_kind == SWM_HOST) {
      SWM_CK(cudaMemcpyAsync(y0, x0, sizeof(c128) * n_inc * N, cudaMemcpyHostToDevice, ctx->stream));
      src = y0;
    }
    const dim3 g((unsigned)ceil_div(N, 256), n_inc);
    k_from_user<<<g, 256, 0, ctx->stream>>>(N, ctx->rowwire, ctx->off, ctx->uoff, src, xin);
    SWM_LAUNCHED();
    if (ctx->prec == SWM_C128)
      k_mult_diag<double><<<g, 256, 0, ctx->stream>>>(N, ctx->rowwire, ctx->off, ctx->m, ctx->diag_b, ctx->full,
                                                      (const c128*)ctx->Z, xin, y0);
    else
      k_mult_diag<float><<<g, 256, 0, ctx->stream>>>(N, ctx->rowwire, ctx->off, ctx->m, ctx->diag_b, ctx->full,
                                                     (const c64*)ctx->Z, xin, y0);
    SWM_LAUNCHED();
    ctx->guess = y0;
  }
  ctx->phase_begin(swm_ctx::PH_SOLVE);
  int rc = ctx->bf16 ? refine_solve(ctx, frames, tol, restart, max_iter)
           : ctx->solver == SWM_SOLVER_GCR      ? gcr_solve(ctx, tol, restart, max_iter)
           : ctx->solver == SWM_SOLVER_BICGSTAB ? bicgstab_solve(ctx, tol, max_iter)
                                                : gmres_solve(ctx, tol, restart, max_iter);
  ctx->phase_end(swm_ctx::PH_SOLVE);
  ctx->guess = nullptr;
  ctx->rhs_frames = nullptr;
  if (!ctx->fused) {
    SWM_CK(cudaStreamSynchronize(ctx->stream));
    ctx->phase_collect();
    ctx->prof_flush();
  }
  if (rc < 0) return rc;
  ctx->stats.n_rhs = n_inc;
  ctx->solved = true;
  if (currents_out) {
    SWM_TRY(ensure_user_offsets(ctx));
    const int64_t N = ctx->N;
    c128* dst = nullptr;
    std::vector<Buf> tmp;
    if (out_kind == SWM_DEVICE)
      dst = (c128*)currents_out;
    else
      SWM_TRY(dalloc(ctx, tmp, (void**)&dst, sizeof(c128) * n_inc * N));
    const dim3 grid((unsigned)ceil_div(N, 256), n_inc);
    if (ctx->prec == SWM_C128)
      k_to_user<double><<<grid, 256, 0, ctx->stream>>>(N, n_inc, ctx->rowwire, ctx->off, ctx->uoff, (const c128*)ctx->Xv,
                                                       dst);
    else
      k_to_user<float><<<grid, 256, 0, ctx->stream>>>(N, n_inc, ctx->rowwire, ctx->off, ctx->uoff, (const c64*)ctx->Xv,
                                                      dst);
    SWM_LAUNCHED();
    if (out_kind == SWM_HOST)
      SWM_CK(cudaMemcpyAsync(currents_out, dst, sizeof(c128) * n_inc * N, cudaMemcpyDeviceToHost, ctx->stream));
    SWM_CK(cudaStreamSynchronize(ctx->stream));
    dfree_group(ctx, tmp);
  }
  return rc;
}

static int rcs_common(swm_ctx* ctx, int n_obs, const double* obs, bool mono, double* sigma_out, int out_kind) {
  if (!ctx) return SWM_EINVAL;
  ctx->err.clear();
  if (!ctx->solved) return ctx->fail(SWM_ESTATE, "RCS requested before swm_solve");
  if (!sigma_out || (out_kind != SWM_HOST && out_kind != SWM_DEVICE)) return ctx->fail(SWM_EINVAL, "bad output");
  if (!mono) {
    if (n_obs < 1 || !obs) return ctx->fail(SWM_EINVAL, "bad observation list");
    for (int i = 0; i < 2 * n_obs; ++i)
      if (!std::isfinite(obs[i])) return ctx->fail(SWM_EINVAL, "non-finite observation angle");
  }
  SWM_TRY(set_device(ctx));
  if (!ctx->fused) ctx->up_used = 0;  // the previous entry point ended with a synchronisation
  ctx->phase_begin(swm_ctx::PH_RCS);
  const int R = ctx->n_rhs;
  const int64_t npairs = mono ? R : (int64_t)R * n_obs;
  std::vector<Buf> tmp;
  double* obs_dev = ctx->inc_dev;
  int stride = 3;
  if (!mono) {
    SWM_TRY(dalloc(ctx, tmp, (void**)&obs_dev, sizeof(double) * 2 * n_obs));
    SWM_TRY(upload(ctx, obs_dev, obs, sizeof(double) * 2 * n_obs));
    stride = 2;
  }
  const size_t sb = ctx->prec == SWM_C64
                        ? far_field_f32_scratch_bytes(ctx, npairs, mono ? R : n_obs)
                        : far_field_scratch_bytes(ctx->nw, npairs);
  void* scratch = nullptr;
  SWM_TRY(dalloc(ctx, tmp, &scratch, sb));
  // the RCS goes straight to the caller's buffer when the GPU can write it (device memory, or
  // page-locked host memory written in place over the host link)
  double* sig = out_kind == SWM_DEVICE ? sigma_out : (double*)device_view(sigma_out);
  const bool sig_direct = sig != nullptr;
  if (!sig_direct) SWM_TRY(dalloc(ctx, tmp, (void**)&sig, sizeof(double) * 2 * npairs));
  std::string err;
  ctx->prof_begin(SWM_K_FAR);
  int rc;
  if (ctx->prec == SWM_C64) {
    rc = far_field_f32_launch(ctx, mono ? R : n_obs, obs_dev, stride, mono, sig, scratch, sb);
  } else {
    rc = far_field_launch(ctx->stream, &ctx->launches, false, true, ctx->Xv, ctx->nw, ctx->N, nullptr, nullptr, ctx->cx,
                          ctx->cy, ctx->cz, ctx->tx, ctx->ty, ctx->tz, ctx->L, ctx->ns, ctx->off, true, ctx->k, R,
                          mono ? R : n_obs, obs_dev, stride, mono, sig, scratch, sb, &err);
    if (rc < 0) ctx->fail(rc, err);
  }
  ctx->prof_end(SWM_K_FAR);
  if (rc < 0) return rc;
  if (!sig_direct)
    SWM_CK(cudaMemcpyAsync(sigma_out, sig, sizeof(double) * 2 * npairs, cudaMemcpyDeviceToHost, ctx->stream));
  ctx->phase_end(swm_ctx::PH_RCS);
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  ctx->phase_collect();
  ctx->prof_flush();
  return SWM_OK;
}

int swm_rcs_bistatic(swm_ctx* ctx, int n_obs, const double* obs, double* sigma_out, int out_kind) {
  return rcs_common(ctx, n_obs, obs, false, sigma_out, out_kind);
}

int swm_rcs_monostatic(swm_ctx* ctx, double* sigma_out, int out_kind) {
  return rcs_common(ctx, 0, nullptr, true, sigma_out, out_kind);
}

int swm_run(swm_ctx* ctx, int64_t nw, const double* centres, const double* dirs, const double* lengths,
            const double* radii, const int32_t* nseg, int mem_kind, double k, double r_c, int precision, int n_inc,
            const double* inc, double tol, int restart, int max_iter, int n_obs, const double* obs,
            double* sigma_out, int out_kind) {
  if (!ctx) return SWM_EINVAL;
  int rc = swm_set_cloud(ctx, nw, centres, dirs, lengths, radii, nseg, mem_kind);
  if (rc < 0) return rc;
  // the host needs nothing from the build's end or the solve until the RCS is read back
  ctx->fused = true;
  ctx->build_check_pending = false;
  ctx->pend.active = false;
  ctx->up_used = 0;  // swm_set_cloud ended with a synchronisation
  rc = swm_build(ctx, k, r_c, precision);
  int solve_rc = SWM_OK;
  if (rc >= 0) {
    solve_rc = swm_solve(ctx, n_inc, inc, tol, restart, max_iter, nullptr, SWM_HOST);
    if (solve_rc >= 0)
      rc = (n_obs == 0 && obs == nullptr) ? swm_rcs_monostatic(ctx, sigma_out, out_kind)
                                          : swm_rcs_bistatic(ctx, n_obs, obs, sigma_out, out_kind);
    else rc = solve_rc;
  }
  ctx->fused = false;
  // every later check after one synchronisation (the RCS call ended with one unless it failed)
  const cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess && rc >= 0) rc = ctx->fail(SWM_ECUDA, std::string("swm_run: ") + cudaGetErrorString(e));
  ctx->phase_collect();
  ctx->prof_flush();
  if (ctx->build_check_pending) {
    ctx->build_check_pending = false;
    const int bc = finish_build_check(ctx);
    if (bc < 0) {
      ctx->built = ctx->solved = false;
      return bc;
    }
  }
  if (ctx->pend.active) {
    solve_rc = finish_solve(ctx);
    if (solve_rc < 0) {
      ctx->solved = false;
      return solve_rc;
    }
  }
  if (rc < 0) return rc;
  return solve_rc;
}

int swm_get_stats(const swm_ctx* ctx, swm_stats* out) {
  if (!ctx || !out) return SWM_EINVAL;
  *out = ctx->stats;
  out->kernel_launches = ctx->launches;
  out->prof_ms = ctx->prof_ms;
  out->prof_launches = ctx->prof_n;
  return SWM_OK;
}

int swm_profile(swm_ctx* ctx, int kernel_class) {
  if (!ctx) return SWM_EINVAL;
  if (kernel_class < SWM_K_NONE || kernel_class > SWM_K_TRANSPOSE) return ctx->fail(SWM_EINVAL, "bad kernel class");
  SWM_TRY(set_device(ctx));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  ctx->prof_flush();
  ctx->prof_cls = kernel_class;
  ctx->prof_ms = 0.0;
  ctx->prof_n = 0;
  return SWM_OK;
}

int swm_get_pattern(swm_ctx* ctx, int64_t* pairs_out) {
  if (!ctx || !pairs_out) return SWM_EINVAL;
  if (!ctx->built) return ctx->fail(SWM_ESTATE, "no built system");
  SWM_TRY(set_device(ctx));
  const int64_t nw = ctx->nw, nb = ctx->nb;
  std::vector<int64_t> rp(nw + 1);
  std::vector<int32_t> col(nb), perm(nw);
  SWM_CK(cudaMemcpyAsync(rp.data(), ctx->row_ptr, sizeof(int64_t) * (nw + 1), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(col.data(), ctx->col, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(perm.data(), ctx->perm, sizeof(int32_t) * nw, cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  std::vector<std::pair<int64_t, int64_t>> pr;
  pr.reserve(nb);
  for (int64_t p = 0; p < nw; ++p)
    for (int64_t b = rp[p]; b < rp[p + 1]; ++b) pr.emplace_back(perm[p], perm[col[b]]);
  std::sort(pr.begin(), pr.end());
  for (int64_t i = 0; i < nb; ++i) {
    pairs_out[2 * i] = pr[i].first;
    pairs_out[2 * i + 1] = pr[i].second;
  }
  return SWM_OK;
}

int swm_get_block(swm_ctx* ctx, int64_t p, int64_t q, double* re_im_out) {
  if (!ctx || !re_im_out) return SWM_EINVAL;
  if (!ctx->built) return ctx->fail(SWM_ESTATE, "no built system");
  if (p < 0 || q < 0 || p >= ctx->nw || q >= ctx->nw) return ctx->fail(SWM_EINVAL, "wire index out of range");
  SWM_TRY(set_device(ctx));
  int32_t ip = 0, iq = 0;
  SWM_CK(cudaMemcpyAsync(&ip, ctx->iperm + p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(&iq, ctx->iperm + q, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  int64_t rp[2];
  int32_t mp = 0, mq = 0, K = 0;
  int64_t rowbase = 0;
  SWM_CK(cudaMemcpyAsync(rp, ctx->row_ptr + ip, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(&mp, ctx->m + ip, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(&mq, ctx->m + iq, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(&K, ctx->full.K + ip, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaMemcpyAsync(&rowbase, ctx->full.rowbase + ip, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  std::vector<int32_t> cols(rp[1] - rp[0]), cps(rp[1] - rp[0]);
  SWM_CK(cudaMemcpyAsync(cols.data(), ctx->col + rp[0], sizeof(int32_t) * cols.size(), cudaMemcpyDeviceToHost,
                         ctx->stream));
  SWM_CK(cudaMemcpyAsync(cps.data(), ctx->full.colpos + rp[0], sizeof(int32_t) * cps.size(), cudaMemcpyDeviceToHost,
                         ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  int64_t b = -1;
  for (size_t i = 0; i < cols.size(); ++i)
    if (cols[i] == iq) b = (int64_t)i;
  if (b < 0) return ctx->fail(SWM_EINVAL, "block not kept");
  const size_t esz = ctx->prec == SWM_C128 ? sizeof(c128) : sizeof(c64);
  std::vector<unsigned char> row(esz * mq);
  for (int i = 0; i < mp; ++i) {
    const int64_t o = rowbase + (int64_t)i * K + cps[b];
    SWM_CK(cudaMemcpyAsync(row.data(), (unsigned char*)ctx->Z + esz * o, esz * mq, cudaMemcpyDeviceToHost, ctx->stream));
    SWM_CK(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < mq; ++j) {
      if (ctx->prec == SWM_C128) {
        c128 z;
        std::memcpy(&z, row.data() + esz * j, sizeof(z));
        re_im_out[2 * (i * mq + j)] = z.re;
        re_im_out[2 * (i * mq + j) + 1] = z.im;
      } else {
        c64 z;
        std::memcpy(&z, row.data() + esz * j, sizeof(z));
        re_im_out[2 * (i * mq + j)] = z.re;
        re_im_out[2 * (i * mq + j) + 1] = z.im;
      }
    }
  }
  return SWM_OK;
}

int swm_get_rhs(swm_ctx* ctx, double* re_im_out) {
  if (!ctx || !re_im_out) return SWM_EINVAL;
  if (!ctx->solved) return ctx->fail(SWM_ESTATE, "no solve yet");
  SWM_TRY(set_device(ctx));
  SWM_TRY(ensure_user_offsets(ctx));
  const int64_t N = ctx->N;
  const int R = ctx->n_rhs;
  std::vector<Buf> tmp;
  c128* dst = nullptr;
  SWM_TRY(dalloc(ctx, tmp, (void**)&dst, sizeof(c128) * R * N));
  const dim3 grid((unsigned)ceil_div(N, 256), R);
  if (ctx->prec == SWM_C128)
    k_to_user<double><<<grid, 256, 0, ctx->stream>>>(N, R, ctx->rowwire, ctx->off, ctx->uoff, (const c128*)ctx->Bv, dst);
  else
    k_to_user<float><<<grid, 256, 0, ctx->stream>>>(N, R, ctx->rowwire, ctx->off, ctx->uoff, (const c64*)ctx->Bv, dst);
  SWM_LAUNCHED();
  SWM_CK(cudaMemcpyAsync(re_im_out, dst, sizeof(c128) * R * N, cudaMemcpyDeviceToHost, ctx->stream));
  SWM_CK(cudaStreamSynchronize(ctx->stream));
  dfree_group(ctx, tmp);
  return SWM_OK;
}

const char* swm_stateless_error(void) { return g_stateless_err.c_str(); }

// The stateless far field: sigma, or with `components` the received components theta_hat . F and
// phi_hat . F (two complex numbers per pair), which sum over disjoint sets of wires.
static int far_field_common(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                            const double* lengths, const int32_t* nseg, const int64_t* off, double k, int n_rhs,
                            const double* currents, int n_obs, const double* obs, double* sigma_out, bool components) {
  g_stateless_err.clear();
  const std::string who = components ? "swm_far_components: " : "swm_far_field: ";
  if (nw < 1 || n_rhs < 1 || n_obs < 1 || n_rhs > 65535 || !centres || !dirs || !lengths || !nseg || !off ||
      !currents || !obs || !sigma_out || !(k > 0.0)) {
    g_stateless_err = who + "bad argument";
    return SWM_EINVAL;
  }
  {
    const void* ptrs[8] = {centres, dirs, lengths, nseg, off, currents, obs, sigma_out};
    if (!all_device_memory(ptrs, 8)) {
      g_stateless_err = who + "every array must be device memory";
      return SWM_EINVAL;
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t N = 0;
  if (cudaMemcpyAsync(&N, off + nw, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    g_stateless_err = who + "cannot read off[nw]";
    return SWM_ECUDA;
  }
  const int64_t npairs = (int64_t)n_rhs * n_obs;
  const size_t sb = far_field_scratch_bytes(nw, npairs);
  void* scratch = nullptr;
  if (cudaMallocAsync(&scratch, sb, st) != cudaSuccess) {
    cudaGetLastError();
    g_stateless_err = who + "scratch allocation failed";
    return SWM_ENOMEM;
  }
  int rc = far_field_launch(st, nullptr, false, true, currents, nw, N, centres, dirs, nullptr, nullptr, nullptr,
                            nullptr, nullptr, nullptr, lengths, nseg, off, false, k, n_rhs, n_obs, obs, 2, false,
                            sigma_out, scratch, sb, &g_stateless_err, components);
  cudaFreeAsync(scratch, st);
  if (rc < 0) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    g_stateless_err = who + cudaGetErrorString(cudaGetLastError());
    return SWM_ECUDA;
  }
  return SWM_OK;
}

int swm_far_field(void* cuda_stream, int64_t nw, const double* centres, const double* dirs, const double* lengths,
                  const int32_t* nseg, const int64_t* off, double k, int n_rhs, const double* currents, int n_obs,
                  const double* obs, double* sigma_out) {
  return far_field_common(cuda_stream, nw, centres, dirs, lengths, nseg, off, k, n_rhs, currents, n_obs, obs,
                          sigma_out, false);
}

int swm_far_components(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                       const double* lengths, const int32_t* nseg, const int64_t* off, double k, int n_rhs,
                       const double* currents, int n_obs, const double* obs, double* comp_out) {
  return far_field_common(cuda_stream, nw, centres, dirs, lengths, nseg, off, k, n_rhs, currents, n_obs, obs,
                          comp_out, true);
}

}  // extern "C"
