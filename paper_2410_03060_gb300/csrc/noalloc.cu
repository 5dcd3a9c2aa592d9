// Allocation-free twin of the stateless far-field entry point (swm_far_field_noalloc).
//
// Some callers cannot allocate device memory when they need the RCS: a process whose device
// memory is fully reserved by another framework's pool, a latency-critical loop that cannot
// afford an allocation or the synchronisation it may bring, or a host that forbids dynamic
// allocation after start-up.  This variant runs the same far-field kernels as swm_far_field but
// takes its scratch (the per-chunk partial sums) from a fixed array compiled into the library
// instead of cudaMallocAsync.
#include <mutex>
#include <string>

#include "common.cuh"
#include "ctx.h"

namespace swm {
namespace {

// 8 MiB of partial sums: 48 bytes per (incidence, observation) pair and wire chunk.  Every GPU
// that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_far_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of g_far_scratch on the current device, looked up once per device (in the
// device's primary context, the one the CUDA runtime makes current).  In host code the symbol
// itself is only a host-side stand-in, never a device address.
int scratch_on_current_device(void** out, std::string* err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    *err = "swm_far_field_noalloc: no usable current device";
    return SWM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_far_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      *err = std::string("swm_far_field_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return SWM_ECUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return SWM_OK;
}

}  // namespace

int far_noalloc_impl(void* cuda_stream, int64_t nw, const double* centres, const double* dirs, const double* lengths,
                     const int32_t* nseg, const int64_t* off, double k, int n_rhs, const double* currents, int n_obs,
                     const double* obs, double* sigma_out, std::string* err);

}  // namespace swm

using namespace swm;

extern "C" {

int swm_far_field_noalloc(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                          const double* lengths, const int32_t* nseg, const int64_t* off, double k, int n_rhs,
                          const double* currents, int n_obs, const double* obs, double* sigma_out) {
  std::string msg;
  const int rc = far_noalloc_impl(cuda_stream, nw, centres, dirs, lengths, nseg, off, k, n_rhs, currents, n_obs, obs,
                                  sigma_out, &msg);
  set_stateless_error(msg);
  return rc;
}

}  // extern "C"

namespace swm {

int far_noalloc_impl(void* cuda_stream, int64_t nw, const double* centres, const double* dirs, const double* lengths,
                     const int32_t* nseg, const int64_t* off, double k, int n_rhs, const double* currents, int n_obs,
                     const double* obs, double* sigma_out, std::string* err) {
  std::string& msg = *err;
  if (nw < 1 || n_rhs < 1 || n_obs < 1 || n_rhs > 65535 || !centres || !dirs || !lengths || !nseg || !off ||
      !currents || !obs || !sigma_out || !(k > 0.0)) {
    msg = "swm_far_field_noalloc: bad argument";
    return SWM_EINVAL;
  }
  {
    const void* ptrs[8] = {centres, dirs, lengths, nseg, off, currents, obs, sigma_out};
    if (!all_device_memory(ptrs, 8)) {
      msg = "swm_far_field_noalloc: every array must be device memory";
      return SWM_EINVAL;
    }
  }
  const int64_t npairs = (int64_t)n_rhs * n_obs;
  const size_t per_chunk = (size_t)npairs * 3 * sizeof(c128);
  if (per_chunk > kNoAllocScratchBytes) {
    msg = "swm_far_field_noalloc: " + std::to_string(n_rhs) + " x " + std::to_string(n_obs) +
            " (incidence, observation) pairs need " + std::to_string(per_chunk) +
            " bytes of scratch; the fixed scratch holds " + std::to_string(kNoAllocScratchBytes) +
            " bytes (at most " + std::to_string(kNoAllocScratchBytes / (3 * sizeof(c128))) + " pairs)";
    return SWM_EINVAL;
  }
  void* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch, err);
  if (rc < 0) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t N = 0;
  if (cudaMemcpyAsync(&N, off + nw, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    msg = std::string("swm_far_field_noalloc: cannot read off[nw]: ") + cudaGetErrorString(cudaGetLastError());
    return SWM_ECUDA;
  }
  // every partial the reduction reads is written by this call, so nothing needs clearing
  rc = far_field_launch(st, nullptr, false, true, currents, nw, N, centres, dirs, nullptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, lengths, nseg, off, false, k, n_rhs, n_obs, obs, 2, false, sigma_out,
                        scratch, kNoAllocScratchBytes, err);
  if (rc < 0) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    msg = std::string("swm_far_field_noalloc: ") + cudaGetErrorString(cudaGetLastError());
    return SWM_ECUDA;
  }
  return SWM_OK;
}

}  // namespace swm
