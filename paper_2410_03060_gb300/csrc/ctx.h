// Host-side state of a swm context and the internal launcher interfaces between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "swm.h"

namespace swm {

// Variable-block-row layout of a block-sparse matrix.  Block-row p holds m_p scalar rows; each
// scalar row is stored contiguously as the concatenation of the block rows of its kept blocks in
// column order, so block-row p occupies m_p * K_p entries starting at rowbase[p] with row stride
// K_p.  Entry (i, j) of block b = (p, q) sits at rowbase[p] + i * K_p + colpos[b] + j.  colmap
// lists, per block-row, the scalar column (internal unknown index) of each of its K_p positions.
struct Layout {
  int32_t* K = nullptr;        // [nw]
  int64_t* rowbase = nullptr;  // [nw + 1]
  int64_t* cmbase = nullptr;   // [nw + 1]
  int32_t* colpos = nullptr;   // [nb], -1 when the block is not stored in this layout
  int32_t* colmap = nullptr;   // [ncm]
  int64_t nval = 0;
  int64_t ncm = 0;
};

// Row descriptor of the stored matrix E: first value, first column-map entry, row length.
struct alignas(16) RowInfo {
  int64_t vb;
  int32_t cmb;
  int32_t K;
};

struct Buf {
  void* p;
  size_t bytes;
};

}  // namespace swm

struct swm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  swm_alloc_fn user_alloc = nullptr;
  swm_free_fn user_free = nullptr;
  void* user_arg = nullptr;
  // device buffers by lifetime: the cloud; the S-NFC pattern and everything indexed by it (kept
  // across builds at the same r_c: frequency sweeps refill only the values); the values at one k;
  // one solve
  std::vector<swm::Buf> cloud_bufs, pattern_bufs, build_bufs, solve_bufs;
  bool pattern_ok = false;  // pattern_bufs hold the pattern of (pattern_rc, pattern_dense)
  double pattern_rc = 0.0;
  bool pattern_dense = false;
  // buffers released by a group wait here for reuse by later allocations on the same stream
  // (stream order makes the reuse safe); they are returned to the allocator by swm_destroy
  std::vector<swm::Buf> free_list;
  std::vector<swm::Buf> kry_bufs;  // Krylov workspace, kept while the problem size stays the same
  void* kry_ws = nullptr;          // host record of that workspace (krylov.cu)
  size_t kry_ws_bytes = 0;
  int64_t launches = 0;

  // phase timing with CUDA events, read after the call's final synchronisation
  enum { PH_NEIGHBOUR, PH_FILL, PH_PRECOND, PH_RHS, PH_SOLVE, PH_RCS, PH_N };
  cudaEvent_t ph_ev[PH_N][2] = {};
  bool ph_rec[PH_N] = {};
  void phase_begin(int i) {
    if (!ph_ev[i][0]) {
      cudaEventCreate(&ph_ev[i][0]);
      cudaEventCreate(&ph_ev[i][1]);
    }
    cudaEventRecord(ph_ev[i][0], stream);
  }
  void phase_end(int i) {
    cudaEventRecord(ph_ev[i][1], stream);
    ph_rec[i] = true;
  }
  void phase_collect() {
    double* dst[PH_N] = {&stats.ms_neighbour, &stats.ms_fill, &stats.ms_precond, &stats.ms_rhs, &stats.ms_solve,
                         &stats.ms_rcs};
    for (int i = 0; i < PH_N; ++i) {
      if (!ph_rec[i]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ph_ev[i][0], ph_ev[i][1]) == cudaSuccess) *dst[i] = ms;
      ph_rec[i] = false;
    }
    cudaGetLastError();
  }

  // cloud, caller order, device
  int64_t nw = 0;
  double *u_c = nullptr, *u_t = nullptr, *u_L = nullptr, *u_a = nullptr;
  int32_t* u_ns = nullptr;
  int max_ns = 0;
  double bbox[6] = {0, 0, 0, 0, 0, 0};  // min xyz, max xyz of the centres

  // built system
  bool built = false;
  double k = 0.0, rc = 0.0;
  int prec = SWM_C128;
  bool dense = false;
  double *cx = nullptr, *cy = nullptr, *cz = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr;
  double *L = nullptr, *a = nullptr;
  int32_t* ns = nullptr;     // segments per internal wire
  int32_t* m = nullptr;      // unknowns per internal wire
  int32_t* perm = nullptr;   // internal wire -> caller wire
  int32_t* iperm = nullptr;  // caller wire -> internal wire
  int64_t* off = nullptr;    // internal unknown offsets [nw + 1]
  int64_t* uoff = nullptr;   // caller-order unknown offset of internal wire p [nw]
  int64_t* uoff_user = nullptr;  // caller-order unknown offsets by caller wire [nw + 1]
  int64_t N = 0;
  int64_t nb = 0, nup = 0;
  int64_t* row_ptr = nullptr;  // [nw + 1]
  int32_t* col = nullptr;      // [nb]
  int64_t* bt = nullptr;       // [nb] index of the transposed block
  int64_t* diag_b = nullptr;   // [nw] index of block (p, p)
  int64_t* ublk = nullptr;     // [nup] blocks (p, q) with q > p
  int64_t* minv_off = nullptr; // [nw + 1] offsets of the m_p x m_p inverse blocks
  int32_t* rowwire = nullptr;  // [N] internal wire of each scalar row
  void* wrec = nullptr;        // [nw] wire records of product form 75 in its order (built by the
                               // first solve that may use it after a pattern build)
  void* rowinfo = nullptr;     // [N] row descriptors of E (value offset, column-map offset, length)
  int64_t nminv = 0;           // entries of the packed self-block inverses
  unsigned long long* d_evals = nullptr;  // fill evaluation counter (device)
  int* d_sing = nullptr;                  // singular self block flag (device)
  void* pinned_state = nullptr;           // two pinned slots for the Krylov state poll
  unsigned* d_arrive = nullptr;           // arrival counter of the cloud-check kernel (kept zero)
  const double* rhs_frames = nullptr;     // b not yet formed: the solver forms it from these frames
  // swm_run: the build's and the persistent solve's final read-backs are left in pinned memory and
  // checked after the run's last synchronisation
  bool fused = false;
  bool build_check_pending = false;
  size_t up_used = 0;  // bytes of the pinned staging area with copies possibly pending
  struct PendingSolve {
    bool active = false;
    int R = 0;
    bool* sync_clean = nullptr;
  } pend;
  int solver = 0;                         // SWM_SOLVER_GMRES or SWM_SOLVER_GCR
  // right-hand sides per block of the fused multi-incidence GMRES step, measured per system shape
  // (N, n_rhs, vector and matrix entry sizes, chunk, restart)
  struct Tuned {
    int64_t shape[6];
    int rb;
  };
  std::vector<Tuned> tuned;
  const void* guess = nullptr;            // during swm_solve_guess: y0 = M x0, complex128 [n_rhs][N]
  void* ffw = nullptr;                    // per-wire float32 far-field data (complex64 path)
  cudaGraphExec_t gm_exec = nullptr;      // captured chunk of GMRES steps and its argument key
  std::vector<unsigned char> gm_key;
  cudaStream_t cap_stream = nullptr;      // private stream for graph capture
  cudaStream_t side = nullptr;            // second stream of the build (self blocks and their inverses)
  cudaEvent_t side_ev[2] = {nullptr, nullptr};  // fork and join of the side stream
  // systems with at least this many unknowns run the Arnoldi step as a streaming product plus
  // separate dots (bandwidth); smaller ones as one fused kernel (latency).  SWM_SPLIT_ROWS overrides.
  int64_t split_rows = int64_t(1) << 19;
  // systems below split_rows with at most 8 right-hand sides solve in one persistent cooperative
  // kernel (SWM_PERSIST=0 turns it off); SM count and cooperative-launch support of the device
  bool persist = true;
  // test hook (SWM_BICGSTAB_MAJOR=1): BiCGSTAB keeps its vectors incidence-major on the complex64
  // path too, as it does on the float64 path and with one incidence
  bool bicg_major = false;
  // CTAs per SM of the incidence-minor BiCGSTAB vector passes (SWM_BICGSTAB_CTAS, default 4)
  int bicg_ctas = 4;
  // test hook (SWM_TEST_BARRIER_EXTRA): grid barriers of the persistent solve wait for this many
  // arrivals more than there are CTAs, so every wait runs out and the solve reports SWM_ETIMEOUT
  int test_barrier_extra = 0;
  int product_form = 0;                   // many right-hand sides: 0 = timed choice, else that form
                                          // (4, 8, 16, 32 incidence-minor, 64, 65, 67 wire-tiled)
  int persist_ctas = 0;                   // CTAs of the persistent solve (0: one per SM)
  int nsm = 0;
  int coop = 0;
  int smem_optin = 0;  // shared memory a CTA may opt in to (bytes)
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  swm::Layout full, offd;
  void* Z = nullptr;     // values of Z in layout `full`
  void* Zp = nullptr;    // values of Z * blockdiag(Z)^-1 without its identity diagonal, layout `offd`
  void* Minv = nullptr;  // inverses of the self blocks
  void* E16 = nullptr;   // precision SWM_BF16: E as complex bfloat16 (inner products of the refinement)
  bool bf16 = false;     // the last build was SWM_BF16 (values complex64, plus E16)

  // last solve
  int n_rhs = 0;
  void* Bv = nullptr;  // right-hand sides [n_rhs][N] (internal order)
  void* Xv = nullptr;  // currents [n_rhs][N] (internal order)
  double* inc_dev = nullptr;
  bool solved = false;

  swm_stats stats{};

  // per-kernel-class event timing (swm_profile)
  int prof_cls = SWM_K_NONE;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  size_t prof_used = 0;
  double prof_ms = 0.0;
  int64_t prof_n = 0;
  void prof_begin(int cls) {
    if (cls != prof_cls) return;
    if (prof_used == prof_ev.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      prof_ev.emplace_back(a, b);
    }
    cudaEventRecord(prof_ev[prof_used].first, stream);
  }
  void prof_end(int cls) {
    if (cls != prof_cls) return;
    cudaEventRecord(prof_ev[prof_used].second, stream);
    ++prof_used;
  }
  // add the recorded intervals (the stream must have been synchronised)
  void prof_flush() {
    for (size_t i = 0; i < prof_used; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, prof_ev[i].first, prof_ev[i].second) == cudaSuccess) prof_ms += ms;
    }
    prof_n += (int64_t)prof_used;
    prof_used = 0;
    cudaGetLastError();
  }

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
};

namespace swm {

// allocation helpers (api.cu)
int dalloc(swm_ctx* ctx, std::vector<Buf>& group, void** out, size_t bytes);
void dfree_group(swm_ctx* ctx, std::vector<Buf>& group);

#define SWM_CK(call)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return ctx->fail(SWM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define SWM_LAUNCHED()                                                                   \
  do {                                                                                   \
    ctx->launches++;                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      return ctx->fail(SWM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

#define SWM_TRY(expr)      \
  do {                     \
    int rc_ = (expr);      \
    if (rc_ < 0) return rc_; \
  } while (0)

// neighbour.cu: a0 + a1 (sort by cell, numbering, S-NFC pattern, layouts)
int build_pattern(swm_ctx* ctx);
// copy n device int64 values to the host with one synchronisation
// launch the bounding-box reduction of the caller centres into out6 (device)
// caller-order unknown offsets, made on first use
int ensure_user_offsets(swm_ctx* ctx);
// precond.cu: read the build's deferred device flags and counters
int finish_build(swm_ctx* ctx);
int finish_build_check(swm_ctx* ctx);
int finish_solve(swm_ctx* ctx);
// scan.cu
int exclusive_scan_i64(swm_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host);
int exclusive_scan_i32_to_i64(swm_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* total_host);
// up to six scans of the same length (one launch when short); inputs int64 (is64) or int32
int exclusive_scan_multi(swm_ctx* ctx, int narr, const void* const* in, const int* is64, int64_t* const* out,
                         int64_t n, int64_t* totals = nullptr);
// fill.cu: a2 + a3
int fill_alloc(swm_ctx* ctx);
int fill_self(swm_ctx* ctx, cudaStream_t s);
int fill_mutual(swm_ctx* ctx);
// precond.cu: a5
int precond_alloc(swm_ctx* ctx);
int precond_invert(swm_ctx* ctx, cudaStream_t s);
int precond_form_E(swm_ctx* ctx);
// rhs_ff.cu: a4 + a7
int compute_rhs(swm_ctx* ctx, int n_inc, const double* inc_dev);
size_t far_field_scratch_bytes(int64_t nw, int64_t npairs);
size_t far_field_f32_scratch_bytes(const swm_ctx* ctx, int64_t npairs, int n_obs);
int far_field_alloc(swm_ctx* ctx);
int prepare_far_field(swm_ctx* ctx, cudaStream_t s);
int far_field_f32_launch(swm_ctx* ctx, int n_obs, const double* obs, int obs_stride, bool mono, double* sigma,
                         void* scratch, size_t scratch_bytes);
int far_field_launch(cudaStream_t st, int64_t* launches, bool cur_c64, bool f64, const void* cur, int64_t nw,
                     int64_t N, const double* c3, const double* t3, const double* cx, const double* cy,
                     const double* cz, const double* tx, const double* ty, const double* tz, const double* Ls,
                     const int32_t* ns, const int64_t* off, bool soa, double k, int n_rhs, int n_obs,
                     const double* obs, int obs_stride, bool mono, double* sigma, void* scratch, size_t scratch_bytes,
                     std::string* err, bool components = false);
// incidence frames on the host: k_hat (propagation, = -arrival) then polarisation e, 6 doubles each
void frames_host(const double* inc, int n, std::vector<double>& out);
// true if every pointer is device or managed memory (api.cu)
bool all_device_memory(const void* const* ptrs, int n);
// error text reported by swm_stateless_error() (api.cu)
void set_stateless_error(const std::string& msg);
// krylov.cu: a6
int gmres_solve(swm_ctx* ctx, double tol, int restart, int max_iter);
int bicgstab_solve(swm_ctx* ctx, double tol, int max_iter);
int build_wire_order(swm_ctx* ctx);
// row descriptors of E (built once per build) and x = M^-1 y into ctx->Xv
int ensure_rowinfo(swm_ctx* ctx);
// y = y0 (ctx->guess, complex128) or 0 at the start of a solve, in the vector precision
int init_y(swm_ctx* ctx, void* Y, bool f64);
// |b_r| of the [n_rhs][N] right-hand sides into bnorm_dev (device), 1 for a zero one
int norms_of_b(swm_ctx* ctx, const void* B, bool f64, double* bnorm_dev);
// Lets kernel `fn` launch with as much dynamic shared memory as a CTA may have on the device
// (smem_optin less its static shared memory).  Always the same value for a kernel, so contexts
// driven from several host threads do not undo each other's setting of this process-wide
// attribute; a launch that asks for less is unaffected.
// Sets a kernel's dynamic shared-memory limit to all the device allows beside its static shared
// memory.  The attribute is process-wide and every caller sets the same value, so contexts on
// concurrent host threads cannot undo one another; it is set once per kernel and device (api.cu
// keeps the table) and the kernel's static shared memory is returned through *static_bytes.
cudaError_t allow_max_dyn_smem(const void* fn, int smem_optin, size_t* static_bytes = nullptr);
// Resident CTAs per SM of a kernel at a block size and dynamic shared memory, queried once per
// kernel, device and shape.
cudaError_t occupancy_cached(const void* fn, int threads, size_t smem, int* blocks);
// pinned host memory of a context (small copies without a staged pageable copy): two slots (128
// bytes in all) for polling the solvers' device state, 64 bytes for the cloud checks and the
// pattern sizes, the persistent solve's state and abort flag, up to kPinnedResidMax float64 values
// read back (relative residuals, build counters), and a staging area for small uploads
// (incidences, observation angles).  Every entry point ends with a stream synchronisation, so an
// area is never rewritten while a copy from it is pending.
constexpr size_t kPollSlotBytes = 65536;
constexpr size_t kIngestSlotOffset = 128;
constexpr size_t kPersistStateOffset = 192;
constexpr size_t kPersistAbortOffset = 224;
constexpr size_t kBuildCountersOffset = 232;  // fill evaluations (8 bytes) and the singular flag (4)
constexpr size_t kPinnedResidOffset = 256;
constexpr size_t kPinnedUpOffset = 32768;
constexpr size_t kPinnedUpBytes = kPollSlotBytes - kPinnedUpOffset;
constexpr int kPinnedResidMax = (int)((kPinnedUpOffset - kPinnedResidOffset) / sizeof(double));
int ensure_poll_slots(swm_ctx* ctx);
int apply_minv(swm_ctx* ctx, const void* Y);
// gcr.cu: the paper's GCR solver (alternative to GMRES)
int gcr_solve(swm_ctx* ctx, double tol, int restart, int max_iter);
// krylov.cu: GMRES on the bfloat16 copy of E (inner solve of the refinement); y-space result
int gmres_inner_bf16(swm_ctx* ctx, double tol, int restart, int max_iter, void** y_out, int* iters);
// Rr = B - (Y + E Y) for every right-hand side in float64 vectors with the complex64 E, one read of
// E shared by all right-hand sides (wire-tiled product, krylov.cu); with Yt (R x N scratch) the
// gathers read y right-hand-side minor
int residual_f64_wire(swm_ctx* ctx, const c128* B, const c128* Y, c128* Rr, c128* Yt);
// Y = X + E X for R right-hand sides in float64 arithmetic with the stored E (complex128 or
// complex64), internal order, every right-hand side (krylov.cu)
int product_f64(swm_ctx* ctx, int R, const c128* X, c128* Y);
// rhs_ff.cu: right-hand sides in float64 into `out` ([n_inc][N], internal order)
int compute_rhs_f64(swm_ctx* ctx, int n_inc, const double* frames_dev, c128* out);
// refine.cu: float64 iterative refinement around bfloat16-storage GMRES (precision SWM_BF16)
int refine_solve(swm_ctx* ctx, const double* frames_dev, double tol, int restart, int max_iter);
// precond.cu: bfloat16 copy of E (ctx->E16) for precision SWM_BF16
int make_e16(swm_ctx* ctx);

}  // namespace swm
