/*
 * swm.h -- C ABI of the GB300 (sm_103a) sparsified thin-wire method-of-moments solver.
 *
 * The library computes the electric currents induced on a cloud of straight, thin, perfectly
 * conducting wires ("chaffs") by plane waves, and the radar cross section (RCS) they scatter,
 * following arXiv 2410.03060 ("Fast algorithm for full-wave EM scattering analysis of large-scale
 * chaff cloud ..."):
 *
 *   - Sec. II-A, Eq. (current_expression) and its footnote: each wire p is cut into n_s(p) equal
 *     segments; the n_s(p) - 1 interior vertices carry rooftop unknowns.  Unknowns are numbered
 *     wire by wire in the caller's wire order: unknown (p, i) has index off_p + i, i = 0..n_s(p)-2,
 *     off_p = sum over wires q < p of (n_s(q) - 1).
 *   - Sec. II-A, Eqs. (TW_EFIE_MOM), (4)-(8): Galerkin testing of the thin-wire EFIE.  The library
 *     solves the scaled system Z jt = b with
 *         b_m  = int Lambda_m(s) t_m . E_inc(r(s)) ds,
 *         Z_mn = (t_m.t_n) int int Lambda_m Lambda_n G - (1/k^2) int int Lambda_m' Lambda_n' G,
 *     G = exp(-j k R)/(4 pi R), R = sqrt(|r - r'|^2 + a^2) (reduced thin-wire kernel).  This is the
 *     paper's Z j = v multiplied by j*omega*mu0, so the physical current in amperes is
 *     jt / (j omega mu0) = -j jt / (k eta0).  Time convention exp(+j omega t).
 *   - Sec. II-B, Eq. (neardef) (S-NFC): the block Z_pq is kept iff the centroid distance
 *     |c_p - c_q| <= r_c (inclusive), every other block is zero.
 *   - Sec. II-B (after Eq. neardef): the block-sparse system is solved iteratively with a
 *     block-diagonal preconditioner; this library uses restarted GMRES, right-preconditioned by
 *     the inverses of the self blocks Z_pp.
 *   - Sec. III-A, III-B: bistatic and monostatic RCS from the far field of the currents.
 *
 * Quadrature (the paper names only "analytic singularity extraction" and "Gaussian quadrature"):
 * different wires use tensor Gauss-Legendre with 4 points per segment (8 when the two wires come
 * closer than the longer segment length); segments of one wire use an exact reduction of the
 * double integral to one dimension, 8 Gauss points per half, and a closed-form static part for
 * coincident or touching segments.  The mutual radius is a^2 = (a_p^2 + a_q^2)/2.
 *
 * Conventions.  Lengths in metres (any unit works if k is in radians per that unit); k in rad/m.
 * Incident plane waves have amplitude 1 V/m.  An incidence is (theta, phi, psi) in radians: the
 * wave ARRIVES from the direction u = (sin th cos ph, sin th sin ph, cos th), i.e. it propagates
 * along -u, and its polarisation is cos(psi) theta_hat + sin(psi) phi_hat of the spherical frame
 * at (theta, phi).  An observation is (theta, phi).  sigma = |e_s . F|^2 / (4 pi) where F is the
 * radiation vector of the currents and e_s is theta_hat (index 0) or phi_hat (index 1) at the
 * observation direction; RCS is in m^2.
 *
 * Memory.  Pointers tagged SWM_HOST are ordinary host memory; SWM_DEVICE pointers are device
 * memory of the context's device (e.g. torch data_ptr()).  The library copies every input it
 * keeps; the caller keeps ownership of every buffer it passes.  Work runs on the context's CUDA
 * stream; calls return after their results are complete in the output buffers.
 *
 * Errors.  Every int-returning call returns SWM_OK (0), a positive warning, or a negative error.
 * On an error the context keeps its previous valid state where possible and swm_last_error()
 * describes the failure.  Nothing throws across the ABI.  A context is not thread-safe: use one
 * context per host thread.
 */
#ifndef SWM_H
#define SWM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SWM_OK 0
#define SWM_ENOTCONV 1 /* warning: GMRES hit max_iter before tol; outputs hold the last iterate */
#define SWM_EINVAL (-1) /* invalid argument (bad size, NaN, non-unit direction, ...) */
#define SWM_ENOMEM (-2) /* device allocation failed */
#define SWM_ECUDA (-3)  /* a CUDA runtime call or kernel failed */
#define SWM_ESTATE (-4) /* call out of order (e.g. solve before build) */
#define SWM_ETIMEOUT (-5) /* a bounded device-side wait ran out (grid barrier of the persistent
                             GMRES kernel, limit 1 s); the context stays usable */

/* memory kinds */
#define SWM_HOST 0
#define SWM_DEVICE 1

/* precision of the fill, the stored blocks and the Krylov vectors */
#define SWM_C128 0 /* plain path: FP64 kernel evaluation, complex128 blocks, complex128 GMRES */
#define SWM_C64 1  /* fast path: FP64 per-block geometry, FP32 kernel evaluation, complex64 blocks
                      and vectors; FP64 dot products, norms, Hessenberg and rotations, except in
                      the persistent solve of small systems, which keeps them in FP32 */
#define SWM_BF16 2 /* mixed path: the SWM_C64 fill and blocks, plus Z M^-1 rounded to complex
                      bfloat16 for the Krylov products; swm_solve runs FP64 iterative refinement
                      (residuals b - Z x with the complex64 blocks, FP64 vectors) around GMRES on
                      the bfloat16 blocks (complex64 vectors; inner tolerance 2e-3, loosened on the
                      last refinement steps to what tol still needs); the GMRES
                      solver is used whatever swm_set_solver chose; currents stored complex64 */

/* limits */
#define SWM_MAX_SEG 16  /* segments per wire: 2 <= n_s <= SWM_MAX_SEG */
#define SWM_MAX_RESTART 128

typedef struct swm_ctx swm_ctx;

typedef struct swm_stats {
  int64_t nw;          /* wires */
  int64_t n;           /* unknowns */
  int64_t nb;          /* kept blocks, full storage, diagonal included */
  int64_t nnz;         /* stored complex entries of Z */
  int n_rhs;           /* incidences of the last solve */
  int iterations;      /* GMRES iterations (matrix-vector products) of the last solve */
  int restarts;        /* restart cycles of the last solve */
  int converged;       /* 1 if every right-hand side reached tol */
  double rel_residual; /* max over right-hand sides of ||b - Z x|| / ||b|| at exit */
  double ms_neighbour; /* phase times of the last build / solve / rcs call (CUDA events) */
  double ms_fill;
  double ms_precond;
  double ms_rhs;
  double ms_solve;
  double ms_rcs;
  int64_t kernel_launches; /* kernels launched by this context since its creation */
  int64_t fill_evals;      /* kernel evaluations of the mutual fill (sum over blocks p < q of
                              n_s(p) n_s(q) n_q^2) in the last build */
  int64_t nnz_offd;        /* stored entries of Z M^-1 without its diagonal blocks */
  int64_t ncm_offd;        /* column-map entries of that matrix (sum over block-rows of K_p) */
  double prof_ms;          /* summed device time of the profiled kernel class (swm_profile) */
  int64_t prof_launches;   /* launches of the profiled kernel class */
  int pattern_reused;      /* 1 if the last build kept the previous S-NFC pattern (same cloud and
                              r_c, e.g. a frequency sweep) and only refilled the values */
  int step_rhs_block;      /* form of the last solve's per-kernel GMRES product: incidences
                              sharing each read of the blocks (1, 4, 8 or 16), 32 for the
                              incidence-minor form, 64, 65 or 67 for the wire-tiled forms (a CTA
                              per group of wires, every incidence sharing its reads of E); as
                              timed on the system the first time a shape was solved on this
                              context */
  int64_t nminv;           /* stored entries of the self-block inverses (sum over wires of m_p^2) */
} swm_stats;

/* kernel classes for swm_profile */
#define SWM_K_NONE 0
#define SWM_K_PAIRS 1       /* S-NFC pair count and write passes */
#define SWM_K_FILL_SELF 2   /* self blocks */
#define SWM_K_FILL_MUTUAL 3 /* mutual blocks */
#define SWM_K_INVERT 4      /* self-block inverses */
#define SWM_K_FORM_E 5      /* Z_pq Z_qq^-1 */
#define SWM_K_RHS 6         /* right-hand sides */
#define SWM_K_APPLY 7       /* block-sparse product w = A u of each Arnoldi step (with the transpose
                               to incidence-minor order when that form runs), and the residual
                               b - A y at each restart */
#define SWM_K_DOTS 8        /* dots of the delayed Gram-Schmidt (Q^H u, Q^H w, |u|^2, u^H w) with the
                               Hessenberg column, rotation and residual estimate they complete */
#define SWM_K_UPDATE 9      /* update of the delayed Gram-Schmidt (q_j and the next vector) */
#define SWM_K_FINISH 10     /* unused (kept so that class numbers stay as they were) */
#define SWM_K_FAR 11        /* far field: partial sums and their reduction to RCS */
#define SWM_K_TRANSPOSE 13  /* copy of the pending vectors to incidence-minor order before the
                               wire-tiled product with two incidences per thread (form 67); the
                               APPLY class then times the product kernel alone */
#define SWM_K_GMRES 12      /* the whole solve as one persistent cooperative kernel (systems below
                               SWM_SPLIT_ROWS unknowns with at most 8 right-hand sides); the
                               per-step classes 7-10 then launch nothing */

/* Create a context on CUDA device `device` that issues all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the context.
 * Environment: SWM_SPLIT_ROWS (default 524288) -- systems with at least this many unknowns never
 * run the persistent solve; SWM_PERSIST (default 1) -- 0 solves small systems with one launch per
 * kernel of each GMRES step instead of the persistent cooperative kernel;
 * SWM_PERSIST_CTAS (default 0 = one per SM) -- CTAs of the persistent solve, at most one per SM;
 * SWM_PRODUCT_FORM (default 0 = timed choice) -- with several incidences, the product form of the
 * per-kernel GMRES (and, for 68-75, of BiCGSTAB) to use instead of timing them: 4, 8 or 16
 * incidences per read of E, 32 the incidence-minor form (12 or more incidences), 64 the
 * wire-tiled form (65: the same with five CTAs per SM; 67: two incidences per thread and the
 * tile's E in shared memory; 68/69: two incidences per thread in packed FP32x2 arithmetic, E
 * staged in shared memory, three CTAs per SM with 48 KB or two with 96 KB; 70/71: the packed form
 * reading E from global memory, three or four CTAs per SM; 72/73: the same in small CTAs of a
 * few whole warps; 74: small CTAs with E and the column map staged by cp.async; 75: 74 over the
 * wires sorted by loop length within windows of 4096);
 * SWM_BICGSTAB_MAJOR (default 0, a test hook) -- 1 keeps BiCGSTAB's vectors incidence-major on the
 * complex64 path (as on the float64 path and with one incidence) instead of incidence-minor;
 * SWM_BICGSTAB_CTAS (default 4, 1-64) -- CTAs per SM of the incidence-minor BiCGSTAB vector passes
 * (their chunks of rows, at least 2048 rows each);
 * SWM_TEST_BARRIER_EXTRA (default 0, a test hook) -- n > 0 makes every grid barrier of the
 * persistent solve wait for n arrivals that never come, so each wait runs out (after 1 s) and the
 * solve returns SWM_ETIMEOUT; all read when the context is created. */
int swm_create(swm_ctx** out, int device, void* cuda_stream);

/* Free every device buffer of the context and the context itself.  NULL is ignored. */
void swm_destroy(swm_ctx* ctx);

/* Message of the last failed call on this context ("" if none).  Valid until the next call. */
const char* swm_last_error(const swm_ctx* ctx);

/* Route the context's device allocations through caller-supplied functions (e.g. a caching
 * allocator).  alloc returns device memory of at least `bytes` usable on `stream` or NULL; free
 * releases it.  Must be called before swm_set_cloud.  Passing NULL functions restores
 * cudaMallocAsync / cudaFreeAsync on the context stream. */
typedef void* (*swm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*swm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);
int swm_set_allocator(swm_ctx* ctx, swm_alloc_fn alloc, swm_free_fn free_fn, void* user);

/* Load a wire cloud (Sec. II-A).  nw >= 1 wires:
 *   centres  nw x 3 float64 (row-major), wire centroids c_p;
 *   dirs     nw x 3 float64, unit directions t_p (|t_p| = 1 within 1e-9);
 *   lengths  nw float64 > 0;
 *   radii    nw float64 > 0;
 *   nseg     nw int32 segment counts, 2 <= nseg <= SWM_MAX_SEG (unknowns per wire = nseg - 1).
 * All five pointers have the same memory kind `mem_kind`.  Replaces any previous cloud and
 * invalidates any built matrix.  SWM_EINVAL on a NaN, a non-unit direction, a non-positive
 * length or radius, or a segment count out of range (checked on the device for SWM_DEVICE). */
int swm_set_cloud(swm_ctx* ctx, int64_t nw, const double* centres, const double* dirs,
                  const double* lengths, const double* radii, const int32_t* nseg, int mem_kind);

/* Build the S-NFC system (Sec. II-B): neighbour search with coupling radius r_c (r_c <= 0 or
 * infinite = entire coupling, every block kept), fill of every kept block at wavenumber k > 0
 * (Eqs. (5)-(8)), and the block-Jacobi preconditioner.  precision is SWM_C128, SWM_C64 or SWM_BF16
 * (see their definitions above; SWM_BF16 also stores Z M^-1 rounded to complex bfloat16).
 * The pattern depends on the cloud and r_c only: a build with the same r_c as the previous one
 * on the same cloud (a frequency sweep: only k changes) keeps the pattern, its index arrays and
 * the wire order, and refills the values (swm_stats.pattern_reused = 1).
 * Device memory: about 16 (c128) or 8 (c64) bytes per stored entry, twice (Z and Z times the
 * preconditioner), plus O(nw + nb) index arrays. */
int swm_build(swm_ctx* ctx, double k, double r_c, int precision);

/* Krylov method of swm_solve (both right-preconditioned by the inverses of the self blocks and
 * minimising the residual over the same Krylov space, restarted every `restart` steps):
 * SWM_SOLVER_GMRES (default) -- restarted GMRES, Hessenberg least squares by Givens rotations;
 * SWM_SOLVER_GCR -- restarted GCR, the method the paper names (Sec. II-B, after Eq. neardef):
 * per step one product, two Gram-Schmidt passes over the stored images A p_i, and an update of
 * the iterate and of the residual, whose norm is then exact; it stores two bases (p_i and A p_i).
 * SWM_SOLVER_BICGSTAB -- BiCGSTAB (van der Vorst 1992), a short-recurrence alternative for the
 * same preconditioned system: per step two products and a fixed number of vector passes (no
 * basis, so `restart` is ignored); max_iter counts its steps (two products each).  On the complex64
 * path with 2 to 256 incidences its vectors are kept incidence-minor, the layout the product
 * gathers from.  It stops when
 * the recursive residual meets tol, then forms the true residual b - Z x and restarts from it
 * where that is still above tol; the reported residuals are the true ones.  Not used with
 * precision SWM_BF16, whose refinement runs GMRES inside.
 * Applies to the following swm_solve calls of this context; SWM_EINVAL for another value. */
#define SWM_SOLVER_GMRES 0
#define SWM_SOLVER_GCR 1
#define SWM_SOLVER_BICGSTAB 2
int swm_set_solver(swm_ctx* ctx, int method);

/* Solve Z jt = b for n_inc >= 1 incidences (Eq. (4) right-hand sides), inc = n_inc x 3 float64
 * (theta, phi, psi) in host memory.  Restarted GMRES(restart) or GCR(restart) (swm_set_solver),
 * 1 <= restart <= SWM_MAX_RESTART, stops when every relative residual ||b - Z x||/||b|| <= tol or
 * after max_iter iterations (SWM_ENOTCONV, last iterate kept).  The currents stay in the context for the RCS calls; if
 * currents_out is not NULL they are also written there as n_inc x N complex128 (interleaved
 * re, im; incidence-major, caller's unknown order), in memory of kind out_kind. */
int swm_solve(swm_ctx* ctx, int n_inc, const double* inc, double tol, int restart, int max_iter,
              double* currents_out, int out_kind);

/* swm_solve from an initial guess x0 (n_inc x N complex128, interleaved re, im; incidence-major,
 * caller's unknown order, memory of kind x0_kind): the Krylov iteration starts from y0 = M x0
 * (M = blockdiag(Z_pp), the right preconditioner) instead of zero; tol stays relative to |b|.
 * No counterpart in the paper: it serves the learned warm start (swm_net_predict).  Otherwise as
 * swm_solve. */
int swm_solve_guess(swm_ctx* ctx, int n_inc, const double* inc, const double* x0, int x0_kind, double tol,
                    int restart, int max_iter, double* currents_out, int out_kind);

/* Learned warm start (no counterpart in the paper): a rotation-invariant neighbourhood network
 * that predicts each wire's current as the isolated-wire current Z_pp^-1 b_p plus three complex
 * sine modes along the wire.  For each of the wire's up to 16 nearest S-NFC partners an MLP
 * (16-128-128-18, SiLU) maps 16 invariant features in the wire's frame (offsets along and across
 * the wire / r_c, direction cosines, lengths / wavelength, the incident polarisation and direction
 * projected on both wires, the incident phase difference, the propagation phase over the
 * distance, a presence flag) to a complex 3 x 3 coupling matrix, applied to the partner's
 * isolated-current mode amplitudes; their sum h and an output MLP (20-256-256-6, SiLU) on
 * [h, 8 own features, own amplitudes] give the mode corrections h + o.  93,720 float32 parameters
 * (W[in][out] then b, layer by layer).  Forward, backward and Adam are the library's kernels.  A
 * network belongs to one device; it reads the geometry, pattern, k, r_c (finite) and block-Jacobi
 * inverses of a built context.  Workspace: about 3 KB per wire-incidence sample (training) on
 * the context's device. */
typedef struct swm_net swm_net;
int64_t swm_net_num_params(void);
int swm_net_create(swm_net** out, int device, void* cuda_stream);
void swm_net_destroy(swm_net* net);
const char* swm_net_last_error(const swm_net* net);
/* parameters in or out (host or device pointer of swm_net_num_params() float32); setting them
 * resets the Adam moments */
int swm_net_set_params(swm_net* net, const float* params, int mem_kind);
int swm_net_get_params(swm_net* net, float* params, int mem_kind);
/* predicted currents x0 (n_inc x N complex128, caller order) for the context's built system */
int swm_net_predict(swm_net* net, swm_ctx* ctx, int n_inc, const double* inc, double* x0_out, int out_kind);
/* one training step on targets x_true (n_inc x N complex128, caller order): loss
 * sum|x0 - x_true|^2 / sum|x_true|^2 to *loss_out, its gradient to grad_out (optional, float32),
 * and with lr > 0 an Adam update (beta 0.9, 0.999, eps 1e-8) of the parameters */
int swm_net_train_step(swm_net* net, swm_ctx* ctx, int n_inc, const double* inc, const double* x_true, int xt_kind,
                       float lr, double* loss_out, float* grad_out);

/* Bistatic RCS (Sec. III-A) of the currents of the last solve at n_obs >= 1 observation
 * directions obs = n_obs x 2 float64 (theta, phi), host memory.  sigma_out receives
 * n_inc x n_obs x 2 float64 (theta- and phi-received), memory of kind out_kind. */
int swm_rcs_bistatic(swm_ctx* ctx, int n_obs, const double* obs, double* sigma_out, int out_kind);

/* The whole path in one call: swm_set_cloud, swm_build, swm_solve (no currents_out) and
 * swm_rcs_bistatic -- or, with n_obs = 0 and obs = NULL, swm_rcs_monostatic (sigma_out then
 * n_inc x 2) -- with the same arguments, meanings and results as those calls made in turn (the
 * paper has no counterpart; this is an entry point of this library).  It synchronises the host only
 * where it needs device results (the cloud's bounding box, the pattern sizes, the RCS): the build's
 * checks and the solver's final state are read after the last synchronisation, so a singular self
 * block is reported (SWM_EINVAL) after the solve and RCS have run on it.  Returns the first error,
 * else the solve's status (SWM_OK or SWM_ENOTCONV).  Statistics as after the separate calls. */
int swm_run(swm_ctx* ctx, int64_t nw, const double* centres, const double* dirs, const double* lengths,
            const double* radii, const int32_t* nseg, int mem_kind, double k, double r_c, int precision, int n_inc,
            const double* inc, double tol, int restart, int max_iter, int n_obs, const double* obs,
            double* sigma_out, int out_kind);

/* Monostatic RCS (Sec. III-B): each incidence observed back along its arrival direction.
 * sigma_out receives n_inc x 2 float64, memory of kind out_kind. */
int swm_rcs_monostatic(swm_ctx* ctx, double* sigma_out, int out_kind);

/* Counters and phase times of the context. */
int swm_get_stats(const swm_ctx* ctx, swm_stats* out);

/* Time every launch of one kernel class (SWM_K_*) with CUDA events on the context stream from now
 * on, adding to stats.prof_ms / stats.prof_launches (both reset by this call).  SWM_K_NONE stops.
 * The events cost a few microseconds of device time per launch of that class only. */
int swm_profile(swm_ctx* ctx, int kernel_class);

/* Kept block pattern of the last build (Eq. neardef) as nb x 2 int64 (p, q) pairs in the
 * caller's wire numbering, host memory of at least 2 * stats.nb entries, rows sorted by p then q. */
int swm_get_pattern(swm_ctx* ctx, int64_t* pairs_out);

/* Block Z_pq (caller's wire numbering) as m_p x m_q complex128, row-major, interleaved re/im,
 * host memory.  SWM_EINVAL if the block was not kept. */
int swm_get_block(swm_ctx* ctx, int64_t p, int64_t q, double* re_im_out);

/* Right-hand sides b of the last solve, n_inc x N complex128 as in swm_solve, host memory. */
int swm_get_rhs(swm_ctx* ctx, double* re_im_out);

/* Stateless far-field RCS of given currents (Sec. III-A), all pointers device memory:
 *   centres, dirs (nw x 3), lengths (nw), nseg (nw) as in swm_set_cloud; off (nw + 1) int64
 *   unknown offsets off_p (off_0 = 0, off_{p+1} = off_p + nseg_p - 1);
 *   currents n_rhs x N complex128 (interleaved); obs n_obs x 2 (theta, phi);
 *   sigma_out n_rhs x n_obs x 2 float64 (theta- and phi-received).
 * SWM_EINVAL if any pointer is not device (or managed) memory.
 * Runs on `cuda_stream` and returns when sigma_out is complete.  Allocates device scratch of
 * about 48 * n_rhs * n_obs * ceil(nw / 256) bytes with cudaMallocAsync and frees it before
 * returning.  Error text (if any) is returned by swm_stateless_error(). */
int swm_far_field(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                  const double* lengths, const int32_t* nseg, const int64_t* off, double k,
                  int n_rhs, const double* currents, int n_obs, const double* obs,
                  double* sigma_out);

/* Allocation-free twin of swm_far_field; the paper has no counterpart (it is a service to
 * callers, not a step of the method).  Same arguments, same results (to rounding: the wire
 * range may be cut into fewer chunks).
 *
 * Who needs it: callers that cannot allocate device memory at the moment they ask for the RCS --
 * a process whose device memory is entirely reserved by another framework's memory pool, a
 * latency-critical loop that cannot afford an allocation or the synchronisation an allocation
 * may bring, or a host that forbids dynamic allocation after start-up.  This entry point makes
 * no cudaMalloc/cudaFree (or any other allocating) call.  Instead its scratch (the per-chunk
 * partial sums) is a fixed 8 MiB array compiled into the library; every GPU that loads the
 * library holds those 8 MiB until the process exits.
 *
 * Limits and rules:
 *   - n_rhs * n_obs <= 174762 (48 bytes of scratch per incidence-observation pair); larger
 *     requests return SWM_EINVAL with the sizes in swm_stateless_error().
 *   - The stream's device must be the current device, in its primary context (the runtime's
 *     default): the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for later calls.
 *   - Every call reads the unknown count off[nw] back to the host and synchronises its stream
 *     before returning, so a call cannot be captured into a CUDA graph.
 *   - Every array must be device memory (SWM_EINVAL otherwise), as for swm_far_field.
 *   - All calls share the one array, and it keeps the last call's contents.  Each call writes
 *     every partial sum it later reads, so nothing has to start at zero; but calls that can
 *     overlap on the GPU (other streams, other host threads) race on the array and must be
 *     serialised by the caller. */
int swm_far_field_noalloc(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                          const double* lengths, const int32_t* nseg, const int64_t* off, double k,
                          int n_rhs, const double* currents, int n_obs, const double* obs,
                          double* sigma_out);

/* Received far-field components of given currents (Sec. III-A), same arguments as swm_far_field
 * but comp_out receives n_rhs x n_obs x 2 complex128 (interleaved re, im): theta_hat . F and
 * phi_hat . F at each observation, F the radiation vector of the currents, so that
 * sigma = |component|^2 / (4 pi).  The components add over disjoint sets of wires: a cloud split
 * over ranks sums them (one all-reduce) and forms sigma afterwards.  Device memory only
 * (SWM_EINVAL otherwise); scratch as swm_far_field. */
int swm_far_components(void* cuda_stream, int64_t nw, const double* centres, const double* dirs,
                       const double* lengths, const int32_t* nseg, const int64_t* off, double k, int n_rhs,
                       const double* currents, int n_obs, const double* obs, double* comp_out);

/* Building blocks of a Krylov solve driven from outside the library on a cloud split over ranks
 * (Sec. II-B: the S-NFC system couples only wires within r_c, so a rank holding its own wires and
 * the wires within r_c of them -- its halo -- has everything its rows need).  All vectors are
 * n_rhs x N complex128 (interleaved re, im), N the context's unknowns, the caller's unknown order.
 * Each call needs a built context, runs on the context's stream, computes in float64 arithmetic
 * with the stored values, and returns when its output is complete.
 *
 * swm_apply: y = A x with A = Z M^-1 = I + E (E = Z blockdiag(Z_pp)^-1 as stored by swm_build),
 *   the operator of the right-preconditioned iteration; every row of the context (a halo wire's
 *   rows lack the couplings outside the context and are to be discarded by the caller).
 *   x and y of kinds x_kind / y_kind (SWM_HOST or SWM_DEVICE).
 * swm_precond_apply: x = M^-1 y = blockdiag(Z_pp)^-1 y, wire by wire (the block-diagonal
 *   preconditioner named after Eq. neardef).
 * swm_rhs: the right-hand sides b (Eq. (4)) of n_inc incidences (host list as in swm_solve). */
int swm_apply(swm_ctx* ctx, int n_rhs, const double* x, int x_kind, double* y, int y_kind);
int swm_precond_apply(swm_ctx* ctx, int n_rhs, const double* y, int y_kind, double* x, int x_kind);
int swm_rhs(swm_ctx* ctx, int n_inc, const double* inc, double* b_out, int out_kind);

/* Vector algebra of classical Gram-Schmidt on device vectors (no counterpart in the paper; the
 * paper's Krylov solver needs it, Sec. II-B).  Q is k or more vectors of n_rhs x n complex128,
 * contiguous (vector i at Q + 2 i n_rhs n doubles); v, out n_rhs x n.  Device memory only
 * (SWM_EINVAL otherwise); k * n_rhs <= 65535.
 * swm_vec_dots: out[i][r] = sum_n conj(Q[i][r][n]) v[r][n], k x n_rhs complex128 to host memory
 *   (partial sums over chunks of rows added in a fixed order).
 * swm_vec_axpy: v[r] -= sum over i < k of coef[i][r] Q[i][r], coef k x n_rhs complex128 (host).
 * swm_vec_scale: out[r] = a[r] v[r], a n_rhs float64 (host). */
int swm_vec_dots(swm_ctx* ctx, int64_t n, int k, int n_rhs, const double* Q, const double* v, double* out);
int swm_vec_axpy(swm_ctx* ctx, int64_t n, int k, int n_rhs, const double* Q, const double* coef, double* v);
int swm_vec_scale(swm_ctx* ctx, int64_t n, int n_rhs, const double* a, const double* v, double* out);

/* Block forms of the same algebra, for block GMRES (one Krylov space shared by S right-hand
 * sides): Q is K vectors of length n (contiguous, vector a at Q + 2 a n doubles), W is S vectors.
 * swm_vec_gram: out[a][b] = sum_n conj(Q[a][n]) W[b][n], K x S complex128 to host memory (partial
 *   sums over chunks of 2048 rows added in a fixed order, float64 throughout).
 * swm_vec_gemm: W[b] -= sum over a < K of Q[a] C[a][b], C K x S complex128 (host).
 * Device memory only (SWM_EINVAL otherwise). */
int swm_vec_gram(swm_ctx* ctx, int64_t n, int K, int S, const double* Q, const double* W, double* out);
int swm_vec_gemm(swm_ctx* ctx, int64_t n, int K, int S, const double* Q, const double* C, double* W);

/* Message of the last failed stateless call on this host thread ("" if none). */
const char* swm_stateless_error(void);

/* Library version string. */
const char* swm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWM_H */
