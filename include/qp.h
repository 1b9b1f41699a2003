/*
 * qp.h -- C ABI of libqpgpu: batched, differentiable FP32 interior-point QP
 * solver with implicit complementarity, for one NVIDIA GB300 (sm_103a).
 *
 * Method: "A Differentiable Interior-Point Method in Single Precision".
 *   Problem (eq. 1):  minimise 1/2 x'Qx + q'x  subject to  A x = b,  G x <= h.
 *   Complementarity is kept on the manifold z .* s = kappa by the softplus
 *   retraction z = b_k(v), s = b_k(-v) (eq. 9-11, App. C); each Newton step
 *   solves eq. 14 by a two-level elimination that keeps every pivot bounded:
 *   rows with W = B_k(v)/B_k(-v) <= tau are eliminated into
 *   K_I = Q + G_I' W_I G_I, the others stay as scaled multipliers beside the
 *   equality rows; K_I and the Schur complement C = D + Y Y' (Y = F L^-T,
 *   F = [G_A; A]) are Cholesky-factored in FP32.  The predictor and
 *   corrector share that factorisation, eq. 7 gives the step length, and the
 *   iterate is retracted (Alg. 1).  Gradients follow Alg. 2 (relax to
 *   kappa_relax) and Alg. 3 (implicit-function-theorem adjoint with the
 *   cached factors).
 *
 * Letters: n variables, n_eq equality rows (A, b), n_ineq inequality rows
 * (G, h).  (The paper writes m for the equality count and p for the
 * inequality count.)
 *
 * Conventions for every call:
 *   - All matrix/vector arguments are FP32 DEVICE pointers owned by the caller,
 *     batch-major and row-major per instance, packed (no padding):
 *       Q[B][n][n] (symmetric, both triangles stored), q[B][n], A[B][n_eq][n],
 *       b[B][n_eq], G[B][n_ineq][n], h[B][n_ineq]; x[B][n], y[B][n_eq],
 *       z[B][n_ineq], s[B][n_ineq]; status[B], iters[B] int32; kkt_res[B].
 *     Gradient outputs have the shapes of the data they differentiate.
 *     Every pointer must be 4-byte aligned; pointers for empty blocks may be NULL.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     enqueue work and return; nothing synchronises except create/destroy.
 *   - Return value: QP_OK or a negative QP_E* code.  Argument errors are
 *     detected on the host before anything is enqueued.  Per-instance
 *     outcomes are written to status[] on the device.
 *   - A handle holds launch configuration for one problem size.  Sizes that
 *     fit one SM's shared memory need no other device memory, so one handle
 *     may serve several streams at once.  Larger sizes (up to n = 256) run a
 *     variant whose matrices live in a device workspace the handle owns
 *     (qp_workspace_bytes); calls through such a handle must not overlap.
 *     The factor cache that the backward pass reuses is caller-owned device
 *     memory (qp_grad_cache_bytes), which keeps each forward/backward pair
 *     independent of any other.
 */
#ifndef QPGPU_QP_H
#define QPGPU_QP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes (API level) ------------------------------------------ */
#define QP_OK 0
#define QP_PENDING 1      /* serving: result not ready yet                    */
#define QP_EINVAL (-1)    /* bad argument (sizes, NULL pointer, alignment)     */
#define QP_ENOMEM (-2)    /* device allocation failed                          */
#define QP_ECUDA (-3)     /* a CUDA runtime call failed                        */
#define QP_EAGAIN (-4)    /* serving: not admissible now, retry later          */
#define QP_ETIMEOUT (-5)  /* serving: a bounded wait ran out                   */
#define QP_ENOTSUP (-6)   /* size or option not supported by this build        */
#define QP_ESTATE (-7)    /* call out of order (e.g. backward before solve)    */

/* ---- per-instance status ------------------------------------------------- */
#define QP_SOLVED 0       /* residual measure below tol (and relax converged)  */
#define QP_MAX_ITER 1     /* max_iter reached                                  */
#define QP_STALLED 2      /* residual measure stopped decreasing               */
#define QP_NUMERICAL 3    /* non-finite value or non-positive Cholesky pivot   */
#define QP_BAD_INPUT 4    /* non-finite problem data                           */

/* ---- options --------------------------------------------------------------- */
#define QP_IMPLICIT 0     /* the paper's implicit complementarity (eq. 9-14)   */
#define QP_STANDARD 1     /* explicit z .* s = kappa, Mehrotra (eq. 6, 8), through
                             the bounded two-level factorisation of QP_IMPLICIT   */
#define QP_STANDARD_SCHUR 2 /* explicit z .* s = kappa, Mehrotra, with eq. 8's
                             partially condensed matrix Q + G' diag(z ./ s) G
                             Cholesky-factored in FP32 as it stands (equality rows
                             by their Schur complement A K^-1 A', no shift, no
                             retry): the standard method the paper compares with;
                             a failed pivot ends the instance as QP_NUMERICAL   */
#define QP_SIGMA_MEHROTRA 0 /* sigma = (mu_aff / kappa)^3 clipped to [0, 1]    */
#define QP_SIGMA_CONSTANT 1 /* sigma = settings.sigma                          */
#define QP_NORM_SCALED 0  /* scaled infinity-norm residual measure             */
#define QP_NORM_ABS 1     /* absolute infinity norms (Alg. 1 as printed)       */
#define QP_GWG_FP32 0     /* K = Q + G'WG formed in FP32                       */
#define QP_GWG_TF32 1     /* G'WG on tensor cores, TF32 inputs, FP32 accumulate */
#define QP_GWG_BF16 2     /* G'WG on tensor cores, BF16 inputs, FP32 accumulate */

/* ---- per-instance diagnostics (qp_handle_set_diag) ------------------------ */
/* bits 0-7: the first stage of the iteration at which a non-finite value (or a
 * failed Cholesky pivot) appeared, in the order of the paper's NaN trace of
 * the standard method (App. D, Table 1); 0 if none. */
#define QP_STAGE_MASK 0xff
#define QP_STAGE_NONE 0
#define QP_STAGE_SCALING 1    /* the Newton matrix's diagonal W = z ./ s (or B_+/B_-) */
#define QP_STAGE_PREDICTOR 2  /* the affine (predictor) solve, its factorisation included */
#define QP_STAGE_CENTERING 3  /* alpha_aff, mu_aff, sigma                              */
#define QP_STAGE_CORRECTOR 4  /* the corrector direction (dx, ds, dz, dy)              */
#define QP_STAGE_LINESEARCH 5 /* the step length alpha and the updated iterate         */
#define QP_STAGE_RELAX 6      /* anywhere in Alg. 2 or the factorisation cached for Alg. 3 */
#define QP_STAGE_BACKWARD 7   /* the adjoint solve of Alg. 3 (qp_backward_batch)       */
#define QP_STAGE_INIT 8       /* the starting point                                    */
#define QP_DIAG_FACTOR_FAILED 0x100  /* a Cholesky pivot was not positive              */
#define QP_DIAG_TC_FALLBACK 0x200    /* tensor-core G'WG ran out of a bounded wait and
                                        the solve continued with FP32 products          */
#define QP_DIAG_STAGE_FALLBACK 0x400 /* bulk-copy staging (of G'WG, or of a back
                                        substitution's factor blocks) ran out of a bounded
                                        wait; that step was finished from global memory   */
#define QP_DIAG_ASYNC_LOST 0x800     /* copies may have been in flight after a bounded
                                        wait: the instance is reported QP_NUMERICAL     */

typedef struct {
  int32_t batch;  /* number of independent QPs (>= 0)        */
  int32_t n;      /* variables (>= 1)                        */
  int32_t n_eq;   /* equality rows (0 <= n_eq <= n)          */
  int32_t n_ineq; /* inequality rows (>= 0)                  */
} qp_dims;

typedef struct {
  float tol;            /* stop when the residual measure < tol (Alg. 1)            */
  int32_t max_iter;     /* Newton iterations of the solve (Alg. 1; paper: 100)      */
  int32_t sigma_mode;   /* QP_SIGMA_*                                               */
  float sigma;          /* constant sigma (QP_SIGMA_CONSTANT)                       */
  float kappa_min;      /* floor on kappa_target (0: 1e-2 * tol)                    */
  float kappa_relax;    /* central-path parameter of the gradients (Alg. 2); 0:
                           gradients at the solution itself                         */
  float relax_tol;      /* Alg. 2 stop tolerance (0: tol / 10); a relaxed measure
                           below tol that has stopped decreasing for 3 iterations
                           (the FP32 floor) also ends the relax                     */
  int32_t relax_max_iter; /* Alg. 2 iteration cap (0: max_iter)                     */
  int32_t formulation;  /* QP_IMPLICIT, QP_STANDARD or QP_STANDARD_SCHUR             */
  int32_t residual_norm; /* QP_NORM_*                                               */
  int32_t gwg_precision; /* QP_GWG_*: TF32 / BF16 put the G'WG products on the tensor
                            cores (FP32 sums) in the large-problem variant; sizes that
                            run on chip accept only QP_GWG_FP32 (QP_ENOTSUP); the
                            server applies it to large-variant requests only         */
  int32_t refine_steps;  /* iterative-refinement sweeps of the adjoint solve of
                            Alg. 3 against the bounded system (default 3)           */
  int32_t warm_start;    /* 1: start from the x, y, z, s passed in (z, s > 0)       */
  int32_t relax_chord;   /* 1: Alg. 2 factors its first iterate only and reuses that
                            factorisation for the following Newton steps (chord
                            steps; Alg. 2's "if not cached"); its polishing step and
                            the factor cached for Alg. 3 are fresh.  0: refactor at
                            every relax iterate (default)                            */
  int32_t refine_forward; /* iterative-refinement sweeps of each Newton solve of Alg. 1
                            and Alg. 2 in the large-problem variant: the residual of
                            the bounded eq. 14 system is formed in FP32 from Q, G, A
                            (no tensor-core products) and corrected with the same
                            factors -- recovers the accuracy of TF32 / BF16 G'WG
                            (default 0; sizes that run on chip ignore it)             */
} qp_settings;

typedef struct qp_handle qp_handle;

/* Fill `s` with the defaults: tol 1e-5, max_iter 100, Mehrotra sigma,
 * sigma 0.1, kappa_min 0 (-> 1e-2 tol), kappa_relax 1e-4, relax_tol 0
 * (-> tol / 10), relax_max_iter 0, implicit, scaled norm, FP32 G'WG, 3
 * refinement sweeps of the adjoint solve, cold start, relax refactors every
 * iterate, no refinement of the forward Newton solves.  (Defaults follow the paper's ablation settings where it states
 * them: max_iter 100, kappa_relax 1e-4.) */
void qp_settings_default(qp_settings* s);

/* Create a solver handle for batches of the given size on the current
 * device.  Allocates device memory only for sizes beyond one SM's shared
 * memory: the workspace of qp_workspace_bytes.  Supported: n <= 256.
 * Returns QP_EINVAL (bad dims), QP_ENOTSUP (size too large for this build),
 * QP_ENOMEM (workspace allocation failed) or QP_ECUDA. */
int qp_handle_create(const qp_dims* dims, qp_handle** out);

/* As qp_handle_create, with the threads per QP of the forward kernel chosen
 * by the caller: 0 automatic (as qp_handle_create: one warp per QP for
 * n <= 32 in batches of 2048 or more, else 128 up to n = 72, else 512), 32
 * (one warp per QP; n <= 32), 128 (n <= 72), 256 (n > 128: two CTAs of the
 * large-problem variant per SM) or 512 (any n: the width the persistent
 * server of qp_serve_create runs every size at, so that a served request
 * equals a batch-1 solve of this width bit for bit).  Sizes whose data do
 * not fit one SM's shared memory at the requested width, and other widths,
 * return QP_ENOTSUP.  Results are the same up to FP32 rounding order. */
int qp_handle_create_threads(const qp_dims* dims, int32_t threads_per_qp, qp_handle** out);

/* Free the handle and its workspace, if any. */
int qp_handle_destroy(qp_handle* h);

/* Launch configuration a handle chose (capacity planning, tests).  Problems
 * with n <= 32 in batches of 2048 or more run one warp (32 threads) per QP,
 * so that many QPs share an SM; other sizes up to n = 72 use 128 threads per
 * QP, larger ones 512. */
typedef struct {
  int32_t fwd_threads;        /* threads per CTA (one CTA per QP) of the forward kernel */
  int32_t fwd_blocks_per_sm;  /* resident forward CTAs per SM                          */
  int32_t bwd_threads;        /* threads per CTA of the backward kernel                 */
  int32_t max_active;         /* amax: inequality rows kept as multipliers at most      */
  int32_t large_variant;      /* 1: matrices in the handle's device workspace           */
  size_t fwd_smem_bytes;      /* dynamic shared memory per forward CTA                  */
} qp_handle_info;

/* Fill `out`.  Returns QP_EINVAL for a null argument. */
int qp_handle_query(const qp_handle* h, qp_handle_info* out);

/* Register a caller-owned DEVICE array diag[batch] (int32, 4-byte aligned)
 * that later qp_solve_batch / qp_backward_batch calls through this handle
 * fill with one diagnostics word per instance (QP_STAGE_* in bits 0-7, the
 * first stage with a non-finite value; QP_DIAG_* flags above them).  The
 * solve writes every word; the backward pass adds QP_STAGE_BACKWARD to words
 * whose stage is still QP_STAGE_NONE when its adjoint solution is not finite
 * or the instance's cache slot cannot be used (NaN gradients).
 * With an array registered the solve also tests each stage's values for
 * finiteness (a few block reductions per iteration); NULL (the default)
 * turns both off.  Returns QP_EINVAL for a null handle or a misaligned
 * pointer. */
int qp_handle_set_diag(qp_handle* h, int32_t* diag);

/* Solve + relax + backward of a batch held in HOST memory: the library copies
 * the data in, runs the kernels and copies the results out, in chunks of
 * about a quarter of the batch (whole waves of resident CTAs) on two
 * streams of its own, so that a chunk's
 * copies overlap the kernels of its neighbours (with page-locked host memory;
 * pageable memory works but serialises the copies).  Blocks until done.
 * Arrays and layouts as qp_solve_batch / qp_backward_batch, all in host
 * memory.  dl_dx NULL: solve only (no relax, no gradients; dQ..dh ignored).
 * y, status, iters, kkt_res and the gradient outputs may be NULL (not
 * copied back).  The first call allocates the handle's device arena for two
 * chunks (inputs, outputs, gradient cache) and the two streams; they are
 * kept until qp_handle_destroy.  Calls through one handle must not overlap.
 * Returns QP_EINVAL / QP_ENOTSUP as qp_solve_batch, QP_ENOMEM, QP_ECUDA. */
int qp_solve_backward_host(qp_handle* h, const qp_settings* settings, const float* Q,
                           const float* q, const float* A, const float* b, const float* G,
                           const float* h_, const float* dl_dx, float* x, float* y, float* z,
                           float* s, int32_t* status, int32_t* iters, float* kkt_res, float* dQ,
                           float* dq, float* dA, float* db, float* dG, float* dh);

/* Bytes of device memory the gradient cache of one solve needs: per
 * instance a header, the Cholesky factor L of K_I = Q + G_I'W_I G_I (packed
 * lower; unpacked for the large-problem variant), Y = F L^-T with
 * F = [G_A; A] (nf = active rows + n_eq rows), the factor of
 * C = D + Y Y' (packed lower; unpacked for the large variant), W (or 1/W),
 * the active-row map, the relaxed point (x, y, z) and one more m-block (the
 * solve keeps the iterate the relax starts from in this slot), each block
 * padded to 16 bytes. */
size_t qp_grad_cache_bytes(const qp_dims* dims);

/* Per-instance shared memory the solve kernel uses, in bytes (0 if the
 * size is unsupported); for capacity planning. */
size_t qp_smem_bytes(int32_t n, int32_t n_eq, int32_t n_ineq);

/* Bytes of device workspace a handle of these dims allocates: 0 when the
 * problem fits one SM's shared memory, else batch x (K, G, A, Y, C of one
 * instance) for the large-problem variant. */
size_t qp_workspace_bytes(const qp_dims* dims);

/* Solve the batch (Alg. 1).  If grad_cache is not NULL (device memory of
 * qp_grad_cache_bytes, 16-byte aligned), also relax each solution to
 * settings->kappa_relax (Alg. 2; kappa_relax = 0 keeps the solution itself),
 * factor the Newton matrix at that point and store the factor, W and the
 * point in grad_cache for qp_backward_batch (Alg. 3).  x, y, z, s receive
 * the solution of Alg. 1 (not the relaxed point); with settings->warm_start
 * they are also read as the starting point.  status/iters/kkt_res may be
 * NULL.  iters counts all Newton iterations (solve + relax); kkt_res is the
 * FP32 residual measure at the returned point.  Instances whose data are
 * not finite get status QP_BAD_INPUT and NaN outputs. */
int qp_solve_batch(qp_handle* h, const qp_settings* settings, const float* Q, const float* q,
                   const float* A, const float* b, const float* G, const float* h_,
                   float* x, float* y, float* z, float* s, int32_t* status, int32_t* iters,
                   float* kkt_res, float* grad_cache, void* stream);

/* Vector-Jacobian product (Alg. 3) of the solve that filled grad_cache:
 * given dl_dx[B][n], writes the gradients of <dl_dx, x(kappa_relax)> with
 * respect to Q (symmetrised, (dx x' + x dx')/2), q, A, b, G and h.  Q, A and
 * G must be the data passed to that solve: the adjoint solve is refined
 * against the Newton system built from them.  Any gradient pointer may be
 * NULL to skip that block.  A cache not written by a solve of this size
 * gives NaN gradients (never an out-of-bounds access); the result is
 * undefined if the cache belongs to a different batch of the same size. */
int qp_backward_batch(qp_handle* h, const float* grad_cache, const float* Q, const float* A,
                      const float* G, const float* dl_dx, float* dQ, float* dq, float* dA,
                      float* db, float* dG, float* dh, void* stream);

/* ---- fixed-scratch variant (an addition of this library; the paper has no
 *      counterpart) -------------------------------------------------------- */

/* Size of the library's fixed device array that holds the factor cache of
 * qp_solve_backward_static: 16 MiB per device (for example 637 instances of
 * n = 50, n_eq = 10, n_ineq = 100; compare qp_grad_cache_bytes). */
#define QP_STATIC_CACHE_BYTES (16 * 1024 * 1024)

/* qp_solve_batch followed by qp_backward_batch, with the factor cache between
 * them held in a fixed device array of the library instead of caller memory,
 * so that the call allocates no memory of any kind.  For callers that cannot
 * supply the cache on the call path: a fixed-rate loop that must not call
 * cudaMalloc there (an allocation can synchronise the device and stall), or a
 * program whose device memory belongs to an arena not lent to libraries.
 * Arguments, outputs and per-instance status are those of the two calls
 * (dl_dx[B][n] is required; gradient pointers may be NULL); instances with
 * non-finite data get NaN gradients.
 * Limit: returns QP_ENOTSUP, with nothing enqueued, when
 * qp_grad_cache_bytes(dims) > QP_STATIC_CACHE_BYTES.  Other argument errors
 * return QP_EINVAL before anything that touches caller memory is enqueued.
 * Every call looks up the array's device address in the current context (so
 * a context that was destroyed and recreated gets the new address); the
 * first call in a context can load the library's device code there, which
 * is when the array is reserved: make that first call before any stream
 * capture is begun.
 * Sharing: every call on a device uses the same array, so calls whose device
 * work can overlap (different streams, unsynchronised host threads) race on
 * it and give undefined results; calls ordered on one stream are safe. */
int qp_solve_backward_static(qp_handle* h, const qp_settings* settings, const float* Q,
                             const float* q, const float* A, const float* b, const float* G,
                             const float* h_, const float* dl_dx, float* x, float* y, float* z,
                             float* s, int32_t* status, int32_t* iters, float* kkt_res,
                             float* dQ, float* dq, float* dA, float* db, float* dG, float* dh,
                             void* stream);

/* ---- serving: continuous batching of single requests ------------------- */

/* A server owns a device arena, a pinned host mirror of it and a scheduler
 * thread; requests of any supported size are submitted one at a time and
 * admitted while their footprint (qp_serve_footprint_bytes) fits the arena.
 * Each request is solved (Alg. 1; with want_grad also relaxed and
 * differentiated, Alg. 2-3) by one CTA.  Two modes:
 *
 * QP_SERVE_LAUNCHES: the scheduler groups waiting requests into launches (the
 * oldest request first, requests of its kernel class in arrival order, up to
 * max_batch and up to the free arena memory) and keeps up to max_inflight
 * launches on the GPU at once, one stream each, so requests that arrive while
 * others run start as soon as a stream and memory free up; a kernel class
 * takes the last free stream only while it has fewer than
 * max(1, max_inflight / 3) launches in flight.  A request's arithmetic is
 * that of qp_solve_batch of its size: results equal solo results bit for bit.
 *
 * QP_SERVE_PERSISTENT: one resident 512-thread CTA per SM loops over a ring of
 * request descriptors that the scheduler publishes in mapped host memory as
 * soon as a request's data are on the device; a free CTA claims the next
 * request while the others are in the middle of theirs, keeps its iterate
 * and factors on the device, runs Alg. 3 for it on 128 or 256 of its threads
 * and writes the outputs straight to mapped host memory.  Every size runs at
 * 512 threads (qp_handle_create_threads(dims, 512)): results equal those of a
 * batch-1 solve of that width and qp_backward_batch bit for bit.  A CTA with
 * no request for idle_ms leaves (the scheduler starts CTAs again when work
 * arrives); while CTAs are resident they hold every SM, so no other kernel of
 * the process runs beside them.  Needs host-native atomics (NVLink-C2C
 * systems); QP_ENOTSUP otherwise.
 *
 * Every wait, on the host and on the device, is bounded. */
typedef struct qp_server qp_server;

#define QP_SERVE_LAUNCHES 0
#define QP_SERVE_PERSISTENT 1

typedef struct {
  size_t hbm_budget_bytes; /* device arena for resident requests (>= 1 MiB)     */
  int32_t max_inflight;    /* launches: launches on the GPU at once, one stream
                              each (1-64)                                         */
  int32_t max_batch;       /* launches: requests per launch                       */
  int32_t max_queue;       /* requests waiting on the host before QP_EAGAIN       */
  qp_settings settings;    /* solver settings of every request (no warm start)    */
  int32_t mode;            /* QP_SERVE_LAUNCHES or QP_SERVE_PERSISTENT            */
  int32_t idle_ms;         /* persistent: a CTA with no request for this long
                              leaves its loop (1-10000)                           */
} qp_serve_config;

typedef struct {
  int32_t n, n_eq, n_ineq; /* sizes of this request                             */
  int32_t want_grad;       /* 1: relax and return the gradients of <dl_dx, x>    */
  /* HOST inputs, copied during qp_serve_submit (layout as qp_solve_batch, one
   * instance); dl_dx[n] when want_grad */
  const float *Q, *q, *A, *b, *G, *h, *dl_dx;
  /* HOST outputs, written by the qp_serve_poll* / qp_serve_wait call that
   * returns this request; each may be NULL; they must stay valid until then */
  float *x, *y, *z, *s;
  float *dQ, *dq, *dA, *db, *dG, *dh;
} qp_request;

typedef struct {
  uint64_t ticket;
  int32_t status;          /* per-instance status (QP_SOLVED, ...)               */
  int32_t iters;
  float kkt_res;
  double t_submit_ms;      /* server clock (ms since qp_serve_create): submitted */
  double t_launch_ms;      /* its launch was issued (persistent: its descriptor
                              was published to the resident CTAs)               */
  double t_done_ms;        /* its results reached host memory (as the scheduler
                              saw them)                                          */
} qp_result;

/* Defaults: 1 GiB arena, 8 launches in flight, 1024 requests per launch,
 * 2^20 queued requests, qp_settings_default, QP_SERVE_PERSISTENT, idle 50 ms. */
void qp_serve_config_default(qp_serve_config* c);

/* Arena bytes one request occupies while resident (data, outputs, gradient
 * outputs and factor cache when want_grad, workspace of the large variant);
 * 0 if the size is unsupported.  The admission unit of the server. */
size_t qp_serve_footprint_bytes(int32_t n, int32_t n_eq, int32_t n_ineq, int32_t want_grad);

/* Allocate the arena and mirror, create the streams and start the scheduler on
 * the current device.  QP_EINVAL (bad config), QP_ENOMEM, QP_ECUDA. */
int qp_serve_create(const qp_serve_config* cfg, qp_server** out);

/* Queue one request (non-blocking: its inputs are copied, the GPU work is
 * issued by the scheduler).  QP_OK with *ticket; QP_EAGAIN if max_queue
 * requests are waiting; QP_ENOTSUP if the size is unsupported or larger than
 * the arena; QP_EINVAL for bad arguments; QP_ECUDA after a device error. */
int qp_serve_submit(qp_server* s, const qp_request* r, uint64_t* ticket);

/* QP_PENDING while the request is queued or running; otherwise writes its
 * outputs, fills *res, retires the ticket and returns QP_OK, or QP_ECUDA when
 * a device error failed its launch (after such an error every request still
 * queued fails the same way, and new submissions return QP_ECUDA).
 * QP_EINVAL for an unknown ticket. */
int qp_serve_poll(qp_server* s, uint64_t ticket, qp_result* res);

/* As qp_serve_poll for the earliest completed request not yet collected;
 * QP_PENDING if none has completed. */
int qp_serve_poll_any(qp_server* s, qp_result* res);

/* Wait at most timeout_ms for the request, then as qp_serve_poll;
 * QP_ETIMEOUT if it has not completed by then. */
int qp_serve_wait(qp_server* s, uint64_t ticket, int32_t timeout_ms, qp_result* res);

/* Stop the scheduler, drain the streams and free everything; tickets not yet
 * collected are dropped. */
int qp_serve_destroy(qp_server* s);

/* Human-readable name of a return or status code. */
const char* qp_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* QPGPU_QP_H */
