/*
 * cluster.h — C ABI of the B300 fuzzy-clustering library (libcluster.so).
 *
 * The library minimises f(U) = ||S - U U^T||_F^2 over row-stochastic
 * membership matrices U (n x k, every row on the probability simplex), the
 * model (P) of arXiv 2506.04045 Sect. 2 written with U = X^T (the paper's X is
 * C x N with columns on the simplex; here n = N articles, k = C clusters).
 * S is a sparse symmetric similarity matrix given in CSR form.  The solver is
 * the paper's parallel FISTA (Algorithm 4) or plain projected gradient
 * (Algorithm 3, momentum off), one fused GPU pass per iteration.
 *
 * Conventions shared by every entry point:
 *  - Pointers marked "device" must be CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns a cluster_status.  Nothing aborts the process; on an
 *    error the call leaves its outputs unspecified and cluster_last_error()
 *    returns a message for the calling thread.
 *  - The caller owns every buffer it passes in; the library owns every
 *    object it returns (free them with the matching destroy/free call).
 *  - Layouts: U, U0 and U_out are n x k row-major float32 (row i = article
 *    i's memberships, stride k).  CSR columns must be sorted and unique within
 *    each row.
 */
#ifndef CLUSTER_H_
#define CLUSTER_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CLUSTER_API __attribute__((visibility("default")))
#else
#define CLUSTER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status codes                                                              */
/* ------------------------------------------------------------------------ */
typedef enum cluster_status {
  CLUSTER_OK = 0,
  CLUSTER_EINVAL = 1,      /* bad argument or input that fails validation      */
  CLUSTER_ENOMEM = 2,      /* device or host allocation failed                 */
  CLUSTER_ECUDA = 3,       /* a CUDA runtime call failed                       */
  CLUSTER_ENONFINITE = 4,  /* NaN/Inf appeared in the iterate (report status)  */
  CLUSTER_EMAXITER = 5,    /* report status: max_iter reached before a stop    */
  CLUSTER_ETIMEOUT = 6,    /* a bounded wait gave up                           */
  CLUSTER_EAGAIN = 7       /* server: the request is still pending             */
} cluster_status;

/* Arithmetic of the fused pass.  FP32: float32 iterate, products with S and
 * Gram matrices accumulated in float32, objective/trace/norm reductions in
 * float64.  MIXED_BF16: the copy of the iterate that the product S*U gathers
 * and the values of S are bfloat16 (round to nearest even); a float32 master
 * iterate is kept for the row-local update; accumulations as in FP32. */
typedef enum cluster_precision {
  CLUSTER_FP32 = 0,
  CLUSTER_MIXED_BF16 = 1
} cluster_precision;

/* Step size tau.  Theorem 2.1 gives convergence of plain projected gradient
 * for tau < 1/L with L = 4 ||S||_2 + 12 n; the experiments (Sect. 5,
 * "Hyperparameters") replace ||S||_2 by ||S||_F.  For the two 1/L rules
 * options.tau is a multiplier on 1/L (0 means 1). */
typedef enum cluster_step_rule {
  CLUSTER_STEP_CONST = 0,       /* tau = options.tau                          */
  CLUSTER_STEP_INV_L_FROB = 1,  /* tau = options.tau / (4 ||S||_F + 12 n)     */
  CLUSTER_STEP_INV_L_SPEC = 2   /* tau = options.tau / (4 ||S||_2 + 12 n),
                                   ||S||_2 by power iteration on the GPU     */
} cluster_step_rule;

/* Stopping rule.  LOSS is the paper's: stop at iteration n once
 * f(Xbar^{n-1}) - f(Xbar^n) <= tol (Algorithm 4 and the prose after it; the
 * output is Xbar^n).  The PG rules use r_n = ||Y^n - Xbar^n||_F / tau, the
 * gradient mapping at the extrapolated point: PG_REL stops once
 * r_n <= tol * r_1, PG_ABS once r_n <= tol (output Xbar^n).  NONE runs
 * max_iter iterations. */
typedef enum cluster_stop_rule {
  CLUSTER_STOP_LOSS = 0,
  CLUSTER_STOP_PG_REL = 1,
  CLUSTER_STOP_PG_ABS = 2,
  CLUSTER_STOP_NONE = 3
} cluster_stop_rule;

/* Sparse symmetric similarity matrix S (n x n) in CSR form.
 * row_ptr: n+1 entries, int32 (index64 = 0) or int64 (index64 = 1),
 * row_ptr[0] = 0, row_ptr[n] = nnz; col: nnz int32 column indices, sorted
 * and unique within each row; val: nnz float32 values.  The paper's S is the
 * citation adjacency (s_ij = 1 if i cites or is cited by j) plus a unit
 * diagonal (Example 4.1); weights other than 1 are accepted. */
typedef struct cluster_csr {
  int64_t n;
  int64_t nnz;
  int32_t index64;
  int32_t _pad;
  const void* row_ptr;
  const int32_t* col;
  const float* val;
} cluster_csr;

typedef struct cluster_options {
  int32_t precision;   /* cluster_precision (default FP32)                      */
  int32_t step_rule;   /* cluster_step_rule (default INV_L_FROB)                */
  int32_t stop_rule;   /* cluster_stop_rule (default LOSS)                      */
  int32_t accel;       /* 1 = FISTA (Algorithm 4), 0 = plain GPA (default 1)    */
  int32_t borrow;      /* 1 = keep the caller's device CSR arrays (they must
                          outlive the context); 0 = copy them (default 0)      */
  int32_t validate;    /* 0 = none; 1 = CSR structure (sorted, in range, unit
                          diagonal present, finite values) and U0 rows on the
                          simplex (default); 2 = also check that S is symmetric */
  double tau;          /* see cluster_step_rule (default 1)                     */
  double tol;          /* stopping tolerance (default 0)                        */
  int64_t max_iter;    /* iteration cap, >= 1 (default 1000)                    */
  int32_t graph_chunk; /* iterations per captured CUDA graph (default 16)      */
  int32_t fused_pass;  /* 0 = split iteration (gather kernel + streaming update
                          kernel, default); 1 = one fused kernel per iteration.
                          Same arithmetic; the Gram partial order differs.      */
  int32_t relabel;     /* 1 = number the articles internally by decreasing
                          degree (default): rows of frequently gathered articles
                          then share cache lines and DRAM pages; inputs and
                          outputs keep the caller's numbering, each row's sum
                          keeps its order, only the Gram partial order differs.
                          0 = keep the caller's numbering.                      */
  int32_t l2_window;   /* 1 = with relabel, keep the gathered rows of the
                          highest-degree articles in a persisting L2 window
                          (half the device's persisting maximum; default);
                          0 = no window.  A cache hint: no value changes.       */
  int32_t update_engine; /* form of the row-local update for 17 <= k <= 64:
                          0 = automatic (default): k <= 32 streams (3) on a
                          solver of at least 2^17 articles; everything else
                          (smaller solvers, batched and served instances,
                          33 <= k <= 64) uses 1 (measured faster there);
                          1 = warp-level mma.sync, blocks of rows;
                          2 = tcgen05.mma with TMEM accumulators, the same
                          blocks, products and order as 1 (the same bits);
                          3 = streaming (k <= 32): one CTA per SM over tiles of
                          128 rows moved by TMA, one thread per row, y G on
                          tcgen05 as 3xTF32 and the Gram matrices as scaled
                          float16 splits with float-pair partials (results
                          within float32 rounding of 1 and 2, not the same
                          bits); a batch or the overlapped pass uses 2 instead.
                          k <= 16 uses mma.sync (k > 8) or float32 FMA, k > 64
                          mma.sync.                                               */
  int32_t overlap;     /* 1 = with the internal numbering and n >= 2^20, run the
                          update of each of 8 row chunks on a second stream as
                          soon as the gather has produced that chunk's rows,
                          beside the gather of the following chunks; 0 = gather,
                          then update (default: the gather slows more beside the
                          update than the overlap saves).  Such problems use 4
                          update blocks per resident block either way, so the
                          two schedules give the same bits.                     */
} cluster_options;

/* Progress of a solve.  Iteration n means the paper's Xbar^n (Xbar^0 = U0). */
typedef struct cluster_report {
  int64_t iters;       /* fused passes (gradient evaluations) executed          */
  int64_t f_iter;      /* index n of the newest iterate whose loss is known    */
  double f;            /* f(Xbar^{f_iter}) in float64, by the trace identity   */
  double trace_SU;     /* sum_i <u_i, (S U)_i> of that iterate                 */
  double gram_fro2;    /* ||U^T U||_F^2 of that iterate                        */
  double pg_norm;      /* newest r_n = ||Y^n - Xbar^n||_F / tau                 */
  double tau;          /* step size in use                                      */
  double L;            /* Lipschitz bound 4 ||S|| + 12 n of the step rule       */
  int64_t out_iter;    /* index of the iterate cluster_get_U returns            */
  int32_t done;        /* 1 once a stop rule, max_iter or a fault ended it      */
  int32_t status;      /* CLUSTER_OK (stopped by its rule / still running),
                          CLUSTER_EMAXITER, or CLUSTER_ENONFINITE              */
} cluster_report;

typedef struct cluster_ctx cluster_ctx;

/* Fill `opt` with the defaults listed in cluster_options. */
CLUSTER_API void cluster_options_default(cluster_options* opt);

/* Message describing the calling thread's most recent error ("" if none).
 * The string stays valid until the thread's next library call. */
CLUSTER_API const char* cluster_last_error(void);

/* Create a solver for S (device CSR) with k clusters (1 <= k <= 128) from
 * the start point U0 (device, n x k; every row must be on the simplex to
 * within 1e-5).  Validates the inputs (EINVAL on failure), computes ||S||_F^2
 * and the step size, numbers the articles internally by degree (opt->relabel;
 * the context then keeps its own renumbered copy of S even with borrow = 1),
 * builds the gather schedule, and evaluates the Gram matrix of U0.  The
 * context keeps its own copy of U0.  With opt->l2_window it raises the
 * context's persisting L2 limit while it lives (restored when the last such
 * solver is destroyed).  Work is enqueued on `stream`; the call returns after
 * it completes.
 * Sect. 3, Algorithm 4 "initialize"; Sect. 5 "Hyperparameters". */
CLUSTER_API cluster_status cluster_init(const cluster_csr* S, int32_t k, const float* U0,
                                        const cluster_options* opt, void* stream,
                                        cluster_ctx** out);

/* Advance by at most `iters` iterations (fewer if a stop rule fires or
 * max_iter is reached), then fill `rep` (may be NULL).  Each iteration is one
 * fused pass over S on the GPU (Algorithm 4's body with the second product
 * with S replaced by linearity); the host synchronises once per call. */
CLUSTER_API cluster_status cluster_step(cluster_ctx* ctx, int64_t iters, cluster_report* rep);

/* Enqueue `iters` iterations on the context's stream and return without
 * synchronising (no report).  For timing loops; call cluster_step(ctx, 0,
 * &rep) afterwards to synchronise and read the state. */
CLUSTER_API cluster_status cluster_enqueue(cluster_ctx* ctx, int64_t iters);

/* Per-kernel timing of the fused iteration, averaged over the launches of
 * one cluster_enqueue_profiled call (milliseconds, CUDA events on the
 * context's stream).  With the overlapped pass (cluster_options.overlap),
 * pass_ms runs from the start to the end of the last gather (hub-row sums
 * included, heavy_ms = 0) and update_ms is the part of the updates after it.
 * pass = the fused pass kernel, heavy = the kernel that
 * computes the partial products of chunked high-degree rows (0 if none),
 * fold = the float64 fold.  heavy_nnz is the number of nonzeros the heavy
 * kernel streams per iteration (the pass kernel streams nnz - heavy_nnz). */
typedef struct cluster_kernel_times {
  double pass_ms;      /* split: the gather kernel S*X; fused: the fused pass    */
  double heavy_ms;     /* split: chunk-sum kernel; fused: chunk partial kernel   */
  double fold_ms;
  double update_ms;    /* split: the streaming update kernel; fused: 0          */
  double total_ms;     /* first event to last event                            */
  int64_t launches;    /* iterations timed                                     */
  int64_t heavy_nnz;
  int64_t heavy_rows;
  int64_t kernels;     /* kernel launches of the library in the call           */
} cluster_kernel_times;

/* Run `iters` iterations launched one kernel at a time (no graph) with CUDA
 * events between the kernels, synchronise, and return the per-kernel
 * averages.  Same kernels and arithmetic as cluster_step; for measurement. */
CLUSTER_API cluster_status cluster_enqueue_profiled(cluster_ctx* ctx, int64_t iters,
                                                    cluster_kernel_times* out);

/* Iterate until the stop rule fires or max_iter is reached, then make sure
 * rep->f is the loss of the returned iterate (one extra objective pass if
 * needed).  Returns CLUSTER_OK; rep->status tells how the run ended. */
CLUSTER_API cluster_status cluster_solve(cluster_ctx* ctx, cluster_report* rep);

/* Current report without doing any work. */
CLUSTER_API cluster_status cluster_get_report(cluster_ctx* ctx, cluster_report* rep);

/* Copy the output iterate (the one rep.out_iter names) into U_out (device,
 * n x k). */
CLUSTER_API cluster_status cluster_get_U(cluster_ctx* ctx, float* U_out);

/* f(U) = ||S||_F^2 + ||U^T U||_F^2 - 2 sum_i <u_i, (S U)_i> in float64
 * (Sect. 3, "Loss Update"), for device S and U (n x k).  Allocates and frees
 * its own scratch; synchronises `stream`.  *f receives the value.  S is
 * trusted, not validated (unlike cluster_init): a column index outside [0, n)
 * or a decreasing row pointer makes the kernels read outside S's arrays. */
CLUSTER_API cluster_status cluster_objective(const cluster_csr* S, int32_t k, const float* U,
                                             void* stream, double* f);

/* The objective f(U) like cluster_objective, but without allocating any
 * memory.  The paper has no counterpart: this entry point is for callers that
 * must not call cudaMalloc at the point where they evaluate f — for instance a
 * service that gives all free device memory to its own pool at start-up, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device.  Its device scratch is one fixed array of about 2.7 MB compiled into
 * the library, which every GPU that loads the library keeps until the process
 * exits.
 * Limits (EINVAL otherwise): k in {2, 4, 8, 16, 32} (U, n x k device, is read
 * in place, 16-byte aligned; 8-byte for k = 2), S with int64 row pointers
 * (index64 = 1), n < 2^31.  Rows are split evenly over the GPU rather than
 * ordered by degree, so graphs with rows of very high degree run slower than
 * with cluster_objective.
 * The call cannot be part of a stream capture (it synchronises `stream` and
 * reads partial sums on the host): on a capturing stream it returns EINVAL
 * and enqueues nothing.  The first call on a device looks up the scratch
 * array's device address for that device (cudaGetSymbolAddress) and keeps it
 * for the life of the process; do not use the library across a
 * cudaDeviceReset (the module is reloaded and the kept address goes stale).  All calls share the one array and each call resets
 * what must start at zero, so calls that overlap on the GPU (other threads,
 * other streams) race and must be serialised by the caller.  S is trusted as
 * in cluster_objective (not validated).  The call synchronises `stream` and
 * writes the value to *f. */
CLUSTER_API cluster_status cluster_objective_static(const cluster_csr* S, int32_t k, const float* U,
                                                    void* stream, double* f);

/* Second-order check (Sect. 4, Theorem 4.1, Eq. "hessian").  In row notation
 * (U = Xbar^T, W = V^T) the Hessian of f at U applied to a direction W is
 *     H[W] = -4 S W + 4 W (U^T U) + 4 U (U^T W + W^T U).
 * The call computes, from one product S W on the device:
 *   HW         (optional) H[W], n x k row-major float32, device;
 *   curvature  (optional) <W, H[W]> in float64, host;
 *   slope      (optional) <grad f(U), W> = <-4 (S U - U U^T U), W> in float64, host.
 * A direction tangent to Omega at U has rows summing to zero (and w_ia >= 0
 * where u_ia = 0); a stationary U with a tangent W of negative curvature is
 * not a local minimum (the 0.5 J saddle of Example 4.1 has curvature -4 along
 * the direction the paper prints).  U and W are n x k row-major float32 device
 * arrays (not modified); S as for cluster_objective (symmetric).  The library
 * allocates and frees its own scratch and synchronises `stream`.  Errors:
 * EINVAL for NULL pointers or k outside [1, 128], ENOMEM, ECUDA. */
CLUSTER_API cluster_status cluster_hessian_apply(const cluster_csr* S, int32_t k, const float* U, const float* W,
                                                 void* stream, float* HW, double* curvature, double* slope);

/* Checkpoint.  The state is everything a resumed run needs to continue bit
 * for bit: the two newest iterates, the stored product S*Xbar^{n-1}, the
 * float64 Gram matrices and scalars.  cluster_state_size gives the byte size;
 * buffers are host memory. */
CLUSTER_API cluster_status cluster_state_size(cluster_ctx* ctx, size_t* bytes);
CLUSTER_API cluster_status cluster_get_state(cluster_ctx* ctx, void* host_buf, size_t bytes);
CLUSTER_API cluster_status cluster_set_state(cluster_ctx* ctx, const void* host_buf, size_t bytes);

/* Test hook for the timeout path.  flags bit 0: the tcgen05 updates (k in
 * 17..32 with update_engine 2, and the streaming update: update_engine 3, or
 * 0 on a solver of at least 2^17 articles) still issue their y G products but
 * withhold
 * the commit that signals their completion, so their bounded waits give up
 * after about one second; the run then ends with report status
 * CLUSTER_ETIMEOUT, out_iter names the last complete iterate and the context
 * stays usable (report, U, checkpoint).  flags 0 restores normal operation.
 * Synchronises the context's stream.  EINVAL for a NULL context, ECUDA. */
CLUSTER_API cluster_status cluster_test_hooks(cluster_ctx* ctx, int32_t flags);

/* Release everything the context owns.  NULL is ignored. */
CLUSTER_API void cluster_destroy(cluster_ctx* ctx);

/* ------------------------------------------------------------------------ */
/* Batched solves                                                            */
/* ------------------------------------------------------------------------ */
/* A batch advances `count` independent instances (each its own S, k and U0,
 * all on the current device) together: instances with the same padded cluster
 * count and precision share one persistent launch per kernel and iteration,
 * and the iteration sequence is captured in a CUDA graph.  Every instance
 * runs exactly the arithmetic, row ranges and reduction order it runs alone
 * (cluster_init with the same options), so its iterates are bit-identical to
 * a solo run.  S: host array of `count` cluster_csr descriptors (device
 * arrays); k: host array; U0: host array of `count` device pointers (n_i x
 * k_i).  opt is shared (fused_pass must be 0).  Inputs are copied as
 * cluster_init copies them (or borrowed with opt->borrow). */
typedef struct cluster_batch cluster_batch;

CLUSTER_API cluster_status cluster_batch_create(int32_t count, const cluster_csr* S, const int32_t* k,
                                                const float* const* U0, const cluster_options* opt,
                                                void* stream, cluster_batch** out);

/* Enqueue `iters` iterations of every unfinished instance (no host sync). */
CLUSTER_API cluster_status cluster_batch_enqueue(cluster_batch* b, int64_t iters);

/* Advance every instance by at most `iters` iterations (instances stop on
 * their own stop rule or max_iter), synchronise, and fill reps[0..count-1]
 * (may be NULL). */
CLUSTER_API cluster_status cluster_batch_step(cluster_batch* b, int64_t iters, cluster_report* reps);

/* Choose, per class, the gather's tile shape (nonzeros per batch of a row,
 * rows per work unit: three candidates, the first the solo solver's) and the
 * launch shapes (resident blocks per SM) of the gather and the update by
 * timing candidates on live iterations: each trial advances every unfinished
 * instance by one iteration, exactly as cluster_batch_step would (no shape
 * changes a value: each row is summed by one team in index order).  About
 * trials x max over classes of (3 x gather occupancy + update occupancy)
 * iterations are used; the CUDA graph is re-captured with the chosen shapes. */
CLUSTER_API cluster_status cluster_batch_autotune(cluster_batch* b, int32_t trials);

/* JSON description of the batch's classes into buf: per class the padded k,
 * precision, instances, gather units, chunked rows, update items, the gather
 * tile shape (shape index, nonzeros per batch, rows per unit) and the launch
 * shapes; after cluster_batch_autotune also each class's gather and update
 * times for the chosen shapes, the class running alone, in milliseconds. */
CLUSTER_API cluster_status cluster_batch_describe(cluster_batch* b, char* buf, size_t len);

/* Copy instance i's output iterate into U_out (device, n_i x k_i). */
CLUSTER_API cluster_status cluster_batch_get_U(cluster_batch* b, int32_t i, float* U_out);

CLUSTER_API void cluster_batch_destroy(cluster_batch* b);

/* ------------------------------------------------------------------------ */
/* Serving with continuous batching                                          */
/* ------------------------------------------------------------------------ */
/* A server owns a worker thread and the current device (at create time).
 * cluster_server_submit copies a request (host CSR, k, host start point) and
 * queues it; the worker admits queued requests in arrival order while their
 * estimated device footprint fits hbm_budget (and max_resident, if set),
 * keeps admitted solves resident, and advances all of them together
 * iters_per_tick iterations per tick through the batched launches.  Solves
 * that stop (their rule or max_iter) are finalised, copied to the host and
 * freed after the tick in which they stop, which admits more requests.  A
 * solve's result does not depend on what else is resident: it equals the same
 * request solved alone with the same options. */
typedef struct cluster_server cluster_server;

typedef struct cluster_server_options {
  cluster_options solve;   /* applied to every request (borrow and fused_pass
                              are set by the server); default stop rule PG_REL,
                              tol 1e-5, max_iter 5000                          */
  size_t hbm_budget;       /* device bytes resident solves may use; 0 = 80% of
                              the free device memory at create time            */
  int32_t iters_per_tick;  /* default 64                                        */
  int32_t max_resident;    /* 0 = no limit besides the budget                   */
  int32_t borrow_host;     /* 1 = submit keeps pointers to the caller's host
                              arrays instead of copying them; they must stay
                              valid until the request's result is taken      */
  int32_t _pad;
  size_t queue_bytes_max;  /* host bytes of copied, not yet admitted requests
                              above which submit refuses with CLUSTER_EAGAIN
                              ("queue full"); an empty queue always accepts
                              one request; 0 = no limit                       */
} cluster_server_options;

typedef struct cluster_server_stats {
  uint64_t submitted, admitted, completed, failed, ticks, rejected;
  int64_t queued, resident;
  size_t resident_bytes, budget_bytes, queued_host_bytes;
  double uptime_s;
} cluster_server_stats;

/* Per-request timing (seconds): queue_s = submit -> admission, run_s =
 * admission -> result on the host, total_s = submit -> result on the host. */
typedef struct cluster_request_times {
  double queue_s, run_s, total_s;
} cluster_request_times;

CLUSTER_API void cluster_server_options_default(cluster_server_options* opt);
CLUSTER_API cluster_status cluster_server_create(const cluster_server_options* opt, cluster_server** out);

/* Queue a request.  S: host CSR (int32 or int64 row pointers), U0: host n x k.
 * The server copies both (the caller's buffers may be reused at once) unless
 * borrow_host is set.  CLUSTER_EAGAIN if the copied-request queue is full. */
CLUSTER_API cluster_status cluster_server_submit(cluster_server* s, const cluster_csr* S, int32_t k,
                                                 const float* U0, uint64_t* ticket);

/* CLUSTER_EAGAIN while pending.  Once finished, returns the solve's status
 * (CLUSTER_OK, or the error that ended it, with cluster_last_error() set),
 * fills U_out (host, n x k), rep and times (each may be NULL) and forgets the
 * ticket. */
CLUSTER_API cluster_status cluster_server_poll(cluster_server* s, uint64_t ticket, float* U_out,
                                               cluster_report* rep, cluster_request_times* times);

/* Like poll but blocks up to timeout_s seconds; CLUSTER_ETIMEOUT if still
 * pending then (the ticket stays valid). */
CLUSTER_API cluster_status cluster_server_wait(cluster_server* s, uint64_t ticket, double timeout_s,
                                               float* U_out, cluster_report* rep, cluster_request_times* times);

CLUSTER_API cluster_status cluster_server_get_stats(cluster_server* s, cluster_server_stats* out);

/* Stop the worker after its current tick; unfinished requests end with
 * CLUSTER_EAGAIN.  Frees everything. */
CLUSTER_API void cluster_server_destroy(cluster_server* s);

/* ------------------------------------------------------------------------ */
/* CSR construction (host)                                                   */
/* ------------------------------------------------------------------------ */
/* Build the symmetric similarity matrix from an edge list (Example 4.1):
 * s_ij = s_ji = w_e for each edge e = (src[e], dst[e]) — "i cites or is cited
 * by j" — keeping the largest weight when a pair repeats.  w may be NULL
 * (all weights 1).  With add_unit_diag != 0 the diagonal is 1 and self-loop
 * edges are ignored; otherwise self-loops keep their largest weight.
 * src/dst/w are host arrays of length m.  On success `out` receives host
 * arrays allocated by the library (int64 row_ptr, index64 = 1, sorted
 * columns); release them with cluster_csr_free.  EINVAL if an endpoint is
 * outside [0, n) or a weight is not finite. */
CLUSTER_API cluster_status cluster_csr_from_edges(int64_t n, int64_t m, const int64_t* src,
                                                  const int64_t* dst, const float* w,
                                                  int32_t add_unit_diag, cluster_csr* out);
CLUSTER_API void cluster_csr_free(cluster_csr* csr);

#ifdef __cplusplus
}
#endif
#endif /* CLUSTER_H_ */
