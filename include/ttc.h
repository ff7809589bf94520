/*
 * ttc.h - C ABI of a GB300 (sm_103a) library for low-TT-rank tensor
 * completion by Preconditioned Riemannian Gradient Descent (PRGD).
 *
 * Problem (Eq. (model: Low TT)): given mode sizes n_1..n_d, TT-ranks
 * r_0..r_d (r_0 = r_d = 1), an index set Omega and observed values y,
 * minimise f(T) = 1/2 ||P_Omega(T - T*)||_F^2 over tensors of TT-rank r.
 * One iteration is Algorithm 2 (Trim skipped, which Section 3.2 allows):
 *   G_l = P_Omega(T_l - T*);  G_{l,i} = eps I + diag(M_i(G_l) M_i(G_l)^T);
 *   W_l = T_l - alpha_l tilde P_T W^{-1} G_l   (Lemma 3.5 closed form);
 *   T_{l+1} = SVD^tt_r(W_l)                      (Algorithm 1 by TT-rounding).
 *
 * Conventions shared by every call:
 *   - indices are 0-based; `idx` is row-major N x d (entry e, mode k at
 *     idx[e*d + k]);
 *   - host core k is a row-major array of shape r[k] x n[k] x r[k+1], the
 *     paper's T_k in R^{r_{k-1} x d_k x r_k} (Section 2, Eq. (TT Core));
 *   - every pointer argument is a HOST pointer unless its name ends in
 *     `_dev`; inputs are copied, outputs go to caller-allocated buffers;
 *   - a context owns its device memory and its CUDA stream use; it is not
 *     thread-safe.  Every call returns a ttc_status (0 = success) and never
 *     exits or throws across the ABI.
 */
#ifndef TTC_H
#define TTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttc_ctx ttc_ctx;

typedef enum {
  TTC_OK = 0,
  TTC_EINVAL = -1,      /* bad argument (sizes, ranks, null pointers, order of calls) */
  TTC_ENOMEM = -2,      /* device or host allocation failed */
  TTC_ERANGE = -3,      /* an index coordinate is negative or >= n_k */
  TTC_EDUP = -4,        /* Omega holds the same index twice (Omega is a set) */
  TTC_ENONFINITE = -5,  /* NaN/Inf in the input values or during an iteration */
  TTC_ENOTCONV = -6,    /* ttc_solve hit max_iter before its tolerance */
  TTC_ETIMEOUT = -7,
  TTC_ECUDA = -8,       /* a CUDA runtime call failed; see ttc_last_cuda_error */
  TTC_EBUSY = -9,
  TTC_EUNSUPPORTED = -10 /* shape outside the compiled limits (order <= 16, rank <= 32) */
} ttc_status;

/* Precision modes. */
enum {
  TTC_PREC_FP64 = 0,   /* every stage in FP64 */
  TTC_PREC_MIXED = 1,  /* FP32 Omega pass (FP32 accumulate); FP64 dense stages;
                          ttc_solve switches the pass to FP64 once the relative
                          residual ||P_Omega(T_l - T*)|| / ||y|| falls below
                          `polish_below` or the stop metric falls below
                          `polish_factor` times its tolerance; a MIXED solve
                          reports convergence only at or after that switch */
  TTC_PREC_FP32 = 2    /* FP32 Omega pass only, never polished */
};

/* Stop rules of ttc_solve. */
enum {
  TTC_STOP_RELERR = 0, /* ||T_l - T*||_F / ||T*||_F <= tol (needs ttc_set_truth) */
  TTC_STOP_STEP = 1,   /* ||T_{l+1} - T_l||_F <= tol * max(1, ||T_l||_F) (Section 5, noise experiment) */
  TTC_STOP_NONE = 2,   /* run exactly max_iter iterations */
  TTC_STOP_RESID = 3   /* ||P_Omega(T_l) - y|| <= tol ||y|| (residual on Omega; no extra kernels) */
};

/* Step-size rules. */
enum {
  TTC_STEP_CONSTANT = 0, /* alpha_l = alpha_scale * sqrt(eps_l) / p (Theorem 4.1 form; alpha_scale / p with
                            the uniform metric) */
  TTC_STEP_STEEPEST = 1  /* alpha_l = ||Z||_W^2 / ||P_Omega Z||_F^2, Z = tilde P_T W^{-1} G_l: the exact line
                            search along the search direction, Eq. (PRGD stepsize) in Section 3.2 */
};

/* Metrics. */
enum {
  TTC_METRIC_PRECOND = 0, /* W_l from G_{l,i} = eps I + diag(M_i(G_l) M_i(G_l)^T) (Section 3.2) */
  TTC_METRIC_UNIFORM = 1  /* G_{l,i} = I: the iteration is RGD (Section 3.1) */
};

/* Retractions. */
enum {
  TTC_RETRACT_PLAIN = 0,   /* T_{l+1} = SVD^tt_r(W_l) (Algorithm 2) */
  TTC_RETRACT_WEIGHTED = 1 /* T_{l+1} = W^{-1/2} SVD^tt_r(W^{1/2} W_l) (Remark 3.6) */
};

/* Arithmetic of the dense stages' slice products (the Grams Lam, Gam, H, Psi, N of Lemma 3.5's
 * projection and Algorithm 1's rounding, and the new cores) when some core rank exceeds 8; the small
 * factorizations (Gram inverses, the bonds' Cholesky factors and SVDs) are not affected. */
enum {
  TTC_DENSE_AUTO = 0, /* FP64 in FP64 steps, float-float in FP32 steps (default) */
  TTC_DENSE_FP64 = 1, /* always FP64 */
  TTC_DENSE_FF = 2    /* always float-float: pairs of floats (48-bit significands) with compensated dot
                         products (Ogita-Rump-Oishi Dot2), ~1e-11 relative to sum |a_i b_i|, FP32's
                         exponent range; on the FP32 pipe, which on GB300 runs ~6x faster per FMA */
};

typedef struct {
  int precision;        /* TTC_PREC_* */
  double eps_rel;       /* eps_l = eps_rel * ||G_l||_F^2 / min_k n_k (reading of Section 3.2) */
  double alpha_scale;   /* alpha_l = alpha_scale * sqrt(eps_l) / p  (Theorem 4.1 form), p = N / d* */
  int eps_frozen;       /* nonzero: keep iteration 0's eps for the whole run */
  double tol;           /* tolerance of the stop rule */
  int max_iter;
  int stop_rule;        /* TTC_STOP_* */
  int check_every;      /* evaluate the stop rule every k iterations (>= 1) */
  double polish_below;  /* MIXED: switch to FP64 once the relative residual is below this */
  int use_graph;        /* nonzero: replay one CUDA graph per iteration */
  int step_rule;        /* TTC_STEP_* */
  int metric;           /* TTC_METRIC_* */
  int retraction;       /* TTC_RETRACT_* */
  double polish_factor; /* MIXED: also switch to FP64 once the stop metric is <= polish_factor * tol
                           (near convergence; needed when noise keeps the residual from falling) */
  int step_fallback;    /* nonzero (default): a solve with the constant step switches to the steepest
                           step for its remaining iterations once the residual norm grows by more
                           than 2x from one read-back to the next (the constant's scale diverges on
                           that problem); the residual is read back every iteration in MIXED mode
                           or with the residual rule, else every check_every iterations */
  int dense_mode;       /* TTC_DENSE_* */
} ttc_options;

typedef struct {
  double eps;           /* eps_l used */
  double alpha;         /* alpha_l used */
  double res_norm;      /* ||P_Omega(T_l - T*)||_F before the step */
  int precision_used;   /* TTC_PREC_FP64 or TTC_PREC_FP32 for the Omega pass of this step */
  int subspace_iters;   /* Jacobi sweeps the retraction's bond SVDs took (all bonds) */
} ttc_step_info;

typedef struct {
  int iters;
  int converged;        /* 1 if the stop rule was met */
  double last_metric;   /* last value of the stop-rule metric */
  double res_norm;      /* residual norm at the last step */
  int polish_iter;      /* first FP64 iteration in MIXED mode (-1: none) */
  int fallback_iter;    /* first iteration with the steepest step after a constant-step divergence
                           (-1: none) */
} ttc_solve_info;

/* Fill `opt` with defaults: MIXED precision, eps_rel 1, alpha_scale 1.5,
 * tol 1e-6, max_iter 500, stop rule RELERR, check_every 1, polish_below 1e-5,
 * polish_factor 10, graphs on, constant step with the divergence fallback,
 * preconditioned metric, plain retraction. */
void ttc_default_options(ttc_options* opt);

/* Create a context for order d (1 < d <= 16), mode sizes n[d] (n_k >= 1),
 * TT-ranks r[d+1] with r[0] = r[d] = 1, 1 <= r[k] <= 32 and
 * r[k] <= min(n_1 ... n_k, n_{k+1} ... n_d) (the dimensions of the k-th
 * unfolding; a larger rank is TTC_EINVAL).  `opt` may be
 * NULL (defaults).  `cuda_stream` (a cudaStream_t, may be NULL) is the stream
 * all work of this context is issued on; NULL makes the context create its
 * own.  On success *out owns the context; free it with ttc_destroy. */
int ttc_create(ttc_ctx** out, int d, const int64_t* n, const int32_t* r,
               const ttc_options* opt, void* cuda_stream);

/* Copy the observations in: N >= 1 index rows idx[N*d] (int32, 0-based) and
 * values y[N] (FP64).  The device validates every coordinate (TTC_ERANGE),
 * rejects repeated indices (TTC_EDUP) and non-finite values
 * (TTC_ENONFINITE), then builds the per-mode layout: packed coordinates and,
 * for each mode k, a stable sort of the entries by x_k into segments
 * (Omega ordered by slice of mode k, ties in input order).  Replaces any
 * previous observations. */
int ttc_set_observations(ttc_ctx* ctx, int64_t N, const int32_t* idx, const double* y);

/* Set the current iterate T_l from host cores (see the layout above). */
int ttc_set_cores(ttc_ctx* ctx, const double* const* cores);

/* Copy the current iterate out to caller-allocated host cores. */
int ttc_get_cores(ttc_ctx* ctx, double* const* cores_out);

/* Ground truth T* as TT cores of ranks rt[d+1] (rt[0] = rt[d] = 1, each
 * <= 32); enables TTC_STOP_RELERR and ttc_relerr. */
int ttc_set_truth(ttc_ctx* ctx, const int32_t* rt, const double* const* cores);

/* One PRGD iteration (Algorithm 2).  alpha <= 0 takes the step-size policy
 * of the options.  With `out` non-NULL the call waits for the iteration and
 * fills `out` (TTC_ENONFINITE if the residual is not finite); with `out` NULL
 * it only enqueues the iteration on the context's stream and returns. */
int ttc_step(ttc_ctx* ctx, double alpha, ttc_step_info* out);

/* Iterate until the options' stop rule holds or max_iter.  Returns TTC_OK
 * when converged (or the rule is NONE), TTC_ENOTCONV otherwise. */
int ttc_solve(ttc_ctx* ctx, ttc_solve_info* out);

/* ||T_l - T*||_F / ||T*||_F for the current iterate (needs ttc_set_truth). */
int ttc_relerr(ttc_ctx* ctx, double* out);

/* Evaluate the current iterate at M index rows (host in, host out), in the
 * given precision (TTC_PREC_FP64 or TTC_PREC_FP32); Eq. (TT Core). */
int ttc_eval(ttc_ctx* ctx, int64_t M, const int32_t* idx, int precision, double* out);

/* Intermediate results, for checking:
 *   ttc_get_residual: g[N] = T(omega) - y(omega) in input order at the
 *     CURRENT iterate (runs one extra sampled pass, which also overwrites the
 *     slice energies and scatter below);
 * and, for the iterate the last ttc_step started from:
 *   ttc_get_slice_energy: s_k[n_k], the mode-k slice energies of G_l
 *     (diag(M_k(G_l) M_k(G_l)^T), Section 3.2);
 *   ttc_get_scatter: E_k, n_k x r_{k-1} x r_k, the sum over the mode-k slice
 *     x of g * (T^{<=k-1})^T (T^{>=k+1})^T at the iterate's own cores (the
 *     sparse factor of Eq. (tsp in nm) before the weight and gauge factors).
 */
int ttc_get_residual(ttc_ctx* ctx, double* g_out);
int ttc_get_slice_energy(ttc_ctx* ctx, int k, double* s_out);
int ttc_get_scatter(ttc_ctx* ctx, int k, double* E_out);

/* Layout of mode k, for checking: perm[N] (input position of the j-th entry
 * in mode-k order: the stable sort by x_k of mode k-1's order, mode 0's of
 * the input order, i.e. lexicographic in (x_k, x_{k-1}, ..., x_0, input
 * position)) and seg_off[n_k + 1] (CSR offsets of the slices). */
int ttc_get_layout(ttc_ctx* ctx, int k, int32_t* perm_out, int64_t* seg_off_out);

/* Kernel timing: when enabled, the dominant kernel of every iteration (the
 * sampled pass over Omega) is bracketed by CUDA events on the context's
 * stream, also inside the replayed CUDA graph (event-record nodes).  Every
 * iteration then waits for that kernel's end event on the host and adds its
 * duration; *ms and *count return the accumulated duration and number of
 * timed launches since the last reset. */
int ttc_profile_enable(ttc_ctx* ctx, int on);
int ttc_profile_read(ttc_ctx* ctx, double* ms, int64_t* count, int reset);

/* Number of kernels this context has launched so far (a graph replay counts
 * every kernel node it runs). */
int ttc_launch_count(ttc_ctx* ctx, int64_t* launches);

/* Device bytes held by the context. */
int ttc_device_bytes(ttc_ctx* ctx, int64_t* bytes);

/* ---- batches -------------------------------------------------------------
 * A batch steps many independent contexts together: one call enqueues one
 * PRGD iteration of every member as ONE CUDA graph launch.  The sampled pass
 * of all members that share a precision and rank bucket runs as one kernel
 * launch (blocks mapped to (member, chunk)).  The dense stages of members of
 * the same order with TT-ranks <= 8 (and not the steepest step) run batched
 * as well, one launch per stage for a chunk of members, with up to four
 * chunks on concurrent streams; other members' dense stages run as parallel
 * branches of the graph on their own streams.  Each member computes exactly
 * what it computes when stepped alone (bitwise).
 * Members must have observations and cores set, must not be stepped on their
 * own while the batch is in use, and must not change their observations or
 * truth afterwards (create a new batch instead).  The batch does not own the
 * members; destroy the batch before them. */
typedef struct ttc_batch ttc_batch;
int ttc_batch_create(ttc_batch** out, ttc_ctx* const* members, int count, void* cuda_stream);
/* Enqueue one iteration of every member on the batch's stream (no wait,
 * except with profiling on, see below). */
int ttc_batch_step(ttc_batch* b);
/* Wait for all work enqueued by the batch. */
int ttc_batch_sync(ttc_batch* b);
/* Lanes (call before the first step; 1 = none): the members are split into
 * `lanes` contiguous groups, each stepped by its own graph on its own
 * stream.  A step forks the lanes from the batch's stream only when they
 * are joined (after creation, ttc_batch_sync or ttc_batch_join), so between
 * joins the lanes run ahead independently: one lane's sampled pass (bound
 * by bandwidth and arithmetic across the GPU) overlaps another lane's dense
 * chain (bound by the latency of its small factorizations).  Each member
 * still computes what it computes alone (bitwise).  With lanes, the
 * batch's stream sees the lanes' work only after ttc_batch_join, which
 * enqueues a wait for all of it on that stream (no host wait); profiling
 * then serialises the lanes (each profiled step waits on the host).
 * Errors: TTC_EINVAL (lanes < 1 or more than the members, or after the
 * first step), TTC_ECUDA. */
int ttc_batch_set_lanes(ttc_batch* b, int lanes);
int ttc_batch_join(ttc_batch* b);
/* Profiling: the batched sampled-pass launch(es) of every step are bracketed
 * by events (graph event-record nodes), and so is the dense part of the step
 * (Lemma 3.5's projection, the step size and Algorithm 1's rounding of every
 * member, from the end of the pass to the join of all members); each step
 * then waits for the last event and adds both durations.
 * ttc_batch_profile_read gives the pass's total, ttc_batch_profile_read_dense
 * the dense part's (ms may be NULL), over `count` steps. */
int ttc_batch_profile_enable(ttc_batch* b, int on);
int ttc_batch_profile_read(ttc_batch* b, double* ms, int64_t* count, int reset);
int ttc_batch_profile_read_dense(ttc_batch* b, double* ms, int64_t* count, int reset);
/* Kernels launched by the batch so far (all graph kernel nodes of each step). */
int ttc_batch_launch_count(ttc_batch* b, int64_t* launches);
void ttc_batch_destroy(ttc_batch* b);

/* Serving: continuous batching of completion requests.
 *
 * A server owns an engine thread that runs requests on the current device.
 * ttc_submit copies a request (shape, Omega, y, starting cores, optional
 * truth and options) into host memory and queues it; the engine admits queued
 * requests in submission order while their device memory fits the budget and
 * fewer than max_slots are active, steps every active request together (one
 * batched iteration per tick, as ttc_batch_step), applies each request's stop
 * rule after every iteration (as ttc_solve: the precision switch of
 * TTC_PREC_MIXED, the check interval, max_iter), and retires finished
 * requests, copying their cores to host memory and freeing their device
 * memory, while the others keep running.  A request's iterates do not depend
 * on which other requests share its ticks: it computes exactly what ttc_solve
 * computes for it alone.  The paper solves one problem at a time; the
 * server is the batching layer around its Algorithm 2.
 *
 * device_mem_budget: bytes of device memory the active requests may hold
 * (0: 80% of the free memory at creation).  A request whose estimate
 * exceeds the budget is rejected by ttc_submit with TTC_ENOMEM.
 * cuda_stream: stream of the batched work (NULL: the server creates one).
 * Errors: TTC_EINVAL (null pointer, max_slots < 1), TTC_ECUDA. */
typedef struct ttc_server ttc_server;
int ttc_server_create(ttc_server** out, size_t device_mem_budget, int max_slots, void* cuda_stream);

/* One request.  All pointers are host pointers, read only during
 * ttc_submit (the server keeps copies).  n[d], r[d+1] and idx[N*d] (row-major
 * multi-indices) as in ttc_create / ttc_set_observations; init[k] the
 * starting cores; truth_r / truth (both NULL, or both set) the reference
 * train for TTC_STOP_RELERR; opt NULL: defaults with TTC_STOP_RESID. */
typedef struct {
  int d;
  const int64_t* n;
  const int32_t* r;
  int64_t N;
  const int32_t* idx;
  const double* y;
  const double* const* init;
  const int32_t* truth_r;
  const double* const* truth;
  const ttc_options* opt;
} ttc_request;

/* Queue a request; *ticket identifies it in ttc_poll.  Errors: TTC_EINVAL
 * (null pointers, bad shape), TTC_EUNSUPPORTED (limits of ttc_create),
 * TTC_ENOMEM (estimate above the budget), TTC_EBUSY (server shutting down).
 * Errors of the data itself (TTC_ERANGE, TTC_EDUP, TTC_ENONFINITE) are found at
 * admission and returned in the request's result. */
int ttc_submit(ttc_server* s, const ttc_request* req, uint64_t* ticket);

typedef struct {
  int status;          /* TTC_OK, TTC_ENOTCONV or the error that ended the request */
  int iters;
  int converged;
  double last_metric;
  double res_norm;     /* ||P_Omega(T_l) - y|| after the last iteration */
  double latency_ms;   /* submission to completion */
  double queue_ms;     /* submission to admission */
  char detail[128];    /* text of the CUDA error when status is TTC_ECUDA, else "" */
} ttc_result;

/* Wait up to timeout_us microseconds (negative: no limit) for a request to
 * finish; then fill `result` (if not NULL) and copy the final cores into
 * cores_out[k] (host buffers of r[k]*n[k]*r[k+1] doubles, or cores_out NULL)
 * and forget the ticket.  Returns TTC_ETIMEOUT if it has not finished (the
 * ticket stays valid), TTC_EINVAL for an unknown ticket; the request's own
 * outcome is result->status. */
int ttc_poll(ttc_server* s, uint64_t ticket, int64_t timeout_us, ttc_result* result,
             double* const* cores_out);

typedef struct {
  int64_t completed;          /* requests finished with TTC_OK or TTC_ENOTCONV */
  int64_t failed;             /* requests ended by another error */
  int64_t queued;             /* waiting for admission now */
  int64_t iterations;         /* request-iterations run */
  int64_t launches;           /* kernels launched by the engine (graph kernel nodes included) */
  double entry_iterations;    /* sum over request-iterations of |Omega| */
  double busy_ms;             /* engine time spent in ticks (step + stop checks) */
  double wall_ms;             /* time since creation */
  double p50_ms, p99_ms, max_ms;   /* latency percentiles of completed requests */
  int64_t rebuilds;           /* batch graph (re)captures: the member set or a member's precision changed */
  double rebuild_ms;          /* engine time spent in them (part of busy_ms) */
  double admit_ms;            /* engine time spent admitting requests (context, layout, uploads) */
} ttc_serving_stats;
int ttc_server_stats(ttc_server* s, ttc_serving_stats* out);

/* Finish every queued and active request, stop the engine and free all.
 * Results not polled are dropped. */
void ttc_server_destroy(ttc_server* s);

/* Allocation-free squared Frobenius distance of two tensor trains (the paper
 * has no counterpart of this call).  For callers that may not allocate
 * device memory themselves, e.g. a real-time loop with a fixed memory budget
 * or code inside a framework that owns every device allocation: the caller
 * passes the inputs and the output in its own device memory, and the call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Inputs: order d (1 <= d <= 16), mode sizes n[d] (host), TT-ranks ra[d+1]
 * and rb[d+1] (host, first and last 1, each <= 32), and host arrays of d
 * DEVICE pointers a_dev[k], b_dev[k] to cores in the host layout of this
 * header (ra[k] x n[k] x ra[k+1] row-major).  Every one of the d* = prod n_k
 * entries is evaluated in FP64, so d* is limited to 2^32 and the work, d*
 * times sum_k (ra[k] ra[k+1] + rb[k] rb[k+1]) FMAs, to 2^34; larger shapes
 * return TTC_EUNSUPPORTED.  Output: out_dev[0] = ||A - B||_F^2, out_dev[1] =
 * ||B||_F^2 (two doubles of device memory), written on `cuda_stream` (NULL:
 * the default stream); the call returns without waiting.
 *
 * Scratch: per-block partial sums live in one fixed 16 KiB device array
 * (1024 partial pairs) that every GPU loading the library holds until the
 * process exits; it is never cleared (each call writes the slots it reads).
 * All calls share it, so calls that overlap on the GPU (different streams or
 * host threads without ordering) race.  The first call on each device looks
 * up the array's device address with that device current and keeps it for
 * the life of the process; make that first call before any stream capture,
 * and do not use the call after a cudaDeviceReset of that device (the kept
 * address belongs to the old context).  Errors: TTC_EINVAL (null pointers,
 * bad ranks), TTC_EUNSUPPORTED (limits above), TTC_ECUDA (launch failure). */
int ttc_tt_dist2_static(int d, const int64_t* n, const int32_t* ra, const double* const* a_dev,
                        const int32_t* rb, const double* const* b_dev, double* out_dev,
                        void* cuda_stream);

void ttc_destroy(ttc_ctx* ctx);

const char* ttc_strerror(int status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* ttc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TTC_H */
