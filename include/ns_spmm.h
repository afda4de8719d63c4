/*
 * ns_spmm.h -- C ABI of the GB300 hybrid sparse x dense matrix multiply.
 *
 * Operation (Section 5.1 of arXiv 2606.22482, "NeutronSparse"):  C = A * B, where A is an
 * m x n sparse matrix in CSR form, B an n x K dense matrix and C the m x K dense result.  The
 * method splits A into dense row-window tiles, run on the matrix engine (here: the tensor
 * cores), and a sparse residual, run on the vector engine (here: the CUDA cores), and runs both
 * from one balanced work list (Sections 5.2, 6 and 7).
 *
 * Conventions shared by every entry point
 *  - All functions return an ns_status_t and never abort the process.  On failure a message is
 *    available from ns_last_error() (thread-local, valid until the next call on that thread).
 *  - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.  Work is
 *    enqueued on the stream; ns_spmm_plan and ns_autotune synchronise it before returning.
 *  - Dense matrices are row-major with a leading dimension in elements (ldb >= K, ldc >= K).
 *    Device pointers to B and C must be 16-byte aligned and ldb, ldc multiples of 8.
 *  - Kernels never trap.  A kernel that detects an internal error or gives up a bounded wait
 *    writes a device status word; the next call on the same object reports it.
 *  - Indices are int32; nnz < 2^31.  m, n < 2^31.
 */
#ifndef NS_SPMM_H
#define NS_SPMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NS_OK = 0,
    NS_ERR_INVALID = 1,     /* bad argument or invalid CSR (unsorted/duplicate/out-of-range column,
                               non-monotone row pointers) */
    NS_ERR_UNSUPPORTED = 2, /* valid but not handled: K % 8 != 0, K > 1024, unaligned B/C */
    NS_ERR_OOM = 3,         /* device or host allocation failed */
    NS_ERR_CUDA = 4,        /* a CUDA runtime call failed; message names it */
    NS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    NS_ERR_AGAIN = 6,       /* serving: queue full, retry later */
    NS_ERR_TOO_LARGE = 7,   /* serving: request footprint exceeds the HBM budget */
    NS_ERR_NOT_FOUND = 8    /* unknown array name / ticket */
} ns_status_t;

/* Storage type of B.  C is always FP32.  NS_BF16 also stores dense-tile values of A in BF16
 * (round to nearest even) and runs those tiles on the tensor cores in BF16 with FP32
 * accumulation; the residual always runs in FP32 with B widened exactly. */
typedef enum { NS_F32 = 0, NS_BF16 = 1 } ns_dtype_t;

typedef void* ns_stream_t;

/* A CSR matrix.  Columns must be sorted ascending and unique inside each row (explicit zeros
 * are structure).  on_device = 1: the three arrays are device pointers that the caller keeps
 * alive and unchanged until every plan made from them is destroyed (plans may reference them);
 * on_device = 0: host arrays, copied during ns_spmm_plan. */
typedef struct {
    int32_t m, n;
    int64_t nnz;
    const int32_t* rowptr; /* m + 1 entries, rowptr[0] = 0, rowptr[m] = nnz */
    const int32_t* colidx; /* nnz entries */
    const float* vals;     /* nnz entries */
    int32_t on_device;
} ns_csr_t;

#define NS_TAU_INF 2147483647

/* Planner and execution parameters (Sections 5.2 and 6.2).  Fill with ns_tune_default() and
 * change fields, or let ns_autotune() choose them.
 *   TM          row-window height: 16, 32 or 64 rows (Section 6.1 windows match the tile's M)
 *   TK          compacted columns per dense tile: 16 or 32
 *   tau_tile    a tile is dense iff its nonzero count >= tau_tile; the integer form of the
 *               density threshold alpha of Eq. 3 (tau = ceil(alpha * TM * TK)).  NS_TAU_INF:
 *               no dense tiles (pure CUDA-core path); <= 1: every compacted tile is dense
 *   tau_row     row extraction (Eq. 4-5): a row with Len <= tau_row goes straight to the residual
 *   tau_col     column extraction inside the kept rows: a column with count <= tau_col goes
 *               to the residual (0 disables the stage)
 *   col_order   order of compacted columns inside a window: 0 count-descending then column,
 *               1 column-ascending
 *   chunk_nnz   W, residual merge items (nonzeros + row ends) per warp chunk, 2..1024
 *   absorb_cap  a dense window also computes its rows' residual when that has <= absorb_cap nnz
 *   group       residual chunks per work item (one per warp of the execute CTA; must be 4)
 *   cost_tc     Eq. 1 weight of one dense-tile element in the work-list order
 *   cost_res    Eq. 1 weight of one residual merge item in the work-list order
 *   l2_hints    1: stream A and C with evict-first and keep B with evict-last L2 policies;
 *               2: as 1, but only the most-gathered B rows (about 80% of L2, counted by the
 *               planner) evict last and the rest evict first (Section 6.2.1 hot-B staging);
 *               0: default caching
 *   TN          execute in column slices of TN (multiple of 8; 0 = K in one pass): each slice
 *               gathers only TN columns of B, so its working set stays in L2 (Section 6.2.2 N
 *               shaping); A is re-read once per slice.  Execution only: plans do not depend on it
 *   reorder     Section 6.1 local reordering (0 = off): inside clusters of reorder * TM
 *               consecutive kept rows (at most 1024 rows), the first unassigned row anchors a
 *               new window and takes the TM - 1 unassigned rows with the largest Jaccard
 *               similarity of kept-column sets (earlier rows first on ties) */
typedef struct {
    int32_t TM, TK, tau_tile, tau_row, tau_col, col_order, chunk_nnz, absorb_cap, group,
        cost_tc, cost_res, l2_hints, TN, reorder;
} ns_tune_t;

void ns_tune_default(ns_tune_t* t);

/* Counts of a plan, named as in the CPU reference partition. */
typedef struct {
    int64_t m, n, nnz, K, b_bf16, TM, TK;
    int64_t m_aic;    /* rows kept for windows after row extraction */
    int64_t n_win;    /* row windows */
    int64_t n_dtiles; /* dense tiles */
    int64_t n_dwin;   /* windows with at least one dense tile (dense work items) */
    int64_t n_dvals;  /* stored dense-tile values incl. padding to 8 per tile */
    int64_t n_res;    /* residual nonzeros */
    int64_t n_rl;     /* rows handled by residual chunks */
    int64_t T;        /* residual merge items */
    int64_t n_chunks; /* residual warp chunks */
    int64_t n_split;  /* rows assembled from several pieces */
    int64_t n_slots;  /* partial-row slots */
    int64_t n_items;  /* work items of the execute launch */
    int64_t device_bytes; /* device memory the plan holds */
} ns_plan_stats_t;

typedef struct ns_plan* ns_plan_t;

/* Build the execution plan of A for dense operands of width K and type b_dtype (Sections 4,
 * 5.2.2, 6.1, 7): validates A, extracts short rows/columns, forms TM-row windows, compacts
 * their columns into TK-wide tiles, bins tiles by density against tau_tile, builds the residual
 * CSR, splits it into nnz-balanced chunks and orders all work items by estimated cost.  Every
 * step runs as device kernels on `s`; the call synchronises `s` (plan sizes are data-dependent).
 * tune == NULL uses ns_tune_default().  The plan owns its device arrays until ns_plan_destroy.
 * Errors: NS_ERR_INVALID (bad CSR or tune), NS_ERR_UNSUPPORTED (K), NS_ERR_OOM, NS_ERR_CUDA. */
ns_status_t ns_spmm_plan(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, const ns_tune_t* tune,
                         ns_stream_t s, ns_plan_t* out);

/* C := A * B (overwrite; every row of C is written) with one persistent launch over the plan's
 * work list (Section 5.1 execution models, Section 7 balanced lists).  B (n x K, b_dtype) and
 * C (m x K, FP32) are device pointers owned by the caller.  Asynchronous on `s`.  Plans are
 * not re-entrant: at most one execute of a given plan may be in flight.
 * Errors: NS_ERR_INVALID, NS_ERR_UNSUPPORTED (alignment), NS_ERR_TIMEOUT / NS_ERR_CUDA from a
 * previous launch of this plan, NS_ERR_CUDA. */
ns_status_t ns_spmm_execute(ns_plan_t p, const void* B, int64_t ldb, float* C, int64_t ldc,
                            ns_stream_t s);

/* One-shot C = A * B from HOST memory: copies A (host CSR), B (host, n x K) to the device, plans,
 * executes and copies C (host, m x K) back, all on `s`; returns after `s` is synchronised.
 * Pinned host buffers give the fastest copies.  Device buffers are cached inside the library
 * between calls (freed by ns_release_cache).  Same errors as plan + execute. */
ns_status_t ns_spmm_host(const ns_csr_t* A, const void* B, int32_t K, ns_dtype_t b_dtype,
                         float* C, const ns_tune_t* tune, ns_stream_t s);
ns_status_t ns_release_cache(void);

ns_status_t ns_plan_stats(ns_plan_t p, ns_plan_stats_t* st);

/* Copy one named plan array to host memory (for comparison with the CPU reference partition and
 * checks of the execute bookkeeping).  Names: aic_rows win_rows win_dptr dwin dwin_absorb
 * dtile_cols dtile_bits dtile_voff dtile_vals dtile_x res_rowptr res_col res_val rl_rows rl_start
 * chunk_b chunk_k0 row_split split_row split_np split_slot split_base queue item_cost.  The
 * partition (Sections 5.2.2, 6.1) is aic_rows, win_rows, win_dptr, dtile_cols, dtile_bits,
 * dtile_voff, dtile_vals and res_*; dtile_x (BF16 plans) holds every dense tile expanded to
 * TM x TK BF16 values in 8 x 8 blocks of 128 bytes (the tensor cores' operand layout); the rest
 * schedules the execute launch.  ns_plan_array_info gives the element count and size; `bytes`
 * must be at least count * esize.  Synchronous. */
ns_status_t ns_plan_array_info(ns_plan_t p, const char* name, int64_t* count, int32_t* esize);
ns_status_t ns_plan_export(ns_plan_t p, const char* name, void* host_dst, int64_t bytes);

ns_status_t ns_plan_destroy(ns_plan_t p);

/* ---------------------------------------------------------------------------------------- */
/* Batched form: many independent SpMMs in one persistent launch, replayed from a CUDA graph. */
/* ---------------------------------------------------------------------------------------- */
typedef struct ns_batch* ns_batch_t;

/* Plan `count` matrices (each with its own K) and merge their work lists into one.  The batch
 * owns the plans.  Errors as ns_spmm_plan; on error nothing is kept. */
ns_status_t ns_batch_plan(const ns_csr_t* As, int32_t count, const int32_t* Ks, ns_dtype_t b_dtype,
                          const ns_tune_t* tune, ns_stream_t s, ns_batch_t* out);

/* C_g := A_g * B_g for every g, in ONE persistent kernel launch.  The launch is captured into a
 * CUDA graph on the first call and replayed afterwards; the operand table is refreshed by one
 * host-to-device copy when pointers change.  Bs[g], Cs[g] are device pointers, ldb = ldc = K_g. */
ns_status_t ns_batch_execute(ns_batch_t b, const void* const* Bs, float* const* Cs, ns_stream_t s);
ns_status_t ns_batch_stats(ns_batch_t b, int64_t* n_items, int64_t* n_graphs);
ns_status_t ns_batch_destroy(ns_batch_t b);

/* The residual chunk size W (chunk_nnz, with absorb_cap = W) for a whole batch: each W in
 * {128, 256, 512, 1024} is planned as a batch from `start` (NULL: defaults) and its launch is
 * timed on Bs / Cs (device pointers as in ns_batch_execute; Cs is overwritten); *out gets start
 * with the fastest W and *best_ms (may be NULL) its launch time.  The best W of one graph alone
 * (ns_autotune) can differ from the batch's, where many small chunks share one launch.
 * Synchronous; errors as ns_batch_plan / ns_batch_execute. */
ns_status_t ns_batch_autotune(const ns_csr_t* As, int32_t count, const int32_t* Ks, ns_dtype_t b_dtype,
                              const ns_tune_t* start, const void* const* Bs, float* const* Cs,
                              ns_stream_t s, ns_tune_t* out, double* best_ms);

/* ---------------------------------------------------------------------------------------- */
/* Autotuner (Section 5.2.1 dry run + Section 8 sweeps).                                     */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
    double p_res;     /* out: measured residual throughput, nonzeros * K per second          */
    double p_tc;      /* out: measured dense-tile throughput, tile elements * K per second   */
    double alpha0;    /* out: Eq. 3 with r = 1: p_res / p_tc                                  */
    double best_ms;   /* out: execute time of the chosen tune                                 */
    int32_t trials;   /* out: configurations timed                                            */
    double plan_runs; /* in: executions per plan over which planning is amortised; the
                         objective is execute_ms + plan_ms / plan_runs (0: 200, the paper's
                         200-epoch GCN setting; 1: a fresh plan for every execute)          */
} ns_tune_report_t;

/* Dry runs on A give p_res (residual-only plan) and p_tc (every compacted tile dense), hence
 * alpha0 and tau0 = ceil(alpha0 * TM * TK); then (TM, TK, tau) candidates around tau0, the two
 * single-engine extremes and column slices TN are planned and timed, and the best by
 * execute_ms + plan_ms / plan_runs is returned in *out.  A must be on the device.  Synchronous;
 * report may be NULL (then plan_runs = 200). */
ns_status_t ns_autotune(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, ns_stream_t s,
                        ns_tune_t* out, ns_tune_report_t* report);

/* Host-side helpers of the cost model (pure functions, no GPU needed). */
double ns_cost_alpha(double p_res, double p_tc, double r);            /* Eq. 3 */
int32_t ns_cost_tau(double alpha, int32_t TM, int32_t TK);           /* ceil(alpha*TM*TK) */
double ns_skew(double dt_tc, double dt_res);                         /* Eq. 6 */

/* ---------------------------------------------------------------------------------------- */
/* Epoch-level re-balance (Section 5.3).                                                     */
/* ---------------------------------------------------------------------------------------- */
/* Each iteration ("epoch") plans A with the current tau, executes C := A*B once with the
 * execute kernel stamping, per item class, the latest end time (globaltimer) of a dense-tile
 * item and of a residual chunk after the earliest CTA start: dt_tc and dt_res.  With
 * Skew = max/min (Eq. 6; infinite when a class is empty) above 1 + eps, work moves away from the
 * class that finishes last: tau is bisected over the open bracket (0, TM*TK + 1) -- a higher tau
 * leaves more tiles to the CUDA cores (the tensor side finished last), a lower one moves tiles to
 * the tensor cores.  Stops when Skew <= 1 + eps, when the bracket is exhausted or after max_iter
 * (at most 16) iterations; *out gets the tau with the shortest max(dt_tc, dt_res).
 * A must be on the device; B (n x K, ld ldb) and C (m x K, ld ldc) are device pointers and C
 * holds A*B on return.  Synchronous.  start may be NULL (defaults; tau = INF starts mid-bracket). */
typedef struct {
    int32_t iterations;   /* out */
    int32_t converged;    /* out: 1 if Skew <= 1 + eps was reached                            */
    int32_t tau[16];      /* out: tau of every iteration                                      */
    double dt_tc_ms[16];  /* out: dense-tile class span, ms                                   */
    double dt_res_ms[16]; /* out: residual class span, ms                                     */
    double skew[16];      /* out: Eq. 6 (0 when a class is empty: read it as unbounded)        */
} ns_rebalance_report_t;

ns_status_t ns_rebalance(const ns_csr_t* A, int32_t K, ns_dtype_t b_dtype, const void* B, int64_t ldb,
                         float* C, int64_t ldc, ns_stream_t s, const ns_tune_t* start, double eps,
                         int32_t max_iter, ns_tune_t* out, ns_rebalance_report_t* report);

/* One bisection step of ns_rebalance (pure, no GPU): from the open bracket (lo, hi), the tau
 * just timed and its class spans, the next bracket and tau.  Returns 1 when the loop ends
 * (balanced within eps, or no integer left in the bracket), 0 to continue. */
int32_t ns_rebalance_next(int32_t lo, int32_t hi, int32_t tau, double dt_tc, double dt_res, double eps,
                          int32_t* lo_out, int32_t* hi_out, int32_t* tau_out);

/* ---------------------------------------------------------------------------------------- */
/* Serving: continuous batching of SpMM requests on one GPU.                                 */
/* ---------------------------------------------------------------------------------------- */
/* A server owns two host threads.  The planner builds the plan of each new (graph, K, dtype)
 * key -- one plan per graph when the tune keeps every nonzero on the CUDA cores (tau_tile =
 * NS_TAU_INF) and l2_hints != 2, since such a plan depends on neither K nor the dtype -- and
 * plans stay resident for later requests.  The worker admits queued requests whose plan is
 * built, in arrival order (a request waiting for its plan lets later ones pass), while slots are
 * free and the request's device footprint (B, C, its plan's partial-row slots and counters) fits the budget
 * beside the resident plans, evicting idle plans least recently used first.  With nothing in
 * flight the oldest request is admitted even if plans of queued requests fill the budget, so the
 * queue always moves.  Every request admitted since the last launch joins one persistent launch
 * per (K, dtype, kernel) group; C is copied back on that launch's stream. */
typedef struct ns_server* ns_server_t;

typedef struct {
    int64_t hbm_budget_bytes; /* admission limit for resident plans + operands                 */
    int32_t max_inflight;     /* requests admitted at once (slots)                               */
    int32_t max_queue;        /* requests waiting for admission before NS_ERR_AGAIN             */
    int32_t max_graphs;       /* resident graph plans kept (LRU beyond)                          */
    ns_tune_t tune;           /* tune used for every plan                                        */
} ns_serve_cfg_t;

/* A request: graph_id names a graph registered with ns_serve_register_graph; B and C are host
 * pointers (row-major, ld = K) that stay valid until the request is reported done. */
typedef struct {
    int32_t graph_id;
    int32_t K;
    ns_dtype_t b_dtype;
    const void* B;
    float* C;
    double t_arrival; /* caller's clock (seconds) at which the request arrived; for latency */
} ns_request_t;

typedef struct {
    double t_admit, t_start, t_done; /* seconds on the server clock (ns_serve_now): admitted,
                                        launched, result in the host buffer                      */
    int32_t status;                  /* ns_status_t of the request                               */
    int32_t plan_built;              /* 1: this request was the first on its plan key (the plan
                                        was built for it)                                         */
    double t_planned;                /* when its plan became ready, if the request waited for it;
                                        0 when the plan was already resident                      */
    double t_h2d, t_exec, t_d2h;     /* on the GPU, mapped to the server clock: its launch's B
                                        uploads done, its launch's kernel done, its C copy done   */
} ns_req_stats_t;

ns_status_t ns_serve_create(const ns_serve_cfg_t* cfg, ns_server_t* out);
/* Register a host CSR graph; the server copies it.  Returns its id in *graph_id. */
ns_status_t ns_serve_register_graph(ns_server_t sv, const ns_csr_t* A, int32_t* graph_id);
/* Queue a request; returns immediately.  NS_ERR_AGAIN if the queue is full, NS_ERR_TOO_LARGE if
 * B + C + the plan estimate already exceed the HBM budget.  A request whose footprint with its
 * built plan exceeds the budget fails later with NS_ERR_TOO_LARGE (reported by ns_serve_poll). */
ns_status_t ns_serve_submit(ns_server_t sv, const ns_request_t* r, uint64_t* ticket);
/* Non-blocking completion check; *done = 1 once C has been written to the host buffer. */
ns_status_t ns_serve_poll(ns_server_t sv, uint64_t ticket, int* done, ns_req_stats_t* st);
double ns_serve_now(void);
ns_status_t ns_serve_destroy(ns_server_t sv);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free SpMM (no counterpart in the paper).                                       */
/* ---------------------------------------------------------------------------------------- */
/* For callers that cannot allocate device memory -- a process whose HBM is already handed to
 * another allocator (a framework's caching allocator, a fixed per-tenant budget), or a
 * latency-critical path that cannot pay the implicit device synchronisation of cudaMalloc and
 * cudaFree.  C := A * B (every row written) on the CUDA cores, straight from the CSR: no plan,
 * no dense tiles, no cudaMalloc/cudaFree and no allocating library call.  Its scratch (work
 * ticket, split-row counters, partial-row slots) lives in one 32 MiB file-scope device array that
 * every GPU loading this library holds until the process exits.
 *   A       device CSR (on_device = 1), sorted unique columns; not validated beyond keeping every
 *           access in bounds.  B (n x K, b_dtype) and C (m x K, FP32): device pointers, 16-byte
 *           aligned, ldb and ldc >= K and multiples of 8.  Asynchronous on `s`.
 *   Limit   2 * ceil((m + nnz) / 256) * K * 4 bytes of partial rows, plus counters, must fit the
 *           32 MiB array (K = 128: m + nnz up to about 8.3 million); beyond it NS_ERR_TOO_LARGE.
 *   The first call on a device resolves the array's device address (cudaGetSymbolAddress) and
 *   caches it: make that first call before any stream capture.  Calls share the array and it
 *   keeps the last call's contents; each call clears its counters first.  Calls that overlap on
 *   the GPU (different streams or threads) race on the array and give wrong results.
 * Errors: NS_ERR_INVALID (also a CSR with n = 0 and nnz > 0), NS_ERR_UNSUPPORTED (K, alignment),
 * NS_ERR_TOO_LARGE, NS_ERR_CUDA. */
ns_status_t ns_spmm_csr_static(const ns_csr_t* A, const void* B, int64_t ldb, float* C, int64_t ldc,
                               int32_t K, ns_dtype_t b_dtype, ns_stream_t s);

/* ---------------------------------------------------------------------------------------- */
/* Diagnostics                                                                               */
/* ---------------------------------------------------------------------------------------- */
const char* ns_last_error(void);
/* Kernels launched by this library in this process (all entry points). */
int64_t ns_launch_count(void);
/* 1 if the library was built for the device it runs on (sm_103a), else 0. */
int32_t ns_device_ok(void);

/* ---------------------------------------------------------------------------------------- */
/* Fault injection on the host (tests; no counterpart in the paper).  Neither faults a GPU:   */
/* they drive the library's error paths the way a failing call or a kernel guard would.      */
/* ---------------------------------------------------------------------------------------- */
/* After `after` more successful device allocations by the library (plans, scratch, served
 * requests), the next one fails as if the device were out of memory, once; after = -1 turns the
 * injection off.  Process-wide. */
ns_status_t ns_inject_alloc_failure(int32_t after);
/* OR `bits` (NS status bits: 2 = a bounded wait gave up, 4 = an index out of range) into the
 * plan's device status word, as a kernel guard would.  Synchronous.  The plan's next execute
 * copies the word back and the execute after it returns NS_ERR_TIMEOUT (bit 2) or NS_ERR_CUDA.
 * Errors: NS_ERR_INVALID (NULL plan, bits outside 2 | 4), NS_ERR_CUDA. */
ns_status_t ns_plan_inject_status(ns_plan_t p, int32_t bits);

#ifdef __cplusplus
}
#endif

#endif /* NS_SPMM_H */
