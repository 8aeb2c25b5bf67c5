/*
 * chordal.h — C ABI of libchordal.so, the GB300 (sm_103a) parallel chordality
 * test of "A Parallel Algorithm to Test Chordality of Graphs" (arXiv:1508.06329).
 *
 * The test has two parts (Section 6): a LexBFS order computed by partition
 * refinement (Sections 4.2 and 6.1), then the perfect-elimination check of
 * that order (Sections 5.2 and 6.2).  G is chordal iff the LexBFS order is a
 * perfect elimination order (Theorem 5.1).
 *
 * Conventions used by every entry point
 *   - Vertex ids are 0-based, 0..n-1.
 *   - Dense graphs: `rows` holds n rows of `words_per_row` uint32 words; bit
 *     (j & 31) of rows[i * words_per_row + (j >> 5)] is 1 iff ij is an edge
 *     (LSB first).  The matrix must be symmetric with a zero diagonal and zero
 *     padding bits; words_per_row >= ceil(n / 32).
 *   - CSR graphs: row_ptr int64[n + 1], col int32[nnz]; each row sorted
 *     ascending, no self-loops, no duplicates, symmetric.
 *   - order int32[n]: order[i] is the i-th visited vertex (the ordering π of
 *     Section 3.1); pos int32[n] is its inverse π^{-1}.
 *   - Tie-break: among the unnumbered vertices whose label is
 *     lexicographically largest, the lowest id is visited first (the paper
 *     leaves the choice open, Section 6.1; this fixes one LexBFS order).
 *   - Witness: when the graph is not chordal, v is the vertex with the
 *     smallest order index whose earlier neighbourhood LN_v is not a clique
 *     (the "first such node" of Section 5.3), p = p(v) is its neighbour with
 *     the largest order index below v's, and u is the smallest id in
 *     (LN_v - {p}) \ N(p).  When chordal, v = p = u = -1.
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  Calls are asynchronous on `stream`
 *     unless the name ends in _host; results are valid after the stream is
 *     synchronised.  The library allocates only its own workspace, held by the
 *     context and grown on demand (device memory, plus pinned host staging).
 *   - Every call returns a cg_status.  On CG_ECUDA / CG_EINVAL,
 *     cg_last_error_string() describes the failure (thread-local).
 *   - A context may be used by one host thread at a time, and its workspace is
 *     shared by its calls: calls whose GPU work may overlap (different streams)
 *     need different contexts.
 */
#ifndef CHORDAL_GB300_H
#define CHORDAL_GB300_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CG_OK = 0,
    CG_EINVAL = 1,    /* bad size, layout or pointer */
    CG_ENOMEM = 2,    /* workspace allocation failed */
    CG_ECUDA = 3,     /* a CUDA call or kernel launch failed */
    CG_ETIMEOUT = 4,  /* a bounded wait (queue drain) expired */
    CG_EAGAIN = 5,    /* queue full / result not ready yet */
} cg_status;

/* Dense bit-packed graph (device memory). */
typedef struct {
    int32_t n;
    int32_t words_per_row;
    const uint32_t *rows;
} cg_dense;

/* CSR graph (device memory). */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col;
} cg_csr;

/* Verdict and witness (see conventions). */
typedef struct {
    int32_t chordal;
    int32_t v, p, u;
} cg_result;

typedef struct {
    int32_t device;          /* CUDA device ordinal the context works on */
    int32_t validate;        /* 1: check sizes and CSR sortedness on entry (costs a sync) */
    int32_t threads_override;/* 0: autotuned CTA size for the LexBFS kernels; else 128..1024 */
    int32_t reserved;
} cg_config;

typedef struct cg_context cg_context;

/* Library version, e.g. "chordal-gb300 0.1.0 (sm_103a)". */
const char *cg_version(void);
/* Last error message of the calling thread ("" if none). */
const char *cg_last_error_string(void);

/* Create / destroy a context.  cfg may be NULL (device 0, defaults).  The
 * context owns device workspace and pinned staging memory; destroy frees it
 * (synchronising the device first). */
int cg_context_create(const cg_config *cfg, cg_context **out);
int cg_context_destroy(cg_context *ctx);

/*
 * LexBFS order of a dense graph (Section 4.2: pick the first vertex of the
 * first class, split every class C into C ∩ N_x placed before C \ N_x;
 * Section 6.1 runs it on the GPU).  One persistent CTA walks all n steps with
 * the partition state in shared memory (n <= 16384), split between shared
 * memory and the workspace (n <= 65520) or in the workspace.
 *   g      device graph, n >= 0, n <= 131072
 *   order  device int32[n] (written)
 *   pos    device int32[n] (written) or NULL
 */
int cg_lexbfs_order_dense(cg_context *ctx, const cg_dense *g, int32_t *order, int32_t *pos,
                          cudaStream_t stream);

/*
 * One sweep of multi-sweep LexBFS on a dense graph: LexBFS (Section 4.2) in
 * which, among the unnumbered vertices with the lexicographically largest
 * label, the one chosen is
 *   CG_TIE_ID       the lowest vertex id (tiebreak unused; as above),
 *   CG_TIE_RANK     the one with the smallest tiebreak[v]; tiebreak is a
 *                   device int32[n] permutation of 0..n-1,
 *   CG_TIE_LAST_IN  the one latest in tiebreak, a device int32[n] vertex
 *                   order (a previous sweep): LexBFS+ of that sweep;
 * and start (-1 = none, else 0 <= start < n) is numbered first.  This is
 * the building block of the multi-sweep algorithms that use LexBFS beyond the
 * chordality test (interval and co-comparability recognition, Section 3.2;
 * the parallel interval test named as future work in Section 8).
 * The graph is relabelled on the GPU (workspace: n * ceil(n/32) * 4 bytes
 * more) and the dense LexBFS runs on the copy.  n <= 131072.  A tiebreak
 * array that is not a permutation gives an unspecified order; with
 * cfg.validate set it returns CG_EINVAL instead (synchronising the stream).
 */
enum { CG_TIE_ID = 0, CG_TIE_RANK = 1, CG_TIE_LAST_IN = 2 };
int cg_lexbfs_sweep_dense(cg_context *ctx, const cg_dense *g, int32_t kind, const int32_t *tiebreak, int32_t start,
                          int32_t *order, int32_t *pos, cudaStream_t stream);

/* The same sweep on a CSR graph (any n the CSR LexBFS takes).  The relabelled
 * copy (new rows renamed and sorted again on the GPU) takes workspace of
 * about 16 (n + 1) + 12 nnz bytes besides the CSR LexBFS state.  tiebreak,
 * start, order and pos as for cg_lexbfs_sweep_dense; cfg.validate also checks
 * the CSR layout. */
int cg_lexbfs_sweep_csr(cg_context *ctx, const cg_csr *g, int32_t kind, const int32_t *tiebreak, int32_t start,
                        int32_t *order, int32_t *pos, cudaStream_t stream);

/*
 * Perfect-elimination check of a caller-given order (Sections 5.2 and 6.2):
 * p(v) = the neighbour of v with the largest order index below v's, then
 * LN_v - {p(v)} ⊆ N(p(v)) for every v.  The order need not be a LexBFS
 * order; for a LexBFS order the verdict is the chordality verdict.
 *   order   device int32[n], a permutation of 0..n-1 (not checked unless
 *           cfg.validate)
 *   parent  device int32[n] (written: p(v) or -1) or NULL
 *   res     device cg_result (written)
 */
int cg_peo_check_dense(cg_context *ctx, const cg_dense *g, const int32_t *order, int32_t *parent,
                       cg_result *res, cudaStream_t stream);

/* The whole test on one dense graph: LexBFS, then the check (Sections 4.2,
 * 5.2-5.3, 6.1-6.2).  The search also records every vertex's parent p(v) and
 * the earlier-than masks; the check stages runs of rows in shared memory when
 * n <= 49152 and the rows are 16-byte aligned with words_per_row a multiple
 * of 4, else it reads them from global memory.
 *   res    device cg_result (written)
 *   order  device int32[n] (written) or NULL */
int cg_chordal_test_dense(cg_context *ctx, const cg_dense *g, cg_result *res, int32_t *order,
                          cudaStream_t stream);

/* The same test with HOST buffers: copies rows (n * words_per_row uint32,
 * preferably pinned) to the device, runs, copies the result (and the order
 * when host_order != NULL) back and synchronises the stream. */
int cg_chordal_test_dense_host(cg_context *ctx, int32_t n, int32_t words_per_row,
                               const uint32_t *host_rows, cg_result *host_res, int32_t *host_order,
                               cudaStream_t stream);

/*
 * Maximum Cardinality Search order of a dense graph (Section 5.1): each step
 * numbers an unnumbered vertex with the most numbered neighbours, the lowest
 * id among equals.  One CTA; per-vertex counts in shared memory (n <= 65520,
 * larger n: CG_EINVAL).  order device int32[n]; pos device int32[n] or NULL.
 */
int cg_mcs_order_dense(cg_context *ctx, const cg_dense *g, int32_t *order, int32_t *pos, cudaStream_t stream);

/* The chordality test with the MCS order (Theorem 5.2: G is chordal iff its
 * MCS order is a perfect elimination order) and the same check and witness
 * convention (the witness refers to the MCS order).  res device cg_result;
 * order device int32[n] or NULL. */
int cg_chordal_test_mcs_dense(cg_context *ctx, const cg_dense *g, cg_result *res, int32_t *order,
                              cudaStream_t stream);

/*
 * LexBFS order of a CSR graph (Section 4.2 in its O(N + M) form: each class a
 * list sorted by id, only the pivot's neighbours move).  One CTA walks the n
 * steps (warp 0; all its warps for rows longer than 32 neighbours) with the
 * partition state in the context workspace: 60 n bytes plus 8 bytes per
 * sort key slot (the next power of two >= n), 68-76 B per vertex.
 *   g      device CSR graph (sorted, symmetric, no loops; checked only when
 *          cfg.validate, which then synchronises the stream)
 *   order  device int32[n] (written);  pos  device int32[n] (written) or NULL
 */
int cg_lexbfs_order_csr(cg_context *ctx, const cg_csr *g, int32_t *order, int32_t *pos, cudaStream_t stream);

/* Perfect-elimination check of a caller-given order on a CSR graph (Sections
 * 5.2, 6.2): LN_v - {p(v)} ⊆ N(p(v)) by binary search in p's sorted row.
 *   order device int32[n] permutation; parent device int32[n] or NULL;
 *   res device cg_result */
int cg_peo_check_csr(cg_context *ctx, const cg_csr *g, const int32_t *order, int32_t *parent, cg_result *res,
                     cudaStream_t stream);

/* The whole test on one CSR graph.  res device cg_result; order device
 * int32[n] or NULL.  CSR graphs with n <= 131072 and at least 64 neighbours
 * per vertex on average (or n <= 4096) are expanded to bit rows in the
 * workspace (n * ceil(n/32) * 4 bytes more) and take the dense kernels, which
 * are faster there; the order and witness are the same (cg_lexbfs_order_csr
 * and cg_chordal_test_csr_host route the same way). */
int cg_chordal_test_csr(cg_context *ctx, const cg_csr *g, cg_result *res, int32_t *order, cudaStream_t stream);

/* The CSR test with HOST buffers (row_ptr int64[n+1], col int32[nnz]); copies
 * in, runs, copies the result (and order when non-NULL) out, synchronises. */
int cg_chordal_test_csr_host(cg_context *ctx, int32_t n, int64_t nnz, const int64_t *host_row_ptr,
                             const int32_t *host_col, cg_result *host_res, int32_t *host_order, cudaStream_t stream);

/*
 * Many dense graphs in one pass (the batching of independent tests): each
 * graph's LexBFS runs in its own CTA of one persistent launch, graphs handed
 * out largest first; the checks of all graphs share one grid.
 *   graphs         HOST array of `count` descriptors whose `rows` are device
 *                  pointers
 *   res            device cg_result[count] (written)
 *   orders         device int32[sum n] (written, graph k at order_offsets[k])
 *                  or NULL
 *   order_offsets  HOST int64[count] or NULL (then graphs are packed in
 *                  input order)
 */
int cg_chordal_test_batch(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *res,
                          int32_t *orders, const int64_t *order_offsets, cudaStream_t stream);

/*
 * The batched test from HOST buffers (the end-to-end form of
 * cg_chordal_test_batch): graph k's rows are host memory (n * words_per_row
 * uint32 each, preferably pinned); the library copies them into its
 * workspace (one asynchronous copy per graph on `stream`), runs the batch as
 * cg_chordal_test_batch does, copies the results back and synchronises the
 * stream.
 *   graphs       HOST array of `count` descriptors whose `rows` are HOST pointers
 *   host_res     HOST cg_result[count] (written)
 *   host_orders  HOST int32[sum n] (written, graphs packed in input order) or NULL
 * Paper context: Section 7 reports GPU times with and without the input's
 * transfer; this entry is the "with" form for many graphs at once.
 */
int cg_chordal_test_batch_host(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *host_res,
                               int32_t *host_orders, cudaStream_t stream);

/*
 * The dense test without any memory allocation (the paper has no counterpart;
 * this is a deployment aid).  For callers that cannot allocate device memory
 * when they call in — a plugin whose host application owns the device memory
 * and forbids allocations after start-up, a latency-critical loop that must
 * never wait in an allocator, or a caller that keeps no cg_context.  Same
 * kernels and results as cg_chordal_test_dense, but the scratch (positions,
 * parents, an order buffer when `order` is NULL, the witness key) comes from
 * one fixed array in the library's device image, about 193 KiB, held on every
 * GPU that loads the library until the process exits.
 *   g      device graph with n <= 16384 (larger n: CG_EINVAL, use
 *          cg_chordal_test_dense)
 *   res    device cg_result (written)
 *   order  device int32[n] (written) or NULL
 * Works on the current CUDA device.  All calls share the array and it keeps
 * the last call's contents (the witness key is reset by every call); calls
 * that overlap on the GPU race on it, so issue them on one stream.  The first
 * call on each device resolves the array's address (cudaGetSymbolAddress);
 * make that first call before any stream capture begins.  The address is
 * kept for the life of the process: it assumes the device's primary context
 * is never reset (after cudaDeviceReset, or under another context made
 * current on the same device, it would be stale).
 */
int cg_chordal_test_dense_noalloc(const cg_dense *g, cg_result *res, int32_t *order, cudaStream_t stream);

/*
 * Serving: a continuous-batching request queue (not part of the paper).
 * Queries arrive one at a time (cg_queue_submit returns at once with a
 * ticket); a worker thread owned by the queue admits pending queries in
 * arrival order — graphs with n <= 4096 and larger graphs in two separate
 * lanes, so short queries never wait behind long ones — into the next batch
 * while the batch fits the queue's device memory budget and one of its
 * `max_inflight` slots is free, launches each
 * batch on its slot's stream (so queries that arrive while others run
 * overlap with them on the GPU), and marks tickets done when the batch's
 * event completes.  Dense queries and CSR queries with n <= 131072 and at
 * least 64 neighbours per vertex on average (or n <= 4096) use the dense
 * kernels (CSR rows are expanded to bits on the device); sparser CSR queries
 * use the CSR kernels.  Results equal those of the single-graph entries.
 * The graph memory of a query must stay valid until its ticket completes.
 * While a queue runs, its context must not be used for autotuning.
 */
enum { CG_GRAPH_DENSE = 0, CG_GRAPH_CSR = 1 };
typedef struct {
    int32_t kind;     /* CG_GRAPH_DENSE or CG_GRAPH_CSR */
    cg_dense dense;   /* used when kind == CG_GRAPH_DENSE (device rows) */
    cg_csr csr;       /* used when kind == CG_GRAPH_CSR (device arrays) */
} cg_graph_ref;

typedef struct {
    int64_t mem_budget_bytes; /* device pool for in-flight batches (0: 4 GiB), allocated at creation */
    int32_t max_inflight;     /* concurrent batches / slot streams (0: 8) */
    int32_t max_batch;        /* queries per batch of graphs with n <= 4096 (0: 1024) */
    int32_t max_pending;      /* queued queries before submit returns CG_EAGAIN (0: 2^20) */
    int32_t max_batch_large;  /* queries per batch of larger graphs (0: 4) */
    int32_t keep_orders;      /* 1: keep each query's LexBFS order (host memory, n int32) until polled */
} cg_queue_config;

typedef struct {
    int64_t submitted, completed, pending, inflight, batches, pool_free_bytes;
} cg_queue_info;

typedef struct cg_queue cg_queue;

int cg_queue_create(cg_context *ctx, const cg_queue_config *cfg, cg_queue **out);
/* CG_EAGAIN when max_pending queries are waiting.  With the context's
 * cfg.validate set, a CSR query's layout is checked here (synchronising a
 * queue-owned stream) and a malformed one returns CG_EINVAL; without it,
 * CSR queries are trusted to be well formed (sorted, symmetric, in range). */
int cg_queue_submit(cg_queue *q, const cg_graph_ref *g, uint64_t *ticket);
/* CG_OK and the result (HOST memory) once done — the ticket is then
 * forgotten; CG_EAGAIN while pending.  order (nullable, HOST int32[n]) gets
 * the query's LexBFS order (Theorem 5.1: the order is part of the result);
 * it needs keep_orders, else CG_EINVAL.  latency_s (nullable) gets
 * submit-to-completion seconds (host steady clock).  A query that can never
 * run completes with the reason: CG_ENOMEM when it exceeds the memory
 * budget, or the status its batch layout failed with. */
int cg_queue_poll(cg_queue *q, uint64_t ticket, cg_result *host_res, int32_t *order, double *latency_s);
/* Waits until every submitted query completed; timeout_ns < 0 waits forever;
 * CG_ETIMEOUT when the time runs out (no GPU wait is involved). */
int cg_queue_drain(cg_queue *q, int64_t timeout_ns);
int cg_queue_stats(cg_queue *q, cg_queue_info *out);
/* Finishes queued work, stops the worker, frees the pool. */
int cg_queue_destroy(cg_queue *q);

/*
 * Per-phase timing (tracing aid; not part of the paper).  When enabled, each
 * call records CUDA events on the stream a phase runs on: around LexBFS
 * launches, around the check (check + finalize), around fused one-CTA
 * kernels, and around whole batch calls.  cg_profile_read waits for the
 * recorded events, returns the sums since the last read and resets them.
 */
typedef struct {
    double lexbfs_ms;        /* summed LexBFS-only kernel time (single graphs, large batch graphs) */
    double check_ms;         /* summed perfect-elimination check time (check + finalize launches) */
    double fused_ms;         /* summed time of one-CTA whole-test kernels (batch buckets) */
    double batch_ms;         /* summed time of whole batch calls / batch plan runs */
    int64_t lexbfs_launches;
    int64_t check_launches;
    int64_t fused_launches;
    int64_t batch_calls;
    int64_t kernel_launches; /* all kernels this library launched since the last read */
} cg_profile;

int cg_profile_enable(cg_context *ctx, int enable);
/* A batch as a reusable plan: the graphs' descriptors and the scratch are
 * uploaded once and the whole launch sequence (size buckets on forked
 * streams) is captured into a CUDA graph; each run replays it on `stream`.
 * The plan records the caller's device pointers (rows, res, orders): they
 * must stay valid, and their contents may change between runs.  Arguments as
 * for cg_chordal_test_batch. */
typedef struct cg_batch_plan cg_batch_plan;
int cg_batch_plan_create(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *res, int32_t *orders,
                         const int64_t *order_offsets, cg_batch_plan **out);
int cg_batch_plan_run(cg_batch_plan *plan, cudaStream_t stream);
int cg_batch_plan_destroy(cg_batch_plan *plan);

/* Autotuner of the batched path: for each size bucket of `graphs`
 * (n <= 16, 32, ..., 4096) times the one-CTA kernel with 64, 128, 256 and
 * 512 threads on `stream` (synchronising) and keeps the fastest in the
 * context.  cg_autotune_get / _set read or restore the table (slots 0..8,
 * 0 = size rule) so callers can persist it. */
int cg_batch_autotune(cg_context *ctx, const cg_dense *graphs, int32_t count, cudaStream_t stream);
int cg_autotune_get(cg_context *ctx, int32_t *threads, int32_t slots);
int cg_autotune_set(cg_context *ctx, const int32_t *threads, int32_t slots);
int cg_profile_read(cg_context *ctx, cg_profile *out);

/*
 * Bounds-checking build (compiled with -DCG_BOUNDS_CHECK into
 * libchordal_debug.so; a debugging aid, not part of the paper): the state
 * arrays of the dense and CSR searches and the check's indices are checked;
 * an out-of-range index is recorded (array code << 56 | index) in a device
 * error word and redirected to a scratch element instead of going out of
 * bounds, and the launching entry point synchronises and returns CG_ECUDA
 * with the description (cg_last_error_string).  cg_version() names the build.
 *   cg_debug_describe  the description of an error word (any build)
 *   cg_debug_inject    makes the next dense LexBFS launch record code (1..255)
 *                      without any out-of-range access, to test the error
 *                      path; CG_EINVAL in the release build
 */
int cg_debug_describe(uint64_t word, char *buf, int32_t len);
int cg_debug_inject(int32_t code);

/*
 * Latency floors of one step of the sequential LexBFS loop (measurement aid,
 * not part of the paper; Section 6.1 runs n dependent steps, so a step's
 * fixed costs bound the whole order).  Synchronises `stream`; allocates and
 * frees its own scratch.
 *   threads      CTA size of the barrier loop, a multiple of 32 in [32, 1024]
 *   iters        barrier-loop iterations, [1, 2^24]; each is two CTA-wide
 *                barriers, the dense step's fixed synchronisation
 *   chain_bytes  footprint of the load chain, [256, 2^32] bytes (rounded down
 *                to a power of two of 128-byte lines): one node per line, in
 *                a scattered single cycle; within L2 (129 MB) every load is an
 *                L2 round trip, far above it mostly a DRAM round trip
 *   loads        dependent loads one thread follows, [1, 2^24]
 * Each time is the best of three, minus the same launch with no work.
 * CG_EINVAL on an argument out of range, CG_ENOMEM / CG_ECUDA otherwise.
 */
typedef struct {
    double barrier_pair_ns;  /* one iteration of two CTA-wide barriers */
    double load_ns;          /* one dependent load (L1 bypassed) */
    int64_t chain_bytes;     /* the chain's footprint after rounding */
} cg_step_floor_info;
int cg_step_floor(cg_context *ctx, int32_t threads, int32_t iters, int64_t chain_bytes, int32_t loads,
                  cudaStream_t stream, cg_step_floor_info *out);

#ifdef __cplusplus
}
#endif
#endif /* CHORDAL_GB300_H */
