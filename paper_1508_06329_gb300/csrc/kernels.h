// kernels.h — host-side launchers shared between the libchordal sources.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cg {

// ---- dense LexBFS (lexbfs_dense.cu)
struct LexPlan {
    int threads;        // CTA size
    bool rows_smem;     // adjacency copied into shared memory
    bool wide_ids;      // 32-bit ids, state in a global workspace
    int split_state;    // 16-bit ids, class ids in shared memory, class arrays partly in a global
                        // workspace: 0 no, else the split layout 2, 3 or 5 (lexbfs_dense.cuh)
    size_t smem_bytes;  // dynamic shared memory per CTA
    size_t gstate_bytes;// global state bytes per CTA (0: none)
    int n_max;          // the largest graph the plan was made for
};

// Picks the kernel variant for graphs of at most n_max vertices.
// threads_override = 0 lets the size rule decide.
int lexbfs_dense_plan(int n_max, int threads_override, LexPlan *plan);

// Runs LexBFS for `count` graphs, one CTA each (grid = min(count, ctas)).
// descs: device array, or nullptr to use `single` (count must be 1).
// work_counter: device int, zeroed by the launcher (dynamic graph hand-out).
// parent (packed by vbase) receives parents when non-null: parent_mode
// kParentMoves records p(v) for every vertex (a store per moved vertex),
// kParentPivots one value per step by position, parent[i] = p(order[i]), or
// kParentUnresolved for the pivots chosen by a class scan.  keys (nullable)
// is set, on the stream after the search, to the check's initial keys:
// keys[0..count) = "no violation", keys[count] = keys[count + 1] = 0.
// emask (nullable): the search also writes each graph's earlier-than masks
// E_b (b >= 1; row b at emask + ebase + b * mask_stride(n): the vertices
// numbered before step 32 b), which the staged check reads.  cpar
// (nullable; n ints per graph at vbase, scratch) makes kParentPivots exact:
// no kParentUnresolved is left.
int lexbfs_dense_launch(const LexPlan &plan, const DenseDesc *descs, DenseDesc single, int count, int ctas,
                        int32_t *order, int32_t *pos, int32_t *parent, void *gstate, int *work_counter,
                        cudaStream_t stream, int parent_mode = 0, unsigned long long *keys = nullptr,
                        uint32_t *emask = nullptr, int32_t *cpar = nullptr);

// Bounds-checking build: the next dense LexBFS launch records `code` (a test
// of the error path); CG_EINVAL in the release build.
int debug_inject(unsigned code);

// ---- dense perfect-elimination check (peo_dense.cu)
// keys: device u64[count], set to ~0 by the launcher.
// parent_known: parent[] already holds p(v) (from the search); otherwise the
// kernel computes it from the rows and writes it.
// emask: workspace for the graphs' earlier-than masks (earlier_mask_words(n)
// words at each desc's ebase; n_max = the largest n), or null for the
// gather-based check.  prefilled (with masks, parent_known false): parent
// already holds p(v) or kParentUnresolved for each v (from the search).
// res: when given, the results are written too (keys then needs count + 1
// entries: the last counts the check's finished blocks); otherwise the
// caller runs finalize_launch.
int peo_dense_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                     const int32_t *order, const int32_t *pos, int32_t *parent, bool parent_known,
                     unsigned long long *keys, int num_sms, cudaStream_t stream, uint32_t *emask = nullptr,
                     int n_max = 0, bool prefilled = false, cg_result *res = nullptr);
int64_t earlier_mask_words(int n);

// The check of orders the dense LexBFS produced under kParentPivots (parents
// by position in ppos, keys initialised by the search), in one launch: one
// block per group of 32 positions (grid ceil(n_max / 32) x count) builds E_b
// in shared memory from pos, resolves the group's open parents (stored back
// into ppos) and checks its positions; its last block writes res.  vec when
// every graph passes peo_rows_vec_ok (rows 16-byte aligned, words_per_row a
// multiple of 4: 128-bit row loads).  A result with chordal = -1 reports a
// check that could not complete (an order or parent value outside 0..n-1).
bool peo_rows_vec_ok(const DenseDesc &d);
int peo_unit_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, bool vec, const int32_t *order,
                    const int32_t *pos, int32_t *ppos, unsigned long long *keys, cg_result *res, cudaStream_t stream);
// The same check with the rows staged in shared memory: persistent blocks
// stage runs of 16 or 32 positions (their rows, the rows of the positions
// just before, and E_b, which the search wrote: lexbfs_dense_launch's emask)
// with bulk copies into two alternating buffers and test row_v & ~row_p & E_b
// there.  Needs peo_stage_ok for every graph (rows suited to bulk copies,
// n <= kStageMaxN), exact parents in ppos (the search's cpar) and the masks
// at each desc's ebase.
constexpr int kStageMaxN = 49152;
bool peo_stage_ok(const DenseDesc &d);
int peo_stage_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, const int32_t *order,
                     int32_t *ppos, const uint32_t *emask, unsigned long long *keys, cg_result *res, int num_sms,
                     cudaStream_t stream);
// sets *flag when order is not a permutation of 0..n-1 (seen: n ints of scratch)
int order_check_launch(int n, const int32_t *order, int *seen, int *flag, int num_sms, cudaStream_t stream);

// pos[order[i]] = i for every graph (order values outside 0..n-1 are skipped).
int invert_order_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                        const int32_t *order, int32_t *pos, int num_sms, cudaStream_t stream);

int finalize_launch(const DenseDesc *descs, DenseDesc single, int count, const unsigned long long *keys,
                    const int32_t *order, const int32_t *parent, cg_result *res, cudaStream_t stream);

// ---- fused small-graph test, one CTA per graph (batch_dense.cu)
constexpr int kFusedMaxN = 4096;
constexpr size_t kFusedSmemLimit = 227 * 1024 - 64;
struct FusedPlan {
    int threads;
    bool rows_smem;
    size_t smem_bytes;
};
// threads = 0 picks by size; otherwise 64, 128, 256 or 512.  The rows are
// copied to shared memory when they fit and rows_smem_allowed.
int fused_dense_plan(int n_max, int threads, FusedPlan *plan, bool rows_smem_allowed = true);
int fused_dense_launch(const FusedPlan &plan, const DenseDesc *descs, int count, int ctas, int32_t *order,
                       int32_t *pos, int32_t *parent, cg_result *res, int *work_counter, cudaStream_t stream);
int fused_ctas_per_sm(const FusedPlan &plan);

// ---- one multi-sweep LexBFS sweep on a dense graph (sweep_dense.cu)
struct SweepBuffers {
    uint32_t *prow;     // relabelled matrix, n * ceil(n/32) words
    int32_t *rankv;     // n each below
    int32_t *newid;
    int32_t *inv;
    int *seen;
    int32_t *order_p;
    int32_t *pos_p;
    int *flag;          // 1 int: set when the tie-break array is not a permutation
};
// new ids from the tie-break array (sets *sb.flag if it is not a permutation)
int sweep_ids_launch(int n, int kind, const int32_t *tiebreak, int start, const SweepBuffers &sb, int num_sms,
                     cudaStream_t stream);
// order[i] = inv[order_p[i]], pos[v] = pos_p[newid[v]]
int sweep_unpermute_launch(int n, const SweepBuffers &sb, int32_t *order, int32_t *pos, int num_sms,
                           cudaStream_t stream);
// ---- the CSR sweep's relabelled copy (sweep_csr.cu): rows renamed by newid and sorted
size_t sweep_csr_workspace_bytes(int64_t n, int64_t nnz);
int sweep_csr_relabel_launch(int n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const SweepBuffers &sb,
                             void *ws, int64_t **rp_new, int32_t **col_new, int num_sms, cudaStream_t stream);
// relabelled matrix, LexBFS on it, order / pos mapped back
int sweep_order_launch(const DenseDesc &d, const LexPlan &plan, void *gstate, int *counter, const SweepBuffers &sb,
                       int32_t *order, int32_t *pos, int num_sms, cudaStream_t stream);

// ---- dense MCS (mcs_dense.cu): one CTA per graph, n <= 65520
int mcs_dense_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, int ctas, int32_t *order,
                     int32_t *pos, int *work_counter, cudaStream_t stream);

// ---- CSR LexBFS (lexbfs_csr.cu): one CTA per graph (warp 0 walks the steps), state in `ws`
size_t lexbfs_csr_workspace_bytes(int64_t n, int64_t max_deg);
int lexbfs_csr_launch(int n, int64_t max_deg, const int64_t *row_ptr, const int32_t *col, int64_t nnz, int32_t *order,
                      int32_t *pos, int32_t *parent, void *ws, int num_sms, cudaStream_t stream);

// ---- CSR check (peo_csr.cu)
int peo_csr_launch(int n, const int64_t *row_ptr, const int32_t *col, const int32_t *order, const int32_t *pos,
                   int32_t *parent, bool parent_known, unsigned long long *key, int num_sms, cudaStream_t stream);
// CSR graphs as bit rows: rows (n * words, words >= ceil(n/32)) are zeroed,
// then each vertex's neighbours are OR-ed into its row (one warp per vertex).
int csr_to_bits_launch(int n, const int64_t *row_ptr, const int32_t *col, uint32_t *rows, int words, int num_sms,
                       cudaStream_t stream);
// CSR graphs dense enough for the dense kernels: n <= kCsrDenseMaxN and at
// least 64 neighbours per vertex on average (or n <= 4096); the single-graph
// CSR entries and the serving queue expand these to bit rows first.
constexpr int kCsrDenseMaxN = 131072;
bool csr_takes_dense_path(int n, int64_t nnz);
// flag (device int) receives an OR of layout violations, 0 when the CSR is well formed.
int validate_csr_launch(int n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, int *flag, int num_sms,
                        cudaStream_t stream);

}  // namespace cg
