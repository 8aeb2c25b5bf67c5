// capi.cu — the extern "C" entry points of libchordal.so (declared in
// include/chordal.h): argument checks, workspace management, launch order.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"

namespace cg {

namespace {
thread_local char g_err[512] = {0};
}

int set_error(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

}  // namespace cg

using namespace cg;

struct cg_context {
    cg_config cfg{};
    int num_sms = 0;
    void *ws = nullptr;          // device workspace
    size_t ws_bytes = 0;
    void *pinned = nullptr;      // pinned host staging for descriptor uploads
    size_t pinned_bytes = 0;
    cudaEvent_t staged{};        // recorded after each staging upload
    bool staged_pending = false;
    // per-phase timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_lex, ev_check;
    int64_t launches = 0;
};

namespace {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Offsets into one workspace allocation.
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = align_up(off, kAlign);
        const size_t o = off;
        off += std::max<size_t>(count, 1) * sizeof(T);
        return o;
    }
};

template <typename T>
T *at(cg_context *ctx, size_t off) {
    return reinterpret_cast<T *>(static_cast<unsigned char *>(ctx->ws) + off);
}

int ensure_ws(cg_context *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return CG_OK;
    // earlier launches may still read the old buffer
    CG_CUDA_TRY(cudaDeviceSynchronize());
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = align_up(std::max(bytes, (size_t)1 << 20), 1 << 20);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return set_error(CG_ENOMEM, "workspace allocation of %zu bytes failed", want);
    }
    ctx->ws_bytes = want;
    return CG_OK;
}

int ensure_pinned(cg_context *ctx, size_t bytes) {
    if (ctx->staged_pending) {
        CG_CUDA_TRY(cudaEventSynchronize(ctx->staged));
        ctx->staged_pending = false;
    }
    if (bytes <= ctx->pinned_bytes) return CG_OK;
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    const size_t want = align_up(std::max(bytes, (size_t)1 << 16), 1 << 16);
    if (cudaMallocHost(&ctx->pinned, want) != cudaSuccess) {
        cudaGetLastError();
        return set_error(CG_ENOMEM, "pinned staging allocation of %zu bytes failed", want);
    }
    ctx->pinned_bytes = want;
    return CG_OK;
}

cudaEvent_t take_event(cg_context *ctx) {
    if (!ctx->ev_free.empty()) {
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e{};
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Brackets one phase with events when profiling is on.
struct PhaseTimer {
    cg_context *ctx;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *list;
    cudaStream_t stream;
    cudaEvent_t a = nullptr;
    PhaseTimer(cg_context *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *l, cudaStream_t s)
        : ctx(c), list(l), stream(s) {
        if (ctx->profiling && (a = take_event(ctx))) cudaEventRecord(a, stream);
    }
    void stop() {
        if (!a) return;
        cudaEvent_t b = take_event(ctx);
        if (b) {
            cudaEventRecord(b, stream);
            list->emplace_back(a, b);
        } else {
            ctx->ev_free.push_back(a);
        }
        a = nullptr;
    }
    ~PhaseTimer() { stop(); }
};

int check_ctx(cg_context *ctx) {
    if (!ctx) return set_error(CG_EINVAL, "null context");
    CG_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
    return CG_OK;
}

int check_dense(const cg_dense *g) {
    if (!g) return set_error(CG_EINVAL, "null graph descriptor");
    if (g->n < 0) return set_error(CG_EINVAL, "n must be >= 0 (got %d)", g->n);
    if (g->n > 0 && !g->rows) return set_error(CG_EINVAL, "null rows pointer");
    if (g->words_per_row < (g->n + 31) / 32)
        return set_error(CG_EINVAL, "words_per_row %d < ceil(n/32) = %d", g->words_per_row, (g->n + 31) / 32);
    return CG_OK;
}

int check_csr(const cg_csr *g) {
    if (!g) return set_error(CG_EINVAL, "null graph descriptor");
    if (g->n < 0) return set_error(CG_EINVAL, "n must be >= 0 (got %d)", g->n);
    if (g->nnz < 0) return set_error(CG_EINVAL, "nnz must be >= 0");
    if (g->n > 0 && !g->row_ptr) return set_error(CG_EINVAL, "null row_ptr");
    if (g->nnz > 0 && !g->col) return set_error(CG_EINVAL, "null col");
    return CG_OK;
}

DenseDesc desc_of(const cg_dense *g, int64_t vbase, int64_t obase) {
    DenseDesc d;
    d.rows = g->rows;
    d.n = g->n;
    d.words = g->words_per_row;
    d.vbase = vbase;
    d.obase = obase;
    return d;
}

// LexBFS and (optionally) the check for one graph given by value.
int run_single_dense(cg_context *ctx, const cg_dense *g, int32_t *order_out, int32_t *pos_out, cg_result *res,
                     int32_t *parent_out, cudaStream_t stream) {
    const int n = g->n;
    LexPlan plan;
    int rc = lexbfs_dense_plan(n, ctx->cfg.threads_override, &plan);
    if (rc) return rc;
    Carve cv;
    const size_t o_order = cv.take<int32_t>(n);
    const size_t o_pos = cv.take<int32_t>(n);
    const size_t o_parent = cv.take<int32_t>(n);
    const size_t o_key = cv.take<unsigned long long>(1);
    const size_t o_counter = cv.take<int>(1);
    const size_t o_gstate = cv.take<unsigned char>(plan.wide_ids ? plan.gstate_bytes : 0);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    int32_t *order = order_out ? order_out : at<int32_t>(ctx, o_order);
    int32_t *pos = pos_out ? pos_out : at<int32_t>(ctx, o_pos);
    int32_t *parent = parent_out ? parent_out : at<int32_t>(ctx, o_parent);
    const DenseDesc d = desc_of(g, 0, 0);
    if (n > 0) {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        rc = lexbfs_dense_launch(plan, nullptr, d, 1, 1, order, pos, res ? parent : nullptr,
                                 plan.wide_ids ? at<void>(ctx, o_gstate) : nullptr, at<int>(ctx, o_counter), stream);
        if (rc) return rc;
        ctx->launches += 1;
    }
    if (!res) return CG_OK;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    if ((rc = peo_dense_launch(nullptr, d, 1, nullptr, n, order, pos, parent, true, key, ctx->num_sms, stream)))
        return rc;
    ctx->launches += n > 0 ? 2 : 1;
    return finalize_launch(nullptr, d, 1, key, order, parent, res, stream);
}

// Optional layout check of a CSR graph (synchronises the stream).
int validate_csr(cg_context *ctx, const cg_csr *g, int *flag_dev, cudaStream_t stream) {
    int rc;
    if ((rc = validate_csr_launch(g->n, g->nnz, g->row_ptr, g->col, flag_dev, ctx->num_sms, stream))) return rc;
    int flag = 0;
    CG_CUDA_TRY(cudaMemcpyAsync(&flag, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CG_CUDA_TRY(cudaStreamSynchronize(stream));
    if (flag)
        return set_error(CG_EINVAL, "CSR layout check failed (flags 0x%x: 1 row_ptr, 2 range, 4 unsorted/duplicate, "
                                    "8 self-loop, 16 not symmetric)", flag);
    return CG_OK;
}

// LexBFS and (optionally) the check for one CSR graph.
int run_single_csr(cg_context *ctx, const cg_csr *g, int32_t *order_out, int32_t *pos_out, cg_result *res,
                   cudaStream_t stream) {
    const int n = g->n;
    Carve cv;
    const size_t o_order = cv.take<int32_t>(n);
    const size_t o_pos = cv.take<int32_t>(n);
    const size_t o_parent = cv.take<int32_t>(n);
    const size_t o_key = cv.take<unsigned long long>(1);
    const size_t o_flag = cv.take<int>(1);
    const size_t o_state = cv.take<unsigned char>(lexbfs_csr_workspace_bytes(n, n));
    int rc;
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    if (ctx->cfg.validate && (rc = validate_csr(ctx, g, at<int>(ctx, o_flag), stream))) return rc;
    int32_t *order = order_out ? order_out : at<int32_t>(ctx, o_order);
    int32_t *pos = pos_out ? pos_out : at<int32_t>(ctx, o_pos);
    int32_t *parent = at<int32_t>(ctx, o_parent);
    if (n > 0) {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        if ((rc = lexbfs_csr_launch(n, n, g->row_ptr, g->col, order, pos, parent, at<void>(ctx, o_state),
                                    ctx->num_sms, stream)))
            return rc;
        ctx->launches += 2;
    }
    if (!res) return CG_OK;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    if ((rc = peo_csr_launch(n, g->row_ptr, g->col, order, pos, parent, true, key, ctx->num_sms, stream))) return rc;
    DenseDesc d{};
    d.n = n;
    ctx->launches += n > 0 ? 2 : 1;
    return finalize_launch(nullptr, d, 1, key, order, parent, res, stream);
}

}  // namespace

extern "C" {

const char *cg_version(void) { return "chordal-gb300 0.1.0 (sm_103a)"; }

const char *cg_last_error_string(void) { return cg::g_err; }

int cg_context_create(const cg_config *cfg, cg_context **out) {
    if (!out) return set_error(CG_EINVAL, "null output pointer");
    *out = nullptr;
    cg_context *ctx = new (std::nothrow) cg_context();
    if (!ctx) return set_error(CG_ENOMEM, "context allocation failed");
    if (cfg) ctx->cfg = *cfg;
    if (ctx->cfg.threads_override && ctx->cfg.threads_override != 128 && ctx->cfg.threads_override != 256 &&
        ctx->cfg.threads_override != 512 && ctx->cfg.threads_override != 1024) {
        delete ctx;
        return set_error(CG_EINVAL, "threads_override must be 0, 128, 256, 512 or 1024");
    }
    cudaError_t e = cudaSetDevice(ctx->cfg.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->cfg.device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete ctx;
        return set_error(CG_ECUDA, "context creation on device %d failed: %s", cfg ? cfg->device : 0,
                         cudaGetErrorString(e));
    }
    *out = ctx;
    return CG_OK;
}

int cg_profile_enable(cg_context *ctx, int enable) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    ctx->profiling = enable != 0;
    return CG_OK;
}

int cg_profile_read(cg_context *ctx, cg_profile *out) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!out) return set_error(CG_EINVAL, "null profile pointer");
    cg_profile p{};
    for (int phase = 0; phase < 2; ++phase) {
        auto &list = phase == 0 ? ctx->ev_lex : ctx->ev_check;
        double sum = 0;
        for (auto &ab : list) {
            CG_CUDA_TRY(cudaEventSynchronize(ab.second));
            float ms = 0.f;
            CG_CUDA_TRY(cudaEventElapsedTime(&ms, ab.first, ab.second));
            sum += ms;
            ctx->ev_free.push_back(ab.first);
            ctx->ev_free.push_back(ab.second);
        }
        (phase == 0 ? p.lexbfs_ms : p.check_ms) = sum;
        (phase == 0 ? p.lexbfs_launches : p.check_launches) = (int64_t)list.size();
        list.clear();
    }
    p.kernel_launches = ctx->launches;
    ctx->launches = 0;
    *out = p;
    return CG_OK;
}

int cg_context_destroy(cg_context *ctx) {
    if (!ctx) return CG_OK;
    cudaSetDevice(ctx->cfg.device);
    cudaDeviceSynchronize();
    for (auto &ab : ctx->ev_lex) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
    for (auto &ab : ctx->ev_check) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    cudaEventDestroy(ctx->staged);
    delete ctx;
    return CG_OK;
}

int cg_lexbfs_order_dense(cg_context *ctx, const cg_dense *g, int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    return run_single_dense(ctx, g, order, pos, nullptr, nullptr, stream);
}

int cg_chordal_test_dense(cg_context *ctx, const cg_dense *g, cg_result *res, int32_t *order, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    return run_single_dense(ctx, g, order, nullptr, res, nullptr, stream);
}

int cg_peo_check_dense(cg_context *ctx, const cg_dense *g, const int32_t *order, int32_t *parent, cg_result *res,
                       cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    const int n = g->n;
    Carve cv;
    const size_t o_pos = cv.take<int32_t>(n);
    const size_t o_parent = cv.take<int32_t>(n);
    const size_t o_key = cv.take<unsigned long long>(1);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    int32_t *pos = at<int32_t>(ctx, o_pos);
    int32_t *par = parent ? parent : at<int32_t>(ctx, o_parent);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    const DenseDesc d = desc_of(g, 0, 0);
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    if ((rc = invert_order_launch(nullptr, d, 1, nullptr, n, order, pos, ctx->num_sms, stream))) return rc;
    if ((rc = peo_dense_launch(nullptr, d, 1, nullptr, n, order, pos, par, false, key, ctx->num_sms, stream)))
        return rc;
    ctx->launches += n > 0 ? 3 : 1;
    return finalize_launch(nullptr, d, 1, key, order, par, res, stream);
}

int cg_chordal_test_dense_host(cg_context *ctx, int32_t n, int32_t words_per_row, const uint32_t *host_rows,
                               cg_result *host_res, int32_t *host_order, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!host_res) return set_error(CG_EINVAL, "null host result pointer");
    cg_dense probe{n, words_per_row, host_rows};
    if ((rc = check_dense(&probe))) return rc;
    LexPlan plan;
    if ((rc = lexbfs_dense_plan(n, ctx->cfg.threads_override, &plan))) return rc;
    // device copies of the inputs and outputs live past the scratch used by run_single_dense
    Carve cv;
    cv.take<int32_t>(n);
    cv.take<int32_t>(n);
    cv.take<int32_t>(n);
    cv.take<unsigned long long>(1);
    cv.take<int>(1);
    cv.take<unsigned char>(plan.wide_ids ? plan.gstate_bytes : 0);
    const size_t bytes_rows = (size_t)n * words_per_row * sizeof(uint32_t);
    const size_t o_rows = cv.take<unsigned char>(bytes_rows);
    const size_t o_res = cv.take<cg_result>(1);
    const size_t o_order = cv.take<int32_t>(n);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    uint32_t *rows = at<uint32_t>(ctx, o_rows);
    cg_result *res = at<cg_result>(ctx, o_res);
    int32_t *order = at<int32_t>(ctx, o_order);
    if (bytes_rows) CG_CUDA_TRY(cudaMemcpyAsync(rows, host_rows, bytes_rows, cudaMemcpyHostToDevice, stream));
    cg_dense g{n, words_per_row, rows};
    if ((rc = run_single_dense(ctx, &g, order, nullptr, res, nullptr, stream))) return rc;
    CG_CUDA_TRY(cudaMemcpyAsync(host_res, res, sizeof(cg_result), cudaMemcpyDeviceToHost, stream));
    if (host_order && n > 0)
        CG_CUDA_TRY(cudaMemcpyAsync(host_order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, stream));
    CG_CUDA_TRY(cudaStreamSynchronize(stream));
    return CG_OK;
}

int cg_lexbfs_order_csr(cg_context *ctx, const cg_csr *g, int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_csr(g))) return rc;
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    return run_single_csr(ctx, g, order, pos, nullptr, stream);
}

int cg_chordal_test_csr(cg_context *ctx, const cg_csr *g, cg_result *res, int32_t *order, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_csr(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    return run_single_csr(ctx, g, order, nullptr, res, stream);
}

int cg_peo_check_csr(cg_context *ctx, const cg_csr *g, const int32_t *order, int32_t *parent, cg_result *res,
                     cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_csr(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    const int n = g->n;
    Carve cv;
    const size_t o_pos = cv.take<int32_t>(n);
    const size_t o_parent = cv.take<int32_t>(n);
    const size_t o_key = cv.take<unsigned long long>(1);
    const size_t o_flag = cv.take<int>(1);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    if (ctx->cfg.validate && (rc = validate_csr(ctx, g, at<int>(ctx, o_flag), stream))) return rc;
    int32_t *pos = at<int32_t>(ctx, o_pos);
    int32_t *par = parent ? parent : at<int32_t>(ctx, o_parent);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    DenseDesc d{};
    d.n = n;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    if ((rc = invert_order_launch(nullptr, d, 1, nullptr, n, order, pos, ctx->num_sms, stream))) return rc;
    if ((rc = peo_csr_launch(n, g->row_ptr, g->col, order, pos, par, false, key, ctx->num_sms, stream))) return rc;
    ctx->launches += n > 0 ? 3 : 1;
    return finalize_launch(nullptr, d, 1, key, order, par, res, stream);
}

int cg_chordal_test_csr_host(cg_context *ctx, int32_t n, int64_t nnz, const int64_t *host_row_ptr,
                             const int32_t *host_col, cg_result *host_res, int32_t *host_order, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!host_res) return set_error(CG_EINVAL, "null host result pointer");
    cg_csr probe{n, nnz, host_row_ptr, host_col};
    if ((rc = check_csr(&probe))) return rc;
    // inputs and outputs sit after the scratch that run_single_csr carves
    Carve cv;
    cv.take<int32_t>(n);
    cv.take<int32_t>(n);
    cv.take<int32_t>(n);
    cv.take<unsigned long long>(1);
    cv.take<int>(1);
    cv.take<unsigned char>(lexbfs_csr_workspace_bytes(n, n));
    const size_t o_rp = cv.take<int64_t>((size_t)n + 1);
    const size_t o_col = cv.take<int32_t>((size_t)nnz);
    const size_t o_res = cv.take<cg_result>(1);
    const size_t o_order = cv.take<int32_t>(n);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    int64_t *rp = at<int64_t>(ctx, o_rp);
    int32_t *col = at<int32_t>(ctx, o_col);
    if (n >= 0)
        CG_CUDA_TRY(cudaMemcpyAsync(rp, host_row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, stream));
    if (nnz > 0) CG_CUDA_TRY(cudaMemcpyAsync(col, host_col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, stream));
    cg_csr g{n, nnz, rp, col};
    cg_result *res = at<cg_result>(ctx, o_res);
    int32_t *order = at<int32_t>(ctx, o_order);
    if ((rc = run_single_csr(ctx, &g, order, nullptr, res, stream))) return rc;
    CG_CUDA_TRY(cudaMemcpyAsync(host_res, res, sizeof(cg_result), cudaMemcpyDeviceToHost, stream));
    if (host_order && n > 0)
        CG_CUDA_TRY(cudaMemcpyAsync(host_order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, stream));
    CG_CUDA_TRY(cudaStreamSynchronize(stream));
    return CG_OK;
}

int cg_chordal_test_batch(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *res, int32_t *orders,
                          const int64_t *order_offsets, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (count < 0) return set_error(CG_EINVAL, "count must be >= 0");
    if (count == 0) return CG_OK;
    if (!graphs || !res) return set_error(CG_EINVAL, "null graphs or result pointer");
    std::vector<DenseDesc> descs(count);
    std::vector<int64_t> voff(count + 1);
    int64_t total = 0;
    int n_max = 0;
    for (int k = 0; k < count; ++k) {
        if ((rc = check_dense(&graphs[k]))) return set_error(rc, "graph %d: %s", k, cg_last_error_string());
        voff[k] = total;
        const int64_t ob = order_offsets ? order_offsets[k] : total;
        if (ob < 0) return set_error(CG_EINVAL, "graph %d: negative order offset", k);
        descs[k] = desc_of(&graphs[k], total, ob);
        total += graphs[k].n;
        n_max = std::max(n_max, graphs[k].n);
    }
    voff[count] = total;
    LexPlan plan;
    if ((rc = lexbfs_dense_plan(n_max, ctx->cfg.threads_override, &plan))) return rc;
    // resident CTAs: shared memory and threads per SM bound the co-resident count
    const int by_smem = plan.smem_bytes ? (int)std::max<size_t>(1, (228 * 1024) / (plan.smem_bytes + 1024)) : 32;
    const int by_threads = std::max(1, 2048 / plan.threads);
    const int ctas = std::max(1, std::min(count, ctx->num_sms * std::min(by_smem, by_threads)));
    Carve cv;
    const size_t o_desc = cv.take<DenseDesc>(count);
    const size_t o_voff = cv.take<int64_t>(count + 1);
    const size_t o_order = cv.take<int32_t>(orders ? 0 : total);
    const size_t o_pos = cv.take<int32_t>(total);
    const size_t o_parent = cv.take<int32_t>(total);
    const size_t o_keys = cv.take<unsigned long long>(count);
    const size_t o_counter = cv.take<int>(1);
    const size_t o_gstate = cv.take<unsigned char>(plan.wide_ids ? plan.gstate_bytes * (size_t)ctas : 0);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    // stage descriptors + offsets in pinned memory, one upload
    const size_t bytes_desc = sizeof(DenseDesc) * count, bytes_voff = sizeof(int64_t) * (count + 1);
    if ((rc = ensure_pinned(ctx, bytes_desc + bytes_voff + 64))) return rc;
    unsigned char *hp = static_cast<unsigned char *>(ctx->pinned);
    std::memcpy(hp, descs.data(), bytes_desc);
    std::memcpy(hp + align_up(bytes_desc, 16), voff.data(), bytes_voff);
    CG_CUDA_TRY(cudaMemcpyAsync(at<void>(ctx, o_desc), hp, bytes_desc, cudaMemcpyHostToDevice, stream));
    CG_CUDA_TRY(cudaMemcpyAsync(at<void>(ctx, o_voff), hp + align_up(bytes_desc, 16), bytes_voff,
                                cudaMemcpyHostToDevice, stream));
    CG_CUDA_TRY(cudaEventRecord(ctx->staged, stream));
    ctx->staged_pending = true;
    const DenseDesc *ddesc = at<DenseDesc>(ctx, o_desc);
    const int64_t *dvoff = at<int64_t>(ctx, o_voff);
    int32_t *order = orders ? orders : at<int32_t>(ctx, o_order);
    int32_t *pos = at<int32_t>(ctx, o_pos);
    int32_t *parent = at<int32_t>(ctx, o_parent);
    unsigned long long *keys = at<unsigned long long>(ctx, o_keys);
    const DenseDesc none{};
    {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        if ((rc = lexbfs_dense_launch(plan, ddesc, none, count, ctas, order, pos, parent,
                                      plan.wide_ids ? at<void>(ctx, o_gstate) : nullptr, at<int>(ctx, o_counter),
                                      stream)))
            return rc;
        ctx->launches += 1;
    }
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    if ((rc = peo_dense_launch(ddesc, none, count, dvoff, total, order, pos, parent, true, keys, ctx->num_sms,
                               stream)))
        return rc;
    ctx->launches += total > 0 ? 2 : 1;
    return finalize_launch(ddesc, none, count, keys, order, parent, res, stream);
}

}  // extern "C"
