// capi.cu — the extern "C" entry points of libchordal.so (declared in
// include/chordal.h): argument checks, workspace management, launch order.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "host.h"

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

const char *cg_debug_array_name(unsigned code) {
    switch (code) {
        case kChkCls: return "dense LexBFS cls";
        case kChkChild: return "dense LexBFS child";
        case kChkFree: return "dense LexBFS free stack";
        case kChkCnext: return "dense LexBFS class next";
        case kChkCprev: return "dense LexBFS class prev";
        case kChkSize: return "dense LexBFS class size";
        case kChkNumbered: return "dense LexBFS numbered mask";
        case kChkRow: return "dense LexBFS pivot row";
        case kChkMoved: return "dense LexBFS moved counts";
        case kChkCsrCls: return "CSR LexBFS cls";
        case kChkCsrVnext: return "CSR LexBFS vnext";
        case kChkCsrVprev: return "CSR LexBFS vprev";
        case kChkCsrCnext: return "CSR LexBFS class next";
        case kChkCsrCprev: return "CSR LexBFS class prev";
        case kChkCsrCfirst: return "CSR LexBFS class first";
        case kChkCsrClast: return "CSR LexBFS class last";
        case kChkCsrCsize: return "CSR LexBFS class size";
        case kChkCsrCmoved: return "CSR LexBFS class moved";
        case kChkCsrCchild: return "CSR LexBFS class child";
        case kChkCsrFree: return "CSR LexBFS free stack";
        case kChkCsrSy: return "CSR LexBFS long-row vertices";
        case kChkCsrSop: return "CSR LexBFS long-row old prev";
        case kChkCsrSon: return "CSR LexBFS long-row old next";
        case kChkCsrSrun: return "CSR LexBFS long-row runs";
        case kChkCsrSkey: return "CSR LexBFS long-row keys";
        case kChkUnitMask: return "check earlier-than mask";
        case kChkUnitPos: return "check pos gather";
        case kChkUnitGroup: return "check order / parent value";
        case kChkInjected: return "injected test entry";
        default: return "unknown array";
    }
}

}  // namespace cg

using namespace cg;

namespace cg {

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

cudaError_t stream_set_create(StreamSet *ss) {
    cudaError_t e = cudaEventCreateWithFlags(&ss->fork, cudaEventDisableTiming);
    for (int i = 0; e == cudaSuccess && i < kBuckets; ++i) e = cudaEventCreateWithFlags(&ss->join[i], cudaEventDisableTiming);
    for (int i = 0; e == cudaSuccess && i < StreamSet::kAux; ++i)
        e = cudaStreamCreateWithFlags(&ss->aux[i], cudaStreamNonBlocking);
    return e;
}

void stream_set_destroy(StreamSet *ss) {
    if (ss->fork) cudaEventDestroy(ss->fork);
    for (int i = 0; i < kBuckets; ++i)
        if (ss->join[i]) cudaEventDestroy(ss->join[i]);
    for (int i = 0; i < StreamSet::kAux; ++i)
        if (ss->aux[i]) cudaStreamDestroy(ss->aux[i]);
    *ss = StreamSet{};
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

PhaseTimer::PhaseTimer(cg_context *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *l, cudaStream_t s)
    : ctx(c), list(l), stream(s) {
    if (ctx && ctx->profiling && (a = take_event(ctx))) cudaEventRecord(a, stream);
}

void PhaseTimer::stop() {
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

DenseDesc desc_of(const cg_dense *g, int64_t vbase, int64_t obase, int32_t rindex) {
    DenseDesc d{};
    d.rows = g->rows;
    d.n = g->n;
    d.words = g->words_per_row;
    d.vbase = vbase;
    d.obase = obase;
    d.rindex = rindex;
    return d;
}

// ---------------------------------------------------------------- batches
// Graphs are grouped into size buckets (b < 9: n in (2^(b+3), 2^(b+4)], i.e.
// up to 16, 32, ..., 4096; b = 9: n > 4096).  Buckets 0..8 run the fused
// one-CTA test; bucket 9 runs the per-graph LexBFS CTA plus the grid-wide
// check.  Within a bucket graphs are sorted largest first, and CTAs take
// them from an atomic counter (longest job first).
int bucket_of(int n) {
    if (n > kFusedMaxN) return 9;
    int b = 0;
    while (b < 8 && n > (16 << b)) ++b;
    return b;
}

int make_layout(cg_context *ctx, const cg_dense *graphs, int32_t count, const int64_t *order_offsets,
                BatchLayout *L) {
    int rc;
    L->count = count;
    L->emask_words = 0;
    std::vector<int> idx(count);
    std::vector<int> bucket(count);
    for (int k = 0; k < count; ++k) {
        if ((rc = check_dense(&graphs[k]))) return set_error(rc, "graph %d: %s", k, cg_last_error_string());
        if (order_offsets && order_offsets[k] < 0) return set_error(CG_EINVAL, "graph %d: negative order offset", k);
        idx[k] = k;
        bucket[k] = bucket_of(graphs[k].n);
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (bucket[a] != bucket[b]) return bucket[a] < bucket[b];
        return graphs[a].n > graphs[b].n;
    });
    L->descs.resize(count);
    L->voff.resize(count + 1);
    int64_t packed = 0, total = 0;
    // packed order offsets follow input order when the caller gives none
    std::vector<int64_t> obase(count);
    for (int k = 0; k < count; ++k) {
        obase[k] = order_offsets ? order_offsets[k] : packed;
        packed += graphs[k].n;
    }
    for (int b = 0; b < kBuckets; ++b) L->bk[b] = BatchLayout::Bucket{};
    for (int j = 0; j < count; ++j) {
        const int k = idx[j];
        L->voff[j] = total;
        L->descs[j] = desc_of(&graphs[k], total, obase[k], k);
        total += graphs[k].n;
    }
    L->voff[count] = total;
    L->total = total;
    int j = 0;
    for (int b = 0; b < kBuckets; ++b) {
        auto &B = L->bk[b];
        B.begin = j;
        while (j < count && bucket[idx[j]] == b) ++j;
        B.end = j;
        if (B.end == B.begin) continue;
        B.nmax = graphs[idx[B.begin]].n;
        B.vbegin = L->voff[B.begin];
        B.vend = L->voff[B.end];
        const int cnt = B.end - B.begin;
        if (b < 9) {
            if ((rc = fused_dense_plan(B.nmax, ctx->tuned_threads[b], &B.fplan))) return rc;
            if (B.fplan.rows_smem) {
                // rows in shared memory make a step faster but can leave one CTA per SM;
                // with more graphs than that wave holds, rows read from L2 (a step
                // ~1.3x slower) and more CTAs per SM take fewer waves
                FusedPlan pg;
                if ((rc = fused_dense_plan(B.nmax, ctx->tuned_threads[b], &pg, false))) return rc;
                const int64_t ws = ceil_div(cnt, (int64_t)ctx->num_sms * fused_ctas_per_sm(B.fplan));
                const int64_t wg = ceil_div(cnt, (int64_t)ctx->num_sms * fused_ctas_per_sm(pg));
                if (wg * 13 < ws * 10) B.fplan = pg;
            }
            B.ctas = std::min(cnt, ctx->num_sms * fused_ctas_per_sm(B.fplan));
        } else {
            if ((rc = lexbfs_dense_plan(B.nmax, ctx->cfg.threads_override, &B.lplan))) return rc;
            B.bulk = true;
            for (int q = B.begin; q < B.end; ++q) B.bulk = B.bulk && peo_rows_vec_ok(L->descs[q]);
            // graphs sorted largest first: nmax bounds the bucket
            B.stage = B.bulk && B.nmax <= kStageMaxN;
            if (B.stage)
                for (int q = B.begin; q < B.end; ++q) {
                    L->descs[q].ebase = L->emask_words;
                    L->emask_words += earlier_mask_words(L->descs[q].n);
                }
            const int by_smem =
                B.lplan.smem_bytes ? (int)std::max<size_t>(1, (228 * 1024) / (B.lplan.smem_bytes + 1024)) : 32;
            const int by_threads = std::max(1, 2048 / B.lplan.threads);
            B.ctas = std::max(1, std::min(cnt, ctx->num_sms * std::min(by_smem, by_threads)));
        }
    }
    return CG_OK;
}

BatchBuffers batch_buffers(const BatchLayout &L, bool need_order) {
    Carve cv;
    BatchBuffers bb{};
    bb.o_desc = cv.take<DenseDesc>(L.count);
    bb.o_voff = cv.take<int64_t>(L.count + 1);
    bb.o_order = cv.take<int32_t>(need_order ? L.total : 0);
    bb.o_pos = cv.take<int32_t>(L.total);
    bb.o_parent = cv.take<int32_t>(L.total);
    bb.o_ppos = cv.take<int32_t>(L.total);
    // + the check's CTA counter and error word (bucket 9 is last)
    bb.o_keys = cv.take<unsigned long long>(L.count + 2);
    bb.o_counter = cv.take<int>(kBuckets * 64);
    const auto &B9 = L.bk[9];
    bb.o_gstate = cv.take<unsigned char>(B9.end > B9.begin ? B9.lplan.gstate_bytes * B9.ctas : 0);
    bb.o_emask = cv.take<uint32_t>(L.emask_words);
    bb.bytes = cv.off;
    return bb;
}

// Enqueues every bucket on the context's forked streams and joins them back
// into `stream`.  base: device allocation laid out by batch_buffers (the
// descriptors and offsets must already be there).
int enqueue_batch(cg_context *ctx, const BatchLayout &L, const BatchBuffers &bb, unsigned char *base,
                  int32_t *orders, cg_result *res, cudaStream_t stream, const StreamSet &ss, bool account) {
    int rc;
    cg_context *tctx = account ? ctx : nullptr;   // timers and launch counts only for the caller's thread
    auto P = [&](size_t off) { return base + off; };
    const DenseDesc *ddesc = reinterpret_cast<const DenseDesc *>(P(bb.o_desc));
    int32_t *order = orders ? orders : reinterpret_cast<int32_t *>(P(bb.o_order));
    int32_t *pos = reinterpret_cast<int32_t *>(P(bb.o_pos));
    int32_t *parent = reinterpret_cast<int32_t *>(P(bb.o_parent));
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(P(bb.o_keys));
    int *counters = reinterpret_cast<int *>(P(bb.o_counter));
    CG_CUDA_TRY(cudaEventRecord(ss.fork, stream));
    int used = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const auto &B = L.bk[b];
        const int cnt = B.end - B.begin;
        if (cnt <= 0) continue;
        cudaStream_t s = ss.aux[used % StreamSet::kAux];
        CG_CUDA_TRY(cudaStreamWaitEvent(s, ss.fork, 0));
        if (b < 9) {
            PhaseTimer pt(tctx, &ctx->ev_fused, s);
            if ((rc = fused_dense_launch(B.fplan, ddesc + B.begin, cnt, B.ctas, order, pos, parent, res,
                                         counters + 64 * b, s)))
                return rc;
            if (account) ctx->launches += 1;
        } else {
            int32_t *ppos = reinterpret_cast<int32_t *>(P(bb.o_ppos));
            uint32_t *emask = B.stage ? reinterpret_cast<uint32_t *>(P(bb.o_emask)) : nullptr;
            {
                PhaseTimer pt(tctx, &ctx->ev_lex, s);
                if ((rc = lexbfs_dense_launch(B.lplan, ddesc + B.begin, DenseDesc{}, cnt, B.ctas, order, pos, ppos,
                                              B.lplan.gstate_bytes ? P(bb.o_gstate) : nullptr, counters + 64 * b, s,
                                              kParentPivots, keys + B.begin, emask, parent)))
                    return rc;
            }
            PhaseTimer pt(tctx, &ctx->ev_check, s);
            // the position-ordered check of this bucket's graphs: rows staged in
            // shared memory with the search's masks, or E_b built from pos
            if (B.stage)
                rc = peo_stage_launch(ddesc + B.begin, DenseDesc{}, cnt, B.nmax, order, ppos, emask,
                                      keys + B.begin, res, ctx->num_sms, s);
            else
                rc = peo_unit_launch(ddesc + B.begin, DenseDesc{}, cnt, B.nmax, B.bulk, order, pos, ppos,
                                     keys + B.begin, res, s);
            if (rc) return rc;
            if (account) ctx->launches += 2;
        }
        CG_CUDA_TRY(cudaEventRecord(ss.join[b], s));
        CG_CUDA_TRY(cudaStreamWaitEvent(stream, ss.join[b], 0));
        ++used;
    }
    return CG_OK;
}

size_t layout_staging_bytes(const BatchLayout &L) {
    return align_up(sizeof(DenseDesc) * L.count, 16) + sizeof(int64_t) * (L.count + 1) + 64;
}

int upload_layout_to(const BatchLayout &L, const BatchBuffers &bb, unsigned char *base, unsigned char *staging,
                     cudaStream_t stream) {
    const size_t bytes_desc = sizeof(DenseDesc) * L.count, bytes_voff = sizeof(int64_t) * (L.count + 1);
    std::memcpy(staging, L.descs.data(), bytes_desc);
    std::memcpy(staging + align_up(bytes_desc, 16), L.voff.data(), bytes_voff);
    CG_CUDA_TRY(cudaMemcpyAsync(base + bb.o_desc, staging, bytes_desc, cudaMemcpyHostToDevice, stream));
    CG_CUDA_TRY(cudaMemcpyAsync(base + bb.o_voff, staging + align_up(bytes_desc, 16), bytes_voff,
                                cudaMemcpyHostToDevice, stream));
    return CG_OK;
}

int upload_layout(cg_context *ctx, const BatchLayout &L, const BatchBuffers &bb, unsigned char *base,
                  cudaStream_t stream) {
    int rc;
    if ((rc = ensure_pinned(ctx, layout_staging_bytes(L)))) return rc;
    if ((rc = upload_layout_to(L, bb, base, static_cast<unsigned char *>(ctx->pinned), stream))) return rc;
    CG_CUDA_TRY(cudaEventRecord(ctx->staged, stream));
    ctx->staged_pending = true;
    return CG_OK;
}

// Workspace layout of run_single_dense (also the start of the host entry's).
struct SingleDenseCarve {
    size_t o_order, o_pos, o_parent, o_ppos, o_key, o_counter, o_gstate, o_emask;
    Carve cv;
    SingleDenseCarve(int n, const LexPlan &plan) {
        o_order = cv.take<int32_t>(n);
        o_pos = cv.take<int32_t>(n);
        o_parent = cv.take<int32_t>(n);
        o_ppos = cv.take<int32_t>(n);
        o_key = cv.take<unsigned long long>(3);   // key, the check's CTA counter, error word
        o_counter = cv.take<int>(1);
        o_gstate = cv.take<unsigned char>(plan.gstate_bytes);
        // the earlier-than masks of the staged check (written by the search)
        o_emask = cv.take<uint32_t>(n > 0 && n <= kStageMaxN ? earlier_mask_words(n) : 0);
    }
};

// LexBFS and (optionally) the check for one graph given by value.
// base: workspace offset where this call's scratch starts (the bytes before
// it belong to the caller, e.g. a CSR graph expanded to bit rows).
int run_single_dense(cg_context *ctx, const cg_dense *g, int32_t *order_out, int32_t *pos_out, cg_result *res,
                     cudaStream_t stream, size_t base = 0) {
    const int n = g->n;
    LexPlan plan;
    int rc = lexbfs_dense_plan(n, ctx->cfg.threads_override, &plan);
    if (rc) return rc;
    const SingleDenseCarve sc(n, plan);
    if ((rc = ensure_ws(ctx, base + sc.cv.off))) return rc;
    int32_t *order = order_out ? order_out : at<int32_t>(ctx, base + sc.o_order);
    int32_t *pos = pos_out ? pos_out : at<int32_t>(ctx, base + sc.o_pos);
    int32_t *parent = at<int32_t>(ctx, base + sc.o_parent);
    unsigned long long *key = at<unsigned long long>(ctx, base + sc.o_key);
    const DenseDesc d = desc_of(g, 0, 0);
    if (n == 0) {
        if (!res) return CG_OK;
        PhaseTimer pt(ctx, &ctx->ev_check, stream);
        ctx->launches += 1;
        return peo_dense_launch(nullptr, d, 1, nullptr, 0, order, pos, parent, true, key, ctx->num_sms, stream,
                                nullptr, 0, false, res);
    }
    // with a result wanted, the search also records the parents of its pivots
    // by position (one store per step) and initialises the check's keys
    int32_t *ppos = at<int32_t>(ctx, base + sc.o_ppos);
    const bool stage = res && peo_stage_ok(d);
    uint32_t *emask = stage ? at<uint32_t>(ctx, base + sc.o_emask) : nullptr;
    {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        rc = lexbfs_dense_launch(plan, nullptr, d, 1, 1, order, pos, res ? ppos : nullptr,
                                 plan.gstate_bytes ? at<void>(ctx, base + sc.o_gstate) : nullptr, at<int>(ctx, base + sc.o_counter),
                                 stream, kParentPivots, res ? key : nullptr, emask, res ? parent : nullptr);
        if (rc) return rc;
        ctx->launches += 1;
    }
    if (!res) return CG_OK;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    ctx->launches += 1;
    if (stage) return peo_stage_launch(nullptr, d, 1, n, order, ppos, emask, key, res, ctx->num_sms, stream);
    return peo_unit_launch(nullptr, d, 1, n, peo_rows_vec_ok(d), order, pos, ppos, key, res, stream);
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

// Workspace layout of run_single_csr: CSR graphs that take the dense path
// (csr_takes_dense_path) are expanded to bit rows first, the others keep the
// CSR search's state.
struct SingleCsrCarve {
    bool dense = false;
    size_t o_flag = 0, o_rows = 0, dense_base = 0;            // dense path
    size_t o_order = 0, o_pos = 0, o_parent = 0, o_key = 0, o_state = 0;   // CSR path
    size_t bytes = 0;
    int init(int n, int64_t nnz, int threads_override) {
        Carve cv;
        dense = n > 0 && csr_takes_dense_path(n, nnz);
        if (dense) {
            const int words = (n + 31) / 32;
            o_flag = cv.take<int>(1);
            o_rows = cv.take<uint32_t>((size_t)n * words);
            dense_base = align_up(cv.off, kAlign);
            LexPlan plan;
            const int rc = lexbfs_dense_plan(n, threads_override, &plan);
            if (rc) return rc;
            bytes = dense_base + SingleDenseCarve(n, plan).cv.off;
            return CG_OK;
        }
        o_order = cv.take<int32_t>(n);
        o_pos = cv.take<int32_t>(n);
        o_parent = cv.take<int32_t>(n);
        o_key = cv.take<unsigned long long>(1);
        o_flag = cv.take<int>(1);
        o_state = cv.take<unsigned char>(lexbfs_csr_workspace_bytes(n, n));
        bytes = cv.off;
        return CG_OK;
    }
};

// LexBFS and (optionally) the check for one CSR graph; base: workspace offset
// where this call's scratch starts (the bytes before it belong to the caller).
int run_single_csr(cg_context *ctx, const cg_csr *g, int32_t *order_out, int32_t *pos_out, cg_result *res,
                   cudaStream_t stream, size_t base = 0) {
    const int n = g->n;
    int rc;
    SingleCsrCarve sc;
    if ((rc = sc.init(n, g->nnz, ctx->cfg.threads_override))) return rc;
    if ((rc = ensure_ws(ctx, base + sc.bytes))) return rc;
    if (ctx->cfg.validate && (rc = validate_csr(ctx, g, at<int>(ctx, base + sc.o_flag), stream))) return rc;
    if (sc.dense) {
        // dense enough for the dense kernels: bit rows in the workspace, then the dense test
        // (same order and witness: both searches take the lowest id among equal labels)
        const int words = (n + 31) / 32;
        uint32_t *rows = at<uint32_t>(ctx, base + sc.o_rows);
        if ((rc = csr_to_bits_launch(n, g->row_ptr, g->col, rows, words, ctx->num_sms, stream))) return rc;
        ctx->launches += 1;
        const cg_dense d{n, words, rows};
        return run_single_dense(ctx, &d, order_out, pos_out, res, stream, base + sc.dense_base);
    }
    int32_t *order = order_out ? order_out : at<int32_t>(ctx, base + sc.o_order);
    int32_t *pos = pos_out ? pos_out : at<int32_t>(ctx, base + sc.o_pos);
    int32_t *parent = at<int32_t>(ctx, base + sc.o_parent);
    if (n > 0) {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        if ((rc = lexbfs_csr_launch(n, n, g->row_ptr, g->col, g->nnz, order, pos, parent,
                                    at<void>(ctx, base + sc.o_state), ctx->num_sms, stream)))
            return rc;
        ctx->launches += 2;
    }
    if (!res) return CG_OK;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    unsigned long long *key = at<unsigned long long>(ctx, base + sc.o_key);
    if ((rc = peo_csr_launch(n, g->row_ptr, g->col, order, pos, parent, true, key, ctx->num_sms, stream))) return rc;
    DenseDesc d{};
    d.n = n;
    ctx->launches += n > 0 ? 2 : 1;
    return finalize_launch(nullptr, d, 1, key, order, parent, res, stream);
}

}  // namespace cg

extern "C" {

#ifdef CG_BOUNDS_CHECK
const char *cg_version(void) { return "chordal-gb300 0.2.0 (sm_103a, bounds-checking build)"; }
#else
const char *cg_version(void) { return "chordal-gb300 0.2.0 (sm_103a)"; }
#endif

int cg_debug_describe(uint64_t word, char *buf, int32_t len) {
    if (!buf || len <= 0) return set_error(CG_EINVAL, "null or empty message buffer");
    if (!word) {
        snprintf(buf, (size_t)len, "no bounds-check error");
        return CG_OK;
    }
    snprintf(buf, (size_t)len, "%s index %llu out of range", cg_debug_array_name((unsigned)(word >> 56)),
             (unsigned long long)(word & ((1ull << 56) - 1)));
    return CG_OK;
}

int cg_debug_inject(int32_t code) {
    if (code <= 0 || code > 255) return set_error(CG_EINVAL, "code must be in 1..255");
    return debug_inject((unsigned)code);
}

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
    if (e == cudaSuccess) e = stream_set_create(&ctx->streams);
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
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *lists[4] = {&ctx->ev_lex, &ctx->ev_check, &ctx->ev_fused,
                                                                  &ctx->ev_batch};
    double *sums[4] = {&p.lexbfs_ms, &p.check_ms, &p.fused_ms, &p.batch_ms};
    int64_t *counts[4] = {&p.lexbfs_launches, &p.check_launches, &p.fused_launches, &p.batch_calls};
    for (int phase = 0; phase < 4; ++phase) {
        auto &list = *lists[phase];
        double sum = 0;
        for (auto &ab : list) {
            CG_CUDA_TRY(cudaEventSynchronize(ab.second));
            float ms = 0.f;
            CG_CUDA_TRY(cudaEventElapsedTime(&ms, ab.first, ab.second));
            sum += ms;
            ctx->ev_free.push_back(ab.first);
            ctx->ev_free.push_back(ab.second);
        }
        *sums[phase] = sum;
        *counts[phase] = (int64_t)list.size();
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
    for (auto *l : {&ctx->ev_lex, &ctx->ev_check, &ctx->ev_fused, &ctx->ev_batch})
        for (auto &ab : *l) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    cudaEventDestroy(ctx->staged);
    stream_set_destroy(&ctx->streams);
    delete ctx;
    return CG_OK;
}

int cg_lexbfs_order_dense(cg_context *ctx, const cg_dense *g, int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    return run_single_dense(ctx, g, order, pos, nullptr, stream);
}

int cg_lexbfs_sweep_dense(cg_context *ctx, const cg_dense *g, int32_t kind, const int32_t *tiebreak, int32_t start,
                          int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    const int n = g->n;
    if (n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    if (kind != CG_TIE_ID && kind != CG_TIE_RANK && kind != CG_TIE_LAST_IN)
        return set_error(CG_EINVAL, "unknown tie-break kind %d", kind);
    if (kind != CG_TIE_ID && n > 0 && !tiebreak) return set_error(CG_EINVAL, "null tie-break array");
    if (start < -1 || (start >= 0 && start >= n)) return set_error(CG_EINVAL, "start %d outside [-1, n)", start);
    if (kind == CG_TIE_ID && start < 0) return run_single_dense(ctx, g, order, pos, nullptr, stream);
    if (n == 0) return CG_OK;
    LexPlan plan;
    if ((rc = lexbfs_dense_plan(n, ctx->cfg.threads_override, &plan))) return rc;
    const size_t wn = (size_t)(n + 31) / 32;
    Carve cv;
    const size_t o_prow = cv.take<uint32_t>((size_t)n * wn);
    const size_t o_rank = cv.take<int32_t>(n), o_newid = cv.take<int32_t>(n), o_inv = cv.take<int32_t>(n);
    const size_t o_seen = cv.take<int>(n), o_order = cv.take<int32_t>(n), o_pos = cv.take<int32_t>(n);
    const size_t o_flag = cv.take<int>(1), o_counter = cv.take<int>(1);
    const size_t o_gstate = cv.take<unsigned char>(plan.gstate_bytes);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    SweepBuffers sb{at<uint32_t>(ctx, o_prow), at<int32_t>(ctx, o_rank), at<int32_t>(ctx, o_newid),
                    at<int32_t>(ctx, o_inv), at<int>(ctx, o_seen), at<int32_t>(ctx, o_order),
                    at<int32_t>(ctx, o_pos), at<int>(ctx, o_flag)};
    PhaseTimer pt(ctx, &ctx->ev_lex, stream);
    if ((rc = sweep_ids_launch(n, kind, tiebreak, start, sb, ctx->num_sms, stream))) return rc;
    if (ctx->cfg.validate) {   // before the search runs on the relabelled copy
        int flag = 0;
        CG_CUDA_TRY(cudaMemcpyAsync(&flag, sb.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CG_CUDA_TRY(cudaStreamSynchronize(stream));
        if (flag) return set_error(CG_EINVAL, "tie-break array is not a permutation of 0..n-1");
    }
    rc = sweep_order_launch(desc_of(g, 0, 0), plan, plan.gstate_bytes ? at<void>(ctx, o_gstate) : nullptr,
                            at<int>(ctx, o_counter), sb, order, pos, ctx->num_sms, stream);
    if (rc) return rc;
    ctx->launches += 5;
    return CG_OK;
}

int cg_lexbfs_sweep_csr(cg_context *ctx, const cg_csr *g, int32_t kind, const int32_t *tiebreak, int32_t start,
                        int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_csr(g))) return rc;
    const int n = g->n;
    if (n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    if (kind != CG_TIE_ID && kind != CG_TIE_RANK && kind != CG_TIE_LAST_IN)
        return set_error(CG_EINVAL, "unknown tie-break kind %d", kind);
    if (kind != CG_TIE_ID && n > 0 && !tiebreak) return set_error(CG_EINVAL, "null tie-break array");
    if (start < -1 || (start >= 0 && start >= n)) return set_error(CG_EINVAL, "start %d outside [-1, n)", start);
    if (kind == CG_TIE_ID && start < 0) return run_single_csr(ctx, g, order, pos, nullptr, stream);
    if (n == 0) return CG_OK;
    Carve cv;
    const size_t o_rank = cv.take<int32_t>(n), o_newid = cv.take<int32_t>(n), o_inv = cv.take<int32_t>(n);
    const size_t o_seen = cv.take<int>(n), o_order = cv.take<int32_t>(n), o_pos = cv.take<int32_t>(n);
    const size_t o_flag = cv.take<int>(1);
    const size_t o_state = cv.take<unsigned char>(lexbfs_csr_workspace_bytes(n, n));
    const size_t o_relabel = cv.take<unsigned char>(sweep_csr_workspace_bytes(n, g->nnz));
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    if (ctx->cfg.validate && (rc = validate_csr(ctx, g, at<int>(ctx, o_flag), stream))) return rc;
    SweepBuffers sb{nullptr, at<int32_t>(ctx, o_rank), at<int32_t>(ctx, o_newid), at<int32_t>(ctx, o_inv),
                    at<int>(ctx, o_seen), at<int32_t>(ctx, o_order), at<int32_t>(ctx, o_pos), at<int>(ctx, o_flag)};
    PhaseTimer pt(ctx, &ctx->ev_lex, stream);
    if ((rc = sweep_ids_launch(n, kind, tiebreak, start, sb, ctx->num_sms, stream))) return rc;
    if (ctx->cfg.validate) {
        int flag = 0;
        CG_CUDA_TRY(cudaMemcpyAsync(&flag, sb.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CG_CUDA_TRY(cudaStreamSynchronize(stream));
        if (flag) return set_error(CG_EINVAL, "tie-break array is not a permutation of 0..n-1");
    }
    int64_t *rp_new = nullptr;
    int32_t *col_new = nullptr;
    if ((rc = sweep_csr_relabel_launch(n, g->nnz, g->row_ptr, g->col, sb, at<void>(ctx, o_relabel), &rp_new,
                                       &col_new, ctx->num_sms, stream)))
        return rc;
    if ((rc = lexbfs_csr_launch(n, n, rp_new, col_new, g->nnz, sb.order_p, sb.pos_p, nullptr, at<void>(ctx, o_state),
                                ctx->num_sms, stream)))
        return rc;
    if ((rc = sweep_unpermute_launch(n, sb, order, pos, ctx->num_sms, stream))) return rc;
    ctx->launches += 14;
    return CG_OK;
}

int cg_chordal_test_dense(cg_context *ctx, const cg_dense *g, cg_result *res, int32_t *order, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    return run_single_dense(ctx, g, order, nullptr, res, stream);
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
    const size_t o_key = cv.take<unsigned long long>(2);
    const size_t o_emask = cv.take<uint32_t>(earlier_mask_words(n));
    const size_t o_flag = cv.take<int>(1);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    int32_t *pos = at<int32_t>(ctx, o_pos);
    int32_t *par = parent ? parent : at<int32_t>(ctx, o_parent);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    const DenseDesc d = desc_of(g, 0, 0);
    if (ctx->cfg.validate) {   // the position buffer doubles as the seen flags
        if ((rc = order_check_launch(n, order, pos, at<int>(ctx, o_flag), ctx->num_sms, stream))) return rc;
        int flag = 0;
        CG_CUDA_TRY(cudaMemcpyAsync(&flag, at<int>(ctx, o_flag), sizeof(int), cudaMemcpyDeviceToHost, stream));
        CG_CUDA_TRY(cudaStreamSynchronize(stream));
        if (flag) return set_error(CG_EINVAL, "order is not a permutation of 0..n-1");
    }
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    // vertices missing from an invalid order keep position -1 and are skipped
    if (n > 0) CG_CUDA_TRY(cudaMemsetAsync(pos, 0xFF, sizeof(int32_t) * (size_t)n, stream));
    if ((rc = invert_order_launch(nullptr, d, 1, nullptr, n, order, pos, ctx->num_sms, stream))) return rc;
    ctx->launches += n > 0 ? 3 : 1;
    return peo_dense_launch(nullptr, d, 1, nullptr, n, order, pos, par, false, key, ctx->num_sms, stream,
                            at<uint32_t>(ctx, o_emask), n, false, res);
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
    Carve cv = SingleDenseCarve(n, plan).cv;
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
    if ((rc = run_single_dense(ctx, &g, order, nullptr, res, stream))) return rc;
    CG_CUDA_TRY(cudaMemcpyAsync(host_res, res, sizeof(cg_result), cudaMemcpyDeviceToHost, stream));
    if (host_order && n > 0)
        CG_CUDA_TRY(cudaMemcpyAsync(host_order, order, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, stream));
    CG_CUDA_TRY(cudaStreamSynchronize(stream));
    return CG_OK;
}

namespace {
// MCS order and (optionally) the check of one dense graph.
int run_mcs_dense(cg_context *ctx, const cg_dense *g, int32_t *order_out, int32_t *pos_out, cg_result *res,
                  cudaStream_t stream) {
    const int n = g->n;
    Carve cv;
    const size_t o_order = cv.take<int32_t>(n);
    const size_t o_pos = cv.take<int32_t>(n);
    const size_t o_parent = cv.take<int32_t>(n);
    const size_t o_key = cv.take<unsigned long long>(2);
    const size_t o_counter = cv.take<int>(1);
    const size_t o_emask = cv.take<uint32_t>(res ? earlier_mask_words(n) : 0);
    int rc;
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    int32_t *order = order_out ? order_out : at<int32_t>(ctx, o_order);
    int32_t *pos = pos_out ? pos_out : at<int32_t>(ctx, o_pos);
    int32_t *parent = at<int32_t>(ctx, o_parent);
    const DenseDesc d = desc_of(g, 0, 0);
    if (n > 0) {
        PhaseTimer pt(ctx, &ctx->ev_lex, stream);
        if ((rc = mcs_dense_launch(nullptr, d, 1, n, 1, order, pos, at<int>(ctx, o_counter), stream))) return rc;
        ctx->launches += 1;
    }
    if (!res) return CG_OK;
    PhaseTimer pt(ctx, &ctx->ev_check, stream);
    unsigned long long *key = at<unsigned long long>(ctx, o_key);
    ctx->launches += n > 0 ? 2 : 1;
    return peo_dense_launch(nullptr, d, 1, nullptr, n, order, pos, parent, false, key, ctx->num_sms, stream,
                            at<uint32_t>(ctx, o_emask), n, false, res);
}
}  // namespace

int cg_mcs_order_dense(cg_context *ctx, const cg_dense *g, int32_t *order, int32_t *pos, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (g->n > 0 && !order) return set_error(CG_EINVAL, "null order pointer");
    return run_mcs_dense(ctx, g, order, pos, nullptr, stream);
}

int cg_chordal_test_mcs_dense(cg_context *ctx, const cg_dense *g, cg_result *res, int32_t *order,
                              cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx)) || (rc = check_dense(g))) return rc;
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    return run_mcs_dense(ctx, g, order, nullptr, res, stream);
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
    // inputs and outputs first; run_single_csr's scratch follows (sized before any copy,
    // so that no workspace growth can drop the copied inputs)
    Carve cv;
    const size_t o_rp = cv.take<int64_t>((size_t)n + 1);
    const size_t o_col = cv.take<int32_t>((size_t)nnz);
    const size_t o_res = cv.take<cg_result>(1);
    const size_t o_order = cv.take<int32_t>(n);
    const size_t base = align_up(cv.off, kAlign);
    SingleCsrCarve scv;
    if ((rc = scv.init(n, nnz, ctx->cfg.threads_override))) return rc;
    if ((rc = ensure_ws(ctx, base + scv.bytes))) return rc;
    int64_t *rp = at<int64_t>(ctx, o_rp);
    int32_t *col = at<int32_t>(ctx, o_col);
    if (n >= 0)
        CG_CUDA_TRY(cudaMemcpyAsync(rp, host_row_ptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, stream));
    if (nnz > 0) CG_CUDA_TRY(cudaMemcpyAsync(col, host_col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, stream));
    cg_csr g{n, nnz, rp, col};
    cg_result *res = at<cg_result>(ctx, o_res);
    int32_t *order = at<int32_t>(ctx, o_order);
    if ((rc = run_single_csr(ctx, &g, order, nullptr, res, stream, base))) return rc;
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
    BatchLayout L;
    if ((rc = make_layout(ctx, graphs, count, order_offsets, &L))) return rc;
    const BatchBuffers bb = batch_buffers(L, orders == nullptr);
    if ((rc = ensure_ws(ctx, bb.bytes))) return rc;
    unsigned char *base = static_cast<unsigned char *>(ctx->ws);
    if ((rc = upload_layout(ctx, L, bb, base, stream))) return rc;
    PhaseTimer pt(ctx, &ctx->ev_batch, stream);
    return enqueue_batch(ctx, L, bb, base, orders, res, stream, ctx->streams, true);
}

// The batch from host buffers: graph k's rows (host memory) are copied into
// the workspace, the batch runs there, and the results (and orders) come back.
int cg_chordal_test_batch_host(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *host_res,
                               int32_t *host_orders, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (count < 0) return set_error(CG_EINVAL, "count must be >= 0");
    if (count == 0) return CG_OK;
    if (!graphs || !host_res) return set_error(CG_EINVAL, "null graphs or host result pointer");
    // the layout depends on the sizes only: a first pass with the host pointers sizes the workspace
    BatchLayout L;
    if ((rc = make_layout(ctx, graphs, count, nullptr, &L))) return rc;
    const BatchBuffers bb = batch_buffers(L, host_orders == nullptr);
    // graphs whose host rows follow each other share one copy of their whole span; a gap
    // between two graphs is copied only when it lies in pages that hold the callers' rows
    // (the next graph starts at most one 4 KiB page after the page where the previous
    // one ends), so no byte outside mapped caller pages is read.  The device copy keeps
    // each graph's offset and its address modulo 256 (alignment for 128-bit loads).
    constexpr uintptr_t kPage = 4096;
    std::vector<int> by_addr(count);
    for (int k = 0; k < count; ++k) by_addr[k] = k;
    auto hbeg = [&](int k) { return reinterpret_cast<uintptr_t>(graphs[k].rows); };
    auto hbytes = [&](int k) { return (size_t)graphs[k].n * (size_t)graphs[k].words_per_row * sizeof(uint32_t); };
    std::stable_sort(by_addr.begin(), by_addr.end(), [&](int a, int b) { return hbeg(a) < hbeg(b); });
    struct Span {
        uintptr_t beg, end;
        size_t off;
    };
    std::vector<Span> spans;
    std::vector<int> span_of(count, -1);
    Carve cv;
    for (int q = 0; q < count; ++q) {
        const int k = by_addr[q];
        if (!hbytes(k)) continue;
        const uintptr_t b = hbeg(k), e = b + hbytes(k);
        if (!spans.empty() && b >= spans.back().end && b / kPage <= (spans.back().end - 1) / kPage + 1) {
            spans.back().end = e;
        } else {
            spans.push_back(Span{b, e, 0});
        }
        span_of[k] = (int)spans.size() - 1;
    }
    for (auto &sp : spans) sp.off = cv.take<unsigned char>((sp.end - sp.beg) + 256) + (sp.beg & 255);
    const size_t o_res = cv.take<cg_result>(count);
    const size_t o_ord = cv.take<int32_t>(host_orders ? L.total : 0);
    const size_t o_bb = cv.take<unsigned char>(bb.bytes);
    if ((rc = ensure_ws(ctx, cv.off))) return rc;
    unsigned char *ws = static_cast<unsigned char *>(ctx->ws);
    for (size_t si = 0; si < spans.size(); ++si) {
        const Span &sp = spans[si];
        cudaError_t e = cudaMemcpyAsync(ws + sp.off, reinterpret_cast<const void *>(sp.beg), sp.end - sp.beg,
                                        cudaMemcpyHostToDevice, stream);
        if (e == cudaErrorInvalidValue) {   // a span across two pinned allocations: copy its graphs one by one
            cudaGetLastError();
            for (int k = 0; k < count; ++k)
                if (span_of[k] == (int)si)
                    CG_CUDA_TRY(cudaMemcpyAsync(ws + sp.off + (hbeg(k) - sp.beg), graphs[k].rows, hbytes(k),
                                                cudaMemcpyHostToDevice, stream));
        } else if (e != cudaSuccess) {
            return set_error(CG_ECUDA, "host-to-device copy of the batch's rows failed: %s", cudaGetErrorString(e));
        }
    }
    std::vector<cg_dense> dev(graphs, graphs + count);
    for (int k = 0; k < count; ++k)
        if (span_of[k] >= 0) {
            const Span &sp = spans[span_of[k]];
            dev[k].rows = reinterpret_cast<const uint32_t *>(ws + sp.off + (hbeg(k) - sp.beg));
        }
    if ((rc = make_layout(ctx, dev.data(), count, nullptr, &L))) return rc;
    cg_result *res = reinterpret_cast<cg_result *>(ws + o_res);
    int32_t *orders = host_orders ? reinterpret_cast<int32_t *>(ws + o_ord) : nullptr;
    unsigned char *base = ws + o_bb;
    if ((rc = upload_layout(ctx, L, bb, base, stream))) return rc;
    {
        PhaseTimer pt(ctx, &ctx->ev_batch, stream);
        if ((rc = enqueue_batch(ctx, L, bb, base, orders, res, stream, ctx->streams, true))) return rc;
    }
    CG_CUDA_TRY(cudaMemcpyAsync(host_res, res, sizeof(cg_result) * count, cudaMemcpyDeviceToHost, stream));
    if (host_orders && L.total > 0)
        CG_CUDA_TRY(cudaMemcpyAsync(host_orders, orders, sizeof(int32_t) * (size_t)L.total, cudaMemcpyDeviceToHost,
                                    stream));
    CG_CUDA_TRY(cudaStreamSynchronize(stream));
    return CG_OK;
}

struct cg_batch_plan {
    cg_context *ctx = nullptr;
    void *mem = nullptr;
    cudaGraph_t graph{};
    cudaGraphExec_t exec{};
    int64_t launches = 0;
};

int cg_batch_plan_create(cg_context *ctx, const cg_dense *graphs, int32_t count, cg_result *res, int32_t *orders,
                         const int64_t *order_offsets, cg_batch_plan **out) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (!out) return set_error(CG_EINVAL, "null output pointer");
    *out = nullptr;
    if (count <= 0 || !graphs || !res) return set_error(CG_EINVAL, "a plan needs count > 0, graphs and res");
    BatchLayout L;
    if ((rc = make_layout(ctx, graphs, count, order_offsets, &L))) return rc;
    const BatchBuffers bb = batch_buffers(L, orders == nullptr);
    cg_batch_plan *plan = new (std::nothrow) cg_batch_plan();
    if (!plan) return set_error(CG_ENOMEM, "plan allocation failed");
    plan->ctx = ctx;
    if (cudaMalloc(&plan->mem, bb.bytes) != cudaSuccess) {
        cudaGetLastError();
        delete plan;
        return set_error(CG_ENOMEM, "plan buffers (%zu bytes) allocation failed", bb.bytes);
    }
    unsigned char *base = static_cast<unsigned char *>(plan->mem);
    cudaStream_t cs = ctx->streams.aux[StreamSet::kAux - 1];
    rc = upload_layout(ctx, L, bb, base, cs);
    if (rc == CG_OK) {
        cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) rc = set_error(CG_ECUDA, "plan upload failed: %s", cudaGetErrorString(e));
    }
    // capture the launch sequence once; runs replay it
    cudaStream_t origin = nullptr;
    if (rc == CG_OK && cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(CG_ECUDA, "stream creation failed");
    if (rc == CG_OK) {
        const int64_t before = ctx->launches;
        const bool prof = ctx->profiling;
        ctx->profiling = false;   // no timing events inside the captured graph
        cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) rc = set_error(CG_ECUDA, "begin capture failed: %s", cudaGetErrorString(e));
        if (rc == CG_OK) {
            const int erc = enqueue_batch(ctx, L, bb, base, orders, res, origin, ctx->streams, true);
            e = cudaStreamEndCapture(origin, &plan->graph);
            if (erc) rc = erc;
            else if (e != cudaSuccess) rc = set_error(CG_ECUDA, "end capture failed: %s", cudaGetErrorString(e));
        }
        plan->launches = ctx->launches - before;
        ctx->launches = before;
        ctx->profiling = prof;
        if (rc == CG_OK && cudaGraphInstantiate(&plan->exec, plan->graph, 0) != cudaSuccess)
            rc = set_error(CG_ECUDA, "graph instantiation failed");
    }
    if (origin) cudaStreamDestroy(origin);
    if (rc) {
        cudaGetLastError();
        if (plan->exec) cudaGraphExecDestroy(plan->exec);
        if (plan->graph) cudaGraphDestroy(plan->graph);
        cudaFree(plan->mem);
        delete plan;
        return rc;
    }
    *out = plan;
    return CG_OK;
}

int cg_batch_plan_run(cg_batch_plan *plan, cudaStream_t stream) {
    if (!plan) return set_error(CG_EINVAL, "null plan");
    int rc;
    if ((rc = check_ctx(plan->ctx))) return rc;
    PhaseTimer pt(plan->ctx, &plan->ctx->ev_batch, stream);
    CG_CUDA_TRY(cudaGraphLaunch(plan->exec, stream));
    plan->ctx->launches += plan->launches;
    return CG_OK;
}

int cg_batch_plan_destroy(cg_batch_plan *plan) {
    if (!plan) return CG_OK;
    cudaSetDevice(plan->ctx->cfg.device);
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->mem) cudaFree(plan->mem);
    delete plan;
    return CG_OK;
}

int cg_batch_autotune(cg_context *ctx, const cg_dense *graphs, int32_t count, cudaStream_t stream) {
    int rc;
    if ((rc = check_ctx(ctx))) return rc;
    if (count <= 0 || !graphs) return set_error(CG_EINVAL, "autotune needs graphs");
    // time each fused bucket alone with each CTA size; keep the fastest
    Carve cv;
    const size_t o_res = cv.take<cg_result>(count);
    const size_t o_rest = cv.take<unsigned char>(0);
    (void)o_rest;
    BatchLayout L0;
    if ((rc = make_layout(ctx, graphs, count, nullptr, &L0))) return rc;
    const BatchBuffers bb0 = batch_buffers(L0, true);
    if ((rc = ensure_ws(ctx, cv.off + bb0.bytes + kAlign))) return rc;
    cg_result *res = at<cg_result>(ctx, o_res);
    unsigned char *base = static_cast<unsigned char *>(ctx->ws) + align_up(cv.off, kAlign);
    cudaEvent_t a, b;
    CG_CUDA_TRY(cudaEventCreate(&a));
    CG_CUDA_TRY(cudaEventCreate(&b));
    const int cands[4] = {64, 128, 256, 512};
    for (int bk = 0; bk < 9; ++bk) {
        const auto &B0 = L0.bk[bk];
        if (B0.end <= B0.begin) continue;
        float best = 1e30f;
        int best_t = 0;
        for (int c : cands) {
            ctx->tuned_threads[bk] = c;
            BatchLayout L;
            if (make_layout(ctx, graphs, count, nullptr, &L) != CG_OK) { cudaGetLastError(); continue; }
            const BatchBuffers bb = batch_buffers(L, true);
            if ((rc = upload_layout(ctx, L, bb, base, stream))) break;
            const auto &B = L.bk[bk];
            int32_t *order = reinterpret_cast<int32_t *>(base + bb.o_order);
            int32_t *pos = reinterpret_cast<int32_t *>(base + bb.o_pos);
            int32_t *parent = reinterpret_cast<int32_t *>(base + bb.o_parent);
            const DenseDesc *dd = reinterpret_cast<const DenseDesc *>(base + bb.o_desc);
            int *ctr = reinterpret_cast<int *>(base + bb.o_counter);
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == CG_OK; ++rep) {   // second run is timed
                cudaEventRecord(a, stream);
                rc = fused_dense_launch(B.fplan, dd + B.begin, B.end - B.begin, B.ctas, order, pos, parent, res, ctr,
                                        stream);
                cudaEventRecord(b, stream);
                cudaEventSynchronize(b);
                cudaEventElapsedTime(&ms, a, b);
            }
            if (rc) break;
            if (ms < best) {
                best = ms;
                best_t = c;
            }
        }
        ctx->tuned_threads[bk] = best_t;
        if (rc) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc;
}

int cg_autotune_get(cg_context *ctx, int32_t *threads, int32_t slots) {
    if (!ctx || !threads) return set_error(CG_EINVAL, "null argument");
    for (int i = 0; i < slots && i < kBuckets; ++i) threads[i] = ctx->tuned_threads[i];
    return CG_OK;
}

int cg_autotune_set(cg_context *ctx, const int32_t *threads, int32_t slots) {
    if (!ctx || !threads) return set_error(CG_EINVAL, "null argument");
    for (int i = 0; i < slots && i < kBuckets; ++i) {
        const int t = threads[i];
        if (i < 9 && t != 0 && t != 64 && t != 128 && t != 256 && t != 512)
            return set_error(CG_EINVAL, "bucket %d: CTA size %d not in {0, 64, 128, 256, 512}", i, t);
        if (i < 9) ctx->tuned_threads[i] = t;
    }
    return CG_OK;
}

}  // extern "C"
