// queue.cu — continuous-batching request queue for chordality queries.
//
// Serving is not part of the paper; it packages the test for a stream of
// independent queries.  A library-owned worker thread:
//   * admits pending requests in arrival order into the next batch while the
//     batch's device memory fits the largest free block of a fixed pool (the
//     memory budget) and a slot (stream) is free — requests that arrive while
//     other batches run are admitted as soon as slots and memory free up;
//   * launches each batch on its slot's stream (size buckets forked onto the
//     slot's own streams), so several batches' kernels share the GPU;
//   * notices completion by polling each slot's event, copies results (already
//     transferred to pinned host memory by the batch) to the ticket table and
//     returns the batch's memory to the pool.
// Two admission lanes keep short queries from waiting on long ones: graphs
// with n <= 4096 are batched up to max_batch per launch, larger graphs up to
// max_batch_large, each lane in arrival order; results of a batch complete
// together.  Dense queries run the one-CTA or LexBFS-CTA + check kernels of
// the batched path.  CSR queries with n <= 131072 and at least 64 neighbours per vertex on
// average (or n <= 4096) are expanded to bit rows on the device first and take
// the same path; sparser CSR queries run the CSR kernels.
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.h"
#include "lexbfs_dense.cuh"

namespace cg {

namespace {


// First-fit allocator over [0, cap) with coalescing frees.
struct PoolAllocator {
    std::map<size_t, size_t> free_;   // offset -> length
    void reset(size_t cap) {
        free_.clear();
        if (cap) free_[0] = cap;
    }
    size_t largest() const {
        size_t m = 0;
        for (auto &kv : free_) m = kv.second > m ? kv.second : m;
        return m;
    }
    size_t alloc(size_t len) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const size_t off = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest) free_[off + len] = rest;
                return off;
            }
        }
        return (size_t)-1;
    }
    void release(size_t off, size_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum Route { kRouteDense = 0, kRouteCsrBits = 1, kRouteCsr = 2 };

struct Request {
    uint64_t ticket;
    cg_graph_ref g;
    Route route;
    size_t mem;
    std::chrono::steady_clock::time_point t_submit;
};

struct Done {
    cg_result res;
    double latency_s;
    int status;
    std::vector<int32_t> order;   // kept when the queue keeps orders
};

struct Slot {
    cudaStream_t stream{};
    StreamSet ss;
    cudaEvent_t done{};
    unsigned char *staging = nullptr;   // pinned: descriptors up, results down
    size_t staging_bytes = 0;
    std::vector<Request> reqs;
    std::vector<const int32_t *> order_dev;   // per request: its order in the pool (kept orders)
    size_t off = 0, bytes = 0;
    bool busy = false;
};

// Admission estimate for one dense test (order, pos, parent, key, descriptor,
// result, and the 32-bit search state above 16,384 vertices).  The exact
// batch size is computed before a batch is admitted.
size_t dense_need(int n) {
    return align_up(3 * (size_t)n * 4 + 64 + 16, kAlign) * 2 +
           (n > 16384 ? align_up(lex_state_bytes<uint32_t>(n), kAlign) : 0);   // covers the split layout too
}

}  // namespace

}  // namespace cg

using namespace cg;

struct cg_queue {
    cg_context *ctx = nullptr;
    cg_queue_config cfg{};
    unsigned char *pool = nullptr;
    size_t pool_bytes = 0;
    PoolAllocator alloc;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;       // work for the worker
    std::condition_variable done_cv;  // completions for drain
    std::deque<Request> pending[2];   // lane 0: n <= 4096, lane 1: larger graphs
    int lane_turn = 0;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, batches = 0;
    size_t inflight = 0;
    bool stop = false;
    std::thread worker;
    // CSR layout checks at submit (cfg.validate): own stream and flag
    std::mutex val_mu;
    cudaStream_t val_stream{};
    int *val_flag = nullptr;
};

namespace {

size_t request_need(const cg_graph_ref &g, Route route) {
    if (route == kRouteDense) return dense_need(g.dense.n);
    const int n = g.csr.n;
    if (route == kRouteCsrBits) return dense_need(n) + align_up((size_t)n * ((n + 31) / 32) * 4, kAlign);
    return align_up(3 * (size_t)n * 4 + 64, kAlign) + align_up(lexbfs_csr_workspace_bytes(n, n), kAlign) + kAlign;
}

// Builds and enqueues one batch on slot s (worker thread, no lock held).
// dry: only compute the device bytes the batch needs (returned in *bytes_out).
int launch_batch(cg_queue *q, Slot &s, bool dry = false, size_t *bytes_out = nullptr) {
    int rc;
    cg_context *ctx = q->ctx;
    if (!dry) {   // the layout must fit the reservation before any work is queued
        size_t exact = 0;
        if ((rc = launch_batch(q, s, true, &exact))) return rc;
        if (exact > s.bytes) return set_error(CG_ENOMEM, "queue batch layout exceeds its reservation");
        s.order_dev.assign(s.reqs.size(), nullptr);
    }
    const bool keep = q->cfg.keep_orders != 0;
    unsigned char *base = dry ? nullptr : q->pool + s.off;
    const int count = (int)s.reqs.size();
    size_t cur = 0;
    auto take = [&](size_t bytes) {
        cur = align_up(cur, kAlign);
        const size_t o = cur;
        cur += bytes > 0 ? bytes : 1;
        return o;
    };
    const size_t o_res = take(sizeof(cg_result) * count);
    cg_result *dres = reinterpret_cast<cg_result *>(base + o_res);
    // dense views of the dense and bit-expanded CSR requests
    std::vector<cg_dense> dense;
    std::vector<int> dense_req;
    for (int i = 0; i < count; ++i) {
        const Request &r = s.reqs[i];
        if (r.route == kRouteDense) {
            dense.push_back(r.g.dense);
            dense_req.push_back(i);
        } else if (r.route == kRouteCsrBits) {
            const int n = r.g.csr.n, words = (n + 31) / 32;
            uint32_t *rows = reinterpret_cast<uint32_t *>(base + take((size_t)n * words * 4));
            if (n > 0 && !dry &&
                (rc = csr_to_bits_launch(n, r.g.csr.row_ptr, r.g.csr.col, rows, words, ctx->num_sms, s.stream)))
                return rc;
            dense.push_back(cg_dense{n, words, rows});
            dense_req.push_back(i);
        }
    }
    if (!dense.empty()) {
        BatchLayout L;
        if ((rc = make_layout(ctx, dense.data(), (int)dense.size(), nullptr, &L))) return rc;
        for (auto &d : L.descs) d.rindex = dense_req[d.rindex];   // result slot = request index
        const BatchBuffers bb = batch_buffers(L, true);
        const size_t o_b = take(bb.bytes);
        unsigned char *bbase = base + o_b;
        if (!dry && keep) {   // the batch's own order buffer packs the graphs in dense-list order
            int64_t off = 0;
            for (size_t j = 0; j < dense.size(); ++j) {
                s.order_dev[dense_req[j]] = reinterpret_cast<const int32_t *>(bbase + bb.o_order) + off;
                off += dense[j].n;
            }
        }
        const size_t need = layout_staging_bytes(L) + sizeof(cg_result) * count + 64;
        if (dry) goto csr_part;
        // staging is sized at queue creation: freeing pinned memory here would synchronise the device
        if (need > s.staging_bytes) return set_error(CG_EINVAL, "batch larger than the slot's staging");
        if ((rc = upload_layout_to(L, bb, bbase, s.staging, s.stream))) return rc;
        if ((rc = enqueue_batch(ctx, L, bb, bbase, nullptr, dres, s.stream, s.ss, false))) return rc;
    } else if (!dry && s.staging_bytes < sizeof(cg_result) * count) {
        return set_error(CG_EINVAL, "batch larger than the slot's staging");
    }
csr_part:
    // sparse CSR requests: one warp each on the slot stream
    for (int i = 0; i < count; ++i) {
        const Request &r = s.reqs[i];
        if (r.route != kRouteCsr) continue;
        const int n = r.g.csr.n;
        int32_t *order = reinterpret_cast<int32_t *>(base + take((size_t)n * 4));
        int32_t *pos = reinterpret_cast<int32_t *>(base + take((size_t)n * 4));
        int32_t *parent = reinterpret_cast<int32_t *>(base + take((size_t)n * 4));
        unsigned long long *key = reinterpret_cast<unsigned long long *>(base + take(8));
        void *state = base + take(lexbfs_csr_workspace_bytes(n, n));
        if (dry) continue;
        if (keep) s.order_dev[i] = order;
        if (n > 0 && (rc = lexbfs_csr_launch(n, n, r.g.csr.row_ptr, r.g.csr.col, r.g.csr.nnz, order, pos, parent, state,
                                             ctx->num_sms, s.stream)))
            return rc;
        if ((rc = peo_csr_launch(n, r.g.csr.row_ptr, r.g.csr.col, order, pos, parent, true, key, ctx->num_sms,
                                 s.stream)))
            return rc;
        DenseDesc d{};
        d.n = n;
        if ((rc = finalize_launch(nullptr, d, 1, key, order, parent, dres + i, s.stream))) return rc;
    }
    if (dry) {
        *bytes_out = align_up(cur, kAlign) + kAlign;
        return CG_OK;
    }
    // results land in the tail of the slot's pinned staging
    cg_result *hres = reinterpret_cast<cg_result *>(s.staging + s.staging_bytes - sizeof(cg_result) * count);
    CG_CUDA_TRY(cudaMemcpyAsync(hres, dres, sizeof(cg_result) * count, cudaMemcpyDeviceToHost, s.stream));
    CG_CUDA_TRY(cudaEventRecord(s.done, s.stream));
    return CG_OK;
}

void worker_loop(cg_queue *q) {
    cudaSetDevice(q->ctx->cfg.device);
    std::unique_lock<std::mutex> lk(q->mu);
    const size_t batch_overhead = 64 * 1024;
    for (;;) {
        bool progressed = false;
        // 1. completions
        for (auto &s : q->slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) continue;
            const auto now = std::chrono::steady_clock::now();
            const int count = (int)s.reqs.size();
            const cg_result *hres =
                reinterpret_cast<const cg_result *>(s.staging + s.staging_bytes - sizeof(cg_result) * count);
            for (int i = 0; i < count; ++i) {
                Done d{};
                d.status = e == cudaSuccess ? CG_OK : CG_ECUDA;
                if (e == cudaSuccess) d.res = hres[i];
                d.latency_s = std::chrono::duration<double>(now - s.reqs[i].t_submit).count();
                const Request &r = s.reqs[i];
                const int n = r.g.kind == CG_GRAPH_DENSE ? r.g.dense.n : r.g.csr.n;
                if (e == cudaSuccess && q->cfg.keep_orders && n > 0 && i < (int)s.order_dev.size() &&
                    s.order_dev[i]) {   // the batch is complete: a plain copy out of its pool memory
                    d.order.resize(n);
                    if (cudaMemcpy(d.order.data(), s.order_dev[i], sizeof(int32_t) * (size_t)n,
                                   cudaMemcpyDeviceToHost) != cudaSuccess) {
                        cudaGetLastError();
                        d.status = CG_ECUDA;
                        d.order.clear();
                    }
                }
                q->done[r.ticket] = std::move(d);
            }
            if (e != cudaSuccess) cudaGetLastError();
            q->alloc.release(s.off, s.bytes);
            q->completed += count;
            q->inflight -= count;
            s.reqs.clear();
            s.busy = false;
            progressed = true;
        }
        if (progressed) q->done_cv.notify_all();
        // 2. admission: two lanes (small graphs batch widely, large graphs in
        //    small groups), each in arrival order, each batch in a free slot
        bool any_busy = false;
        for (auto &s : q->slots) any_busy = any_busy || s.busy;
        bool launched = false;
        for (int lane = 0; lane < 2; ++lane) {
            const int ln = (q->lane_turn + lane) & 1;
            std::deque<Request> &pend = q->pending[ln];
            if (pend.empty()) continue;
            Slot *free_slot = nullptr;
            for (auto &s : q->slots)
                if (!s.busy) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot) break;
            const size_t room = q->alloc.largest();
            const int cap = ln == 0 ? q->cfg.max_batch : q->cfg.max_batch_large;
            size_t total = batch_overhead;
            std::vector<Request> take;
            while (!pend.empty() && (int)take.size() < cap) {
                const Request &r = pend.front();
                if (total + r.mem + 4 * kAlign > room) break;
                total += r.mem + 4 * kAlign;
                take.push_back(r);
                pend.pop_front();
            }
            // exact device bytes of the candidate batch: halve it until it fits
            Slot probe;
            int dry_rc = CG_OK;
            char dry_msg[256] = {0};
            while (!take.empty()) {
                probe.reqs = take;
                size_t exact = 0;
                const int prc = launch_batch(q, probe, true, &exact);
                if (prc != CG_OK) {   // kept: if the batch shrinks to nothing, this is why
                    dry_rc = prc;
                    snprintf(dry_msg, sizeof(dry_msg), "%s", cg_last_error_string());
                    exact = (size_t)-1;
                }
                if (exact <= room) {
                    total = exact;
                    break;
                }
                const size_t keep = take.size() / 2;
                for (size_t i = take.size(); i > keep; --i) pend.push_front(take[i - 1]);
                take.resize(keep);
            }
            if (take.empty()) {
                if (!any_busy && !launched) {
                    // the head request alone cannot run: its layout failed, or it exceeds the whole budget
                    Request r = pend.front();
                    pend.pop_front();
                    Done d{};
                    d.status = dry_rc != CG_OK ? dry_rc : CG_ENOMEM;
                    if (dry_rc != CG_OK) set_error(dry_rc, "%s", dry_msg);
                    d.res = cg_result{-1, -1, -1, -1};
                    q->done[r.ticket] = d;
                    q->completed += 1;
                    q->done_cv.notify_all();
                    launched = true;
                }
                continue;
            }
            const size_t off = q->alloc.alloc(total);
            Slot &s = *free_slot;
            s.reqs = std::move(take);
            s.off = off;
            s.bytes = total;
            s.busy = true;
            any_busy = true;
            launched = true;
            q->inflight += s.reqs.size();
            q->batches += 1;
            lk.unlock();
            const int rc = launch_batch(q, s);
            lk.lock();
            if (rc != CG_OK) {
                // the batch never reaches the GPU: fail its requests
                cudaStreamSynchronize(s.stream);
                for (auto &r : s.reqs) {
                    Done d{};
                    d.status = rc;
                    d.res = cg_result{-1, -1, -1, -1};
                    q->done[r.ticket] = d;
                }
                q->alloc.release(s.off, s.bytes);
                q->completed += s.reqs.size();
                q->inflight -= s.reqs.size();
                s.reqs.clear();
                s.busy = false;
                q->done_cv.notify_all();
            }
        }
        q->lane_turn ^= 1;
        if (launched) continue;
        const bool nothing_pending = q->pending[0].empty() && q->pending[1].empty();
        if (q->stop && nothing_pending && !any_busy) break;
        if (any_busy)
            q->cv.wait_for(lk, std::chrono::microseconds(20));
        else
            q->cv.wait(lk, [&] { return q->stop || !q->pending[0].empty() || !q->pending[1].empty(); });
    }
}

}  // namespace

extern "C" {

int cg_queue_create(cg_context *ctx, const cg_queue_config *cfg, cg_queue **out) {
    if (!ctx || !out) return set_error(CG_EINVAL, "null argument");
    *out = nullptr;
    CG_CUDA_TRY(cudaSetDevice(ctx->cfg.device));
    cg_queue *q = new (std::nothrow) cg_queue();
    if (!q) return set_error(CG_ENOMEM, "queue allocation failed");
    q->ctx = ctx;
    if (cfg) q->cfg = *cfg;
    if (q->cfg.mem_budget_bytes <= 0) q->cfg.mem_budget_bytes = (int64_t)4 << 30;
    if (q->cfg.max_inflight <= 0) q->cfg.max_inflight = 8;
    if (q->cfg.max_batch <= 0) q->cfg.max_batch = 1024;
    if (q->cfg.max_pending <= 0) q->cfg.max_pending = 1 << 20;
    if (q->cfg.max_batch_large <= 0) q->cfg.max_batch_large = 4;
    q->pool_bytes = align_up((size_t)q->cfg.mem_budget_bytes, kAlign);
    if (cudaMalloc(&q->pool, q->pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        const size_t want = q->pool_bytes;
        delete q;
        return set_error(CG_ENOMEM, "queue pool of %zu bytes could not be allocated", want);
    }
    q->alloc.reset(q->pool_bytes);
    if (cudaStreamCreateWithFlags(&q->val_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&q->val_flag, 256) != cudaSuccess) {
        cudaGetLastError();
        if (q->val_stream) cudaStreamDestroy(q->val_stream);
        cudaFree(q->pool);
        delete q;
        return set_error(CG_ECUDA, "queue validation stream setup failed");
    }
    q->slots.resize(q->cfg.max_inflight);
    // pinned staging per slot, sized once for the largest batch: descriptors,
    // offsets and results
    const int most = q->cfg.max_batch > q->cfg.max_batch_large ? q->cfg.max_batch : q->cfg.max_batch_large;
    const size_t staging = align_up((sizeof(DenseDesc) + sizeof(int64_t) + sizeof(cg_result)) * (most + 1) + 256, 4096);
    for (auto &s : q->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = stream_set_create(&s.ss);
        if (e == cudaSuccess) e = cudaMallocHost(&s.staging, staging);
        if (e == cudaSuccess) s.staging_bytes = staging;
        if (e != cudaSuccess) {
            set_error(CG_ECUDA, "queue stream setup failed: %s", cudaGetErrorString(e));
            for (auto &t : q->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
                if (t.staging) cudaFreeHost(t.staging);
                stream_set_destroy(&t.ss);
            }
            cudaStreamDestroy(q->val_stream);
            cudaFree(q->val_flag);
            cudaFree(q->pool);
            delete q;
            return CG_ECUDA;
        }
    }
    q->worker = std::thread(worker_loop, q);
    *out = q;
    return CG_OK;
}

int cg_queue_submit(cg_queue *q, const cg_graph_ref *g, uint64_t *ticket) {
    if (!q || !g || !ticket) return set_error(CG_EINVAL, "null argument");
    int rc;
    Route route;
    if (g->kind == CG_GRAPH_DENSE) {
        if ((rc = check_dense(&g->dense))) return rc;
        if (g->dense.n > kCsrDenseMaxN) return set_error(CG_EINVAL, "dense queries support n <= %d", kCsrDenseMaxN);
        route = kRouteDense;
    } else if (g->kind == CG_GRAPH_CSR) {
        if ((rc = check_csr(&g->csr))) return rc;
        if (q->ctx->cfg.validate) {   // the CSR kernels index by row_ptr and col: check the layout first
            std::lock_guard<std::mutex> vl(q->val_mu);
            CG_CUDA_TRY(cudaSetDevice(q->ctx->cfg.device));
            if ((rc = validate_csr_launch(g->csr.n, g->csr.nnz, g->csr.row_ptr, g->csr.col, q->val_flag,
                                          q->ctx->num_sms, q->val_stream)))
                return rc;
            int flag = 0;
            CG_CUDA_TRY(cudaMemcpyAsync(&flag, q->val_flag, sizeof(int), cudaMemcpyDeviceToHost, q->val_stream));
            CG_CUDA_TRY(cudaStreamSynchronize(q->val_stream));
            if (flag)
                return set_error(CG_EINVAL, "CSR layout check failed (flags 0x%x: 1 row_ptr, 2 range, "
                                            "4 unsorted/duplicate, 8 self-loop, 16 not symmetric)", flag);
        }
        route = csr_takes_dense_path(g->csr.n, g->csr.nnz) ? kRouteCsrBits : kRouteCsr;
    } else {
        return set_error(CG_EINVAL, "unknown graph kind %d", g->kind);
    }
    Request r;
    r.g = *g;
    r.route = route;
    r.mem = request_need(*g, route);
    r.t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(q->mu);
        if (q->stop) return set_error(CG_EINVAL, "queue is shutting down");
        if ((int64_t)(q->pending[0].size() + q->pending[1].size()) >= q->cfg.max_pending)
            return set_error(CG_EAGAIN, "queue full (%d pending)", q->cfg.max_pending);
        r.ticket = q->next_ticket++;
        const int n = g->kind == CG_GRAPH_DENSE ? g->dense.n : g->csr.n;
        q->pending[n <= kFusedMaxN ? 0 : 1].push_back(r);
        q->submitted += 1;
    }
    q->cv.notify_one();
    *ticket = r.ticket;
    return CG_OK;
}

int cg_queue_poll(cg_queue *q, uint64_t ticket, cg_result *host_res, int32_t *order, double *latency_s) {
    if (!q) return set_error(CG_EINVAL, "null queue");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->done.find(ticket);
    if (it == q->done.end()) {
        if (ticket == 0 || ticket >= q->next_ticket) return set_error(CG_EINVAL, "unknown ticket %llu",
                                                                      (unsigned long long)ticket);
        return CG_EAGAIN;
    }
    if (order && !q->cfg.keep_orders)
        return set_error(CG_EINVAL, "the queue keeps no orders (cg_queue_config.keep_orders = 0)");
    const Done d = std::move(it->second);
    q->done.erase(it);
    if (host_res) *host_res = d.res;
    if (latency_s) *latency_s = d.latency_s;
    if (order && !d.order.empty()) std::memcpy(order, d.order.data(), sizeof(int32_t) * d.order.size());
    if (d.status != CG_OK) return set_error(d.status, "request %llu failed", (unsigned long long)ticket);
    return CG_OK;
}

int cg_queue_drain(cg_queue *q, int64_t timeout_ns) {
    if (!q) return set_error(CG_EINVAL, "null queue");
    std::unique_lock<std::mutex> lk(q->mu);
    const auto pred = [&] { return q->completed >= q->submitted; };
    if (timeout_ns < 0) {
        q->done_cv.wait(lk, pred);
        return CG_OK;
    }
    if (!q->done_cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred))
        return set_error(CG_ETIMEOUT, "drain timed out with %llu requests outstanding",
                         (unsigned long long)(q->submitted - q->completed));
    return CG_OK;
}

int cg_queue_stats(cg_queue *q, cg_queue_info *out) {
    if (!q || !out) return set_error(CG_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(q->mu);
    out->submitted = (int64_t)q->submitted;
    out->completed = (int64_t)q->completed;
    out->pending = (int64_t)(q->pending[0].size() + q->pending[1].size());
    out->inflight = (int64_t)q->inflight;
    out->batches = (int64_t)q->batches;
    out->pool_free_bytes = (int64_t)q->alloc.largest();
    return CG_OK;
}

int cg_queue_destroy(cg_queue *q) {
    if (!q) return CG_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
    }
    q->cv.notify_all();
    if (q->worker.joinable()) q->worker.join();
    cudaSetDevice(q->ctx->cfg.device);
    for (auto &s : q->slots) {
        if (s.stream) {
            cudaStreamSynchronize(s.stream);
            cudaStreamDestroy(s.stream);
        }
        if (s.done) cudaEventDestroy(s.done);
        stream_set_destroy(&s.ss);
        if (s.staging) cudaFreeHost(s.staging);
    }
    if (q->val_stream) cudaStreamDestroy(q->val_stream);
    cudaFree(q->val_flag);
    cudaFree(q->pool);
    delete q;
    return CG_OK;
}

}  // extern "C"
