// host.h — host-side state and helpers shared by the libchordal sources
// (context, workspace carving, batch layout and launch sequencing).
#pragma once
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include "kernels.h"

namespace cg {

constexpr int kBuckets = 10;   // size buckets of a batch: n <= 16, 32, ..., 4096, then n > 4096
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Streams a batch forks its size buckets onto, and the fork / join events.
struct StreamSet {
    static constexpr int kAux = 8;
    cudaStream_t aux[kAux]{};
    cudaEvent_t fork{};
    cudaEvent_t join[kBuckets]{};
};
cudaError_t stream_set_create(StreamSet *ss);
void stream_set_destroy(StreamSet *ss);

}  // namespace cg

struct cg_context {
    cg_config cfg{};
    int num_sms = 0;
    void *ws = nullptr;          // device workspace
    size_t ws_bytes = 0;
    void *pinned = nullptr;      // pinned host staging for descriptor uploads
    size_t pinned_bytes = 0;
    cudaEvent_t staged{};        // recorded after each staging upload
    bool staged_pending = false;
    cg::StreamSet streams;       // forked streams of batch calls
    int tuned_threads[cg::kBuckets]{};   // 0 = size rule
    // per-phase timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_lex, ev_check, ev_fused, ev_batch;
    int64_t launches = 0;
};

namespace cg {

// Offsets into one workspace allocation.
struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t count) {
        off = align_up(off, kAlign);
        const size_t o = off;
        off += (count > 0 ? count : 1) * sizeof(T);
        return o;
    }
};

template <typename T>
T *at(cg_context *ctx, size_t off) {
    return reinterpret_cast<T *>(static_cast<unsigned char *>(ctx->ws) + off);
}

// Brackets one phase with events when profiling is on (ctx may be null: no-op).
struct PhaseTimer {
    cg_context *ctx;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *list;
    cudaStream_t stream;
    cudaEvent_t a = nullptr;
    PhaseTimer(cg_context *c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *l, cudaStream_t s);
    void stop();
    ~PhaseTimer() { stop(); }
};

int check_dense(const cg_dense *g);
int check_csr(const cg_csr *g);
DenseDesc desc_of(const cg_dense *g, int64_t vbase, int64_t obase, int32_t rindex = 0);
int bucket_of(int n);

// A batch sorted into size buckets (largest graph first inside each bucket).
struct BatchLayout {
    struct Bucket {
        int begin = 0, end = 0, nmax = 0;
        FusedPlan fplan{};
        LexPlan lplan{};
        int ctas = 0;
        bool bulk = false;              // bucket 9: every graph's rows suit 128-bit loads
        bool stage = false;             // bucket 9: the staged check (masks written by the search)
        int64_t vbegin = 0, vend = 0;   // packed vertex range
    };
    int count = 0;
    std::vector<DenseDesc> descs;      // bucket order
    std::vector<int64_t> voff;         // packed vertex offset of each desc (+ total)
    Bucket bk[kBuckets];
    int64_t total = 0;
    int64_t emask_words = 0;           // earlier-than masks of the staged bucket's graphs (at each ebase)
};

// Device buffers a batch needs (offsets into one allocation).
struct BatchBuffers {
    size_t o_desc, o_voff, o_order, o_pos, o_parent, o_ppos, o_keys, o_counter, o_gstate, o_emask, bytes;
};

int make_layout(cg_context *ctx, const cg_dense *graphs, int32_t count, const int64_t *order_offsets,
                BatchLayout *L);
BatchBuffers batch_buffers(const BatchLayout &L, bool need_order);
// Launches every bucket on ss's streams, forked from and joined back into
// `stream`.  account: record phase timers / launch counts in ctx (only from
// the thread that owns ctx).
int enqueue_batch(cg_context *ctx, const BatchLayout &L, const BatchBuffers &bb, unsigned char *base,
                  int32_t *orders, cg_result *res, cudaStream_t stream, const StreamSet &ss, bool account);
size_t layout_staging_bytes(const BatchLayout &L);
// Copies descriptors and offsets through `staging` (pinned host) to the device.
int upload_layout_to(const BatchLayout &L, const BatchBuffers &bb, unsigned char *base, unsigned char *staging,
                     cudaStream_t stream);

}  // namespace cg
