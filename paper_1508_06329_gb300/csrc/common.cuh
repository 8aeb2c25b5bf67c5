// common.cuh — shared helpers of the libchordal CUDA sources (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "chordal.h"

namespace cg {

constexpr int kWarp = 32;

// Records a message for cg_last_error_string() and returns the status.
int set_error(int status, const char *fmt, ...);

#define CG_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::cg::set_error(CG_ECUDA, "%s failed: %s (%s:%d)", #expr,              \
                                   cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)

#define CG_LAUNCH_CHECK(what)                                                              \
    do {                                                                                   \
        cudaError_t e_ = cudaGetLastError();                                               \
        if (e_ != cudaSuccess)                                                             \
            return ::cg::set_error(CG_ECUDA, "launch of %s failed: %s", what,             \
                                   cudaGetErrorString(e_));                                \
    } while (0)

// Asks L2 to fetch [p, p + bytes) (bulk prefetch, no completion tracking).
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---- bulk copies global -> shared memory (cp.async.bulk, completed on an mbarrier)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t arrivals) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}

// Makes shared-memory writes of the generic proxy (and an mbarrier's
// initialisation) visible to the bulk-copy engine.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of bulk-copy data for the phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Copies `bytes` (a multiple of 16; both addresses 16-byte aligned) from
// global memory into this CTA's shared memory; completion counts on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_parity(unsigned long long *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// `limit` polls (each poll may suspend the thread for a short while) and
// returns false then.
__device__ __forceinline__ bool mbar_wait_parity_bounded(unsigned long long *bar, uint32_t parity,
                                                         uint32_t limit = 1u << 22) {
    for (uint32_t k = 0; k < limit; ++k)
        if (mbar_try_wait_parity(bar, parity)) return true;
    return false;
}

// Spreads bulk L2 prefetches of a contiguous range over the CTA's threads.
template <int T>
__device__ __forceinline__ void prefetch_range_l2(const void *base, size_t bytes) {
    constexpr uint32_t kChunk = 32768;
    const uintptr_t a = reinterpret_cast<uintptr_t>(base);
    const uintptr_t a16 = (a + 15) & ~uintptr_t(15);
    if (bytes <= (size_t)(a16 - a)) return;
    size_t left = (bytes - (a16 - a)) & ~size_t(15);
    const size_t chunks = (left + kChunk - 1) / kChunk;
    for (size_t c = threadIdx.x; c < chunks; c += T) {
        const size_t off = c * kChunk;
        const uint32_t len = (uint32_t)((left - off) < kChunk ? (left - off) : kChunk);
        prefetch_l2_bulk(reinterpret_cast<const void *>(a16 + off), len);
    }
}

// Parent value meaning "not known yet": the dense check finds it.
constexpr int kParentUnresolved = -2;

// How the dense LexBFS records parents (when given a parent array).
constexpr int kParentMoves = 0;        // every moved vertex: parent[y] = pivot
constexpr int kParentExact = 1;        // once per pivot, exact (per-class parents)

// Per-graph descriptor as the kernels see it (device memory).
struct DenseDesc {
    const uint32_t *rows;   // n * words
    int32_t n;
    int32_t words;
    int64_t vbase;          // offset of this graph's vertices in the packed pos / parent workspace
    int64_t obase;          // offset of this graph's order in the caller's order array
    int32_t rindex;         // slot of this graph's result
    int32_t pad;
    int64_t ebase;          // word offset of this graph's earlier-than masks in the check's mask buffer
};

// Per-launch buffers of the search that feed the position-ordered check
// (indexed like pos / parent by each graph's vbase; masks by its ebase).
struct CheckFeed {
    int32_t *cpar;                // per-class parents (scratch)
    int32_t *ppos;                // parents by position
    uint32_t *emask;              // earlier-than masks
    unsigned long long *keys;     // [count] witness keys, [count] block counter, [count + 1] error word
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Row stride (words) of a graph's earlier-than masks: ceil(n/32) rounded up to
// a multiple of 4, so every mask row starts on a 16-byte boundary.
__host__ __device__ inline int mask_stride(int n) { return (((n + 31) >> 5) + 3) & ~3; }

}  // namespace cg
