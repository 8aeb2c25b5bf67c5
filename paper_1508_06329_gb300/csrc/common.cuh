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
constexpr int kParentMoves = 0;        // every moved vertex: parent[v] = pivot
constexpr int kParentPivots = 1;       // once per step, by position: parent[i], or kParentUnresolved

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


__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Row stride (words) of a graph's earlier-than masks: ceil(n/32) rounded up to
// a multiple of 4, so every mask row starts on a 16-byte boundary.
__host__ __device__ inline int mask_stride(int n) { return (((n + 31) >> 5) + 3) & ~3; }

}  // namespace cg
