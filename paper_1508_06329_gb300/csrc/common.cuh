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

// Describes a bounds-check error word (host side; the release build never sets one).
const char *cg_debug_array_name(unsigned code);

#ifdef CG_BOUNDS_CHECK
// After a launch: synchronise, read and clear this translation unit's error word.
// (Skipped while the stream is being captured into a CUDA graph: a batch plan
// replays unchecked launches.)
#define CG_DEBUG_CHECK(stream, what)                                                        \
    do {                                                                                    \
        cudaStreamCaptureStatus cs_ = cudaStreamCaptureStatusNone;                          \
        if (cudaStreamIsCapturing(stream, &cs_) != cudaSuccess || cs_ != cudaStreamCaptureStatusNone) break; \
        cudaError_t e_ = cudaStreamSynchronize(stream);                                     \
        unsigned long long w_ = 0, z_ = 0;                                                  \
        if (e_ == cudaSuccess) e_ = cudaMemcpyFromSymbol(&w_, ::cg::cg_dbg_word, sizeof(w_)); \
        if (e_ == cudaSuccess && w_) e_ = cudaMemcpyToSymbol(::cg::cg_dbg_word, &z_, sizeof(z_)); \
        if (e_ != cudaSuccess)                                                              \
            return ::cg::set_error(CG_ECUDA, "%s: %s", what, cudaGetErrorString(e_));      \
        if (w_)                                                                             \
            return ::cg::set_error(CG_ECUDA, "bounds check in %s: %s index %llu out of range", what, \
                                   ::cg::cg_debug_array_name((unsigned)(w_ >> 56)),        \
                                   (unsigned long long)(w_ & ((1ull << 56) - 1)));          \
    } while (0)
#else
#define CG_DEBUG_CHECK(stream, what) \
    do {                             \
    } while (0)
#endif

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

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- per-thread asynchronous copies global -> shared memory (cp.async, 16 bytes,
// cached in L2 only), waited for by commit group
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's most recent commit groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
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

// ---- bounds-checking build (-DCG_BOUNDS_CHECK)
// The state arrays of the searches and the check are declared CG_ARR(T): a
// plain pointer in the release build; in the bounds-checking build a pointer
// with its length, whose operator[] records an out-of-range index in the
// translation unit's error word (array code and index; the first one wins)
// and redirects the access to a scratch element instead of going out of
// bounds.  Each launcher then synchronises and turns a non-zero word into
// CG_ECUDA with a description (CG_DEBUG_CHECK).
#ifdef CG_BOUNDS_CHECK
static __device__ unsigned long long cg_dbg_word;       // this translation unit's error word
static __device__ unsigned long long cg_dbg_sink[2];    // target of redirected accesses

__device__ __forceinline__ void cg_dbg_record(unsigned code, unsigned long long idx) {
    atomicCAS(&cg_dbg_word, 0ull, ((unsigned long long)(code & 0xFFu) << 56) | (idx & ((1ull << 56) - 1)));
}

template <typename T>
struct Chk {
    T *p;
    unsigned long long n;
    unsigned code;
    __device__ T &operator[](long long i) const {
        if ((unsigned long long)i >= n) {
            cg_dbg_record(code, (unsigned long long)i);
            return *reinterpret_cast<T *>(cg_dbg_sink);
        }
        return p[i];
    }
    __host__ __device__ operator T *() const { return p; }
};
template <typename T>
__device__ __forceinline__ Chk<T> cg_arr(T *p, unsigned long long n, unsigned code) {
    return Chk<T>{p, n, code};
}
#define CG_ARR(T) ::cg::Chk<T>
#else
template <typename T>
__device__ __forceinline__ T *cg_arr(T *p, unsigned long long, unsigned) {
    return p;
}
#define CG_ARR(T) T *
#endif

// Array codes of the bounds-checking build (the high byte of the error word).
enum : unsigned {
    kChkCls = 1, kChkChild, kChkFree, kChkCnext, kChkCprev, kChkSize, kChkNumbered, kChkRow, kChkMoved,
    kChkCsrCls = 16, kChkCsrVnext, kChkCsrVprev, kChkCsrCnext, kChkCsrCprev, kChkCsrCfirst, kChkCsrClast,
    kChkCsrCsize, kChkCsrCmoved, kChkCsrCchild, kChkCsrFree, kChkCsrSy, kChkCsrSop, kChkCsrSon, kChkCsrSrun,
    kChkCsrSkey,
    kChkUnitMask = 40, kChkUnitPos, kChkUnitRow, kChkUnitGroup,
    kChkInjected = 255,
};

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
