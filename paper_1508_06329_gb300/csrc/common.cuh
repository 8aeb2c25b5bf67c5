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

// Per-graph descriptor as the kernels see it (device memory).
struct DenseDesc {
    const uint32_t *rows;   // n * words
    int32_t n;
    int32_t words;
    int64_t vbase;          // offset of this graph's vertices in the packed pos / parent workspace
    int64_t obase;          // offset of this graph's order in the caller's order array
    int32_t rindex;         // slot of this graph's result
    int32_t pad;
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace cg
