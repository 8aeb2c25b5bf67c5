// floor.cu — latency floors that bound one step of the sequential LexBFS
// loop (Section 6.1: n dependent steps): an empty loop of CTA-wide barriers,
// and a chain of dependent global loads (one memory round trip each).
// Measurement aid only; the chordality path never calls it.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "host.h"

namespace cg {
namespace {

constexpr int kLineInts = 32;   // one chain node per 128-byte line

// Two CTA-wide barriers per iteration: the synchronisation a dense LexBFS
// step cannot avoid (pivot known, then the refined classes published).
__global__ void __launch_bounds__(1024) barrier_pair_kernel(int32_t iters, int32_t *sink) {
    for (int32_t i = 0; i < iters; ++i) {
        asm volatile("bar.sync 0;" ::: "memory");
        asm volatile("bar.sync 0;" ::: "memory");
    }
    if (threadIdx.x == 0) sink[0] = iters;
}

// Chain node k (at int index k * 32) points to node (a k + c) mod 2^bits.
// With c odd and a = 1 mod 4 this map is one cycle through all 2^bits nodes
// (Hull-Dobell full-period condition), so a walk visits lines in a
// scattered order without repeating one before it has seen them all.
__global__ void chain_init_kernel(int32_t *next, int bits) {
    const uint64_t nodes = 1ull << bits, mask = nodes - 1;
    const uint64_t a = 6364136223846793005ull, c = 1442695040888963407ull;
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nodes;
         k += (uint64_t)gridDim.x * blockDim.x)
        next[k * kLineInts] = (int32_t)(((a * k + c) & mask) * kLineInts);
}

// One thread follows `loads` dependent loads (L2-cached, L1 bypassed),
// starting where the previous walk stopped (at[0], a chain index), so that
// repeated walks of a chain larger than L2 keep meeting lines not yet read.
__global__ void chain_walk_kernel(const int32_t *__restrict__ next, int32_t loads, int32_t *at) {
    int32_t i = at[0];
    for (int32_t k = 0; k < loads; ++k) i = __ldcg(next + i);
    at[0] = i;
}

// Smallest of `reps` timings (ms) of launch() on `stream`.
template <typename F>
int best_ms(cudaStream_t stream, int reps, F launch, float *out) {
    cudaEvent_t a, b;
    CG_CUDA_TRY(cudaEventCreate(&a));
    CG_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    int rc = CG_OK;
    for (int r = 0; r < reps && rc == CG_OK; ++r) {
        cudaEventRecord(a, stream);
        launch();
        cudaEventRecord(b, stream);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess)
            rc = set_error(CG_ECUDA, "step floor timing failed: %s", cudaGetErrorString(e));
        else if (ms < best)
            best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *out = best;
    return rc;
}

}  // namespace
}  // namespace cg

extern "C" int cg_step_floor(cg_context *ctx, int32_t threads, int32_t iters, int64_t chain_bytes,
                             int32_t loads, cudaStream_t stream, cg_step_floor_info *out) {
    using namespace cg;
    if (!ctx) return set_error(CG_EINVAL, "null context");
    if (!out) return set_error(CG_EINVAL, "null result pointer");
    if (threads < 32 || threads > 1024 || threads % 32)
        return set_error(CG_EINVAL, "threads must be a multiple of 32 in [32, 1024] (got %d)", threads);
    if (iters < 1 || iters > (1 << 24)) return set_error(CG_EINVAL, "iters must be in [1, 2^24] (got %d)", iters);
    if (loads < 1 || loads > (1 << 24)) return set_error(CG_EINVAL, "loads must be in [1, 2^24] (got %d)", loads);
    if (chain_bytes < 256 || chain_bytes > (int64_t(1) << 32))
        return set_error(CG_EINVAL, "chain_bytes must be in [256, 2^32] (got %lld)", (long long)chain_bytes);
    CG_CUDA_TRY(cudaSetDevice(ctx->cfg.device));

    int bits = 1;   // largest power-of-two node count whose lines fit chain_bytes
    while ((int64_t(128) << (bits + 1)) <= chain_bytes) ++bits;
    const size_t bytes = size_t(128) << bits;   // node index * 32 < 2^30: fits int32
    int32_t *buf = nullptr, *sink = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess || cudaMalloc(&sink, 2 * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return set_error(CG_ENOMEM, "step floor scratch allocation (%zu bytes) failed", bytes);
    }
    int rc = CG_OK;
    float t_bar = 0.f, t_bar0 = 0.f, t_walk = 0.f, t_walk0 = 0.f;
    const int reps = 3;
    chain_init_kernel<<<ctx->num_sms * 4, 256, 0, stream>>>(buf, bits);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(sink, 0, 2 * sizeof(int32_t), stream);   // walks start at node 0
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) rc = set_error(CG_ECUDA, "chain init failed: %s", cudaGetErrorString(e));
    // The init kernel's writes leave a chain that fits L2 resident there.
    if (rc == CG_OK)
        rc = best_ms(stream, reps, [&] { barrier_pair_kernel<<<1, threads, 0, stream>>>(iters, sink + 1); }, &t_bar);
    if (rc == CG_OK)
        rc = best_ms(stream, reps, [&] { barrier_pair_kernel<<<1, threads, 0, stream>>>(0, sink + 1); }, &t_bar0);
    if (rc == CG_OK)
        rc = best_ms(stream, reps, [&] { chain_walk_kernel<<<1, 1, 0, stream>>>(buf, loads, sink); }, &t_walk);
    if (rc == CG_OK)
        rc = best_ms(stream, reps, [&] { chain_walk_kernel<<<1, 1, 0, stream>>>(buf, 0, sink); }, &t_walk0);
    cudaFree(buf);
    cudaFree(sink);
    if (rc != CG_OK) return rc;
    out->barrier_pair_ns = (double)std::max(t_bar - t_bar0, 0.f) * 1e6 / iters;
    out->load_ns = (double)std::max(t_walk - t_walk0, 0.f) * 1e6 / loads;
    out->chain_bytes = (int64_t)bytes;
    return CG_OK;
}
