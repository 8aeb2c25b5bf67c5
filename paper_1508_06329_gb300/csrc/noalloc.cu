// noalloc.cu — cg_chordal_test_dense_noalloc: the dense chordality test for
// callers that must not allocate memory at call time.
//
// Who needs it: code that cannot call cudaMalloc (or any allocating routine)
// when it runs — for example a plugin inside a host application that owns
// the device memory pool and forbids allocations after start-up, a
// latency-critical loop that must never block in the allocator, or a caller
// that has no library context to keep a workspace in.  This entry point takes
// the scratch the test needs (vertex positions, parents, an order buffer when
// the caller passes none, and the witness key) from one fixed array compiled
// into the library's device image instead of a context workspace.
//
// Limits and sharing:
//   * n <= kNoallocMaxN (16,384): the LexBFS state then lives in shared memory
//     and the scratch array is 3 * 64 KiB + 512 B (about 193 KiB).  Every GPU
//     that loads the library holds this array until the process exits.
//   * All calls share the one array and it keeps the last call's contents;
//     the witness key is re-initialised by every call before it is used.
//     Calls that overlap on the GPU (different streams, different host
//     threads) race on the array: serialise them on one stream.
//   * The first call on a device resolves the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make
//     that first call before any stream capture begins.  The address is kept
//     for the life of the process, which assumes the device's primary context
//     is never reset: after cudaDeviceReset (or with another context made
//     current on the device) the kept address would be stale.
#include <atomic>
#include <mutex>

#include "kernels.h"

namespace cg {
namespace {

constexpr int kNoallocMaxN = 16384;
constexpr size_t kVecBytes = (size_t)kNoallocMaxN * sizeof(int32_t);   // 64 KiB, 256-aligned
constexpr size_t kOffPos = 0;
constexpr size_t kOffParent = kOffPos + kVecBytes;
constexpr size_t kOffOrder = kOffParent + kVecBytes;
constexpr size_t kOffKey = kOffOrder + kVecBytes;
constexpr size_t kOffCounter = kOffKey + 256;
constexpr size_t kScratchBytes = kOffCounter + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
std::atomic<unsigned char *> g_scratch_addr[kMaxDevices];
std::atomic<int> g_num_sms[kMaxDevices];

// Resolves (once per device) the device address of the scratch array.
int scratch_for_current_device(unsigned char **out, int *num_sms) {
    int dev = 0;
    CG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(CG_EINVAL, "device ordinal %d out of range", dev);
    unsigned char *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        p = g_scratch_addr[dev].load(std::memory_order_acquire);
        if (!p) {
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess || !addr)
                return set_error(CG_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed on device %d: %s",
                                 dev, cudaGetErrorString(e));
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess)
                return set_error(CG_ECUDA, "cudaDeviceGetAttribute failed on device %d: %s", dev,
                                 cudaGetErrorString(e));
            g_num_sms[dev].store(sms, std::memory_order_relaxed);
            p = static_cast<unsigned char *>(addr);
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    *num_sms = g_num_sms[dev].load(std::memory_order_relaxed);
    return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" int cg_chordal_test_dense_noalloc(const cg_dense *g, cg_result *res, int32_t *order,
                                             cudaStream_t stream) {
    if (!g) return set_error(CG_EINVAL, "null graph descriptor");
    if (!res) return set_error(CG_EINVAL, "null result pointer");
    if (g->n < 0) return set_error(CG_EINVAL, "n must be >= 0 (got %d)", g->n);
    if (g->n > kNoallocMaxN)
        return set_error(CG_EINVAL,
                         "n = %d exceeds the no-allocation limit of %d vertices; use cg_chordal_test_dense",
                         g->n, kNoallocMaxN);
    if (g->n > 0 && !g->rows) return set_error(CG_EINVAL, "null rows pointer");
    if (g->words_per_row < (g->n + 31) / 32)
        return set_error(CG_EINVAL, "words_per_row %d < ceil(n/32) = %d", g->words_per_row, (g->n + 31) / 32);
    unsigned char *scratch = nullptr;
    int num_sms = 0;
    int rc = scratch_for_current_device(&scratch, &num_sms);
    if (rc) return rc;
    const int n = g->n;
    LexPlan plan;
    if ((rc = lexbfs_dense_plan(n, 0, &plan))) return rc;
    if (plan.gstate_bytes) return set_error(CG_EINVAL, "no-allocation path needs the shared-memory variant");
    int32_t *pos = reinterpret_cast<int32_t *>(scratch + kOffPos);
    int32_t *parent = reinterpret_cast<int32_t *>(scratch + kOffParent);
    int32_t *ord = order ? order : reinterpret_cast<int32_t *>(scratch + kOffOrder);
    unsigned long long *key = reinterpret_cast<unsigned long long *>(scratch + kOffKey);
    int *counter = reinterpret_cast<int *>(scratch + kOffCounter);
    DenseDesc d{};
    d.rows = g->rows;
    d.n = n;
    d.words = g->words_per_row;
    d.vbase = 0;
    d.obase = 0;
    if (n > 0 && (rc = lexbfs_dense_launch(plan, nullptr, d, 1, 1, ord, pos, parent, nullptr, counter, stream)))
        return rc;
    // peo_dense_launch resets the key to its "no violation" value before the check
    if ((rc = peo_dense_launch(nullptr, d, 1, nullptr, n, ord, pos, parent, true, key, num_sms, stream))) return rc;
    return finalize_launch(nullptr, d, 1, key, ord, parent, res, stream);
}
