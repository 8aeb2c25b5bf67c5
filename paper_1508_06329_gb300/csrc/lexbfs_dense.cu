// lexbfs_dense.cu — kernels and launcher of the one-CTA-per-graph dense LexBFS.
#include <algorithm>

#include "kernels.h"
#include "lexbfs_dense.cuh"

namespace cg {

#ifdef CG_BOUNDS_CHECK
// A code set by cg_debug_inject: the next dense LexBFS launch records it as a
// bounds-check error without touching memory out of range (a test of the
// status path).
static __device__ unsigned cg_dbg_inject_code;
#endif

namespace {

constexpr size_t kSmemLimit = 227 * 1024;   // opt-in dynamic shared memory per CTA (sm_100 family)
constexpr int kSmemMaxN = 16384;             // 16-bit ids, whole state in shared memory
constexpr int kSplitMaxN = 65520;            // 16-bit ids, class ids in shared memory, class arrays global
constexpr int kWideMaxN = 131072;            // 32-bit ids: 4 words per thread at 1024 threads

template <typename Id, int T, int WPT, int LPW, bool ROWS_SMEM, int SPLIT = 0>
__global__ void __launch_bounds__(T) lexbfs_dense_kernel(const DenseDesc *__restrict__ descs, DenseDesc single,
                                                         int count, int32_t *__restrict__ order,
                                                         int32_t *__restrict__ pos, int32_t *__restrict__ parent,
                                                         int pmode, unsigned char *gstate, size_t gstate_stride,
                                                         int *work_counter, uint32_t *emask,
                                                         int32_t *cpar, bool cpar_smem) {
    extern __shared__ __align__(16) unsigned char smem[];
    LexScalars *sc = reinterpret_cast<LexScalars *>(smem);
    unsigned char *free_smem = smem + kLexScalarBytes;
#ifdef CG_BOUNDS_CHECK
    if (blockIdx.x == 0 && threadIdx.x == 0 && cg_dbg_inject_code) {
        cg_dbg_record(cg_dbg_inject_code, 0ull);
        cg_dbg_inject_code = 0u;
    }
#endif
    for (;;) {
        if (threadIdx.x == 0) sc->next_graph = count == 1 ? (int)blockIdx.x : atomicAdd(work_counter, 1);
        __syncthreads();
        const int gi = sc->next_graph;
        __syncthreads();
        if (gi >= count) break;
        const DenseDesc d = descs ? descs[gi] : single;
        const int n = d.n;
        LexState<Id> st;
        unsigned char *p = free_smem;
        // where the state lives is fixed per variant at compile time, so every
        // state access compiles to a shared- or a global-memory instruction
        // (a runtime choice leaves generic loads, stores and atomics)
        if constexpr (SPLIT != 0) {   // split layouts 1..3
            st = lex_state_carve_split<Id, SPLIT>(p, gstate + (size_t)blockIdx.x * gstate_stride, n);
            p += lex_split_smem_bytes<Id>(n, SPLIT);
        } else if constexpr (sizeof(Id) == 4) {   // 32-bit ids: the whole state in the workspace
            st = lex_state_carve<Id>(gstate + (size_t)blockIdx.x * gstate_stride, n);
        } else {
            st = lex_state_carve<Id>(p, n);
            p += lex_state_bytes<Id>(n);
        }
        const uint32_t *rows = d.rows;
        int stride = d.words;
        if (!ROWS_SMEM) prefetch_range_l2<T>(d.rows, (size_t)n * d.words * sizeof(uint32_t));
        if (ROWS_SMEM) {
            const int wn = (n + 31) >> 5;
            uint32_t *srows = reinterpret_cast<uint32_t *>(p);
            const int64_t total = (int64_t)n * wn;
            for (int64_t k = threadIdx.x; k < total; k += T) {
                const int r = (int)(k / wn), w = (int)(k - (int64_t)r * wn);
                srows[k] = __ldg(d.rows + (size_t)r * d.words + w);
            }
            rows = srows;
            stride = wn;
            p += ((size_t)n * wn * sizeof(uint32_t) + 15) & ~size_t(15);
            __syncthreads();
        }
        // the per-class last pivot: in shared memory when it fits beside the state
        int32_t *cp = cpar ? (cpar_smem ? reinterpret_cast<int32_t *>(p) : cpar + d.vbase) : nullptr;
        lexbfs_cta<Id, T, WPT, LPW, layout_mv(SPLIT) ? 1 : layout_arr(SPLIT) ? 2 : 0>(rows, stride, n, st, sc, order + d.obase, pos ? pos + d.vbase : nullptr,
                                    parent ? parent + d.vbase : nullptr, pmode, emask ? emask + d.ebase : nullptr,
                                    cp);
        __syncthreads();
        if (count == 1) break;
    }
}

template <typename Id, int T, int WPT, int LPW, bool ROWS_SMEM, int SPLIT = 0>
int launch_variant(const LexPlan &plan, const DenseDesc *descs, DenseDesc single, int count, int ctas,
                   int32_t *order, int32_t *pos, int32_t *parent, int pmode, void *gstate,
                   int *work_counter, cudaStream_t stream, unsigned long long *keys, uint32_t *emask,
                   int32_t *cpar) {
    auto kern = lexbfs_dense_kernel<Id, T, WPT, LPW, ROWS_SMEM, SPLIT>;
    // cpar in shared memory when it fits (one store per split class per step:
    // in global memory it cost ~0.2 us per step on G(n, 0.5), n = 10,000)
    const size_t cpar_bytes = cpar ? ((size_t)plan.n_max * sizeof(int32_t) + 15) & ~size_t(15) : 0;
    const bool cpar_smem = cpar && !SPLIT && sizeof(Id) == 2 && plan.smem_bytes + cpar_bytes <= kSmemLimit;
    const size_t smem = plan.smem_bytes + (cpar_smem ? cpar_bytes : 0);
    CG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (count > 1) CG_CUDA_TRY(cudaMemsetAsync(work_counter, 0, sizeof(int), stream));
    kern<<<ctas, T, smem, stream>>>(descs, single, count, order, pos, parent, pmode,
                                    static_cast<unsigned char *>(gstate), plan.gstate_bytes, work_counter, emask,
                                    cpar, cpar_smem);
    if (keys) {   // the check's initial keys: "no violation", then the CTA counter and error word
        CG_CUDA_TRY(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * count, stream));
        CG_CUDA_TRY(cudaMemsetAsync(keys + count, 0, 2 * sizeof(unsigned long long), stream));
    }
    CG_LAUNCH_CHECK("lexbfs_dense_kernel");
    CG_DEBUG_CHECK(stream, "lexbfs_dense_kernel");
    return CG_OK;
}

}  // namespace

int lexbfs_dense_plan(int n_max, int threads_override, LexPlan *plan) {
    if (n_max < 0 || n_max > kWideMaxN)
        return set_error(CG_EINVAL, "dense LexBFS supports n <= %d (got %d); use the CSR entry points", kWideMaxN,
                         n_max);
    LexPlan p{};
    const int n = std::max(n_max, 1);
    const int wn = (n + 31) / 32;
    if (n <= kSmemMaxN) {
        const size_t state = lex_state_bytes<uint16_t>(n);
        const size_t rows = ((size_t)n * wn * 4 + 15) & ~size_t(15);
        p.wide_ids = false;
        p.rows_smem = kLexScalarBytes + state + rows <= kSmemLimit;
        // measured on GB300 (subtree, clique, tree, G(n, 0.1) graphs): 512 threads
        // up to ~1,500 vertices, 1024 above (more lanes per row word shorten the
        // per-step bit loops more than the extra warps cost at the barriers)
        int th = n <= 1536 ? 512 : 1024;
        if (threads_override) th = threads_override;
        // words per thread must cover the row
        while ((int64_t)th * (th == 128 ? 4 : th == 256 ? 2 : 1) < wn) th *= 2;
        p.threads = std::min(th, 1024);
        p.smem_bytes = kLexScalarBytes + state + (p.rows_smem ? rows : 0);
        p.gstate_bytes = 0;
    } else if (n <= kSplitMaxN) {
        p.wide_ids = false;
        p.rows_smem = false;
        p.threads = 1024;
        // as much of the per-class state in shared memory as fits
        p.split_state = kLayoutSplitArr;
        for (int l : {kLayoutSplitMvChild, kLayoutSplitMv})
            if (kLexScalarBytes + lex_split_smem_bytes<uint16_t>(n, l) <= kSmemLimit) {
                p.split_state = l;
                break;
            }
        p.smem_bytes = kLexScalarBytes + lex_split_smem_bytes<uint16_t>(n, p.split_state);
        p.gstate_bytes = lex_split_global_bytes<uint16_t>(n, p.split_state);
    } else {
        p.wide_ids = true;
        p.rows_smem = false;
        p.threads = 1024;
        p.smem_bytes = kLexScalarBytes;
        p.gstate_bytes = (lex_state_bytes<uint32_t>(n) + 255) & ~size_t(255);
    }
    if (p.threads != 128 && p.threads != 256 && p.threads != 512 && p.threads != 1024)
        return set_error(CG_EINVAL, "unsupported CTA size %d", p.threads);
    p.n_max = n;
    *plan = p;
    return CG_OK;
}

int lexbfs_dense_launch(const LexPlan &plan, const DenseDesc *descs, DenseDesc single, int count, int ctas,
                        int32_t *order, int32_t *pos, int32_t *parent, void *gstate, int *work_counter,
                        cudaStream_t stream, int parent_mode, unsigned long long *keys, uint32_t *emask,
                        int32_t *cpar) {
    if (count <= 0) return CG_OK;
    if (emask && (reinterpret_cast<uintptr_t>(emask) & 15) != 0)
        return set_error(CG_EINVAL, "earlier-than mask buffer not 16-byte aligned");
    ctas = std::max(1, std::min(ctas, count));
    auto go = [&](auto launch, void *gs) {
        return launch(plan, descs, single, count, ctas, order, pos, parent, parent_mode, gs, work_counter, stream,
                      keys, emask, cpar);
    };
    if (plan.split_state == kLayoutSplitMvChild)
        return go(launch_variant<uint16_t, 1024, 2, 1, false, kLayoutSplitMvChild>, gstate);
    if (plan.split_state == kLayoutSplitMv) return go(launch_variant<uint16_t, 1024, 2, 1, false, kLayoutSplitMv>, gstate);
    if (plan.split_state) return go(launch_variant<uint16_t, 1024, 2, 1, false, kLayoutSplitArr>, gstate);
    if (plan.wide_ids) return go(launch_variant<uint32_t, 1024, 4, 1, false>, gstate);
    switch (plan.threads) {
        case 128:
            return plan.rows_smem ? go(launch_variant<uint16_t, 128, 4, 1, true>, nullptr)
                                  : go(launch_variant<uint16_t, 128, 4, 1, false>, nullptr);
        case 256:
            return plan.rows_smem ? go(launch_variant<uint16_t, 256, 2, 1, true>, nullptr)
                                  : go(launch_variant<uint16_t, 256, 2, 1, false>, nullptr);
        case 512:
            return plan.rows_smem ? go(launch_variant<uint16_t, 512, 1, 1, true>, nullptr)
                                  : go(launch_variant<uint16_t, 512, 1, 1, false>, nullptr);
        default:
            return go(launch_variant<uint16_t, 1024, 1, 2, false>, nullptr);
    }
}

int debug_inject(unsigned code) {
#ifdef CG_BOUNDS_CHECK
    CG_CUDA_TRY(cudaMemcpyToSymbol(cg_dbg_inject_code, &code, sizeof(code)));
    return CG_OK;
#else
    (void)code;
    return set_error(CG_EINVAL, "not a bounds-checking build (CG_BOUNDS_CHECK)");
#endif
}

}  // namespace cg
