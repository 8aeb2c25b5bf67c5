// batch_dense.cu — the whole chordality test of one small dense graph in one
// CTA, many graphs per launch (the batched path).
//
// Each CTA takes graphs from an atomic counter (graphs pre-sorted largest
// first by the host), runs the partition-refinement LexBFS of
// lexbfs_dense.cuh, then the perfect-elimination check of Sections 5.2 / 6.2
// on the same graph: its warps take vertices v, read p = p(v) (recorded by
// the search) and scan row_v & ~row_p for an earlier vertex other than p; the
// CTA keeps the first violation in order with a shared 64-bit atomicMin on
// (pos(v) << 32 | u) and writes (chordal, v, p, u).  When the rows fit, they
// are copied to shared memory once and serve both phases; positions and
// parents are staged in the search's (then unused) shared arrays.
#include <algorithm>

#include "kernels.h"
#include "lexbfs_dense.cuh"

namespace cg {

namespace {

constexpr uint16_t kNoParent16 = 0xFFFFu;

template <int T>
__device__ void check_cta(const uint32_t *__restrict__ rows, int stride, int n, const uint16_t *__restrict__ spos,
                          const uint16_t *__restrict__ spar, unsigned long long *skey) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = T / 32;
    const int wn = (n + 31) >> 5;
    const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
    for (int v = warp; v < n; v += kWarps) {
        const uint16_t p16 = spar[v];
        if (p16 == kNoParent16) continue;
        const int p = p16;
        const unsigned pv = spos[v];
        const uint32_t *rv = rows + (size_t)v * stride;
        const uint32_t *rp = rows + (size_t)p * stride;
        unsigned umin = kNoVertex;
        for (int w = lane; w < wn && umin == kNoVertex; w += 32) {
            uint32_t bits = rv[w] & ~rp[w];
            if (w == wn - 1) bits &= lastmask;
            if (w == (p >> 5)) bits &= ~(1u << (p & 31));
            while (bits) {
                const int u = (w << 5) + (__ffs(bits) - 1);
                bits &= bits - 1;
                if (spos[u] < pv) {
                    umin = (unsigned)u;
                    break;
                }
            }
        }
        umin = __reduce_min_sync(0xFFFFFFFFu, umin);
        if (lane == 0 && umin != kNoVertex) atomicMin(skey, ((unsigned long long)pv << 32) | umin);
    }
}

template <int T, int WPT, int LPW, bool ROWS_SMEM>
__global__ void __launch_bounds__(T) chordal_dense_fused_kernel(const DenseDesc *__restrict__ descs, int count,
                                                                int32_t *__restrict__ order,
                                                                int32_t *__restrict__ pos,
                                                                int32_t *__restrict__ parent,
                                                                cg_result *__restrict__ res, int *work_counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    LexScalars *sc = reinterpret_cast<LexScalars *>(smem);
    __shared__ unsigned long long skey;
    for (;;) {
        if (threadIdx.x == 0) sc->next_graph = atomicAdd(work_counter, 1);
        __syncthreads();
        const int gi = sc->next_graph;
        __syncthreads();
        if (gi >= count) break;
        const DenseDesc d = descs[gi];
        const int n = d.n;
        unsigned char *p = smem + kLexScalarBytes;
        LexState<uint16_t> st = lex_state_carve<uint16_t>(p, n);
        p += lex_state_bytes<uint16_t>(n);
        const uint32_t *rows = d.rows;
        int stride = d.words;
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
            __syncthreads();
        } else {
            prefetch_range_l2<T>(d.rows, (size_t)n * d.words * sizeof(uint32_t));
        }
        int32_t *ord = order + d.obase;
        int32_t *pg = pos + d.vbase;
        int32_t *par = parent + d.vbase;
        lexbfs_cta<uint16_t, T, WPT, LPW>(rows, stride, n, st, sc, ord, pg, par);
        __syncthreads();
        // positions and parents into the search's shared arrays (no longer used)
        uint16_t *spos = st.cls;
        uint16_t *spar = st.child;
        for (int v = threadIdx.x; v < n; v += T) {
            spos[v] = (uint16_t)pg[v];
            const int pp = par[v];
            spar[v] = pp < 0 ? kNoParent16 : (uint16_t)pp;
        }
        if (threadIdx.x == 0) skey = ~0ull;
        __syncthreads();
        check_cta<T>(rows, stride, n, spos, spar, &skey);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long k = skey;
            cg_result r;
            if (k == ~0ull) {
                r.chordal = 1;
                r.v = r.p = r.u = -1;
            } else {
                r.chordal = 0;
                r.v = ord[(int)(k >> 32)];
                r.p = spar[r.v];
                r.u = (int)(k & 0xFFFFFFFFu);
            }
            res[d.rindex] = r;
        }
        __syncthreads();
    }
}

template <int T, int WPT, int LPW, bool ROWS_SMEM>
int launch_fused(const FusedPlan &plan, const DenseDesc *descs, int count, int ctas, int32_t *order, int32_t *pos,
                 int32_t *parent, cg_result *res, int *work_counter, cudaStream_t stream) {
    auto kern = chordal_dense_fused_kernel<T, WPT, LPW, ROWS_SMEM>;
    CG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes));
    CG_CUDA_TRY(cudaMemsetAsync(work_counter, 0, sizeof(int), stream));
    kern<<<ctas, T, plan.smem_bytes, stream>>>(descs, count, order, pos, parent, res, work_counter);
    CG_LAUNCH_CHECK("chordal_dense_fused_kernel");
    CG_DEBUG_CHECK(stream, "chordal_dense_fused_kernel");
    return CG_OK;
}

}  // namespace

int fused_dense_plan(int n_max, int threads, FusedPlan *plan, bool rows_smem_allowed) {
    if (n_max < 0 || n_max > kFusedMaxN)
        return set_error(CG_EINVAL, "fused batch path supports n <= %d (got %d)", kFusedMaxN, n_max);
    const int n = std::max(n_max, 1);
    const int wn = (n + 31) / 32;
    FusedPlan p{};
    const size_t state = lex_state_bytes<uint16_t>(n);
    const size_t rows = (size_t)n * wn * 4;
    p.rows_smem = rows_smem_allowed && kLexScalarBytes + state + rows <= kFusedSmemLimit;
    if (threads == 0) threads = n <= 256 ? 64 : (n <= 1024 ? 128 : 256);
    if (threads != 64 && threads != 128 && threads != 256 && threads != 512)
        return set_error(CG_EINVAL, "fused batch path: unsupported CTA size %d", threads);
    p.threads = threads;
    p.smem_bytes = kLexScalarBytes + state + (p.rows_smem ? rows : 0);
    *plan = p;
    return CG_OK;
}

int fused_dense_launch(const FusedPlan &plan, const DenseDesc *descs, int count, int ctas, int32_t *order,
                       int32_t *pos, int32_t *parent, cg_result *res, int *work_counter, cudaStream_t stream) {
    if (count <= 0) return CG_OK;
    ctas = std::max(1, std::min(ctas, count));
    // words per thread slice: T * WPT / LPW must cover ceil(kFusedMaxN / 32) = 128 words
#define CG_FUSED_CASE(TT, WW)                                                                                  \
    case TT:                                                                                                   \
        return plan.rows_smem ? launch_fused<TT, WW, 1, true>(plan, descs, count, ctas, order, pos, parent, res, \
                                                               work_counter, stream)                           \
                              : launch_fused<TT, WW, 1, false>(plan, descs, count, ctas, order, pos, parent, res, \
                                                                work_counter, stream);
    switch (plan.threads) {
        CG_FUSED_CASE(64, 2)
        CG_FUSED_CASE(128, 1)
        CG_FUSED_CASE(256, 1)
        CG_FUSED_CASE(512, 1)
        default:
            return set_error(CG_EINVAL, "fused batch path: unsupported CTA size %d", plan.threads);
    }
#undef CG_FUSED_CASE
}

int fused_ctas_per_sm(const FusedPlan &plan) {
    const int by_smem = (int)std::max<size_t>(1, (228 * 1024) / (plan.smem_bytes + 1024 + 16));
    const int by_threads = std::max(1, 2048 / plan.threads);
    return std::max(1, std::min(std::min(by_smem, by_threads), 32));
}

}  // namespace cg
