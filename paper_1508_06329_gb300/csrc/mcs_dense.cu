// mcs_dense.cu — Maximum Cardinality Search on dense graphs, one CTA per graph.
//
// Method (Section 5.1; Tarjan and Yannakakis): every unnumbered vertex carries
// the number of its numbered neighbours; each step numbers a vertex with the
// largest count (lowest id among equals, as for LexBFS) and counts it at its
// unnumbered neighbours.  By Theorem 5.2 the graph is chordal iff the MCS
// order is a perfect elimination order, so the same check follows.
//
// GPU form: counts as 16-bit values in shared memory (n <= 65,520 fits) with a
// numbered bitmask.  Thread t owns a bit slice of row words (as in the LexBFS
// kernel) and keeps in a register the largest key (count << 16 | 65535 - v)
// of the unnumbered vertices of its slice.  A step: the owners of the pivot's
// unnumbered neighbours raise their counts and keys; the owner of the pivot's
// own slice (or, for slices longer than 4 bits, that thread's warp) rescans
// it; a block-wide max of the keys (warp max, one barrier,
// then every warp reduces the warp maxima) names the next pivot.  One
// __syncthreads per step.  The pivot's row is the one load on the step's
// critical path: a graph whose rows fit beside the counts is first copied into
// shared memory (n <= ~1,340); a larger one is bulk-prefetched into L2.
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kMcsMaxN = 65520;
constexpr size_t kMcsSmemRows = 200 * 1024;   // dynamic shared memory limit for the row copy

template <int T, int WPT, bool WARP_RESCAN>
__global__ void __launch_bounds__(T) mcs_dense_kernel(const DenseDesc *__restrict__ descs, DenseDesc single, int count,
                                                      int32_t *__restrict__ order, int32_t *__restrict__ pos,
                                                      int *work_counter, uint32_t smem_bytes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned red[2][T / 32];
    __shared__ int next_graph;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (;;) {
        if (t == 0) next_graph = count == 1 ? (int)blockIdx.x : atomicAdd(work_counter, 1);
        __syncthreads();
        const int gi = next_graph;
        __syncthreads();
        if (gi >= count) break;
        const DenseDesc d = descs ? descs[gi] : single;
        const int n = d.n;
        if (n <= 0) {
            if (count == 1) break;
            continue;
        }
        int32_t *ord = order + d.obase;
        int32_t *ps = pos ? pos + d.vbase : nullptr;
        const int wn = (n + 31) >> 5;
        const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
        const size_t label_bytes = ((size_t)n * 2 + 15) & ~size_t(15);
        const size_t state_bytes = label_bytes + (size_t)wn * 4;
        uint16_t *label = reinterpret_cast<uint16_t *>(smem);
        uint32_t *numbered = reinterpret_cast<uint32_t *>(smem + label_bytes);
        const uint32_t *rows = d.rows;
        int stride = d.words;
        const size_t rows_off = (state_bytes + 15) & ~size_t(15);
        if (rows_off + (size_t)n * wn * 4 <= smem_bytes) {   // compact copy (stride wn) beside the counts
            uint32_t *rs = reinterpret_cast<uint32_t *>(smem + rows_off);
            for (int v = warp; v < n; v += T / 32)
                for (int w = lane; w < wn; w += 32) rs[(size_t)v * wn + w] = __ldg(d.rows + (size_t)v * d.words + w);
            rows = rs;
            stride = wn;
        } else {
            prefetch_range_l2<T>(d.rows, (size_t)n * d.words * sizeof(uint32_t));
        }
        int lpw = 1;
        while (lpw < 32 && T / (lpw * 2) >= wn) lpw *= 2;
        const int kGroups = T / lpw, kSlice = 32 / lpw;
        const int lpwShift = __ffs(lpw) - 1, sliceShift = __ffs(kSlice) - 1, groupShift = __ffs(kGroups) - 1;
        const int wt = t / lpw, sl = t % lpw;
        const uint32_t part = lpw == 1 ? 0xFFFFFFFFu : (((1u << kSlice) - 1u) << (sl * kSlice));
        for (int v = t; v < n; v += T) label[v] = 0;
        for (int w = t; w < wn; w += T) numbered[w] = 0u;
        // initial keys: count 0, so the lowest id of each slice
        unsigned kmax[WPT];
        uint32_t row[WPT];
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const int w = k * kGroups + wt;
            uint32_t valid = w < wn ? (w == wn - 1 ? lastmask : 0xFFFFFFFFu) & part : 0u;
            kmax[k] = valid ? (65535u - (unsigned)((w << 5) + __ffs(valid) - 1)) : 0u;
        }
        int x = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < WPT; ++k) {   // row of vertex 0, the first pivot
            const int w = k * kGroups + wt;
            row[k] = w < wn ? rows[w] & part : 0u;
        }
        for (int i = 0; i < n; ++i) {
            const int slot = i & 1;
            if (t == 0) {
                ord[i] = x;
                if (ps) ps[x] = i;
            }
            unsigned best = 0u;
            if constexpr (!WARP_RESCAN) {
                // short slices: the owner of x's slice recomputes its maximum without x
#pragma unroll
                for (int k = 0; k < WPT; ++k) {
                    const int w = k * kGroups + wt;
                    if (w < wn) {
                        uint32_t nb = numbered[w];
                        const bool mine = w == (x >> 5) && ((part >> (x & 31)) & 1u);
                        if (mine) {
                            nb |= 1u << (x & 31);
                            numbered[w] = nb;
                        }
                        uint32_t bits = row[k] & ~nb;   // unnumbered neighbours of x in this slice
                        if (w == wn - 1) bits &= lastmask;
                        while (bits) {
                            const int y = (w << 5) + __ffs(bits) - 1;
                            bits &= bits - 1;
                            const unsigned c = (unsigned)label[y] + 1u;
                            label[y] = (uint16_t)c;
                            const unsigned key = (c << 16) | (65535u - (unsigned)y);
                            kmax[k] = key > kmax[k] ? key : kmax[k];
                        }
                        if (mine) {
                            uint32_t live = ~nb & part;
                            if (w == wn - 1) live &= lastmask;
                            unsigned m = 0u;
                            while (live) {
                                const int y = (w << 5) + __ffs(live) - 1;
                                live &= live - 1;
                                const unsigned key = ((unsigned)label[y] << 16) | (65535u - (unsigned)y);
                                m = key > m ? key : m;
                            }
                            kmax[k] = m;
                        }
                    }
                    best = kmax[k] > best ? kmax[k] : best;
                }
            } else {
                // long slices: the warp of x's owner recomputes that slice's
                // maximum without x, one lane per vertex.  x's slice: word xw,
                // slice xs, held by thread xt as its item xk (lpw, kSlice and
                // kGroups are powers of two).
                const int xw = x >> 5, xs = (x & 31) >> sliceShift;
                const int xk = xw >> groupShift, xt = ((xw & (kGroups - 1)) << lpwShift) + xs;
#pragma unroll
                for (int k = 0; k < WPT; ++k) {
                    const int w = k * kGroups + wt;
                    if (w < wn) {
                        uint32_t nb = numbered[w];
                        if (t == xt && k == xk) {
                            nb |= 1u << (x & 31);
                            numbered[w] = nb;
                        }
                        uint32_t bits = row[k] & ~nb;
                        if (w == wn - 1) bits &= lastmask;
                        unsigned km = kmax[k];
                        while (bits) {
                            const int y = (w << 5) + __ffs(bits) - 1;
                            bits &= bits - 1;
                            const unsigned c = (unsigned)label[y] + 1u;
                            label[y] = (uint16_t)c;
                            km = max(km, (c << 16) | (65535u - (unsigned)y));
                        }
                        kmax[k] = km;
                    }
                }
                if ((xt >> 5) == warp) {
                    __syncwarp();
                    const int y = (xw << 5) + xs * kSlice + lane;
                    unsigned key = 0u;
                    if (lane < kSlice && y < n && !((numbered[xw] >> (y & 31)) & 1u))
                        key = ((unsigned)label[y] << 16) | (65535u - (unsigned)y);
                    key = __reduce_max_sync(0xFFFFFFFFu, key);
#pragma unroll
                    for (int k = 0; k < WPT; ++k)
                        if (t == xt && k == xk) kmax[k] = key;
                }
#pragma unroll
                for (int k = 0; k < WPT; ++k) best = kmax[k] > best ? kmax[k] : best;
            }
            best = __reduce_max_sync(0xFFFFFFFFu, best);
            if (lane == 0) red[slot][warp] = best;
            __syncthreads();
            const unsigned r = lane < T / 32 ? red[slot][lane] : 0u;
            const unsigned top = __reduce_max_sync(0xFFFFFFFFu, r);
            if (i + 1 == n) break;
            x = (int)(65535u - (top & 0xFFFFu));
            if (x >= n) x = n - 1;   // unreachable while an unnumbered vertex remains; keeps loads in bounds
#pragma unroll
            for (int k = 0; k < WPT; ++k) {
                const int w = k * kGroups + wt;
                row[k] = w < wn ? rows[(size_t)x * stride + w] & part : 0u;
            }
        }
        __syncthreads();
        if (count == 1) break;
    }
}

// Lanes per row word as the kernel chooses them for n (the smallest power of
// two whose word groups still cover the row).
int mcs_lpw(int T, int n) {
    const int wn = (n + 31) / 32;
    int lpw = 1;
    while (lpw < 32 && T / (lpw * 2) >= wn) lpw *= 2;
    return lpw;
}

template <int T, int WPT>
int launch_mcs(size_t smem, const DenseDesc *descs, DenseDesc single, int count, int n_max, int ctas,
               int32_t *order, int32_t *pos, int *work_counter, cudaStream_t stream) {
    // slices of more than 4 bits are rescanned by a warp, shorter ones by their owner
    auto kern = 32 / mcs_lpw(T, n_max) > 4 ? mcs_dense_kernel<T, WPT, true> : mcs_dense_kernel<T, WPT, false>;
    CG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (count > 1) CG_CUDA_TRY(cudaMemsetAsync(work_counter, 0, sizeof(int), stream));
    kern<<<ctas, T, smem, stream>>>(descs, single, count, order, pos, work_counter, (uint32_t)smem);
    CG_LAUNCH_CHECK("mcs_dense_kernel");
    return CG_OK;
}

}  // namespace

int mcs_dense_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, int ctas, int32_t *order,
                     int32_t *pos, int *work_counter, cudaStream_t stream) {
    if (count <= 0 || n_max <= 0) return CG_OK;
    if (n_max > kMcsMaxN) return set_error(CG_EINVAL, "dense MCS supports n <= %d (got %d)", kMcsMaxN, n_max);
    // counts + numbered bits; with the rows too when they fit (n <= ~1,340)
    const size_t wn = (size_t)(n_max + 31) / 32;
    const size_t state = ((((size_t)n_max * 2 + 15) & ~size_t(15)) + wn * 4 + 15) & ~size_t(15);
    const size_t with_rows = state + (size_t)n_max * wn * 4;
    const size_t smem = with_rows <= kMcsSmemRows ? with_rows : state;
    ctas = std::max(1, std::min(ctas, count));
    auto go = [&](auto launch) {
        return launch(smem, descs, single, count, n_max, ctas, order, pos, work_counter, stream);
    };
    if (n_max <= 2048) return go(launch_mcs<512, 1>);
    if (n_max <= 32768) return go(launch_mcs<1024, 1>);
    return go(launch_mcs<1024, 2>);
}

}  // namespace cg
