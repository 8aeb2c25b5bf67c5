// peo_dense.cu — perfect-elimination check of dense graphs (Sections 5.2, 6.2).
//
// Three forms of the same test.  The check of the search's own order, with
// exact parents and the earlier-than masks written by the search, is
// peo_stage_kernel (rows staged in shared memory; further below) or, for
// graphs beyond its size or with rows unsuited to 16-byte copies,
// peo_unit_kernel.  The check of a caller-given order (and of an MCS order)
// is the general form described here.
//
// For every vertex v (one warp per vertex, all graphs of a bucket in one grid):
//   p(v)  = the neighbour of v with the largest order index below pos(v)
//           (the paper's preparationLNandP kernel);
//   bad   = (LN_v - {p}) \ N(p), evaluated word by word as row_v & ~row_p and
//           kept only for bits u != p with pos(u) < pos(v) (the paper's
//           testing kernel, with p itself excluded).
// GPU form: peo_prep_kernel builds "earlier-than" masks (E_b: the vertices
// numbered before position 32 b, one bit row per group of 32 positions) and,
// one thread per vertex, finds p(v) among the 32 positions before pos(v)
// (where it lies for ~95% of the vertices of a LexBFS order); the check warp
// then streams row v, row p(v) and E_b (restricting to earlier vertices is a
// word-wise AND, no pos gathers) and finds the remaining parents by probing
// groups of 32 positions and a binary search over the masks.  Without masks
// (the fixed-scratch entry point) p(v) comes from the caller or from pos
// gathers over row v.
// The first violation in order is found by an atomicMin over the 64-bit
// key (pos(v) << 32 | u), u being the lowest id of bad(v); the finalize
// kernel turns each graph's key into (chordal, v, p, u).
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kPeoThreads = 256;

constexpr int kRC = 8;    // row words per lane held in registers (256 words = 8,192 vertices per chunk)

// "Earlier-than" masks: for each group b of 32 positions, E_b has bit u set
// iff pos(u) < 32 b.  ceil(n/32) rows of mask_stride(n) words per graph at
// emask + ebase, row b = E_b.
constexpr int kMaskRows = 8;          // rows b per mask tile
constexpr int kScan = 32;             // positions a prep thread scans for p(v)

// (chordal, v, p, u) from a graph's key (pos(v*) << 32 | u*, or ~0 when chordal).
__device__ __forceinline__ void write_result(const DenseDesc &d, unsigned long long k, const int32_t *order,
                                             const int32_t *parent, cg_result *out) {
    cg_result r;
    if (k == ~0ull) {
        r.chordal = 1;
        r.v = r.p = r.u = -1;
    } else {
        r.chordal = 0;
        r.v = order[d.obase + (int)(k >> 32)];
        r.p = parent[d.vbase + r.v];
        r.u = (int)(k & 0xFFFFFFFFu);
    }
    *out = r;
}

// p(v) by gathering pos over every neighbour: max pos(u) < pos(v).
__device__ __forceinline__ int parent_by_gather(const uint32_t *__restrict__ rv, int wn, uint32_t lastmask,
                                                const int32_t *__restrict__ pos_g, int pv, int lane) {
    int best = -1;
    for (int w = lane; w < wn; w += 32) {
        uint32_t bits = __ldg(rv + w);
        if (w == wn - 1) bits &= lastmask;
        while (bits) {
            const int u = (w << 5) + (__ffs(bits) - 1);
            bits &= bits - 1;
            const int pu = __ldg(pos_g + u);
            if (pu < pv && pu > best) best = pu;
        }
    }
    return __reduce_max_sync(0xFFFFFFFFu, best);
}

// |row ∩ mask| over the whole row (warp-wide sum).
__device__ __forceinline__ int count_in(const uint32_t *__restrict__ row, const uint32_t *__restrict__ mask, int wn,
                                        int lane) {
    int c = 0;
    for (int w = lane; w < wn; w += 32) c += __popc(__ldg(row + w) & __ldg(mask + w));
    return __reduce_add_sync(0xFFFFFFFFu, c);
}

__device__ __forceinline__ bool has_bit(const uint32_t *__restrict__ row, int u) {
    return (__ldg(row + (u >> 5)) >> (u & 31)) & 1u;
}

// emask: the "earlier-than" masks (built by peo_prep_kernel), or null.  With
// masks, LN_v = row_v & (E_b | {order[32b .. pos(v) - 1]}) for b = pos(v) / 32,
// so the subset test streams row v, row p(v) and E_b with no pos gathers, and
// p(v) is found by probing the order backwards from pos(v) in groups of 32
// (after kProbe groups without a neighbour, a binary search over the masks
// finds the last group that holds one).
template <bool PARENT_KNOWN>
__global__ void __launch_bounds__(kPeoThreads, 4) peo_dense_kernel(const DenseDesc *__restrict__ descs,
                                                                DenseDesc single, int count,
                                                                const int64_t *__restrict__ voff, int64_t total,
                                                                const int32_t *__restrict__ order,
                                                                const int32_t *__restrict__ pos,
                                                                int32_t *__restrict__ parent,
                                                                const uint32_t *__restrict__ emask,
                                                                unsigned long long *__restrict__ keys,
                                                                cg_result *__restrict__ res) {
    constexpr int kProbe = 4;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t vbase0 = descs ? __ldg(voff) : 0;   // voff may be a slice of a larger offset table
    for (int64_t gr = warp; gr < total; gr += nwarps) {
        const int64_t gv = gr + vbase0;
        int gi = 0;
        if (descs) {
            int lo = 0, hi = count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(voff + mid) <= gv) lo = mid; else hi = mid;
            }
            gi = lo;
        }
        const DenseDesc d = descs ? descs[gi] : single;
        const int v = (int)(gv - (descs ? __ldg(voff + gi) : 0));
        const int wn = (d.n + 31) >> 5;
        const uint32_t lastmask = (d.n & 31) ? ((1u << (d.n & 31)) - 1u) : 0xFFFFFFFFu;
        const int32_t *pos_g = pos + d.vbase;
        const int32_t *ord_g = order + d.obase;
        const int pv = __ldg(pos_g + v);
        if (pv < 0 || pv >= d.n) continue;   // not in the order (only for an invalid caller order)
        const uint32_t *rv = d.rows + (size_t)v * d.words;
        const int es = mask_stride(d.n);
        const uint32_t *E = emask ? emask + d.ebase + (size_t)(pv >> 5) * es : nullptr;

        uint32_t ae[kRC];   // row_v & E_b of one chunk
        auto load_ae = [&](int w0) {
#pragma unroll
            for (int k = 0; k < kRC; ++k) {
                const int w = w0 + k * 32 + lane;
                ae[k] = w < wn ? __ldg(rv + w) & (E ? __ldg(E + w) : 0xFFFFFFFFu) : 0u;
            }
        };
        // the vertices at positions 32b .. pos(v) - 1 (not in E_b), one per lane
        const int a0 = pv & ~31;
        int ux = -1;
        bool xin = false;   // ux is a neighbour of v
        if (E && lane < pv - a0) {
            ux = __ldg(ord_g + a0 + lane);
            xin = (unsigned)ux < (unsigned)d.n && has_bit(rv, ux);
        }
        int p;
        if (PARENT_KNOWN || E) {
            // known, or found by peo_prep_kernel's scan of the last kScan positions
            p = __ldg(parent + d.vbase + v);
        }
        if (!PARENT_KNOWN) {
            if (E) {
                if (p == kParentUnresolved) {   // warp-wide: groups of 32 positions, then the masks
                    p = -1;
                    int c = (pv >> 5) - 1;
                    for (int r = 0; c >= 0 && r < kProbe; --c, ++r) {
                        const int u = __ldg(ord_g + c * 32 + lane);   // c * 32 + 31 < pos(v)
                        const unsigned hit = __ballot_sync(0xFFFFFFFFu, (unsigned)u < (unsigned)d.n && has_bit(rv, u));
                        if (hit) {
                            p = __shfl_sync(0xFFFFFFFFu, u, 31 - __clz(hit));
                            break;
                        }
                    }
                    if (p < 0 && c >= 0) {
                        // groups 0..c remain: F(g) = |row_v ∩ E_g| is nondecreasing in g; the
                        // parent's group is the last g <= c with F(g) < F(c + 1)
                        const int total = count_in(rv, emask + d.ebase + (size_t)(c + 1) * es, wn, lane);
                        if (total > 0) {
                            int lo = 0, hi = c + 1;   // F(lo) < total = F(hi)
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (count_in(rv, emask + d.ebase + (size_t)mid * es, wn, lane) == total) hi = mid;
                                else lo = mid;
                            }
                            const int u = __ldg(ord_g + lo * 32 + lane);
                            const unsigned hit =
                                __ballot_sync(0xFFFFFFFFu, (unsigned)u < (unsigned)d.n && has_bit(rv, u));
                            if (hit) p = __shfl_sync(0xFFFFFFFFu, u, 31 - __clz(hit));
                        }
                    }
                    if (lane == 0) parent[d.vbase + v] = p;
                }
            } else {
                const int best = parent_by_gather(rv, wn, lastmask, pos_g, pv, lane);
                p = best >= 0 ? __ldg(ord_g + best) : -1;
                if (lane == 0) parent[d.vbase + v] = p;
            }
        }
        if (p < 0 || p >= d.n) continue;

        // LN_v - {p} ⊆ N(p): the lowest id among earlier vertices of row_v & ~row_p other than p
        const uint32_t *rp = d.rows + (size_t)p * d.words;
        unsigned xmin = 0xFFFFFFFFu;   // among the vertices at positions 32b .. pos(v) - 1
        if (E) {
            const bool bad = xin && ux != p && !has_bit(rp, ux);
            xmin = __reduce_min_sync(0xFFFFFFFFu, bad ? (unsigned)ux : 0xFFFFFFFFu);
        }
        unsigned umin = 0xFFFFFFFFu;   // among the rest (E_b, or by pos gathers without masks)
        for (int w0 = 0; w0 < wn && umin == 0xFFFFFFFFu; w0 += 32 * kRC) {
            load_ae(w0);
            uint32_t bp[kRC];
#pragma unroll
            for (int k = 0; k < kRC; ++k) {
                const int w = w0 + k * 32 + lane;
                bp[k] = w < wn ? __ldg(rp + w) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kRC; ++k) {
                const int w = w0 + k * 32 + lane;
                uint32_t bits = ae[k] & ~bp[k];
                if (w == wn - 1) bits &= lastmask;
                if (w == (p >> 5)) bits &= ~(1u << (p & 31));
                if (E) {
                    if (bits && umin == 0xFFFFFFFFu) umin = (unsigned)((w << 5) + __ffs(bits) - 1);
                } else {
                    while (bits && umin == 0xFFFFFFFFu) {
                        const int u = (w << 5) + (__ffs(bits) - 1);
                        bits &= bits - 1;
                        if (__ldg(pos_g + u) < pv) umin = (unsigned)u;
                    }
                }
            }
            umin = __reduce_min_sync(0xFFFFFFFFu, umin);
        }
        umin = min(umin, xmin);
        if (lane == 0 && umin != 0xFFFFFFFFu)
            atomicMin(keys + gi, ((unsigned long long)(unsigned)pv << 32) | umin);
    }
    if (res) {   // the last block to finish turns the keys into results (keys[count] counts blocks)
        __shared__ bool last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(keys + count, 1ull) == (unsigned long long)gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            for (int g = threadIdx.x; g < count; g += blockDim.x)
                write_result(descs ? descs[g] : single, atomicAdd(keys + g, 0ull), order, parent,
                             res + (descs ? descs[g].rindex : g));
        }
    }
}

// Flags an order that is not a permutation of 0..n-1 (seen[] zeroed).
__global__ void order_check_kernel(int n, const int32_t *__restrict__ order, int *__restrict__ seen,
                                   int *__restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = order[i];
        if (x < 0 || x >= n || atomicExch(&seen[x], 1) != 0) atomicOr(flag, 1);
    }
}

// Blocks [0, mask_blocks) of a launch build a graph's earlier-than masks E_b
// from pos: one warp per tile of 32 words w (a lane per word, holding the
// position groups pos(u) / 32 of its 32 vertices) by kMaskRows rows b, so the
// stores of a row are coalesced.
__device__ void build_mask_tiles(const DenseDesc &d, const int32_t *__restrict__ pos_g, uint32_t *__restrict__ emask,
                                 int mask_blocks) {
    const int n = d.n;
    const int wn = (n + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int wcols = (wn + 31) >> 5, brows = (wn + kMaskRows - 1) / kMaskRows;
    const int64_t tiles = (int64_t)wcols * brows;
    uint32_t *E = emask + d.ebase;
    const int es = mask_stride(n);
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < tiles;
         tile += ((int64_t)mask_blocks * blockDim.x) >> 5) {
        const int wc = (int)(tile % wcols), br = (int)(tile / wcols);
        const int w = (wc << 5) + lane;
        uint32_t grp[32];   // position group of vertex 32 w + k (0xFFFFFFFF past n: never earlier)
        if (w < wn && (w << 5) + 32 <= n && ((reinterpret_cast<uintptr_t>(pos_g) & 15) == 0)) {
            const int4 *q = reinterpret_cast<const int4 *>(pos_g + (w << 5));
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int4 t4 = __ldg(q + k);
                grp[4 * k] = (uint32_t)t4.x >> 5;
                grp[4 * k + 1] = (uint32_t)t4.y >> 5;
                grp[4 * k + 2] = (uint32_t)t4.z >> 5;
                grp[4 * k + 3] = (uint32_t)t4.w >> 5;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int u = (w << 5) + k;
                grp[k] = (w < wn && u < n) ? (uint32_t)__ldg(pos_g + u) >> 5 : 0xFFFFFFFFu;
            }
        }
        const int b0 = br * kMaskRows, b1 = min(b0 + kMaskRows, wn);
        for (int b = b0; b < b1; ++b) {
            uint32_t word = 0u;
#pragma unroll
            for (int k = 0; k < 32; ++k) word |= (grp[k] < (uint32_t)b ? 1u : 0u) << k;
            if (w < wn) E[(size_t)b * es + w] = word;
        }
    }
}

// The check's preparation, one launch per bucket of graphs (blockIdx.y =
// graph): blocks [0, mask_blocks) build E_b, one warp per tile of 32 words w
// (a lane per word, holding the position groups pos(u) / 32 of its 32
// vertices) by kMaskRows rows b, so the stores of a row are coalesced; with
// PARENTS, the other blocks give each vertex v whose parent is not known yet
// (all of them, or with prefilled those marked kParentUnresolved) a thread
// that scans the kScan positions before pos(v), 8 independent probes at a
// time, for the latest neighbour: p(v), -1 (none exists) or kParentUnresolved
// (left to the check's warp).
template <bool PARENTS>
__global__ void peo_prep_kernel(const DenseDesc *__restrict__ descs, DenseDesc single,
                                const int32_t *__restrict__ order, const int32_t *__restrict__ pos,
                                int32_t *__restrict__ parent, uint32_t *__restrict__ emask, int mask_blocks,
                                bool prefilled, unsigned long long *__restrict__ keys) {
    if (keys && blockIdx.x == 0 && threadIdx.x == 0) {   // "no violation" key, and the check's block counter
        keys[blockIdx.y] = ~0ull;
        if (blockIdx.y == 0) keys[gridDim.y] = 0ull;
    }
    const DenseDesc d = descs ? descs[blockIdx.y] : single;
    const int n = d.n;
    const int32_t *pos_g = pos + d.vbase;
    if ((int)blockIdx.x < mask_blocks) {
        build_mask_tiles(d, pos_g, emask, mask_blocks);
        return;
    }
    if (!PARENTS) return;
    const int32_t *ord_g = order + d.obase;
    const int stride = (gridDim.x - mask_blocks) * blockDim.x;
    for (int v = (blockIdx.x - mask_blocks) * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (prefilled && parent[d.vbase + v] != kParentUnresolved) continue;
        const int pv = __ldg(pos_g + v);
        if (pv < 0 || pv >= n) continue;   // skipped by the check as well
        const uint32_t *rv = d.rows + (size_t)v * d.words;
        const int jmin = max(0, pv - kScan);
        int p = -1;
        for (int j = pv - 1; j >= jmin && p < 0; j -= 8) {
            int u[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u[q] = j - q >= jmin ? __ldg(ord_g + j - q) : -1;
            bool h[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) h[q] = (unsigned)u[q] < (unsigned)n && has_bit(rv, u[q]);
#pragma unroll
            for (int q = 7; q >= 0; --q)
                if (h[q]) p = u[q];   // the latest (smallest q) wins
        }
        if (p < 0 && jmin > 0) p = kParentUnresolved;
        parent[d.vbase + v] = p;
    }
}

__global__ void finalize_kernel(const DenseDesc *__restrict__ descs, DenseDesc single, int count,
                                const unsigned long long *__restrict__ keys, const int32_t *__restrict__ order,
                                const int32_t *__restrict__ parent, cg_result *__restrict__ res) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= count) return;
    const DenseDesc d = descs ? descs[gi] : single;
    write_result(d, keys[gi], order, parent, res + (descs ? d.rindex : gi));
}

__global__ void invert_order_kernel(const DenseDesc *__restrict__ descs, DenseDesc single, int count,
                                    const int64_t *__restrict__ voff, int64_t total,
                                    const int32_t *__restrict__ order, int32_t *__restrict__ pos) {
    const int64_t vbase0 = descs ? __ldg(voff) : 0;
    for (int64_t gr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gr < total;
         gr += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gv = gr + vbase0;
        int gi = 0;
        if (descs) {
            int lo = 0, hi = count;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(voff + mid) <= gv) lo = mid; else hi = mid;
            }
            gi = lo;
        }
        const DenseDesc d = descs ? descs[gi] : single;
        const int i = (int)(gv - (descs ? __ldg(voff + gi) : 0));
        const int x = order[d.obase + i];
        if (x >= 0 && x < d.n) pos[d.vbase + x] = i;
    }
}

constexpr unsigned kNoBad = 0xFFFFFFFFu;    // no bad vertex found

// (chordal, v, p, u) from a key, with the parent by position; chordal = -1
// when the check could not complete (err != 0: 1 a bounded wait gave up, 2 an
// order or parent value outside 0..n-1).
__device__ __forceinline__ void write_result_ppos(const DenseDesc &d, unsigned long long k, unsigned long long err,
                                                  const int32_t *order, const int32_t *ppos, cg_result *out) {
    cg_result r;
    if (err) {
        r.chordal = -1;
        r.v = r.p = r.u = -1;
    } else if (k == ~0ull) {
        r.chordal = 1;
        r.v = r.p = r.u = -1;
    } else {
        const int i = (int)(k >> 32);
        r.chordal = 0;
        r.v = order[d.obase + i];
        r.p = ppos[d.vbase + i];
        r.u = (int)(k & 0xFFFFFFFFu);
    }
    *out = r;
}

constexpr int kPosChunk = 4;   // uint4 loads per lane per array and pass (512 row words)

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// ---- the check of a search's own order: one block per group of 32 positions
//
// Block (b, g) takes positions 32 b .. 32 b + 31 of graph g (blockIdx.y):
//   1. it builds E_b, the vertices numbered before position 32 b, in shared
//      memory from pos (a word per thread and pass: the pos of its 32
//      vertices against 32 b; pos is small enough to stay in L1);
//   2. it resolves the parents the search left open in the group
//      (kParentUnresolved: pivots taken from the class after the top one),
//      one vertex per warp: p(v) is the earlier neighbour with the largest
//      position, from pos gathered over row v (row words loaded first, then
//      one predicated load per bit position);
//   3. each warp checks four of the positions: the lowest bit of row_v &
//      ~row_p & E_b other than p (row v and row p loaded 128 bits per lane,
//      E_b read from shared memory), plus the group's own earlier positions
//      one per lane; the first violation in order is kept by an atomicMin of
//      (pos(v) << 32 | u) and the last block writes the results.
constexpr int kUnitThreads = 256;
constexpr int kUnitWarps = kUnitThreads / 32;
constexpr int kGatherWords = 16;   // row words per lane held at once by a gathering warp

template <bool VEC>
__global__ void __launch_bounds__(kUnitThreads) peo_unit_kernel(const DenseDesc *__restrict__ descs, DenseDesc single,
                                                                int count, const int32_t *__restrict__ order,
                                                                const int32_t *__restrict__ pos,
                                                                int32_t *__restrict__ ppos,
                                                                unsigned long long *__restrict__ keys,
                                                                cg_result *__restrict__ res) {
    extern __shared__ __align__(16) uint32_t sE[];   // mask_stride(n) words
    __shared__ int s_v[32], s_p[32];
    __shared__ unsigned s_open;
    __shared__ bool s_last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int gi = blockIdx.y;
    const DenseDesc d = descs ? descs[gi] : single;
    const int n = d.n;
    const int g0 = (int)blockIdx.x << 5;
    if (g0 < n) {
        const int wn = (n + 31) >> 5;
        const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
        const int32_t *pos_g = pos + d.vbase;
        const int32_t *ord_g = order + d.obase;
        int32_t *pp_g = ppos + d.vbase;
        if (warp == 0) {   // the group's vertices and parents (values outside 0..n-1 are reported)
            int v = g0 + lane < n ? __ldg(ord_g + g0 + lane) : -1;
            int p = g0 + lane < n ? __ldg(pp_g + g0 + lane) : -1;
            const bool bad =
                g0 + lane < n && ((unsigned)v >= (unsigned)n || p >= n || (p < -1 && p != kParentUnresolved));
            if (bad) {
                atomicOr(keys + count + 1, 2ull);
#ifdef CG_BOUNDS_CHECK
                cg_dbg_record(kChkUnitGroup, (unsigned long long)(g0 + lane));
#endif
                v = 0;
                p = -1;
            }
            s_v[lane] = v;
            s_p[lane] = p;
            const unsigned open = __ballot_sync(0xFFFFFFFFu, p == kParentUnresolved);
            if (lane == 0) s_open = open;
        }
        // E_b from pos: bit k of word w is set iff pos(32 w + k) < 32 b
        const bool vecpos = ((reinterpret_cast<uintptr_t>(pos_g) & 15) == 0);
        for (int w = t; w < wn; w += kUnitThreads) {
            uint32_t word = 0u;
            if (vecpos && (w << 5) + 32 <= n) {
                const int4 *q = reinterpret_cast<const int4 *>(pos_g + (w << 5));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int4 p4 = __ldg(q + k);
                    word |= (p4.x < g0 ? 1u : 0u) << (4 * k) | (p4.y < g0 ? 1u : 0u) << (4 * k + 1) |
                            (p4.z < g0 ? 1u : 0u) << (4 * k + 2) | (p4.w < g0 ? 1u : 0u) << (4 * k + 3);
                }
            } else {
                for (int k = 0; k < 32 && (w << 5) + k < n; ++k)
                    word |= (__ldg(pos_g + (w << 5) + k) < g0 ? 1u : 0u) << k;
            }
            sE[w] = word;
        }
        __syncthreads();
        // open parents, one vertex per warp
        unsigned open = s_open;
        for (int r = 0; open; ++r) {
            const int j = __ffs(open) - 1;
            open &= open - 1;
            if ((r % kUnitWarps) != warp) continue;
            const int iv = g0 + j;
            const uint32_t *rv = d.rows + (size_t)s_v[j] * d.words;
            int best = -1;
            for (int w0 = 0; w0 < wn; w0 += 32 * kGatherWords) {   // the row words first, then the pos loads
                uint32_t rw[kGatherWords];
#pragma unroll
                for (int k = 0; k < kGatherWords; ++k) {
                    const int w = w0 + lane + 32 * k;
                    rw[k] = w < wn ? __ldg(rv + w) : 0u;
                    if (w == wn - 1) rw[k] &= lastmask;
                }
#pragma unroll
                for (int k = 0; k < kGatherWords; ++k) {
                    const int w = w0 + lane + 32 * k;
                    int pu[32];
#ifdef CG_BOUNDS_CHECK
                    if (rw[k] && (w << 5) + 31 - __clz(rw[k]) >= n) {
                        cg_dbg_record(kChkUnitPos, (unsigned long long)((w << 5) + 31 - __clz(rw[k])));
                        rw[k] = 0u;
                    }
#endif
#pragma unroll
                    for (int b = 0; b < 32; ++b) pu[b] = (rw[k] >> b) & 1u ? __ldg(pos_g + (w << 5) + b) : -1;
#pragma unroll
                    for (int b = 0; b < 32; ++b)
                        if (pu[b] < iv && pu[b] > best) best = pu[b];
                }
            }
            best = __reduce_max_sync(0xFFFFFFFFu, best);
            if (lane == 0) {   // also stored for the witness (the last block reads it after the counter)
                const int pj = best >= 0 ? __ldg(ord_g + best) : -1;
                s_p[j] = pj;
                pp_g[iv] = pj;
            }
        }
        __syncthreads();
        // the check, four positions per warp
        for (int j = warp; j < 32 && g0 + j < n; j += kUnitWarps) {
            const int i = g0 + j;
            const int p = s_p[j];
            if (p < 0) continue;   // no earlier neighbour: LN_v is empty
            const uint32_t *rv = d.rows + (size_t)s_v[j] * d.words;
            const uint32_t *rp = d.rows + (size_t)p * d.words;
            unsigned m = kNoBad;
            for (int c = 0; c < wn; c += 128 * kPosChunk) {
                uint4 a[kPosChunk], b[kPosChunk];
#pragma unroll
                for (int it = 0; it < kPosChunk; ++it) {
                    const int w = c + 128 * it + 4 * lane;
                    if (w < wn) {
                        if (VEC) {   // rows padded to 4 words: the whole uint4 is in bounds
                            a[it] = ldg4(rv + w);
                            b[it] = ldg4(rp + w);
                        } else {
                            a[it] = make_uint4(__ldg(rv + w), w + 1 < wn ? __ldg(rv + w + 1) : 0u,
                                               w + 2 < wn ? __ldg(rv + w + 2) : 0u,
                                               w + 3 < wn ? __ldg(rv + w + 3) : 0u);
                            b[it] = make_uint4(__ldg(rp + w), w + 1 < wn ? __ldg(rp + w + 1) : 0u,
                                               w + 2 < wn ? __ldg(rp + w + 2) : 0u,
                                               w + 3 < wn ? __ldg(rp + w + 3) : 0u);
                        }
                    } else {
                        a[it] = b[it] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
#pragma unroll
                for (int it = 0; it < kPosChunk; ++it) {   // a lane's words rise with (it, k): its first hit is its lowest
                    const int w4 = c + 128 * it + 4 * lane;
#ifdef CG_BOUNDS_CHECK
                    if (w4 < wn && w4 + 3 >= mask_stride(n)) cg_dbg_record(kChkUnitMask, (unsigned long long)w4);
#endif
                    const uint4 e = w4 < wn ? *reinterpret_cast<const uint4 *>(sE + w4) : make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t aa[4] = {a[it].x, a[it].y, a[it].z, a[it].w};
                    const uint32_t bb[4] = {b[it].x, b[it].y, b[it].z, b[it].w};
                    const uint32_t ee[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int w = w4 + k;
                        uint32_t bits = w < wn ? aa[k] & ~bb[k] & ee[k] : 0u;
                        if (w == wn - 1) bits &= lastmask;
                        if (w == (p >> 5)) bits &= ~(1u << (p & 31));
                        if (bits && m == kNoBad) m = (unsigned)((w << 5) + __ffs(bits) - 1);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, m != kNoBad)) break;   // later chunks hold higher ids
            }
            // the group's own earlier positions 32 b .. i - 1, one per lane
            if (lane < j) {
                const int u = s_v[lane];
                if (u != p) {
                    const uint32_t bit = 1u << (u & 31);
                    if ((__ldg(rv + (u >> 5)) & bit) && !(__ldg(rp + (u >> 5)) & bit)) m = min(m, (unsigned)u);
                }
            }
            m = __reduce_min_sync(0xFFFFFFFFu, m);
            if (lane == 0 && m != kNoBad) atomicMin(keys + gi, ((unsigned long long)(unsigned)i << 32) | m);
        }
    }
    // the last block to finish turns the keys into results (keys[count] counts blocks)
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(keys + count, 1ull) == (unsigned long long)gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const unsigned long long err = atomicAdd(keys + count + 1, 0ull);
        for (int g = t; g < count; g += kUnitThreads)
            write_result_ppos(descs ? descs[g] : single, atomicAdd(keys + g, 0ull), err, order, ppos,
                              res + (descs ? descs[g].rindex : g));
    }
}

// ---- the check of a search's own order, rows staged in shared memory
//
// For almost every vertex of a LexBFS order, p(v) is the vertex numbered just
// before it, so the rows of a run of positions hold nearly all the parent
// rows too.  A unit is P consecutive positions s0 .. s0 + P - 1 inside one
// group b of 32 positions (P = 16 or 32).  Each block is persistent over the
// units blockIdx.x, blockIdx.x + gridDim.x, ... of graph blockIdx.y, with two
// shared-memory buffers: while it checks unit k, the 16-byte asynchronous
// copies (cp.async, every thread, one commit group per unit) of unit k + 1
// are in flight, warp 0 has written the vertices of unit k + 2 and holds
// those of unit k + 3 in registers.
//   * a unit's buffer: the rows of positions s0 - 1 .. s0 + P - 1 (slot s =
//     position s0 - 1 + s) and E_b (the earlier-than mask the search wrote at
//     step 32 b, zero padded; zero for b = 0); its meta data: the vertices,
//     their exact parents (from the search) and the group's 32 vertices;
//   * checking position i = s0 + j (P / 8 per warp): the lowest bit of
//     row_v & ~row_p & E_b other than p, 128-bit shared-memory loads (row p
//     from its slot, or from global memory when p was numbered before
//     s0 - 1), plus the group's own earlier positions 32 b .. i - 1 one per
//     lane; the first violation in order is kept by an atomicMin of
//     (pos(v) << 32 | u) and the last block writes the results.
// Every row is read from L2 about once; the masks are 1/P of a row per
// position.  (One bulk copy per row, cp.async.bulk on an mbarrier, moved the
// same bytes about three times slower: the block's bulk copies completed one
// after another.)
constexpr int kStageThreads = 256;
constexpr int kStageWarps = kStageThreads / 32;

__device__ __forceinline__ uint4 lds4(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }

template <int P>
struct StageMeta {
    int v[P + 1];   // vertex of slot s (-1: none)
    int p[P];       // p(v) of position s0 + j (-1: no earlier neighbour)
    int grp[32];    // vertices of the group's positions 32 b .. 32 b + 31
    int s0, npos;
};

template <int P>
__global__ void __launch_bounds__(kStageThreads) peo_stage_kernel(const DenseDesc *__restrict__ descs,
                                                                  DenseDesc single, int count,
                                                                  const int32_t *__restrict__ order,
                                                                  const int32_t *__restrict__ ppos,
                                                                  const uint32_t *__restrict__ emask,
                                                                  unsigned long long *__restrict__ keys,
                                                                  cg_result *__restrict__ res) {
    constexpr int kSlots = P + 2;   // P + 1 rows and E_b
    extern __shared__ __align__(128) uint32_t sbuf[];   // 2 buffers x kSlots slots x mask_stride(n) words
    __shared__ StageMeta<P> meta[3];
    __shared__ bool s_last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int gi = blockIdx.y;
    const DenseDesc d = descs ? descs[gi] : single;
    const int n = d.n;
    const int units = (n + P - 1) / P;
    const int nk = (int)blockIdx.x < units ? (units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (nk > 0) {
        const int sw = mask_stride(n);   // slot stride: ceil(n/32) rounded up to 4 words (16 bytes)
        const int q4 = sw >> 2;          // 16-byte chunks per slot
        const int32_t *ord_g = order + d.obase;
        const int32_t *pp_g = ppos + d.vbase;
        const uint32_t *E_g = emask + d.ebase;
        // warp 0's registers: a unit ahead (lane l: the vertex and parent of
        // position s0 + l, the group's vertex 32 b + l; lane 0 also the vertex
        // of position s0 - 1)
        int rv_ = -1, rp_ = -1, rg_ = -1, r0_ = -1;
        auto load_unit = [&](int k) {   // warp 0: global loads, not waited for here
            const int s0 = ((int)blockIdx.x + k * (int)gridDim.x) * P, g0 = s0 & ~31;
            rv_ = lane < P && s0 + lane < n ? __ldg(ord_g + s0 + lane) : -1;
            rp_ = lane < P && s0 + lane < n ? __ldg(pp_g + s0 + lane) : -1;
            rg_ = g0 + lane < n ? __ldg(ord_g + g0 + lane) : -1;
            r0_ = lane == 0 && s0 > 0 ? __ldg(ord_g + s0 - 1) : -1;
        };
        auto write_meta = [&](int k) {   // warp 0: registers -> meta[k % 3]
            StageMeta<P> &m = meta[k % 3];
            const int s0 = ((int)blockIdx.x + k * (int)gridDim.x) * P;
            const int npos = min(P, n - s0);
            int v = rv_, p = rp_, gv = rg_, v0 = r0_;
            // values outside 0..n-1 (only if the buffers were overwritten, or a
            // parent left open) are reported, never used
            const bool bad = (unsigned)(v + 1) > (unsigned)n || (unsigned)(gv + 1) > (unsigned)n ||
                             (unsigned)(v0 + 1) > (unsigned)n || (lane < npos && (v < 0 || p >= n || p < -1));
            if (bad) {
                atomicOr(keys + count + 1, 2ull);
#ifdef CG_BOUNDS_CHECK
                cg_dbg_record(kChkUnitGroup, (unsigned long long)(s0 + lane));
#endif
                if ((unsigned)(v + 1) > (unsigned)n) v = -1;
                if ((unsigned)(gv + 1) > (unsigned)n) gv = -1;
                if ((unsigned)(v0 + 1) > (unsigned)n) v0 = -1;
                if (p >= n || p < -1) p = -1;
            }
            if (lane < P) {
                m.v[lane + 1] = v;
                m.p[lane] = v >= 0 ? p : -1;
            }
            if (lane == 0) {
                m.v[0] = v0;
                m.s0 = s0;
                m.npos = npos;
            }
            m.grp[lane] = gv;
        };
        auto issue_unit = [&](int k) {   // every thread: its 16-byte chunks of unit k, one commit group
            const StageMeta<P> &m = meta[k % 3];
            uint32_t *buf = sbuf + (size_t)(k & 1) * kSlots * sw;
            const int b = m.s0 >> 5;
            for (int slot = warp; slot < kSlots; slot += kStageWarps) {   // a warp per slot, a lane per chunk
                uint32_t *dst = buf + (size_t)slot * sw;
                const uint32_t *src = nullptr;
                if (slot <= P) {
                    const int v = m.v[slot];
                    if (v >= 0) src = d.rows + (size_t)v * d.words;
                } else if (b > 0) {
                    src = E_g + (size_t)b * sw;
                }
                if (src) {
                    for (int c = lane; c < q4; c += 32) cp_async16(dst + 4 * c, src + 4 * c);
                } else if (slot > P) {   // E_0: nothing precedes position 0
                    for (int c = lane; c < q4; c += 32)
                        *reinterpret_cast<uint4 *>(dst + 4 * c) = make_uint4(0u, 0u, 0u, 0u);
                }
            }
            cp_async_commit();
        };
        if (warp == 0) {
            load_unit(0);
            write_meta(0);
            if (nk > 1) {
                load_unit(1);
                write_meta(1);
            }
            if (nk > 2) load_unit(2);
        }
        __syncthreads();   // meta[0], meta[1]
        issue_unit(0);
        for (int k = 0; k < nk; ++k) {
            if (k + 1 < nk) issue_unit(k + 1);
            else cp_async_commit();   // an empty group keeps the count uniform
            if (warp == 0 && k + 2 < nk) {
                write_meta(k + 2);
                if (k + 3 < nk) load_unit(k + 3);
            }
            cp_async_wait<1>();   // this thread's copies of unit k have landed
            __syncthreads();      // everyone's
            const StageMeta<P> &m = meta[k % 3];
            const uint32_t *buf = sbuf + (size_t)(k & 1) * kSlots * sw;
            const uint32_t *E = buf + (size_t)(P + 1) * sw;
            const int s0 = m.s0, g0 = s0 & ~31;
            for (int j = warp; j < m.npos; j += kStageWarps) {
                const int p = m.p[j];
                if (p < 0) continue;   // no earlier neighbour: LN_v is empty
                const uint32_t *rv = buf + (size_t)(j + 1) * sw;
                // row p: a staged slot 0..j when p sits there, else global memory
                const unsigned at = __ballot_sync(0xFFFFFFFFu, lane <= j && m.v[lane] == p);
                const uint32_t *rps = at ? buf + (size_t)(__ffs(at) - 1) * sw : nullptr;
                const uint32_t *rpg = d.rows + (size_t)p * d.words;
                const int pw4 = (p >> 5) & ~3, pk = (p >> 5) & 3;
                const uint32_t keep = ~(1u << (p & 31));
                unsigned mn = kNoBad;
                for (int c = 0; c < sw; c += 128) {   // warp-uniform trip count; 4 words per lane
                    const int w4 = c + 4 * lane;
                    uint32_t b0 = 0u, b1 = 0u, b2 = 0u, b3 = 0u;
                    if (w4 < sw) {   // E_b is zero past n: padding bits and words drop out
                        const uint4 a = lds4(rv + w4), e = lds4(E + w4);
                        const uint4 q = rps ? lds4(rps + w4) : ldg4(rpg + w4);
                        b0 = a.x & ~q.x & e.x;
                        b1 = a.y & ~q.y & e.y;
                        b2 = a.z & ~q.z & e.z;
                        b3 = a.w & ~q.w & e.w;
                        if (w4 == pw4) {   // p itself is not tested
                            if (pk == 0) b0 &= keep;
                            else if (pk == 1) b1 &= keep;
                            else if (pk == 2) b2 &= keep;
                            else b3 &= keep;
                        }
                    }
                    if (b0 | b1 | b2 | b3) {   // this lane's lowest bad id in the chunk
                        const int kk = b0 ? 0 : b1 ? 1 : b2 ? 2 : 3;
                        const uint32_t bits = b0 ? b0 : b1 ? b1 : b2 ? b2 : b3;
                        mn = (unsigned)(((w4 + kk) << 5) + __ffs(bits) - 1);
                    }
                    if (__any_sync(0xFFFFFFFFu, mn != kNoBad)) break;   // later chunks hold higher ids
                }
                // the group's own earlier positions 32 b .. i - 1, one per lane
                if (lane < s0 + j - g0) {
                    const int u = m.grp[lane];
                    if (u >= 0 && u != p) {
                        const uint32_t bit = 1u << (u & 31);
                        const uint32_t pw = rps ? rps[u >> 5] : __ldg(rpg + (u >> 5));
                        if ((rv[u >> 5] & bit) && !(pw & bit)) mn = min(mn, (unsigned)u);
                    }
                }
                mn = __reduce_min_sync(0xFFFFFFFFu, mn);
                if (lane == 0 && mn != kNoBad)
                    atomicMin(keys + gi, ((unsigned long long)(unsigned)(s0 + j) << 32) | mn);
            }
            __syncthreads();   // buffer k & 1 and meta[k % 3] are free again
        }
    }
    // the last block to finish turns the keys into results (keys[count] counts blocks)
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(keys + count, 1ull) == (unsigned long long)gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const unsigned long long err = atomicAdd(keys + count + 1, 0ull);
        for (int g = t; g < count; g += kStageThreads)
            write_result_ppos(descs ? descs[g] : single, atomicAdd(keys + g, 0ull), err, order, ppos,
                              res + (descs ? descs[g].rindex : g));
    }
}

}  // namespace

int invert_order_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                        const int32_t *order, int32_t *pos, int num_sms, cudaStream_t stream) {
    if (total <= 0) return CG_OK;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), (int64_t)num_sms * 8));
    invert_order_kernel<<<blocks, 256, 0, stream>>>(descs, single, count, voff, total, order, pos);
    CG_LAUNCH_CHECK("invert_order_kernel");
    return CG_OK;
}

int order_check_launch(int n, const int32_t *order, int *seen, int *flag, int num_sms, cudaStream_t stream) {
    CG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), stream));
    if (n <= 0) return CG_OK;
    CG_CUDA_TRY(cudaMemsetAsync(seen, 0, sizeof(int) * (size_t)n, stream));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms * 4));
    order_check_kernel<<<blocks, 256, 0, stream>>>(n, order, seen, flag);
    CG_LAUNCH_CHECK("order_check_kernel");
    return CG_OK;
}

int64_t earlier_mask_words(int n) {
    const int64_t wn = (n + 31) / 32;
    return wn * mask_stride(n);
}

int peo_dense_launch(const DenseDesc *descs, DenseDesc single, int count, const int64_t *voff, int64_t total,
                     const int32_t *order, const int32_t *pos, int32_t *parent, bool parent_known,
                     unsigned long long *keys, int num_sms, cudaStream_t stream, uint32_t *emask, int n_max,
                     bool prefilled, cg_result *res) {
    if (count <= 0) return CG_OK;
    const bool fused = emask && res && total > 0;   // keys initialised by the prep kernel, results by the check
    if (!fused) CG_CUDA_TRY(cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * count, stream));
    if (total <= 0) return res ? finalize_launch(descs, single, count, keys, order, parent, res, stream) : CG_OK;
    if (emask) {
        if (count > 65535) return set_error(CG_EINVAL, "too many graphs for one mask launch (%d)", count);
        const int64_t wn = (n_max + 31) / 32;
        const int64_t tiles = ceil_div(wn, 32) * ceil_div(wn, kMaskRows);   // one warp per tile
        const int mask_blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(tiles, 8), (int64_t)num_sms * 4));
        const int parent_blocks =
            parent_known ? 0 : (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_max, 256), (int64_t)num_sms * 4));
        const dim3 grid(mask_blocks + parent_blocks, count);
        unsigned long long *kinit = fused ? keys : nullptr;
        if (parent_known)
            peo_prep_kernel<false><<<grid, 256, 0, stream>>>(descs, single, order, pos, parent, emask, mask_blocks,
                                                             false, kinit);
        else
            peo_prep_kernel<true><<<grid, 256, 0, stream>>>(descs, single, order, pos, parent, emask, mask_blocks,
                                                            prefilled, kinit);
        CG_LAUNCH_CHECK("peo_prep_kernel");
    }
    const int64_t warps_needed = total;
    const int64_t blocks_needed = ceil_div(warps_needed, kPeoThreads / 32);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)num_sms * 8));
    cg_result *fres = fused ? res : nullptr;
    if (parent_known)
        peo_dense_kernel<true><<<blocks, kPeoThreads, 0, stream>>>(descs, single, count, voff, total, order, pos,
                                                                   parent, emask, keys, fres);
    else
        peo_dense_kernel<false><<<blocks, kPeoThreads, 0, stream>>>(descs, single, count, voff, total, order, pos,
                                                                    parent, emask, keys, fres);
    CG_LAUNCH_CHECK("peo_dense_kernel");
    if (res && !fused) return finalize_launch(descs, single, count, keys, order, parent, res, stream);
    return CG_OK;
}

int peo_unit_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, bool vec, const int32_t *order,
                    const int32_t *pos, int32_t *ppos, unsigned long long *keys, cg_result *res, cudaStream_t stream) {
    if (count <= 0 || n_max <= 0) return set_error(CG_EINVAL, "position-ordered check needs vertices");
    if (count > 65535) return set_error(CG_EINVAL, "too many graphs for one check launch (%d)", count);
    const dim3 grid((unsigned)ceil_div(n_max, 32), (unsigned)count);
    const size_t smem = (size_t)mask_stride(n_max) * sizeof(uint32_t);
    if (vec) {
        if (smem > 48 * 1024)
            CG_CUDA_TRY(cudaFuncSetAttribute(peo_unit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        peo_unit_kernel<true><<<grid, kUnitThreads, smem, stream>>>(descs, single, count, order, pos, ppos, keys, res);
    } else {
        if (smem > 48 * 1024)
            CG_CUDA_TRY(cudaFuncSetAttribute(peo_unit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
        peo_unit_kernel<false><<<grid, kUnitThreads, smem, stream>>>(descs, single, count, order, pos, ppos, keys,
                                                                     res);
    }
    CG_LAUNCH_CHECK("peo_unit_kernel");
    CG_DEBUG_CHECK(stream, "peo_unit_kernel");
    return CG_OK;
}

bool peo_rows_vec_ok(const DenseDesc &d) {
    return (reinterpret_cast<uintptr_t>(d.rows) & 15) == 0 && (d.words & 3) == 0;
}

bool peo_stage_ok(const DenseDesc &d) { return d.n > 0 && d.n <= kStageMaxN && peo_rows_vec_ok(d); }

namespace {
// Dynamic shared memory of the staged check for units of P positions.
size_t stage_smem_bytes(int P, int n_max) { return 2 * (size_t)(P + 2) * mask_stride(n_max) * sizeof(uint32_t); }
}  // namespace

int peo_stage_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, const int32_t *order,
                     int32_t *ppos, const uint32_t *emask, unsigned long long *keys, cg_result *res, int num_sms,
                     cudaStream_t stream) {
    if (count <= 0 || n_max <= 0 || n_max > kStageMaxN)
        return set_error(CG_EINVAL, "staged check needs 1..%d vertices (got %d)", kStageMaxN, n_max);
    if (count > 65535) return set_error(CG_EINVAL, "too many graphs for one check launch (%d)", count);
    if (!emask || (reinterpret_cast<uintptr_t>(emask) & 15) != 0)
        return set_error(CG_EINVAL, "staged check needs a 16-byte aligned mask buffer");
    // units of 16 positions (more resident blocks per SM) unless 32 keep as many warps resident
    auto per_sm_of = [](size_t smem) {
        return (int)std::min<size_t>(2048 / kStageThreads, (228 * 1024) / (smem + 2048));
    };
    const int P = per_sm_of(stage_smem_bytes(32, n_max)) >= per_sm_of(stage_smem_bytes(16, n_max)) ? 32 : 16;
    const size_t smem = stage_smem_bytes(P, n_max);
    const int per_sm = std::max(1, per_sm_of(smem));
    const int64_t units = ceil_div(n_max, P);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(units, ceil_div((int64_t)num_sms * per_sm, count)));
    const dim3 grid((unsigned)blocks, (unsigned)count);
    if (P == 32) {
        CG_CUDA_TRY(cudaFuncSetAttribute(peo_stage_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        peo_stage_kernel<32><<<grid, kStageThreads, smem, stream>>>(descs, single, count, order, ppos, emask, keys, res);
    } else {
        CG_CUDA_TRY(cudaFuncSetAttribute(peo_stage_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        peo_stage_kernel<16><<<grid, kStageThreads, smem, stream>>>(descs, single, count, order, ppos, emask, keys, res);
    }
    CG_LAUNCH_CHECK("peo_stage_kernel");
    CG_DEBUG_CHECK(stream, "peo_stage_kernel");
    return CG_OK;
}

int finalize_launch(const DenseDesc *descs, DenseDesc single, int count, const unsigned long long *keys,
                    const int32_t *order, const int32_t *parent, cg_result *res, cudaStream_t stream) {
    if (count <= 0) return CG_OK;
    finalize_kernel<<<(int)ceil_div(count, 128), 128, 0, stream>>>(descs, single, count, keys, order, parent, res);
    CG_LAUNCH_CHECK("finalize_kernel");
    return CG_OK;
}

}  // namespace cg
