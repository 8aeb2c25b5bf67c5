// peo_dense.cu — perfect-elimination check of dense graphs (Sections 5.2, 6.2).
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
constexpr int kMaskRows = 32;         // rows b per mask tile
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
    const int wn = (n + 31) >> 5;
    const int32_t *pos_g = pos + d.vbase;
    if ((int)blockIdx.x < mask_blocks) {
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

// ---- the check of a search's own order, positions in order (fed by the search)
//
// One CTA takes kSub consecutive positions s0 .. s0 + kSub - 1 of one graph
// (blockIdx.y).  The search left p(v) by position (exact), the order, and
// E_b for the group b = s0 / 32 (the vertices numbered before position 32 b),
// so nothing is searched here: the CTA stages, per round of kChunkWords row
// words, row v of each of its positions, row p(v) of the parents that are not
// among its own vertices (for a LexBFS order p(v) is mostly the previous
// pivot, i.e. the row staged just before) and the mask row E_b in shared
// memory — one bulk copy each, all completing on one mbarrier — then each
// warp tests its vertices:
//   bad(v) = (row_v & ~row_p & E_b, without p) ∪ {u at positions 32 b ..
//            pos(v) - 1 : u ∈ N(v), u != p, u ∉ N(p)}
// and the first violation in order is kept by a 64-bit atomicMin of
// (pos(v) << 32 | min bad(v)).  The last CTA to finish writes the results.
constexpr unsigned kNoBad = 0xFFFFFFFFu;    // no bad vertex found
constexpr int kGrpThreads = 256;
constexpr int kSub = 16;                       // positions per CTA (2 per warp)
constexpr int kExt = 8;                        // staged parent rows outside the CTA's own rows
constexpr int kChunkWords = 512;               // row words staged per row and round (2 KiB)
constexpr int kMaskSlot = kSub + kExt;         // slot of E_b
constexpr int kSlots = kSub + kExt + 1;
constexpr size_t kGrpSmemBytes = (size_t)kSlots * kChunkWords * sizeof(uint32_t);

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

template <bool BULK>
__global__ void __launch_bounds__(kGrpThreads) peo_group_kernel(const DenseDesc *__restrict__ descs, DenseDesc single,
                                                                int count, const int32_t *__restrict__ order,
                                                                const int32_t *__restrict__ ppos,
                                                                const uint32_t *__restrict__ emask,
                                                                unsigned long long *__restrict__ keys,
                                                                cg_result *__restrict__ res) {
    extern __shared__ __align__(128) uint32_t sbuf[];   // kSlots rows of kChunkWords words
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_v[32];         // vertices at the group's 32 positions (-1 past n)
    __shared__ int s_p[kSub];       // p(v) of the CTA's positions (-1: none)
    __shared__ int s_src[kSub];     // slot holding row p(v): j' < kSub own, kSub + e staged, -1 global
    __shared__ int s_ext[kExt];     // vertex of each staged parent slot
    __shared__ int s_next;
    __shared__ bool s_last;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int gi = blockIdx.y;
    const DenseDesc d = descs ? descs[gi] : single;
    const int n = d.n;
    const int s0 = blockIdx.x * kSub;
    if (s0 < n) {
        const int wn = (n + 31) >> 5;
        const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;
        const int gstart = s0 & ~31;
        const int nsub = min(kSub, n - s0);
        // order and parents come from the search; a value outside 0..n-1 (only
        // possible if those buffers were overwritten) is reported, never used
        if (t < 32) {
            int v = gstart + t < n ? __ldg(order + d.obase + gstart + t) : -1;
            if (gstart + t < n && (unsigned)v >= (unsigned)n) {
                atomicOr(keys + count + 1, 2ull);
                v = 0;
            }
            s_v[t] = v;
        } else if (t < 32 + kSub) {
            const int j = t - 32;
            int p = j < nsub ? __ldg(ppos + d.vbase + s0 + j) : -1;
            if (p >= n || p < -1) {
                atomicOr(keys + count + 1, 2ull);
                p = -1;
            }
            s_p[j] = p;
        } else if (t == 32 + kSub) {
            s_next = 0;
            if (BULK) {
                mbar_init(&bar, 1);
                fence_proxy_async_smem();
            }
        }
        __syncthreads();
        if (t < kSub) {   // where row p(v) comes from: p precedes v, so an own row has a lower slot
            const int p = s_p[t];
            int src = -1;
            if (p >= 0) {
                for (int k = 0; k < t; ++k)
                    if (s_v[s0 - gstart + k] == p) src = k;
                if (src < 0) {
                    const int e = atomicAdd(&s_next, 1);
                    if (e < kExt) {
                        src = kSub + e;
                        s_ext[e] = p;
                    }
                }
            }
            s_src[t] = src;
        }
        __syncthreads();
        const int next = min(s_next, kExt);
        const uint32_t *Eg = emask + d.ebase + (size_t)(s0 >> 5) * mask_stride(n);
        unsigned umin[2] = {kNoBad, kNoBad};   // vertices j = warp and warp + 8
        bool failed = false;
        int round = 0;
        for (int c0 = 0; c0 < wn; c0 += kChunkWords, ++round) {
            const int cw = min(kChunkWords, wn - c0);
            if (BULK) {
                if (t == 0) {
                    const uint32_t bytes = (uint32_t)((cw + 3) & ~3) * 4u;   // within the padded row (words % 4 == 0)
                    mbar_arrive_expect_tx(&bar, bytes * (uint32_t)(nsub + next + 1));
                    for (int j = 0; j < nsub; ++j)
                        bulk_copy_g2s(sbuf + j * kChunkWords, d.rows + (size_t)s_v[s0 - gstart + j] * d.words + c0,
                                      bytes, &bar);
                    for (int e = 0; e < next; ++e)
                        bulk_copy_g2s(sbuf + (kSub + e) * kChunkWords, d.rows + (size_t)s_ext[e] * d.words + c0, bytes,
                                      &bar);
                    bulk_copy_g2s(sbuf + kMaskSlot * kChunkWords, Eg + c0, bytes, &bar);
                }
                if (!mbar_wait_parity_bounded(&bar, round & 1)) failed = true;
            } else {
                const int rows_used = nsub + next + 1;
                for (int idx = t; idx < rows_used * cw; idx += kGrpThreads) {
                    const int r = idx / cw, w = idx - r * cw;
                    const uint32_t *src;
                    int slot;
                    if (r < nsub) {
                        slot = r;
                        src = d.rows + (size_t)s_v[s0 - gstart + r] * d.words;
                    } else if (r < nsub + next) {
                        slot = kSub + (r - nsub);
                        src = d.rows + (size_t)s_ext[r - nsub] * d.words;
                    } else {
                        slot = kMaskSlot;
                        src = Eg;
                    }
                    sbuf[slot * kChunkWords + w] = __ldg(src + c0 + w);
                }
                __syncthreads();
            }
            if (__syncthreads_or(failed)) {   // a bounded wait gave up: report, do not test
                if (t == 0) atomicOr(keys + count + 1, 1ull);
                break;
            }
            const uint32_t *E = sbuf + kMaskSlot * kChunkWords;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = warp + 8 * q;
                if (j >= nsub || umin[q] != kNoBad) continue;   // a hit in an earlier round has a lower id
                const int p = s_p[j];
                if (p < 0) continue;   // no earlier neighbour: LN_v is empty
                const uint32_t *rv = sbuf + j * kChunkWords;
                const int src = s_src[j];
                const uint32_t *rps = src >= 0 ? sbuf + src * kChunkWords : nullptr;
                const uint32_t *rpg = d.rows + (size_t)p * d.words + c0;
                // earlier groups: the lowest bit of row_v & ~row_p & E_b, p excluded
                unsigned m = kNoBad;
                for (int w0 = 0; w0 < cw; w0 += 32) {   // warp-uniform trip count
                    const int w = w0 + lane;
                    if (w < cw) {
                        const int gw = c0 + w;
                        uint32_t bits = rv[w] & ~(rps ? rps[w] : __ldg(rpg + w)) & E[w];
                        if (gw == wn - 1) bits &= lastmask;
                        if (gw == (p >> 5)) bits &= ~(1u << (p & 31));
                        if (bits) m = (unsigned)((gw << 5) + __ffs(bits) - 1);
                    }
                    if (__any_sync(0xFFFFFFFFu, m != kNoBad)) break;   // later words hold higher ids
                }
                // the group's own earlier positions 32 b .. pos(v) - 1, one per lane
                if (gstart + lane < s0 + j) {
                    const int u = s_v[lane];
                    const int uw = (u >> 5) - c0;
                    if (uw >= 0 && uw < cw && u != p) {
                        const uint32_t bit = 1u << (u & 31);
                        const uint32_t pw = rps ? rps[uw] : __ldg(rpg + uw);
                        if ((rv[uw] & bit) && !(pw & bit)) m = min(m, (unsigned)u);
                    }
                }
                m = __reduce_min_sync(0xFFFFFFFFu, m);
                umin[q] = m;
            }
            if (c0 + kChunkWords < wn) {   // the next round overwrites the staged rows
                __syncthreads();
                if (BULK) fence_proxy_async_smem();
            }
        }
        if (lane == 0 && !failed) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = warp + 8 * q;
                if (j < nsub && umin[q] != kNoBad)
                    atomicMin(keys + gi, ((unsigned long long)(unsigned)(s0 + j) << 32) | umin[q]);
            }
        }
    }
    // the last CTA to finish turns the keys into results (keys[count] counts CTAs)
    __syncthreads();
    if (t == 0) {
        __threadfence();
        s_last = atomicAdd(keys + count, 1ull) == (unsigned long long)gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        const unsigned long long err = atomicAdd(keys + count + 1, 0ull);
        for (int g = t; g < count; g += kGrpThreads)
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

bool peo_group_bulk_ok(const DenseDesc &d) {
    return (reinterpret_cast<uintptr_t>(d.rows) & 15) == 0 && (d.words & 3) == 0 && (d.ebase & 3) == 0;
}

int peo_group_launch(const DenseDesc *descs, DenseDesc single, int count, int n_max, bool bulk, const int32_t *order,
                     const int32_t *ppos, const uint32_t *emask, unsigned long long *keys, cg_result *res,
                     cudaStream_t stream) {
    if (count <= 0 || n_max <= 0) return set_error(CG_EINVAL, "position-ordered check needs count, n > 0");
    if (count > 65535) return set_error(CG_EINVAL, "too many graphs for one check launch (%d)", count);
    if ((reinterpret_cast<uintptr_t>(emask) & 15) != 0) return set_error(CG_EINVAL, "mask buffer not 16-byte aligned");
    const dim3 grid((unsigned)ceil_div(n_max, kSub), (unsigned)count);
    if (bulk) {
        CG_CUDA_TRY(cudaFuncSetAttribute(peo_group_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGrpSmemBytes));
        peo_group_kernel<true><<<grid, kGrpThreads, kGrpSmemBytes, stream>>>(descs, single, count, order, ppos, emask,
                                                                             keys, res);
    } else {
        CG_CUDA_TRY(cudaFuncSetAttribute(peo_group_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kGrpSmemBytes));
        peo_group_kernel<false><<<grid, kGrpThreads, kGrpSmemBytes, stream>>>(descs, single, count, order, ppos,
                                                                              emask, keys, res);
    }
    CG_LAUNCH_CHECK("peo_group_kernel");
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
