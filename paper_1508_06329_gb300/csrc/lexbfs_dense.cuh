// lexbfs_dense.cuh — LexBFS by partition refinement, one CTA per graph.
//
// Method (Section 4.2 of the paper; its GPU form in Section 6.1): the
// unnumbered vertices are partitioned into classes ordered top first.  Each
// step visits the first vertex x of the first class, then replaces every
// class C by C ∩ N_x followed by C \ N_x (Observation 6.2: the new class goes
// right before the class it came from).  Within a class vertices are kept in
// id order, so the visited vertex is the lowest id of the top class.
//
// GPU form used here (differs from the paper's four kernels per step, whose
// racy pick and racy set creation are replaced by deterministic rules):
//   * state: cls[v] (class id per vertex), a doubly linked class list with a
//     head sentinel, and per class one word packing (size, moved-this-step);
//     everything sits in shared memory for n <= 16384 (16-bit ids), otherwise
//     in a global workspace (32-bit ids);
//   * the pivot row is read word-parallel (thread t owns words t, t+T, ...);
//     each unnumbered neighbour y bumps the moved count of its class with a
//     shared-memory atomic; the first arrival per class is its allocator;
//   * allocators split a class only when it loses some but not all members
//     (C ∩ N_x and C \ N_x both non-empty), taking a fresh id from a free
//     stack and linking it right before C;  a class that moves entirely keeps
//     its id and place;
//   * the relabel cls[y] = child[cls[y]] of a step's moved vertices is
//     deferred to the next step and done by the thread owning y's word;
//   * the next pivot is the lowest moved vertex of the top class (an atomicMin
//     collected while splitting), or of the class after it when the top class
//     empties; only when neither class lost members is a class scan needed.
//     A known pivot's row is requested right after the first barrier, so its
//     load overlaps the list update, the second barrier and the next step's
//     relabel pass.  Two __syncthreads per step;
//   * a shared bitmask of numbered vertices filters each pivot row, so only
//     unnumbered neighbours are visited; the deferred relabel and the split
//     are two short loops over a word's bits, and a thread posts only its
//     first (lowest) candidate of the top class to the pivot atomicMin;
//   * parents: p(y) of the perfect-elimination check (Section 5.2), y's
//     neighbour with the largest order index below its own, is the last pivot
//     that moved y.  kParentMoves stores it for every moved vertex (one store
//     per edge; the one-CTA fused test wants all parents).  kParentPivots
//     stores one value per step, by position (parent[i] = p(order[i])): a
//     pivot chosen among the moved vertices has the current pivot as parent;
//     one chosen by a class scan gets kParentUnresolved and the check finds
//     it, unless cpar is given: the members of a class share one label and
//     so one latest numbered neighbour, the pivot that last moved them,
//     which cpar[c] records (set by the allocators when a class is split off
//     or moves whole).  A pivot scanned from the top class f shares the
//     current pivot's parent; one scanned from the class after it reads
//     cpar there (loaded by thread 0 at the start of the step);
//   * with emask, the numbered bitmask at the start of every step 32 b
//     (b >= 1) is also written out as E_b, the vertices numbered before
//     position 32 b: the staged check reads one mask row per 32 positions
//     instead of building it from pos;
//   * the graph's rows are bulk-prefetched into L2 when the CTA starts.
#pragma once
#include "common.cuh"

namespace cg {

template <typename Id>
struct IdTraits;
template <>
struct IdTraits<uint16_t> {
    using Sz = uint32_t;
    static constexpr int kShift = 16;
    static constexpr uint32_t kMask = 0xFFFFu;
};
template <>
struct IdTraits<uint32_t> {
    using Sz = unsigned long long;
    static constexpr int kShift = 32;
    static constexpr unsigned long long kMask = 0xFFFFFFFFull;
};

template <typename Id>
struct LexState {
    CG_ARR(typename IdTraits<Id>::Sz) sz;  // [n]     size | moved-this-step << kShift (size only with mvw)
    CG_ARR(uint32_t) mvw;                  // [(n+1)/2] moved-this-step, two 16-bit counts per word (split layouts 2, 3)
    CG_ARR(uint16_t) mvh;                  // [n]     the same counts as 16-bit entries (stores)
    CG_ARR(uint32_t) arrived;              // [ceil(n/32)] class c's bit: a member moved this step (layout 5)
    CG_ARR(Id) cls;                        // [n]     class of each vertex, kNumbered once visited
    CG_ARR(Id) child;                      // [n]     class receiving a class's pivot neighbours
    CG_ARR(Id) freel;                      // [n]     stack of unused class ids
    CG_ARR(Id) cnext;                      // [n + 1] class list; index n is the head sentinel
    CG_ARR(Id) cprev;                      // [n + 1]
    CG_ARR(uint32_t) numbered;             // [ceil(n/32)] bit v set once v is visited
};

struct LexScalars {
    int free_top;
    int next_graph;
    unsigned front_min[2];
    unsigned second_min[2];
    unsigned split[2];   // a class was split in the step of this parity (its moved vertices need a relabel)
    unsigned red[32];
};

constexpr unsigned kNoVertex = 0xFFFFFFFFu;

// How lexbfs_cta records parents (when given a parent array).

template <typename Id>
__host__ __device__ inline size_t lex_state_bytes(int n) {
    using Sz = typename IdTraits<Id>::Sz;
    size_t b = (size_t)n * sizeof(Sz) + (size_t)n * sizeof(Id) * 3 + (size_t)(n + 1) * sizeof(Id) * 2;
    b = (b + 15) & ~size_t(15);
    b += (size_t)((n + 31) / 32) * sizeof(uint32_t);   // numbered bitmask
    return (b + 15) & ~size_t(15);
}

template <typename Id>
__device__ inline LexState<Id> lex_state_carve(unsigned char *base, int n) {
    using Sz = typename IdTraits<Id>::Sz;
    LexState<Id> s;
    s.sz = cg_arr(reinterpret_cast<Sz *>(base), n, kChkSize);
    Id *p = reinterpret_cast<Id *>(base + (size_t)n * sizeof(Sz));
    s.cls = cg_arr(p, n, kChkCls);
    s.child = cg_arr(p + n, n, kChkChild);
    s.freel = cg_arr(p + 2 * (size_t)n, n, kChkFree);
    s.cnext = cg_arr(p + 3 * (size_t)n, n + 1, kChkCnext);
    s.cprev = cg_arr(p + 4 * (size_t)n + 1, n + 1, kChkCprev);
    size_t b = (size_t)n * sizeof(Sz) + (size_t)n * sizeof(Id) * 3 + (size_t)(n + 1) * sizeof(Id) * 2;
    s.numbered = cg_arr(reinterpret_cast<uint32_t *>(base + ((b + 15) & ~size_t(15))), (n + 31) / 32, kChkNumbered);
    return s;
}

constexpr size_t kLexScalarBytes = (sizeof(LexScalars) + 15) & ~size_t(15);

// Split layouts for graphs too large for the whole state in shared memory but
// within 16-bit ids.  The per-vertex class ids and the numbered bitmask (read
// and written for every moved vertex and by class scans) always stay in
// shared memory; of the per-class state, what a moved vertex touches goes
// there too as far as it fits, the rest (sizes, the free stack and the class
// list, touched once per split class) to a global workspace:
//   layout 3 (n <= 37,920): the moved counts (16 bits each, two per word for
//     the shared atomics) and the children;
//   layout 2 (n <= 56,312): the moved counts;
//   layout 5 (n <= 65,520): one "arrived" bit per class (the first moved
//     member's atomicOr elects the class's allocator); the counts are added
//     to the packed global size words without a return value.
// (Arrival bits with the children in shared memory and the counts in global
// memory, measured on GB300 for 37,921..54,656 vertices, matched layout 2 on
// a sparse graph but were ~1.4x slower per step on a dense one, whose moved
// vertices pile onto few global count words.)
constexpr int kLayoutSplitMv = 2, kLayoutSplitMvChild = 3, kLayoutSplitArr = 5;
__host__ __device__ constexpr bool layout_mv(int l) { return l == kLayoutSplitMv || l == kLayoutSplitMvChild; }
__host__ __device__ constexpr bool layout_child(int l) { return l == kLayoutSplitMvChild; }
__host__ __device__ constexpr bool layout_arr(int l) { return l == kLayoutSplitArr; }

template <typename Id>
__host__ __device__ inline size_t lex_split_smem_bytes(int n, int layout) {
    size_t b = ((size_t)n * sizeof(Id) + 15) & ~size_t(15);
    b += ((size_t)((n + 31) / 32) * sizeof(uint32_t) + 15) & ~size_t(15);
    if (layout_mv(layout)) b += ((size_t)((n + 1) / 2) * sizeof(uint32_t) + 15) & ~size_t(15);
    if (layout_arr(layout)) b += ((size_t)((n + 31) / 32) * sizeof(uint32_t) + 15) & ~size_t(15);
    if (layout_child(layout)) b += ((size_t)n * sizeof(Id) + 15) & ~size_t(15);
    return b;
}

template <typename Id>
__host__ __device__ inline size_t lex_split_global_bytes(int n, int layout) {
    using Sz = typename IdTraits<Id>::Sz;
    const size_t child = layout_child(layout) ? 0 : 1;
    const size_t b = (size_t)n * sizeof(Sz) + (size_t)n * sizeof(Id) * (1 + child) + (size_t)(n + 1) * sizeof(Id) * 2;
    return (b + 255) & ~size_t(255);
}

template <typename Id, int LAYOUT>
__device__ inline LexState<Id> lex_state_carve_split(unsigned char *smem, unsigned char *gmem, int n) {
    using Sz = typename IdTraits<Id>::Sz;
    LexState<Id> s;
    unsigned char *q = smem;
    s.cls = cg_arr(reinterpret_cast<Id *>(q), n, kChkCls);
    q += ((size_t)n * sizeof(Id) + 15) & ~size_t(15);
    s.numbered = cg_arr(reinterpret_cast<uint32_t *>(q), (n + 31) / 32, kChkNumbered);
    q += ((size_t)((n + 31) / 32) * sizeof(uint32_t) + 15) & ~size_t(15);
    if constexpr (layout_mv(LAYOUT)) {
        s.mvw = cg_arr(reinterpret_cast<uint32_t *>(q), (n + 1) / 2, kChkMoved);
        s.mvh = cg_arr(reinterpret_cast<uint16_t *>(q), n, kChkMoved);
        q += ((size_t)((n + 1) / 2) * sizeof(uint32_t) + 15) & ~size_t(15);
    }
    if constexpr (layout_arr(LAYOUT)) {
        s.arrived = cg_arr(reinterpret_cast<uint32_t *>(q), (n + 31) / 32, kChkMoved);
        q += ((size_t)((n + 31) / 32) * sizeof(uint32_t) + 15) & ~size_t(15);
    }
    s.sz = cg_arr(reinterpret_cast<Sz *>(gmem), n, kChkSize);
    Id *p = reinterpret_cast<Id *>(gmem + (size_t)n * sizeof(Sz));
    if constexpr (layout_child(LAYOUT)) {
        s.child = cg_arr(reinterpret_cast<Id *>(q), n, kChkChild);
    } else {
        s.child = cg_arr(p, n, kChkChild);
        p += n;
    }
    s.freel = cg_arr(p, n, kChkFree);
    s.cnext = cg_arr(p + n, n + 1, kChkCnext);
    s.cprev = cg_arr(p + 2 * (size_t)n + 1, n + 1, kChkCprev);
    return s;
}

// Word w of row x as stored, 0 for w >= wn: nothing touches the loaded value
// here, so the warp does not wait for it until the word is first used
// (padding bits are cleared there).
__device__ __forceinline__ uint32_t row_raw(const uint32_t *__restrict__ rows, int stride, int x, int w, int wn) {
    uint32_t v = 0u;
#ifdef CG_BOUNDS_CHECK
    if (w < wn && x < 0) {   // x < n holds when x comes from the state arrays
        cg_dbg_record(kChkRow, (unsigned long long)(unsigned)x);
        return 0u;
    }
#endif
    if (w < wn) v = rows[(size_t)x * stride + w];
    return v;
}

// One CTA computes the LexBFS order of one graph.  rows/stride address the
// adjacency (global memory, or a compact shared-memory copy).  parent may be
// null; otherwise it receives p(v) (-1 when v has no earlier neighbour):
// under kParentMoves as parent[v], under kParentPivots as parent[i] =
// p(order[i]) or kParentUnresolved.  lpw >= LPW threads
// share each row word (thread t takes bit slice t % lpw of word t / lpw +
// k * T / lpw), which shortens the serial bit loop; lpw grows while T / lpw
// still covers the row.
// MV: where the moved counts live: 0 in the packed size words, 1 in the
// 16-bit counts of st.mvw (split layouts 2, 3), 2 in the packed size words
// with the allocator elected by st.arrived (split layout 5).
template <typename Id, int T, int WPT, int LPW, int MV = 0>
__device__ void lexbfs_cta(const uint32_t *__restrict__ rows, int stride, int n, LexState<Id> st,
                           LexScalars *sc, int32_t *__restrict__ order, int32_t *__restrict__ pos,
                           int32_t *__restrict__ parent, int pmode = kParentMoves,
                           uint32_t *__restrict__ emask = nullptr, int32_t *__restrict__ cpar = nullptr) {
    using Tr = IdTraits<Id>;
    using Sz = typename Tr::Sz;
    const Id kNumbered = (Id)~(Id)0;
    const Id kNone = (Id)(kNumbered - 1);
    const int t = threadIdx.x;
    if (n <= 0) return;
    const int wn = (n + 31) >> 5;
    // lanes per word: at least LPW, more while the row still has a word slot
    // per thread group, so short rows spread their bits over all threads
    int lpw = LPW;
    while (lpw < 32 && T / (lpw * 2) >= wn) lpw *= 2;
    const int kGroups = T / lpw;                // word slots per k
    const int kSlice = 32 / lpw;                // bits per thread
    const int wt = t / lpw;
    const uint32_t part = lpw == 1 ? 0xFFFFFFFFu
                                   : ((kSlice == 32 ? 0xFFFFFFFFu : ((1u << kSlice) - 1u)) << ((t % lpw) * kSlice));
    const Id HEAD = (Id)n;
    const uint32_t lastmask = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xFFFFFFFFu;

    for (int v = t; v < n; v += T) {
        st.cls[v] = 0;
        if (parent && pmode == kParentMoves) parent[v] = -1;
    }
    for (int k = t; k < n - 1; k += T) st.freel[k] = (Id)(k + 1);
    for (int w = t; w < wn; w += T) st.numbered[w] = 0u;
    if constexpr (MV == 1)
        for (int w = t; w < (n + 1) / 2; w += T) st.mvw[w] = 0u;
    if constexpr (MV == 2)
        for (int w = t; w < (n + 31) / 32; w += T) st.arrived[w] = 0u;
    if (t == 0) {
        st.sz[0] = (Sz)n;
        st.cnext[HEAD] = 0;
        st.cprev[0] = HEAD;
        st.cnext[0] = kNone;
        sc->free_top = n - 1;
        sc->front_min[0] = sc->front_min[1] = kNoVertex;
        sc->second_min[0] = sc->second_min[1] = kNoVertex;
        sc->split[0] = sc->split[1] = 0u;
        if (cpar) cpar[0] = -1;   // class 0 (all vertices) has no numbered neighbour
    }
    uint32_t rA[WPT], rB[WPT], rC[WPT], amask[WPT];   // previous / current / next pivot row, as loaded
    int x = 0;
#pragma unroll
    for (int k = 0; k < WPT; ++k) {
        const int w = k * kGroups + wt;
        rB[k] = row_raw(rows, stride, x, w, wn);
        rA[k] = 0u;
        rC[k] = 0u;
        amask[k] = 0u;
    }
    Id pending_free = kNone;
    int par_x = -1;   // p(x) of the current pivot (thread 0, kParentPivots)
    __syncthreads();

    // adds k to class c's moved count; true for the first arrival of the step
    // (that thread allocates for the class)
    auto moved_add = [&](Id c, unsigned k) -> bool {
        if constexpr (MV == 1) {
            const unsigned sh = (unsigned)(c & 1) << 4;
            return ((atomicAdd(&st.mvw[c >> 1], k << sh) >> sh) & 0xFFFFu) == 0u;
        } else if constexpr (MV == 2) {
            atomicAdd(&st.sz[c], (Sz)k << Tr::kShift);   // no return value: the chain does not wait for it
            const uint32_t bit = 1u << (c & 31);
            return (atomicOr(&st.arrived[c >> 5], bit) & bit) == 0u;
        } else {
            return (atomicAdd(&st.sz[c], (Sz)k << Tr::kShift) >> Tr::kShift) == 0;
        }
    };
    auto step = [&](const int i, uint32_t (&row_prev)[WPT], uint32_t (&row_cur)[WPT],
                    uint32_t (&row_nxt)[WPT]) -> bool {
        const int slot = i & 1;
        const Id f = st.cnext[HEAD];
        const Id g = st.cnext[f];
        const Sz fsz = MV == 1 ? st.sz[f] : st.sz[f] & Tr::kMask;  // still counts x
        // uniform shortcuts: when the previous step split no class, every class
        // that moved kept its id and the relabel is a no-op; when f is the only
        // class, every unnumbered neighbour of x is in f and a warp adds its
        // count to f with one atomic (cliques take this path at every step)
        const bool relabel = sc->split[slot ^ 1] != 0u;
        const bool single = g == kNone;
        // parent of a pivot scanned from g (thread 0; used after barrier A, so the load overlaps phase S)
        const int cpar_g = t == 0 && cpar && g != kNone ? cpar[g] : kParentUnresolved;

        // E_b = the vertices numbered before x, written at every step 32 b
        // (x's own bit may already be set by a thread of phase S, so it is cleared)
        if (emask && (i & 31) == 0 && i > 0) {
            const int xw = x >> 5;
            uint32_t *eb = emask + (size_t)(i >> 5) * mask_stride(n);
            for (int w = t; w < mask_stride(n); w += T) {   // padding words past ceil(n/32) are zero
                const uint32_t nb = w < wn ? st.numbered[w] : 0u;
                eb[w] = w == xw ? nb & ~(1u << (x & 31)) : nb;
            }
        }
        // ---- phase S: deferred relabel, number x, split by N(x)
        if (t == 0) {
            if (pending_free != kNone) {
                st.freel[sc->free_top] = pending_free;
                sc->free_top += 1;
                pending_free = kNone;
            }
            order[i] = x;
            if (pos) pos[x] = i;
            if (parent && pmode == kParentPivots) parent[i] = par_x;
        }
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const int w = k * kGroups + wt;
            uint32_t am = 0u;
            if (w < wn) {
                const uint32_t prev = row_prev[k];
                uint32_t nb = st.numbered[w];
                // relabel pass: vertices moved by the previous pivot take their new class
                uint32_t bits = relabel ? prev : 0u;
                while (bits) {
                    const int y = (w << 5) + (__ffs(bits) - 1);
                    bits &= bits - 1;
                    st.cls[y] = st.child[st.cls[y]];
                }
                uint32_t rw = row_cur[k];   // first use of the pivot row's word
                if (w == wn - 1) rw &= lastmask;
                const uint32_t cur = rw & part & ~nb;  // unnumbered neighbours of x
                // split pass: count moved members per class; a lane's first moved
                // member of the top class (or of the next one) is its pivot candidate
                bits = single ? 0u : cur;
                if (single && parent && pmode == kParentMoves)
                    for (uint32_t pb = cur; pb; pb &= pb - 1) parent[(w << 5) + (__ffs(pb) - 1)] = x;
                bool f_done = false, g_done = false;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    const uint32_t bit = 1u << b;
                    bits &= bits - 1;
                    const int y = (w << 5) + b;
                    const Id c = st.cls[y];
                    if (moved_add(c, 1u)) am |= bit;
                    if (!f_done && c == f) {
                        atomicMin(&sc->front_min[slot], (unsigned)y);
                        f_done = true;
                    } else if (!g_done && c == g) {
                        atomicMin(&sc->second_min[slot], (unsigned)y);
                        g_done = true;
                    }
                    if (parent && pmode == kParentMoves) parent[y] = x;
                }
                if (w == (x >> 5) && ((part >> (x & 31)) & 1u)) {
                    st.cls[x] = kNumbered;
                    st.numbered[w] = nb | (1u << (x & 31));
                }
                row_cur[k] = cur;
            }
            if (single) {   // warp-uniform: the warp's count of f's moved members in one atomic
                const uint32_t cur = w < wn ? row_cur[k] : 0u;
                const unsigned total = __reduce_add_sync(0xFFFFFFFFu, (unsigned)__popc(cur));
                const unsigned lanes = __ballot_sync(0xFFFFFFFFu, cur != 0u);
                if (lanes && (t & 31) == __ffs(lanes) - 1) {   // the warp's lowest moved vertex
                    if (moved_add(f, total)) am = cur & (0u - cur);   // first arrival allocates
                    atomicMin(&sc->front_min[slot], (unsigned)((w << 5) + __ffs(cur) - 1));
                }
            }
            amask[k] = am;
        }
        __syncthreads();  // A

        // ---- phase D: next pivot (uniform decision)
        const unsigned fmin = sc->front_min[slot];
        const unsigned gmin = sc->second_min[slot];
        const bool fempty = (fsz == 1);
        int mode;  // 0 pivot known, 1 scan class f, 2 scan class g, 3 finished
        unsigned xn = 0;
        Id target = 0;
        if (fmin != kNoVertex) {
            mode = 0;
            xn = fmin;
        } else if (!fempty) {
            mode = 1;
            target = f;
        } else if (g == kNone) {
            mode = 3;
        } else if (gmin != kNoVertex) {
            mode = 0;
            xn = gmin;
        } else {
            mode = 2;
            target = g;
        }
        // a moved pivot's parent is x; one scanned from f shares x's; one from g has g's
        if (t == 0) par_x = mode == 0 ? x : mode == 1 && cpar ? par_x : cpar_g;
        if (mode == 0) {
#pragma unroll
            for (int k = 0; k < WPT; ++k) row_nxt[k] = row_raw(rows, stride, (int)xn, k * kGroups + wt, wn);
        }

        // ---- phase A: allocate / link split classes
#pragma unroll
        for (int k = 0; k < WPT; ++k) {
            const int w = k * kGroups + wt;
            uint32_t am = amask[k];
            while (am) {
                const int y = (w << 5) + (__ffs(am) - 1);
                am &= am - 1;
                const Id c = st.cls[y];  // class before this step's move (relabel is deferred)
                Sz mv, size;
                if constexpr (MV == 1) {
                    mv = (st.mvw[c >> 1] >> ((c & 1) << 4)) & 0xFFFFu;
                    size = st.sz[c] - (c == f ? 1 : 0);
                    st.mvh[c] = 0;   // the moved count restarts (the other half of the word is another class's)
                } else {
                    if constexpr (MV == 2) atomicAnd(&st.arrived[c >> 5], ~(1u << (c & 31)));
                    const Sz s = st.sz[c];
                    mv = s >> Tr::kShift;
                    size = (s & Tr::kMask) - (c == f ? 1 : 0);
                }
                if (mv == size) {
                    st.child[c] = c;
                    st.sz[c] = size;
                    if (cpar) cpar[c] = x;
                    if (fempty && c == g) {
                        st.cnext[HEAD] = g;
                        st.cprev[g] = HEAD;
                    }
                } else {
                    const int idx = atomicSub(&sc->free_top, 1) - 1;
                    sc->split[slot] = 1u;
                    const Id cn = st.freel[idx];
                    if (cpar) cpar[cn] = x;
                    st.child[c] = cn;
                    st.sz[cn] = mv;
                    st.sz[c] = size - mv;
                    Id p = st.cprev[c];
                    if (fempty && p == f) p = HEAD;
                    st.cnext[p] = cn;
                    st.cprev[cn] = p;
                    st.cnext[cn] = c;
                    st.cprev[c] = cn;
                }
            }
        }
        if (t == 0) {
            if (fmin == kNoVertex) st.sz[f] = fsz - 1;
            if (fempty) {
                pending_free = f;
                if (g == kNone || gmin == kNoVertex) {
                    st.cnext[HEAD] = g;
                    if (g != kNone) st.cprev[g] = HEAD;
                }
            }
            sc->front_min[slot ^ 1] = kNoVertex;
            sc->split[slot ^ 1] = 0u;   // read at the start of this step by every thread (before barrier A)
            sc->second_min[slot ^ 1] = kNoVertex;
        }
        // class scan for the next pivot, overlapping phase A (cls is not written there)
        if (mode == 1 || mode == 2) {
            unsigned best = kNoVertex;
            for (int v = t; v < n; v += T)
                if (st.cls[v] == target) {
                    best = (unsigned)v;
                    break;
                }
            best = __reduce_min_sync(0xFFFFFFFFu, best);
            if ((t & 31) == 0) sc->red[t >> 5] = best;
        }
        __syncthreads();  // B
        if (mode == 3) return false;
        if (mode != 0) {
            const unsigned r = (t & 31) < (T / 32) ? sc->red[t & 31] : kNoVertex;
            xn = __reduce_min_sync(0xFFFFFFFFu, r);
#pragma unroll
            for (int k = 0; k < WPT; ++k) row_nxt[k] = row_raw(rows, stride, (int)xn, k * kGroups + wt, wn);
        }
        x = (int)xn;
        return true;
    };
    if constexpr (WPT == 1) {
        // one row word per thread: three registers rotate through the roles
        // previous / current / next pivot row (the loop is unrolled three
        // times), so no register copy at the end of a step waits for the next
        // row's load; the load is first consumed in the next step's split pass,
        // after its relabel pass (9% faster per step on GB300 at N = 16,384)
        for (int i = 0; i < n; i += 3) {
            if (!step(i, rA, rB, rC) || i + 1 >= n) break;
            if (!step(i + 1, rB, rC, rA) || i + 2 >= n) break;
            if (!step(i + 2, rC, rA, rB)) break;
        }
    } else {   // several words per thread: the rotation would spill, so the rows are copied
        for (int i = 0; i < n; ++i) {
            if (!step(i, rA, rB, rC)) break;
#pragma unroll
            for (int k = 0; k < WPT; ++k) {
                rA[k] = rB[k];
                rB[k] = rC[k];
            }
        }
    }
}

}  // namespace cg
