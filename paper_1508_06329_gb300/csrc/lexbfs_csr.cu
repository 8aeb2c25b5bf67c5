// lexbfs_csr.cu — LexBFS by partition refinement on CSR graphs (sparse).
//
// Method: Section 4.2 (Habib, McConnell, Paul and Viennot's partition
// refinement): visit the first vertex x of the first class, then replace every
// class C by C ∩ N_x placed before C \ N_x.  Its O(N + M) form keeps each
// class as a list sorted by vertex id and moves only the neighbours of x.
//
// GPU form (one CTA per graph, whose warp 0 walks the steps; the state of n
// vertices lives in a global workspace and stays L2-resident, and the graph
// is bulk-prefetched into L2 at launch):
//   * cls[v], and per class a doubly linked member list sorted by id
//     (vnext/vprev, cfirst/clast), its size, and the class list
//     (cnext/cprev, head sentinel n) ordered top first; a free stack of ids;
//   * the pick is cfirst[cnext[head]] — the lowest id of the top class, O(1);
//   * the unnumbered neighbours of x (CSR rows are sorted, so they arrive in
//     increasing id order) are processed 32 at a time; lanes holding members
//     of the same class are grouped with __match_any_sync;
//   * a class that loses only some members splits: the moved members, still
//     in id order, form the new class placed right before it; their removal
//     from the old list is done per maximal run of consecutive moved members
//     (a run ends where a member's old successor is not the next moved member
//     of the same class), linking the run's outer neighbours directly;
//   * a class that moves entirely keeps its id, list and place;
//   * rows of at most 32 neighbours take a register-only single pass by one
//     warp; a longer row is handled by the whole CTA (the other warps wait at
//     a named barrier during the short steps): its unnumbered neighbours are
//     sorted by (class, row position), so that each class's moved members are
//     adjacent and in id order, then every member links to its neighbours in
//     the sorted array, a block-wide max-scan finds the start of each run of
//     list-consecutive moved members, and the run ends unlink the runs.
// parent[y] = x is recorded for every moved y: the last pivot that moves y is
// p(y) of the perfect-elimination check (Section 5.2).
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kNone = -1;
constexpr int kNumberedCls = -2;
constexpr unsigned kFull = 0xFFFFFFFFu;

#ifdef CG_BOUNDS_CHECK
// the bounds-checking build: every state array carries its length
struct CsrState {
    CG_ARR(int) cls;                        // [n] class of each vertex
    CG_ARR(int) vnext;                      // [n] member lists
    CG_ARR(int) vprev;                      // [n]
    CG_ARR(int) cnext;                      // [n + 1] class list, index n = head sentinel
    CG_ARR(int) cprev;                      // [n + 1]
    CG_ARR(int) cfirst;                     // [n] per class: first, last member, size
    CG_ARR(int) clast;                      // [n]
    CG_ARR(int) csize;                      // [n]
    CG_ARR(int) cmoved;                     // [n] long-row step: moved count (0 between steps)
    CG_ARR(int) cchild;                     // [n] long-row step: new id (kNone between steps)
    CG_ARR(int) freel;                      // [n] free class ids
    CG_ARR(int) sy;                         // [max_deg] long-row scratch by row position / sorted index
    CG_ARR(int) sop;                        // [max_deg]
    CG_ARR(int) son;                        // [max_deg]
    CG_ARR(int) srun;                       // [max_deg]
    CG_ARR(unsigned long long) skey;        // [next pow2 >= max_deg] (class << 32 | row position) keys
};

constexpr int kCsrArrays = 11;
constexpr int kCsrThreads = 1024;      // the CTA of the search: warp 0 walks the steps
constexpr int kSortSmem = 4096;        // keys sorted in shared memory up to this many

__host__ __device__ inline int64_t pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

__device__ inline CsrState csr_state_carve(int *base, int64_t n, int64_t max_deg) {
    CsrState s;
    int *p = base;
    const int64_t stride = ((n + 1 + 31) / 32) * 32;
    // kCsrArrays blocks of stride ints, in this order
    s.cls = cg_arr(p, n, kChkCsrCls); p += stride;
    s.vnext = cg_arr(p, n, kChkCsrVnext); p += stride;
    s.vprev = cg_arr(p, n, kChkCsrVprev); p += stride;
    s.cnext = cg_arr(p, n + 1, kChkCsrCnext); p += stride;
    s.cprev = cg_arr(p, n + 1, kChkCsrCprev); p += stride;
    s.cfirst = cg_arr(p, n, kChkCsrCfirst); p += stride;
    s.clast = cg_arr(p, n, kChkCsrClast); p += stride;
    s.csize = cg_arr(p, n, kChkCsrCsize); p += stride;
    s.cmoved = cg_arr(p, n, kChkCsrCmoved); p += stride;
    s.cchild = cg_arr(p, n, kChkCsrCchild); p += stride;
    s.freel = cg_arr(p, n, kChkCsrFree); p += stride;
    const int64_t ds = (((max_deg > 1 ? max_deg : 1) + 31) / 32) * 32;
    const int64_t md = max_deg > 1 ? max_deg : 1;
    s.sy = cg_arr(p, md, kChkCsrSy); p += ds;
    s.sop = cg_arr(p, md, kChkCsrSop); p += ds;
    s.son = cg_arr(p, md, kChkCsrSon); p += ds;
    s.srun = cg_arr(p, md, kChkCsrSrun); p += ds;
    // p stays 8-byte aligned: every block is 32 ints
    s.skey = cg_arr(reinterpret_cast<unsigned long long *>(p), pow2_at_least(md), kChkCsrSkey);
    return s;
}

#else
struct CsrState {
    int *cls, *vnext, *vprev;               // [n]
    int *cnext, *cprev;                     // [n + 1], index n = head sentinel
    int *cfirst, *clast, *csize;            // [n]
    int *cmoved, *cchild;                   // [n]  long-row step: moved count, new id (0 / kNone between steps)
    int *freel;                             // [n]
    int *sy, *sop, *son, *srun;             // [max_deg] long-row scratch by row position / sorted index
    unsigned long long *skey;               // [next pow2 >= max_deg] (class << 32 | row position) keys
};

constexpr int kCsrArrays = 11;
constexpr int kCsrThreads = 1024;      // the CTA of the search: warp 0 walks the steps
constexpr int kSortSmem = 4096;        // keys sorted in shared memory up to this many

__host__ __device__ inline int64_t pow2_at_least(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

__device__ inline CsrState csr_state_carve(int *base, int64_t n, int64_t max_deg) {
    CsrState s;
    int *p = base;
    const int64_t stride = ((n + 1 + 31) / 32) * 32;
    int **arrs[kCsrArrays] = {&s.cls,   &s.vnext,  &s.vprev,  &s.cnext,  &s.cprev, &s.cfirst,
                              &s.clast, &s.csize,  &s.cmoved, &s.cchild, &s.freel};
    for (int a = 0; a < kCsrArrays; ++a) {
        *arrs[a] = p;
        p += stride;
    }
    const int64_t ds = (((max_deg > 1 ? max_deg : 1) + 31) / 32) * 32;
    s.sy = p; p += ds;
    s.sop = p; p += ds;
    s.son = p; p += ds;
    s.srun = p; p += ds;
    s.skey = reinterpret_cast<unsigned long long *>(p);   // p stays 8-byte aligned: every block is 32 ints
    return s;
}

#endif

__host__ inline size_t csr_state_stride_bytes(int64_t n, int64_t max_deg) {
    const int64_t stride = ((n + 1 + 31) / 32) * 32;
    const int64_t ds = ((std::max<int64_t>(max_deg, 1) + 31) / 32) * 32;
    return (size_t)(kCsrArrays * stride + 4 * ds) * sizeof(int) +
           (size_t)pow2_at_least(std::max<int64_t>(max_deg, 1)) * sizeof(unsigned long long);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_gt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ int highest_lane(unsigned m) { return 31 - __clz(m); }

// Initial state: one class (id 0) holding 0..n-1 in id order.
__global__ void csr_init_kernel(int *ws, int64_t n, int64_t max_deg, int32_t *parent) {
    CsrState s = csr_state_carve(ws, n, max_deg);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        s.cls[v] = 0;
        s.vnext[v] = v + 1 < n ? (int)(v + 1) : kNone;
        s.vprev[v] = (int)v - 1;
        s.cmoved[v] = 0;
        s.cchild[v] = kNone;
        s.freel[v] = (int)(v + 1);   // entries 0..n-2 used: ids 1..n-1
        if (parent) parent[v] = -1;
        if (v == 0) {
            s.cfirst[0] = 0;
            s.clast[0] = (int)(n - 1);
            s.csize[0] = (int)n;
            s.cnext[n] = 0;
            s.cprev[0] = (int)n;
            s.cnext[0] = kNone;
        }
    }
}

// Shared parameters of a long-row step.
struct LongShared {
    int64_t beg, end;
    int x, free_top, nvalid, done;
    int carry;            // run-start scan carry
    int wmax[32];         // per-warp maxima of the scan
};

__device__ __forceinline__ void bar_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kCsrThreads) : "memory");
}

// Sorts key[0..p) ascending (p a power of two), all threads of the CTA.
__device__ void cta_sort_keys(unsigned long long *key, int64_t p) {
    for (int64_t k = 2; k <= p; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const unsigned long long a = key[i], b = key[l];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// The same network for p > kSortSmem keys in global memory: the passes with
// a stride below kSortSmem pair keys inside one aligned tile of kSortSmem
// keys, so they run on a shared-memory copy of each tile (the first log2 of
// them for every k up to the tile size, the rest after each k's global passes).
__device__ void cta_sort_keys_tiled(unsigned long long *key, int64_t p, unsigned long long *tile) {
    const int T = blockDim.x;
    auto tile_passes = [&](int64_t t0, int64_t k_lo, int64_t k_hi, int64_t j_first) {
        for (int li = threadIdx.x; li < kSortSmem; li += T) tile[li] = key[t0 + li];
        __syncthreads();
        for (int64_t k = k_lo; k <= k_hi; k <<= 1) {
            for (int64_t j = (k == k_lo ? j_first : (k >> 1)); j > 0; j >>= 1) {
                for (int li = threadIdx.x; li < kSortSmem; li += T) {
                    const int l = li ^ (int)j;
                    if (l > li) {
                        const unsigned long long a = tile[li], b = tile[l];
                        if ((a > b) == (((t0 + li) & k) == 0)) {
                            tile[li] = b;
                            tile[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int li = threadIdx.x; li < kSortSmem; li += T) key[t0 + li] = tile[li];
        __syncthreads();
    };
    for (int64_t t0 = 0; t0 < p; t0 += kSortSmem) tile_passes(t0, 2, kSortSmem, 1);   // k = 2 .. tile size
    for (int64_t k = 2 * kSortSmem; k <= p; k <<= 1) {
        for (int64_t j = k >> 1; j >= kSortSmem; j >>= 1) {
            for (int64_t i = threadIdx.x; i < p; i += T) {
                const int64_t l = i ^ j;
                if (l > i) {
                    const unsigned long long a = key[i], b = key[l];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
        for (int64_t t0 = 0; t0 < p; t0 += kSortSmem) tile_passes(t0, k, k, kSortSmem >> 1);
    }
}

// One long-row step for pivot sh->x (row [sh->beg, sh->end)), the whole CTA;
// x's own bookkeeping is done.  The unnumbered neighbours, keyed by (class,
// row position) and sorted, put each class's moved members next to each other
// in id order (rows are sorted); the first key of a class decides the split
// (moved < size: a new class from the free stack, linked before it), every
// moved member links to its sorted neighbours of the same class, a max-scan of
// run starts (a member whose predecessor in the old list is not the previous
// moved member) gives each run end the run's outer left neighbour, and the run
// ends unlink the runs from the old list.  cmoved / cchild return to 0 / kNone.
__device__ void long_row_step(const CsrState &s, const int32_t *__restrict__ col, int32_t *__restrict__ parent,
                              LongShared *sh) {
    __shared__ unsigned long long skeys[kSortSmem];
    const int t = threadIdx.x, T = blockDim.x;
    const int x = sh->x;
    const int64_t beg = sh->beg;
    const int d = (int)(sh->end - beg);
    const int64_t p = pow2_at_least(d);
    unsigned long long *key = p <= kSortSmem ? skeys : s.skey;
    constexpr unsigned long long kInf = ~0ull;
    for (int64_t k = t; k < p; k += T) {
        unsigned long long e = kInf;
        if (k < d) {
            const int y = col[beg + k];
            const int c = s.cls[y];
            if (c != kNumberedCls) {
                e = ((unsigned long long)(unsigned)c << 32) | (unsigned)k;
                s.sy[k] = y;
                s.sop[k] = s.vprev[y];
                s.son[k] = s.vnext[y];
                atomicAdd(&s.cmoved[c], 1);
                atomicAdd(&sh->nvalid, 1);
                if (parent) parent[y] = x;
            }
        }
        key[k] = e;
    }
    __syncthreads();
    if (p <= kSortSmem) cta_sort_keys(key, p);
    else cta_sort_keys_tiled(key, p, skeys);
    const int K = sh->nvalid;
    auto cls_of = [&](int k) { return (int)(key[k] >> 32); };
    auto pos_of = [&](int k) { return (int)(key[k] & 0xFFFFFFFFu); };
    // class firsts: split decision, new id, insertion before the old class
    for (int k = t; k < K; k += T) {
        const int c = cls_of(k);
        if (k > 0 && cls_of(k - 1) == c) continue;
        const int m = s.cmoved[c], sz = s.csize[c];
        if (m < sz) {
            const int cn = s.freel[atomicSub(&sh->free_top, 1) - 1];
            s.cchild[c] = cn;
            const int pc = s.cprev[c];
            s.cnext[pc] = cn;
            s.cprev[cn] = pc;
            s.cnext[cn] = c;
            s.cprev[c] = cn;
            s.cfirst[cn] = s.sy[pos_of(k)];
            s.csize[cn] = m;
            s.csize[c] = sz - m;
        }
    }
    __syncthreads();
    // run starts and their max-scan over the sorted array (runs never cross classes)
    if (t == 0) sh->carry = -1;
    __syncthreads();
    for (int base = 0; base < K; base += T) {
        const int k = base + t;
        int v = -1;
        if (k < K) {
            const int c = cls_of(k);
            if (s.cchild[c] != kNone) {
                const int py = (k > 0 && cls_of(k - 1) == c) ? s.sy[pos_of(k - 1)] : kNone;
                if (py == kNone || s.sop[pos_of(k)] != py) v = k;
            }
        }
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if ((t & 31) >= o) incl = max(incl, y);
        }
        if ((t & 31) == 31) sh->wmax[t >> 5] = incl;
        __syncthreads();
        int before = sh->carry;
        for (int w = 0; w < (t >> 5); ++w) before = max(before, sh->wmax[w]);
        if (k < K) s.srun[k] = max(before, incl);
        __syncthreads();
        if (t == 0) {
            int m = sh->carry;
            for (int w = 0; w < (T >> 5); ++w) m = max(m, sh->wmax[w]);
            sh->carry = m;
        }
        __syncthreads();
    }
    // links of the moved members, the new lists' last members, the runs unlinked
    for (int k = t; k < K; k += T) {
        const int c = cls_of(k);
        const int cn = s.cchild[c];
        if (cn == kNone) continue;
        const int j = pos_of(k);
        const int y = s.sy[j];
        const bool has_prev = k > 0 && cls_of(k - 1) == c;
        const bool has_next = k + 1 < K && cls_of(k + 1) == c;
        const int py = has_prev ? s.sy[pos_of(k - 1)] : kNone;
        const int ny = has_next ? s.sy[pos_of(k + 1)] : kNone;
        const int on = s.son[j];
        s.vprev[y] = py;
        s.vnext[y] = ny;
        s.cls[y] = cn;
        if (!has_next) s.clast[cn] = y;
        if (ny == kNone || on != ny) {   // run end: link the run's outer neighbours
            const int L = s.sop[pos_of(s.srun[k])], R = on;
            if (L == kNone) s.cfirst[c] = R; else s.vnext[L] = R;
            if (R == kNone) s.clast[c] = L; else s.vprev[R] = L;
        }
    }
    __syncthreads();
    for (int k = t; k < K; k += T) {   // per-class step state back to its resting values
        const int c = cls_of(k);
        if (k > 0 && cls_of(k - 1) == c) continue;
        s.cmoved[c] = 0;
        s.cchild[c] = kNone;
    }
    if (t == 0) sh->nvalid = 0;
    __syncthreads();
}

// One warp walks all n steps; the other warps of the CTA join the long-row steps.

__global__ void __launch_bounds__(kCsrThreads) lexbfs_csr_kernel(int *ws, int n, int64_t max_deg,
                                                                 const int64_t *__restrict__ row_ptr,
                                                                 const int32_t *__restrict__ col, int64_t nnz,
                                                                 int32_t *__restrict__ order, int32_t *__restrict__ pos,
                                                                 int32_t *__restrict__ parent) {
    CsrState s = csr_state_carve(ws, n, max_deg);
    __shared__ LongShared shs;
    LongShared *sh = &shs;
    if (threadIdx.x == 0) {
        sh->done = 0;
        sh->nvalid = 0;
    }
    // Every row is read once, when its vertex is the pivot, so its first read
    // would be a DRAM miss on the step's dependent chain: pull row_ptr and col
    // into L2 (bulk prefetch, no completion wait) while the search starts.
    prefetch_range_l2<kCsrThreads>(row_ptr, (size_t)(n + 1) * sizeof(int64_t));
    prefetch_range_l2<kCsrThreads>(col, (size_t)nnz * sizeof(int32_t));
    __syncthreads();
    if (threadIdx.x >= 32) {   // helper warps: join the long-row steps, then leave when warp 0 is done
        for (;;) {
            bar_sync(1);
            if (sh->done) return;
            long_row_step(s, col, parent, sh);
        }
    }
    const int lane = threadIdx.x;
    const int HEAD = n;
    int free_top = n - 1;
    int x = 0;
    // the pivot's row, fetched ahead when the pivot is known early
    int64_t pbeg = row_ptr[0], pend = row_ptr[1];
    int pcol = (pend - pbeg <= 32 && pbeg + lane < pend) ? col[pbeg + lane] : -1;
    // the pivot's class, its successor in that class and the class size, carried
    // in registers from the step that chose the pivot (it computed them), which
    // saves two dependent loads at the start of most steps
    bool carry = false;
    int cf_f = 0, cf_nx = 0, cf_size = 0;
    // the class after the pivot's class, carried from a step whose next pivot
    // was the first member of the untouched class after its own (the common
    // case on sparse graphs): that step read it and corrected it for its own
    // splits; it is needed when the pivot's class holds only the pivot
    bool ga_known = false;
    int ga = kNone;
    for (int i = 0; i < n; ++i) {
        // ---- number x (the first member of the top class f)
        const int f = carry ? cf_f : s.cls[x];
        const int nx = carry ? cf_nx : s.vnext[x];
        const int fsize = (carry ? cf_size : s.csize[f]) - 1;
        // x's successor's successor: the carry when that successor is the next pivot
        const int nnx = nx != kNone ? s.vnext[nx] : kNone;
        carry = false;
        // when f holds only x, the class after it becomes the top class (the load
        // is waited for only after the neighbours' classes have been gathered)
        const int g_after = nx == kNone ? (ga_known ? ga : s.cnext[f]) : kNone;
        ga_known = false;
        // that class's first member, read ahead: when x has no neighbour in
        // it, it is the next pivot (and the class is untouched by this step)
        const int d_first = g_after != kNone ? s.cfirst[g_after] : kNone;
        // x's bookkeeping (lane 0); deferred in the single-chunk path so that it
        // does not wait for g_after
        auto number_x = [&]() {
            if (lane == 0) {
                order[i] = x;
                if (pos) pos[x] = i;
                s.cls[x] = kNumberedCls;
                s.csize[f] = fsize;
                if (nx == kNone) {  // f held only x: drop it
                    s.cnext[HEAD] = g_after;
                    if (g_after != kNone) s.cprev[g_after] = HEAD;
                    s.freel[free_top - 1] = f;
                } else {
                    s.cfirst[f] = nx;
                    s.vprev[nx] = kNone;
                }
            }
            __syncwarp();
        };
        if (nx == kNone) free_top += 1;   // f goes back on the free stack
        const int64_t beg = pbeg, end = pend;
        int next_x = -1;   // set when the single-chunk path finds the next pivot itself

        if (end - beg <= 32) {
            // ---- single chunk: everything in registers
            const int64_t j = beg + lane;
            const bool inrow = j < end;
            const int y = inrow ? pcol : -1;
            // the top of the free stack, one id per lane (lane 0: f when it was just freed)
            const int ftop = free_top - 1 - lane;
            int fl = ftop >= 0 ? s.freel[ftop] : 0;
            if (lane == 0 && nx == kNone) fl = f;
            const int c0 = inrow ? s.cls[y] : kNumberedCls;
            // the list links, gathered with the classes (x's successor loses x as predecessor)
            int op = inrow ? s.vprev[y] : 0;
            const int on = inrow ? s.vnext[y] : 0;
            if (y == nx) op = kNone;
            const bool valid = inrow && c0 != kNumberedCls;
            // the neighbour's class size and predecessor, read before x is
            // numbered: f has lost x, and a dropped f makes the head g_after's
            // predecessor
            int csz = 0, cpv = 0;
            if (valid) {
                csz = c0 == f ? fsize : s.csize[c0];
                cpv = (nx == kNone && c0 == g_after) ? HEAD : s.cprev[c0];
                if (parent) parent[y] = x;
            }
            // next pivot: the lowest moved vertex of the top class f; else f's
            // next member; else (f emptied) the lowest moved vertex of the class
            // after f, or its first member
            int src_lane = -1;     // lane holding the next pivot when it is a moved vertex
            bool via_nx = false;   // the next pivot is x's successor in f (f did not split)
            bool via_ga = false;   // the next pivot is the first member of the untouched class after f
            int d_nx = kNone, d_size = 0, d_ga = kNone;
            {
                const unsigned inf = __ballot_sync(kFull, valid && c0 == f);
                if (inf) {
                    src_lane = __ffs(inf) - 1;
                    next_x = __shfl_sync(kFull, y, src_lane);
                } else if (nx != kNone) {
                    next_x = nx;
                    via_nx = true;
                } else if (g_after != kNone) {
                    const unsigned ing = __ballot_sync(kFull, valid && c0 == g_after);
                    if (ing) {
                        src_lane = __ffs(ing) - 1;
                        next_x = __shfl_sync(kFull, y, src_lane);
                    } else {
                        next_x = d_first;
                        via_ga = true;
                        d_size = s.csize[g_after];
                        d_ga = s.cnext[g_after];
                    }
                }
                if (next_x >= 0) {   // fetch its row now, overlapping the rest of the step
                    pbeg = row_ptr[next_x];
                    pend = row_ptr[next_x + 1];
                    if (via_ga) d_nx = s.vnext[next_x];
                    pcol = (pend - pbeg <= 32 && pbeg + lane < pend) ? col[pbeg + lane] : -1;
                }
            }
            number_x();
            const unsigned grp = __match_any_sync(kFull, valid ? c0 : kNumberedCls);
            const unsigned vmask = __ballot_sync(kFull, valid);
            const unsigned g = valid ? grp : 0u;
            const int moved = __popc(g);
            const bool first = valid && (g & lanemask_lt()) == 0;
            const bool split = valid && moved < csz;
            // allocate one id per split class (its first member's lane)
            const unsigned need = __ballot_sync(kFull, first && split);
            const int rank = __popc(need & lanemask_lt());
            int cn = __shfl_sync(kFull, fl, rank & 31);
            if (!(first && split)) cn = 0;
            free_top -= __popc(need);
            // every member learns its class's new id from the first member
            const int src = valid ? (__ffs(g) - 1) : lane;
            cn = __shfl_sync(kFull, cn, src);
            const unsigned lower = g & lanemask_lt();
            const unsigned higher = g & lanemask_gt();
            const int py_lane = lower ? highest_lane(lower) : lane;
            const int ny_lane = higher ? (__ffs(higher) - 1) : lane;
            const int py_v = __shfl_sync(kFull, y, py_lane);
            const int ny_v = __shfl_sync(kFull, y, ny_lane);
            const int py = lower ? py_v : kNone;
            const int ny = higher ? ny_v : kNone;
            const bool is_start = split && (py == kNone || op != py);
            const bool is_end = split && (ny == kNone || on != ny);
            const unsigned starts = __ballot_sync(kFull, is_start);
            const unsigned s_le = g & starts & (lanemask_lt() | (1u << lane));
            const int l_lane = s_le ? highest_lane(s_le) : lane;
            const int lval = __shfl_sync(kFull, op, l_lane);
            const int last_lane = valid ? highest_lane(g) : lane;
            const int last_y = __shfl_sync(kFull, y, last_lane);
            // the next pivot's class, successor and class size after this step
            if (src_lane >= 0) {
                cf_f = __shfl_sync(kFull, split ? cn : c0, src_lane);
                cf_nx = __shfl_sync(kFull, split ? ny : on, src_lane);
                cf_size = __shfl_sync(kFull, split ? moved : csz, src_lane);
                carry = true;
            } else if (via_nx) {
                cf_f = f;
                cf_nx = nnx;
                cf_size = fsize;
                carry = true;
            } else if (via_ga) {
                cf_f = g_after;
                cf_nx = d_nx;
                cf_size = d_size;
                carry = true;
                // the class after g_after once this step's new classes are in
                // place: a split class there now has its new part in front
                const unsigned hit = __ballot_sync(kFull, split && c0 == d_ga);
                ga = hit ? __shfl_sync(kFull, cn, __ffs(hit) - 1) : d_ga;
                ga_known = true;
            }
            __syncwarp();
            if (first && split) {
                s.cnext[cpv] = cn;
                s.cprev[cn] = cpv;
                s.cnext[cn] = c0;
                s.cprev[c0] = cn;
                s.cfirst[cn] = y;
                s.clast[cn] = last_y;
                s.csize[cn] = moved;
                s.csize[c0] = csz - moved;
            }
            if (is_end) {
                const int L = lval, R = on;
                if (L == kNone) s.cfirst[c0] = R; else s.vnext[L] = R;
                if (R == kNone) s.clast[c0] = L; else s.vprev[R] = L;
            }
            if (split) {
                s.vprev[y] = py;
                s.vnext[y] = ny;
                s.cls[y] = cn;
            }
            (void)vmask;
        } else {
            number_x();
            // ---- long row: the whole CTA (the other warps wait at barrier 1)
            if (lane == 0) {
                sh->x = x;
                sh->beg = beg;
                sh->end = end;
                sh->free_top = free_top;
            }
            __syncwarp();
            bar_sync(1);
            long_row_step(s, col, parent, sh);
            free_top = sh->free_top;
        }
        __syncwarp();
        // ---- next pivot: first member of the top class
        if (i + 1 < n) {
            if (next_x < 0) {
                const int top = s.cnext[HEAD];
                next_x = s.cfirst[top];
                pbeg = row_ptr[next_x];
                pend = row_ptr[next_x + 1];
                pcol = (pend - pbeg <= 32 && pbeg + lane < pend) ? col[pbeg + lane] : -1;
            }
            x = next_x;
        }
    }
    if (lane == 0) sh->done = 1;
    __syncwarp();
    bar_sync(1);
}

}  // namespace

size_t lexbfs_csr_workspace_bytes(int64_t n, int64_t max_deg) { return csr_state_stride_bytes(n, max_deg) + 256; }

int lexbfs_csr_launch(int n, int64_t max_deg, const int64_t *row_ptr, const int32_t *col, int64_t nnz, int32_t *order,
                      int32_t *pos, int32_t *parent, void *ws, int num_sms, cudaStream_t stream) {
    if (n <= 0) return CG_OK;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms * 4));
    csr_init_kernel<<<blocks, 256, 0, stream>>>(static_cast<int *>(ws), n, max_deg, parent);
    CG_LAUNCH_CHECK("csr_init_kernel");
    lexbfs_csr_kernel<<<1, kCsrThreads, 0, stream>>>(static_cast<int *>(ws), n, max_deg, row_ptr, col, nnz, order,
                                                     pos, parent);
    CG_LAUNCH_CHECK("lexbfs_csr_kernel");
    CG_DEBUG_CHECK(stream, "lexbfs_csr_kernel");
    return CG_OK;
}

}  // namespace cg
