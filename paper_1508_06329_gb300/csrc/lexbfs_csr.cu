// lexbfs_csr.cu — LexBFS by partition refinement on CSR graphs (sparse).
//
// Method: Section 4.2 (Habib, McConnell, Paul and Viennot's partition
// refinement): visit the first vertex x of the first class, then replace every
// class C by C ∩ N_x placed before C \ N_x.  Its O(N + M) form keeps each
// class as a list sorted by vertex id and moves only the neighbours of x.
//
// GPU form (one warp per graph; the state of n vertices lives in a global
// workspace and stays L2-resident):
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
//   * rows longer than 32 neighbours use per-class carries (counts, next/prev
//     member, open run) stamped with the step number, in four passes; rows of
//     at most 32 neighbours take a register-only single pass.
// parent[y] = x is recorded for every moved y: the last pivot that moves y is
// p(y) of the perfect-elimination check (Section 5.2).
#include <algorithm>

#include "kernels.h"

namespace cg {

namespace {

constexpr int kNone = -1;
constexpr int kNumberedCls = -2;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct CsrState {
    int *cls, *vnext, *vprev;               // [n]
    int *cnext, *cprev;                     // [n + 1], index n = head sentinel
    int *cfirst, *clast, *csize;            // [n]
    int *cmoved, *cstamp;                   // [n]  moved count of the step in cstamp
    int *cfirst_idx, *clast_idx, *cchild;   // [n]  per-step carries
    int *cprev_y, *crun_l;                  // [n]
    int *freel;                             // [n]
    int *sy, *sc, *sop, *son, *snext;       // [max_deg] per-step neighbour scratch
};

constexpr int kCsrArrays = 16;

__device__ inline CsrState csr_state_carve(int *base, int64_t n, int64_t max_deg) {
    CsrState s;
    int *p = base;
    const int64_t stride = ((n + 1 + 31) / 32) * 32;
    int **arrs[kCsrArrays] = {&s.cls,    &s.vnext,     &s.vprev,     &s.cnext,  &s.cprev,   &s.cfirst,
                              &s.clast,  &s.csize,     &s.cmoved,    &s.cstamp, &s.cfirst_idx, &s.clast_idx,
                              &s.cchild, &s.cprev_y,   &s.crun_l,    &s.freel};
    for (int a = 0; a < kCsrArrays; ++a) {
        *arrs[a] = p;
        p += stride;
    }
    const int64_t ds = (((max_deg > 1 ? max_deg : 1) + 31) / 32) * 32;
    s.sy = p; p += ds;
    s.sc = p; p += ds;
    s.sop = p; p += ds;
    s.son = p; p += ds;
    s.snext = p;
    return s;
}

__host__ inline size_t csr_state_stride_bytes(int64_t n, int64_t max_deg) {
    const int64_t stride = ((n + 1 + 31) / 32) * 32;
    const int64_t ds = ((std::max<int64_t>(max_deg, 1) + 31) / 32) * 32;
    return (size_t)(kCsrArrays * stride + 5 * ds) * sizeof(int);
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
        s.cstamp[v] = -1;
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

// One warp walks all n steps.
__global__ void __launch_bounds__(32) lexbfs_csr_kernel(int *ws, int n, int64_t max_deg,
                                                        const int64_t *__restrict__ row_ptr,
                                                        const int32_t *__restrict__ col, int32_t *__restrict__ order,
                                                        int32_t *__restrict__ pos, int32_t *__restrict__ parent) {
    CsrState s = csr_state_carve(ws, n, max_deg);
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
        const int g_after = nx == kNone ? s.cnext[f] : kNone;
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
            // next pivot: the lowest moved vertex of the top class f; else f's
            // next member; else (f emptied) the lowest moved vertex of the class
            // after f, or its first member
            int src_lane = -1;     // lane holding the next pivot when it is a moved vertex
            bool via_nx = false;   // the next pivot is x's successor in f (f did not split)
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
                    if (ing) src_lane = __ffs(ing) - 1;
                    next_x = ing ? __shfl_sync(kFull, y, src_lane) : s.cfirst[g_after];
                }
                if (next_x >= 0) {   // fetch its row now, overlapping the rest of the step
                    pbeg = row_ptr[next_x];
                    pend = row_ptr[next_x + 1];
                    pcol = (pend - pbeg <= 32 && pbeg + lane < pend) ? col[pbeg + lane] : -1;
                }
            }
            number_x();
            int csz = 0, cpv = 0;
            if (valid) {
                csz = s.csize[c0];
                cpv = s.cprev[c0];
                if (parent) parent[y] = x;
            }
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
            // ---- long row: four passes over 32-wide chunks with per-class carries
            // pass A: compact the unnumbered neighbours, save old links, count per class
            int k = 0;
            for (int64_t base = beg; base < end; base += 32) {
                const int64_t j = base + lane;
                const bool inrow = j < end;
                const int y = inrow ? col[j] : -1;
                const int c = inrow ? s.cls[y] : kNumberedCls;
                const bool valid = inrow && c != kNumberedCls;
                const unsigned m = __ballot_sync(kFull, valid);
                const int idx = k + __popc(m & lanemask_lt());
                const unsigned grp = __match_any_sync(kFull, valid ? c : kNumberedCls);
                if (valid) {
                    s.sy[idx] = y;
                    s.sc[idx] = c;
                    s.sop[idx] = s.vprev[y];
                    s.son[idx] = s.vnext[y];
                    if (parent) parent[y] = x;
                    if ((grp & lanemask_lt()) == 0) {  // group leader
                        const int cnt = __popc(grp);
                        if (s.cstamp[c] != i) {
                            s.cstamp[c] = i;
                            s.cmoved[c] = cnt;
                            s.cfirst_idx[c] = kNone;
                            s.cchild[c] = kNone;
                            s.cprev_y[c] = kNone;
                            s.crun_l[c] = kNone;
                        } else {
                            s.cmoved[c] += cnt;
                        }
                    }
                }
                k += __popc(m);
                __syncwarp();
            }
            const int nchunks = (k + 31) / 32;
            // pass B (reverse): next member index of the same class; first / last index per class
            for (int ch = nchunks - 1; ch >= 0; --ch) {
                const int idx = ch * 32 + lane;
                const bool valid = idx < k;
                const int c = valid ? s.sc[idx] : kNumberedCls;
                const unsigned grp = __match_any_sync(kFull, valid ? c : kNumberedCls);
                const unsigned g = valid ? grp : 0u;
                const unsigned higher = g & lanemask_gt();
                int carry = kNone;
                if (valid && !higher) carry = s.cfirst_idx[c];   // the class's lowest index in later chunks
                __syncwarp();
                if (valid) {
                    s.snext[idx] = higher ? ch * 32 + (__ffs(higher) - 1) : carry;
                    if (!higher && carry == kNone) s.clast_idx[c] = idx;   // last member of the class
                    if ((g & lanemask_lt()) == 0) s.cfirst_idx[c] = idx;
                }
                __syncwarp();
            }
            // pass C: one allocation per split class, at its first member
            for (int ch = 0; ch < nchunks; ++ch) {
                const int idx = ch * 32 + lane;
                const bool valid = idx < k;
                const int c = valid ? s.sc[idx] : 0;
                const bool first = valid && s.cfirst_idx[c] == idx;
                int moved = 0, size = 0;
                if (first) {
                    moved = s.cmoved[c];
                    size = s.csize[c];
                }
                const bool split = first && moved < size;
                const unsigned need = __ballot_sync(kFull, split);
                const int rank = __popc(need & lanemask_lt());
                if (split) {
                    const int cn = s.freel[free_top - 1 - rank];
                    const int p = s.cprev[c];
                    s.cnext[p] = cn;
                    s.cprev[cn] = p;
                    s.cnext[cn] = c;
                    s.cprev[c] = cn;
                    s.cfirst[cn] = s.sy[idx];
                    s.clast[cn] = s.sy[s.clast_idx[c]];
                    s.csize[cn] = moved;
                    s.csize[c] = size - moved;
                    s.cchild[c] = cn;
                }
                free_top -= __popc(need);
                __syncwarp();
            }
            // pass D: unlink moved runs from the old lists, link the new lists
            for (int ch = 0; ch < nchunks; ++ch) {
                const int idx = ch * 32 + lane;
                const bool inr = idx < k;
                const int c = inr ? s.sc[idx] : kNumberedCls;
                const int cn = inr ? s.cchild[c] : kNone;
                const bool split = inr && cn != kNone;
                const unsigned grp = __match_any_sync(kFull, split ? c : kNumberedCls);
                const unsigned g = split ? grp : 0u;
                int y = 0, op = 0, on = 0, ny = kNone, carry_py = kNone, carry_l = kNone;
                if (split) {
                    y = s.sy[idx];
                    op = s.sop[idx];
                    on = s.son[idx];
                    const int nidx = s.snext[idx];
                    ny = nidx >= 0 ? s.sy[nidx] : kNone;
                    if ((g & lanemask_lt()) == 0) {
                        carry_py = s.cprev_y[c];
                        carry_l = s.crun_l[c];
                    }
                }
                const unsigned lower = g & lanemask_lt();
                const int lead = split ? (__ffs(g) - 1) : lane;
                carry_py = __shfl_sync(kFull, carry_py, lead);
                carry_l = __shfl_sync(kFull, carry_l, lead);
                const int py_v = __shfl_sync(kFull, y, lower ? highest_lane(lower) : lane);
                const int py = lower ? py_v : carry_py;
                const bool is_start = split && (py == kNone || op != py);
                const bool is_end = split && (ny == kNone || on != ny);
                const unsigned starts = __ballot_sync(kFull, is_start);
                const unsigned s_le = g & starts & (lanemask_lt() | (1u << lane));
                const int lv = __shfl_sync(kFull, op, s_le ? highest_lane(s_le) : lane);
                const int lval = s_le ? lv : carry_l;
                __syncwarp();
                if (is_end) {
                    const int L = lval, R = on;
                    if (L == kNone) s.cfirst[c] = R; else s.vnext[L] = R;
                    if (R == kNone) s.clast[c] = L; else s.vprev[R] = L;
                }
                if (split) {
                    s.vprev[y] = py;
                    s.vnext[y] = ny;
                    s.cls[y] = cn;
                    if (lane == highest_lane(g)) {   // carries for the next chunk
                        s.cprev_y[c] = y;
                        s.crun_l[c] = lval;
                    }
                }
                __syncwarp();
            }
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
}

}  // namespace

size_t lexbfs_csr_workspace_bytes(int64_t n, int64_t max_deg) { return csr_state_stride_bytes(n, max_deg) + 256; }

int lexbfs_csr_launch(int n, int64_t max_deg, const int64_t *row_ptr, const int32_t *col, int32_t *order,
                      int32_t *pos, int32_t *parent, void *ws, int num_sms, cudaStream_t stream) {
    if (n <= 0) return CG_OK;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms * 4));
    csr_init_kernel<<<blocks, 256, 0, stream>>>(static_cast<int *>(ws), n, max_deg, parent);
    CG_LAUNCH_CHECK("csr_init_kernel");
    lexbfs_csr_kernel<<<1, 32, 0, stream>>>(static_cast<int *>(ws), n, max_deg, row_ptr, col, order, pos, parent);
    CG_LAUNCH_CHECK("lexbfs_csr_kernel");
    return CG_OK;
}

}  // namespace cg
