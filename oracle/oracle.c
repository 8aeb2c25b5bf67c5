/*
 * oracle.c — plain sequential CPU oracle for the chordality test.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference arm may load this library.  It shares no code with
 * the CUDA path.
 *
 * What it computes (0-based vertex ids, LSB-first bit rows or sorted CSR):
 *   1. LexBFS by partition refinement (Section 4.2, the algorithm of Habib,
 *      McConnell, Paul and Viennot): the unnumbered vertices form one doubly
 *      linked sequence cut into classes, classes ordered top first.  Each
 *      step takes the first vertex x of the first class, numbers it, and for
 *      every class C replaces C by C ∩ N_x followed by C \ N_x.  The sequence
 *      starts as 0..N-1 and neighbours of x are moved in increasing id order,
 *      appended to the tail of the new class, so every class stays sorted by
 *      id and "first vertex of the first class" is the lowest id among the
 *      vertices with the lexicographically largest label.
 *   2. The perfect-elimination check (Section 5.2, "chordalityTest"): for
 *      each v, p(v) is the neighbour of v with the largest order index below
 *      that of v, and the test is LN_v - {p(v)} ⊆ N(p(v)).  Every member of
 *      LN_v - {p} precedes p, so membership in N(p) and in LN_p coincide.
 *   3. The witness: v* = the violating vertex with the smallest order index
 *      (the "first such node" of the correctness proof in Section 5.3),
 *      p* = p(v*), u* = the smallest id in (LN_v* - {p*}) \ N(p*).
 * Result array: {chordal, v*, p*, u*}; (v*, p*, u*) = -1 when chordal.
 * Complexity O(N + M) (plus a binary search per tested edge).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------- input */

/* Sorted adjacency (CSR) from LSB-first bit rows; caller frees *rp, *col. */
static int dense_to_lists(int32_t n, int32_t words, const uint32_t *rows, int64_t **rp_out,
                          int32_t **col_out) {
    int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
    if (!rp) return -1;
    rp[0] = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t c = 0;
        for (int32_t w = 0; w < words; ++w) c += __builtin_popcount(rows[(int64_t)v * words + w]);
        rp[v + 1] = rp[v] + c;
    }
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (rp[n] > 0 ? rp[n] : 1));
    if (!col) { free(rp); return -1; }
    for (int32_t v = 0; v < n; ++v) {
        int64_t k = rp[v];
        for (int32_t w = 0; w < words; ++w) {
            uint32_t bits = rows[(int64_t)v * words + w];
            while (bits) {
                col[k++] = (w << 5) + __builtin_ctz(bits);
                bits &= bits - 1;
            }
        }
    }
    *rp_out = rp;
    *col_out = col;
    return 0;
}

/* ----------------------------------------------------------------- LexBFS */

typedef struct {
    int32_t *vnext, *vprev, *cls;
    int32_t *cfirst, *clast, *cnext, *cprev, *cstamp, *cchild;
    int32_t *freestack;
    int32_t nfree, chead;
} lexbfs_state;

static void vl_unlink(lexbfs_state *s, int32_t y) {
    int32_t p = s->vprev[y], q = s->vnext[y];
    if (p >= 0) s->vnext[p] = q;
    if (q >= 0) s->vprev[q] = p;
    s->vprev[y] = s->vnext[y] = -1;
}
static void vl_insert_after(lexbfs_state *s, int32_t a, int32_t y) {
    int32_t q = s->vnext[a];
    s->vnext[a] = y; s->vprev[y] = a; s->vnext[y] = q;
    if (q >= 0) s->vprev[q] = y;
}
static void vl_insert_before(lexbfs_state *s, int32_t b, int32_t y) {
    int32_t p = s->vprev[b];
    s->vprev[b] = y; s->vnext[y] = b; s->vprev[y] = p;
    if (p >= 0) s->vnext[p] = y;
}
static void cl_unlink(lexbfs_state *s, int32_t c) {
    int32_t p = s->cprev[c], q = s->cnext[c];
    if (p >= 0) s->cnext[p] = q; else s->chead = q;
    if (q >= 0) s->cprev[q] = p;
    s->freestack[s->nfree++] = c;
}
static int32_t cl_new_before(lexbfs_state *s, int32_t c) {
    int32_t d = s->freestack[--s->nfree];
    int32_t p = s->cprev[c];
    s->cprev[d] = p; s->cnext[d] = c; s->cprev[c] = d;
    if (p >= 0) s->cnext[p] = d; else s->chead = d;
    s->cfirst[d] = s->clast[d] = -1;
    s->cstamp[d] = -1;
    return d;
}

/* Remove y from its class's first/last bookkeeping (vertex links still valid).
 * Returns 1 if the class became empty. */
static int class_detach(lexbfs_state *s, int32_t c, int32_t y) {
    if (s->cfirst[c] == y && s->clast[c] == y) { s->cfirst[c] = s->clast[c] = -1; return 1; }
    if (s->cfirst[c] == y) s->cfirst[c] = s->vnext[y];
    else if (s->clast[c] == y) s->clast[c] = s->vprev[y];
    return 0;
}

/* Partition refinement from the initial sequence seq (one class holding the
 * vertices in that order).  Each row of (rp, col) must list the neighbours in
 * the order of their positions in seq, so that moved vertices keep that order
 * inside every class. */
static int hmpv_lexbfs(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *seq, int32_t *order) {
    lexbfs_state s;
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * 10 + 64);
    if (!mem) return -2;
    s.vnext = mem; s.vprev = mem + n; s.cls = mem + 2 * (size_t)n;
    s.cfirst = mem + 3 * (size_t)n; s.clast = mem + 4 * (size_t)n; s.cnext = mem + 5 * (size_t)n;
    s.cprev = mem + 6 * (size_t)n; s.cstamp = mem + 7 * (size_t)n; s.cchild = mem + 8 * (size_t)n;
    s.freestack = mem + 9 * (size_t)n;
    uint8_t *numbered = (uint8_t *)calloc(n, 1);
    if (!numbered) { free(mem); return -2; }
    /* one class (id 0) holding the vertices in the order of seq */
    for (int32_t k = 0; k < n; ++k) {
        int32_t v = seq[k];
        s.vprev[v] = k > 0 ? seq[k - 1] : -1;
        s.vnext[v] = k + 1 < n ? seq[k + 1] : -1;
        s.cls[v] = 0;
    }
    s.cfirst[0] = seq[0]; s.clast[0] = seq[n - 1]; s.cnext[0] = s.cprev[0] = -1; s.cstamp[0] = -1;
    s.chead = 0;
    s.nfree = 0;
    for (int32_t c = n - 1; c >= 1; --c) s.freestack[s.nfree++] = c;

    for (int32_t i = 0; i < n; ++i) {
        /* pick: first vertex of the first class */
        int32_t c0 = s.chead;
        int32_t x = s.cfirst[c0];
        order[i] = x;
        numbered[x] = 1;
        if (class_detach(&s, c0, x)) cl_unlink(&s, c0);
        vl_unlink(&s, x);
        /* refine: each class C -> (C ∩ N_x) placed before (C \ N_x) */
        for (int64_t e = rp[x]; e < rp[x + 1]; ++e) {
            int32_t y = col[e];
            if (numbered[y]) continue;
            int32_t c = s.cls[y];
            if (s.cstamp[c] != i) {
                int32_t d = cl_new_before(&s, c);
                s.cstamp[c] = i;
                s.cstamp[d] = i;
                s.cchild[c] = d;
            }
            int32_t d = s.cchild[c];
            int was_first = s.cfirst[c] == y;
            int emptied = class_detach(&s, c, y);
            if (s.clast[d] >= 0) {
                vl_unlink(&s, y);
                vl_insert_after(&s, s.clast[d], y);
            } else if (!emptied && !was_first) {
                vl_unlink(&s, y);
                vl_insert_before(&s, s.cfirst[c], y);
            } /* else: y already sits where the new class begins */
            s.cls[y] = d;
            if (s.cfirst[d] < 0) s.cfirst[d] = y;
            s.clast[d] = y;
            if (emptied) cl_unlink(&s, c);
        }
    }
    free(numbered);
    free(mem);
    return 0;
}

int or_lexbfs_csr(int32_t n, const int64_t *rp, const int32_t *col, int32_t *order) {
    if (n < 0) return -1;
    if (n == 0) return 0;
    int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!seq) return -2;
    for (int32_t v = 0; v < n; ++v) seq[v] = v;   /* rows are sorted by id already */
    int rc = hmpv_lexbfs(n, rp, col, seq, order);
    free(seq);
    return rc;
}

/*
 * LexBFS with a caller-given tie-break (the building block of multi-sweep
 * LexBFS): among the unnumbered vertices with the lexicographically largest
 * label, the one with the smallest rank[v] is numbered; start >= 0 is numbered
 * first.  rank must be a permutation of 0..n-1 (else -4).  This is Section
 * 4.2's refinement started from the single class ordered by (start first,
 * then rank), with every neighbour list taken in that same order.
 */
static const int32_t *g_sort_key;
static int by_key(const void *a, const void *b) {
    int32_t ka = g_sort_key[*(const int32_t *)a], kb = g_sort_key[*(const int32_t *)b];
    return (ka > kb) - (ka < kb);
}

int or_lexbfs_rank_csr(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *rank, int32_t start,
                       int32_t *order) {
    if (n < 0 || start >= n) return -1;
    if (n == 0) return 0;
    int32_t *key = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *col2 = (int32_t *)malloc(sizeof(int32_t) * (rp[n] > 0 ? rp[n] : 1));
    if (!key || !seq || !col2) { free(key); free(seq); free(col2); return -2; }
    for (int32_t v = 0; v < n; ++v) seq[v] = -1;
    for (int32_t v = 0; v < n; ++v) {
        int32_t r = rank ? rank[v] : v;
        if (r < 0 || r >= n || seq[r] >= 0) { free(key); free(seq); free(col2); return -4; }
        seq[r] = v;
        key[v] = v == start ? -1 : r;
    }
    if (start >= 0) {   /* move start to the front of the sequence */
        int32_t r = rank ? rank[start] : start;
        for (int32_t k = r; k > 0; --k) seq[k] = seq[k - 1];
        seq[0] = start;
    }
    g_sort_key = key;
    for (int32_t v = 0; v < n; ++v) {
        memcpy(col2 + rp[v], col + rp[v], sizeof(int32_t) * (size_t)(rp[v + 1] - rp[v]));
        qsort(col2 + rp[v], (size_t)(rp[v + 1] - rp[v]), sizeof(int32_t), by_key);
    }
    int rc = hmpv_lexbfs(n, rp, col2, seq, order);
    free(key); free(seq); free(col2);
    return rc;
}

int or_lexbfs_rank_dense(int32_t n, int32_t words, const uint32_t *rows, const int32_t *rank, int32_t start,
                         int32_t *order) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    if (n == 0) return 0;
    int64_t *rp; int32_t *col;
    if (dense_to_lists(n, words, rows, &rp, &col)) return -2;
    int rc = or_lexbfs_rank_csr(n, rp, col, rank, start, order);
    free(rp); free(col);
    return rc;
}

int or_lexbfs_dense(int32_t n, int32_t words, const uint32_t *rows, int32_t *order) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    if (n == 0) return 0;
    int64_t *rp; int32_t *col;
    if (dense_to_lists(n, words, rows, &rp, &col)) return -2;
    int rc = or_lexbfs_csr(n, rp, col, order);
    free(rp); free(col);
    return rc;
}

/* ------------------------------------------------------------------- MCS */

/*
 * Maximum Cardinality Search (Section 5.1): every unnumbered vertex carries the
 * number of its numbered neighbours; each step numbers a vertex with the
 * largest count, the lowest id among equals, and counts it at its unnumbered
 * neighbours.  A binary max-heap of (count, -id) with lazy deletion: a vertex
 * re-enters the heap on every increment and stale entries are skipped.
 */
typedef struct { int32_t label, v; } heap_item;

static int item_above(heap_item a, heap_item b) {
    return a.label > b.label || (a.label == b.label && a.v < b.v);
}

int or_mcs_csr(int32_t n, const int64_t *rp, const int32_t *col, int32_t *order) {
    if (n < 0) return -1;
    if (n == 0) return 0;
    int64_t cap = n + (rp[n] > 0 ? rp[n] : 0) + 1;
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * cap);
    int32_t *label = (int32_t *)calloc(n, sizeof(int32_t));
    uint8_t *numbered = (uint8_t *)calloc(n, 1);
    if (!h || !label || !numbered) { free(h); free(label); free(numbered); return -2; }
    int64_t hn = 0;
    for (int32_t v = 0; v < n; ++v) {   /* equal labels: ascending ids form a valid heap */
        h[hn].label = 0; h[hn].v = v; ++hn;
    }
    for (int32_t i = 0; i < n; ++i) {
        int32_t x = -1;
        while (hn > 0) {
            heap_item top = h[0];
            /* pop */
            h[0] = h[--hn];
            for (int64_t k = 0;;) {
                int64_t l = 2 * k + 1, r = l + 1, m = k;
                if (l < hn && item_above(h[l], h[m])) m = l;
                if (r < hn && item_above(h[r], h[m])) m = r;
                if (m == k) break;
                heap_item t = h[k]; h[k] = h[m]; h[m] = t; k = m;
            }
            if (!numbered[top.v] && top.label == label[top.v]) { x = top.v; break; }
        }
        if (x < 0) { free(h); free(label); free(numbered); return -3; }
        order[i] = x;
        numbered[x] = 1;
        for (int64_t e = rp[x]; e < rp[x + 1]; ++e) {
            int32_t y = col[e];
            if (numbered[y]) continue;
            label[y] += 1;
            /* push (label[y], y) */
            int64_t k = hn++;
            h[k].label = label[y]; h[k].v = y;
            while (k > 0) {
                int64_t pidx = (k - 1) / 2;
                if (!item_above(h[k], h[pidx])) break;
                heap_item t = h[k]; h[k] = h[pidx]; h[pidx] = t; k = pidx;
            }
        }
    }
    free(h); free(label); free(numbered);
    return 0;
}

int or_mcs_dense(int32_t n, int32_t words, const uint32_t *rows, int32_t *order) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    if (n == 0) return 0;
    int64_t *rp; int32_t *col;
    if (dense_to_lists(n, words, rows, &rp, &col)) return -2;
    int rc = or_mcs_csr(n, rp, col, order);
    free(rp); free(col);
    return rc;
}

/* ------------------------------------------------------- perfect elimination */

static int adjacent_sorted(const int64_t *rp, const int32_t *col, int32_t a, int32_t b) {
    int64_t lo = rp[a], hi = rp[a + 1];
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < rp[a + 1] && col[lo] == b;
}

/* parent[v] = p(v) (or -1) for every v; result = {chordal, v*, p*, u*}. */
int or_peo_check_csr(int32_t n, const int64_t *rp, const int32_t *col, const int32_t *order,
                     int32_t *parent, int32_t *result) {
    result[0] = 1; result[1] = result[2] = result[3] = -1;
    if (n <= 0) return n < 0 ? -1 : 0;
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!pos) return -2;
    for (int32_t i = 0; i < n; ++i) pos[i] = -1;
    for (int32_t i = 0; i < n; ++i) {
        if (order[i] < 0 || order[i] >= n || pos[order[i]] >= 0) { free(pos); return -1; }
        pos[order[i]] = i;
    }
    /* p(v): rightmost earlier neighbour */
    for (int32_t v = 0; v < n; ++v) {
        int32_t p = -1;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t u = col[e];
            if (pos[u] < pos[v] && (p < 0 || pos[u] > pos[p])) p = u;
        }
        parent[v] = p;
    }
    /* LN_v - {p} ⊆ N(p), vertices visited in order; first failure is v* */
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = order[i], p = parent[v];
        if (p < 0) continue;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            int32_t u = col[e];   /* ascending ids: first hit is u* */
            if (pos[u] < pos[v] && u != p && !adjacent_sorted(rp, col, p, u)) {
                result[0] = 0; result[1] = v; result[2] = p; result[3] = u;
                free(pos);
                return 0;
            }
        }
    }
    free(pos);
    return 0;
}

int or_peo_check_dense(int32_t n, int32_t words, const uint32_t *rows, const int32_t *order,
                       int32_t *parent, int32_t *result) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    result[0] = 1; result[1] = result[2] = result[3] = -1;
    if (n == 0) return 0;
    int64_t *rp; int32_t *col;
    if (dense_to_lists(n, words, rows, &rp, &col)) return -2;
    int rc = or_peo_check_csr(n, rp, col, order, parent, result);
    free(rp); free(col);
    return rc;
}

/* The whole test: LexBFS order, then the perfect-elimination check. */
int or_chordal_test_csr(int32_t n, const int64_t *rp, const int32_t *col, int32_t *order,
                        int32_t *parent, int32_t *result) {
    int rc = or_lexbfs_csr(n, rp, col, order);
    if (rc) return rc;
    return or_peo_check_csr(n, rp, col, order, parent, result);
}

int or_chordal_test_dense(int32_t n, int32_t words, const uint32_t *rows, int32_t *order,
                          int32_t *parent, int32_t *result) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    result[0] = 1; result[1] = result[2] = result[3] = -1;
    if (n == 0) return 0;
    int64_t *rp; int32_t *col;
    if (dense_to_lists(n, words, rows, &rp, &col)) return -2;
    int rc = or_chordal_test_csr(n, rp, col, order, parent, result);
    free(rp); free(col);
    return rc;
}
