/*
 * graphgen.c — seeded synthetic graph generators for the chordality test.
 *
 * This module only builds inputs.  It contains none of the method's arithmetic
 * (no LexBFS, no perfect-elimination check); both the CPU oracle and the GPU
 * path consume what it produces.  Every generator is deterministic for a given
 * seed on any platform: integer arithmetic only, xoshiro256** seeded through
 * splitmix64 (Blackman & Vigna, "Scrambled linear pseudorandom number
 * generators", 2018; splitmix64 from Steele, Lea & Flood, OOPSLA 2014).
 *
 * Graph families (the workloads of the paper's Section 7 have no published
 * generator parameters; these are seeded stand-ins):
 *   - subtree-intersection graphs (Gavril's characterisation of chordal graphs:
 *     the intersection graph of subtrees of a tree is chordal);
 *   - planted induced chordless cycle C_k (k >= 4 makes the graph non-chordal);
 *   - cycle-closing extra edges: uv added only when u and v are connected in
 *     G - (N(u) ∩ N(v)); a shortest such path plus uv is a chordless cycle of
 *     length >= 4, so the result is non-chordal;
 *   - chordal graphs built along a reversed perfect elimination order: each new
 *     vertex joins a clique {w} ∪ (subset of the earlier neighbourhood of w);
 *   - Erdős–Rényi G(n, p) graphs.
 *
 * Dense layout: rows[i * words + (j >> 5)] bit (j & 31) is 1 iff ij is an edge;
 * symmetric, zero diagonal, zero padding bits.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform integer in [0, n), n >= 1 (multiply-high reduction) */
static uint64_t rng_below(gg_rng *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* uniform integer in [lo, hi] */
static int64_t rng_range(gg_rng *r, int64_t lo, int64_t hi) {
    return lo + (int64_t)rng_below(r, (uint64_t)(hi - lo + 1));
}

/* exported raw stream (lets Python draw from the same generator family) */
void gg_stream(uint64_t seed, uint64_t *out, int64_t count) {
    gg_rng r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < count; ++i) out[i] = rng_next(&r);
}

static inline void set_edge(uint32_t *rows, int32_t words, int32_t a, int32_t b) {
    rows[(int64_t)a * words + (b >> 5)] |= 1u << (b & 31);
    rows[(int64_t)b * words + (a >> 5)] |= 1u << (a & 31);
}
static inline void clear_edge(uint32_t *rows, int32_t words, int32_t a, int32_t b) {
    rows[(int64_t)a * words + (b >> 5)] &= ~(1u << (b & 31));
    rows[(int64_t)b * words + (a >> 5)] &= ~(1u << (a & 31));
}
static inline int has_edge(const uint32_t *rows, int32_t words, int32_t a, int32_t b) {
    return (rows[(int64_t)a * words + (b >> 5)] >> (b & 31)) & 1u;
}

/*
 * Subtree-intersection graph.  A random recursive tree on `tree_nodes` nodes
 * (node k > 0 hangs below a uniform node in [0, k)).  Vertex i owns a subtree of
 * size s ~ U{smin..smax} (capped at tree_nodes) grown from a uniform root by
 * repeatedly adding a uniform node of the current frontier.  ij is an edge iff
 * the two subtrees share a tree node.  rows must be zeroed by the caller.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int gg_subtree_dense(int32_t n, int32_t tree_nodes, int32_t smin, int32_t smax,
                     uint64_t seed, uint32_t *rows, int32_t words) {
    if (n < 0 || tree_nodes < 1 || smin < 1 || smax < smin || words < (n + 31) / 32) return -1;
    if (n == 0) return 0;
    gg_rng r;
    rng_seed(&r, seed);
    int32_t t = tree_nodes;
    /* tree adjacency as CSR */
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * t);
    int32_t *deg = (int32_t *)calloc(t + 1, sizeof(int32_t));
    par[0] = -1;
    for (int32_t k = 1; k < t; ++k) {
        par[k] = (int32_t)rng_below(&r, (uint64_t)k);
        deg[k]++;
        deg[par[k]]++;
    }
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * (t + 1));
    tp[0] = 0;
    for (int32_t k = 0; k < t; ++k) tp[k + 1] = tp[k] + deg[k];
    int32_t *tadj = (int32_t *)malloc(sizeof(int32_t) * (tp[t] > 0 ? tp[t] : 1));
    int32_t *fill = (int32_t *)calloc(t, sizeof(int32_t));
    for (int32_t k = 1; k < t; ++k) {
        tadj[tp[k] + fill[k]++] = par[k];
        tadj[tp[par[k]] + fill[par[k]]++] = k;
    }
    /* grow subtrees; record node lists */
    int32_t cap = smax < t ? smax : t;
    int32_t *nodes = (int32_t *)malloc(sizeof(int32_t) * (int64_t)n * cap);
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *in_sub = (int32_t *)malloc(sizeof(int32_t) * t);   /* stamp = vertex+1 */
    int32_t *in_fr = (int32_t *)malloc(sizeof(int32_t) * t);
    int32_t *front = (int32_t *)malloc(sizeof(int32_t) * t);
    for (int32_t k = 0; k < t; ++k) in_sub[k] = in_fr[k] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t s = (int32_t)rng_range(&r, smin, smax);
        if (s > t) s = t;
        int32_t *nd = nodes + (int64_t)i * cap;
        int32_t c = 0, nf = 0;
        int32_t root = (int32_t)rng_below(&r, (uint64_t)t);
        int32_t stamp = i + 1;
        nd[c++] = root;
        in_sub[root] = stamp;
        for (int32_t e = tp[root]; e < tp[root + 1]; ++e) {
            int32_t q = tadj[e];
            if (in_fr[q] != stamp) { in_fr[q] = stamp; front[nf++] = q; }
        }
        while (c < s && nf > 0) {
            int32_t pick = (int32_t)rng_below(&r, (uint64_t)nf);
            int32_t q = front[pick];
            front[pick] = front[--nf];
            in_sub[q] = stamp;
            nd[c++] = q;
            for (int32_t e = tp[q]; e < tp[q + 1]; ++e) {
                int32_t z = tadj[e];
                if (in_sub[z] != stamp && in_fr[z] != stamp) { in_fr[z] = stamp; front[nf++] = z; }
            }
        }
        cnt[i] = c;
    }
    /* membership bitsets per tree node, then row_i = OR over its nodes */
    uint32_t *member = (uint32_t *)calloc((size_t)t * words, sizeof(uint32_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t a = 0; a < cnt[i]; ++a) {
            int32_t k = nodes[(int64_t)i * cap + a];
            member[(int64_t)k * words + (i >> 5)] |= 1u << (i & 31);
        }
    for (int32_t i = 0; i < n; ++i) {
        uint32_t *row = rows + (int64_t)i * words;
        for (int32_t a = 0; a < cnt[i]; ++a) {
            const uint32_t *m = member + (int64_t)nodes[(int64_t)i * cap + a] * words;
            for (int32_t w = 0; w < words; ++w) row[w] |= m[w];
        }
        row[i >> 5] &= ~(1u << (i & 31));
    }
    free(member); free(front); free(in_fr); free(in_sub); free(cnt); free(nodes);
    free(fill); free(tadj); free(tp); free(deg); free(par);
    return 0;
}

/* Erdős–Rényi G(n, p) with p = p_num / 2^32.  rows must be zeroed. */
int gg_random_dense(int32_t n, uint32_t p_num, uint64_t seed, uint32_t *rows, int32_t words) {
    if (n < 0 || words < (n + 31) / 32) return -1;
    gg_rng r;
    rng_seed(&r, seed);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = a + 1; b < n; ++b)
            if ((uint32_t)(rng_next(&r) >> 32) < p_num) set_edge(rows, words, a, b);
    return 0;
}

/*
 * Plant an induced chordless cycle C_k: choose k distinct uniform vertices
 * v_0..v_{k-1}, delete every edge among them, then add v_j v_{j+1 mod k}.
 * The induced subgraph on those vertices is exactly C_k.  verts_out[k] gets
 * the chosen vertices in cycle order.  Returns 0, or -1 on bad arguments.
 */
int gg_plant_cycle_dense(int32_t n, int32_t words, uint32_t *rows, int32_t k,
                         uint64_t seed, int32_t *verts_out) {
    if (k < 3 || k > n) return -1;
    gg_rng r;
    rng_seed(&r, seed);
    /* partial Fisher-Yates over a scratch permutation */
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * n);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = 0; i < k; ++i) {
        int32_t j = i + (int32_t)rng_below(&r, (uint64_t)(n - i));
        int32_t tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    for (int32_t a = 0; a < k; ++a)
        for (int32_t b = a + 1; b < k; ++b) clear_edge(rows, words, perm[a], perm[b]);
    for (int32_t a = 0; a < k; ++a) set_edge(rows, words, perm[a], perm[(a + 1) % k]);
    if (verts_out) memcpy(verts_out, perm, sizeof(int32_t) * k);
    free(perm);
    return 0;
}

/* BFS in the dense graph from s, forbidding vertices whose bit is set in
 * `blocked` (s and target are never blocked).  Returns 1 iff target reached. */
static int dense_connected_avoiding(int32_t n, int32_t words, const uint32_t *rows, int32_t s,
                                    int32_t target, const uint32_t *blocked, uint32_t *seen,
                                    int32_t *queue) {
    memcpy(seen, blocked, sizeof(uint32_t) * words);
    seen[s >> 5] |= 1u << (s & 31);
    int32_t head = 0, tail = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t a = queue[head++];
        const uint32_t *row = rows + (int64_t)a * words;
        for (int32_t w = 0; w < words; ++w) {
            uint32_t fresh = row[w] & ~seen[w];
            while (fresh) {
                int32_t b = (w << 5) + __builtin_ctz(fresh);
                fresh &= fresh - 1;
                if (b == target) return 1;
                seen[b >> 5] |= 1u << (b & 31);
                queue[tail++] = b;
            }
        }
    }
    (void)n;
    return 0;
}

/*
 * Add up to r cycle-closing edges.  Each candidate uv is a uniform non-adjacent
 * pair that is connected in G - (N(u) ∩ N(v)), checked in the current graph
 * (including edges added before).  pairs_out[2*j], pairs_out[2*j+1] receive the
 * added edges.  Gives up after max_tries candidates.  Returns #edges added.
 */
int gg_close_cycles_dense(int32_t n, int32_t words, uint32_t *rows, int32_t r_edges,
                          uint64_t seed, int32_t max_tries, int32_t *pairs_out) {
    if (n < 4) return 0;
    gg_rng r;
    rng_seed(&r, seed);
    uint32_t *blocked = (uint32_t *)malloc(sizeof(uint32_t) * words);
    uint32_t *seen = (uint32_t *)malloc(sizeof(uint32_t) * words);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t added = 0, tries = 0;
    while (added < r_edges && tries < max_tries) {
        ++tries;
        int32_t u = (int32_t)rng_below(&r, (uint64_t)n);
        int32_t v = (int32_t)rng_below(&r, (uint64_t)n);
        if (u == v || has_edge(rows, words, u, v)) continue;
        const uint32_t *ru = rows + (int64_t)u * words, *rv = rows + (int64_t)v * words;
        for (int32_t w = 0; w < words; ++w) blocked[w] = ru[w] & rv[w];
        if (!dense_connected_avoiding(n, words, rows, u, v, blocked, seen, queue)) continue;
        set_edge(rows, words, u, v);
        if (pairs_out) { pairs_out[2 * added] = u; pairs_out[2 * added + 1] = v; }
        ++added;
    }
    free(queue); free(seen); free(blocked);
    return added;
}

/*
 * Chordal graph along a reversed perfect elimination order.  Vertex 0 starts
 * alone; vertex t >= 1 draws a clique size s ~ U{1..smax}, then draws uniform
 * earlier vertices w until |LN(w)| >= s - 1 (at most 64 draws; after that s is
 * capped at |LN(w)| + 1), and joins K = {w} ∪ (uniform (s-1)-subset of LN(w)).
 * LN(w), w's neighbourhood among earlier vertices, is a clique by
 * construction, so K is a clique and |K| = s.  Emits edges (t, k) for k in K.
 * Returns #edges, or -1 if cap is too small.  Vertex ids are construction
 * order; callers may relabel.
 */
int64_t gg_peo_edges(int32_t n, int32_t smax, uint64_t seed, int32_t *eu, int32_t *ev, int64_t cap) {
    if (n <= 0 || smax < 1) return 0;
    gg_rng r;
    rng_seed(&r, seed);
    /* LN lists: vertex t's list is lnbuf[t*smax .. t*smax + lncnt[t]) */
    int32_t *lncnt = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *lnbuf = (int32_t *)malloc(sizeof(int32_t) * (int64_t)n * smax);
    int32_t *cpy = (int32_t *)malloc(sizeof(int32_t) * smax);
    int64_t m = 0;
    lncnt[0] = 0;
    for (int32_t t = 1; t < n; ++t) {
        int32_t s = (int32_t)rng_range(&r, 1, smax);
        int32_t w = 0;
        for (int tries = 0; tries < 64; ++tries) {
            w = (int32_t)rng_below(&r, (uint64_t)t);
            if (lncnt[w] >= s - 1) break;
        }
        int32_t L = lncnt[w];
        int32_t take = s - 1 < L ? s - 1 : L;
        memcpy(cpy, lnbuf + (int64_t)w * smax, sizeof(int32_t) * L);
        for (int32_t a = 0; a < take; ++a) {
            int32_t b = a + (int32_t)rng_below(&r, (uint64_t)(L - a));
            int32_t x = cpy[a]; cpy[a] = cpy[b]; cpy[b] = x;
        }
        int32_t *mine = lnbuf + (int64_t)t * smax;
        mine[0] = w;
        for (int32_t a = 0; a < take; ++a) mine[a + 1] = cpy[a];
        lncnt[t] = take + 1;
        if (m + take + 1 > cap) { m = -1; break; }
        for (int32_t a = 0; a <= take; ++a) { eu[m] = t; ev[m] = mine[a]; ++m; }
    }
    free(cpy); free(lnbuf); free(lncnt);
    return m;
}

/* ---- CSR helpers for cycle closing on sparse graphs ---------------------- */

static int csr_adjacent(const int64_t *rp, const int32_t *col, int32_t a, int32_t b,
                        const int32_t *extra, int32_t nextra) {
    int64_t lo = rp[a], hi = rp[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    if (lo < rp[a + 1] && col[lo] == b) return 1;
    for (int32_t j = 0; j < nextra; ++j)
        if ((extra[2 * j] == a && extra[2 * j + 1] == b) || (extra[2 * j] == b && extra[2 * j + 1] == a)) return 1;
    return 0;
}

/*
 * Cycle-closing edges on a CSR graph (sorted rows).  Same rule as the dense
 * version; edges added so far are kept in pairs_out and honoured by the
 * adjacency test and the BFS.  Returns #edges added.
 */
int gg_close_cycles_csr(int32_t n, const int64_t *rp, const int32_t *col, int32_t r_edges,
                        uint64_t seed, int32_t max_tries, int32_t *pairs_out) {
    if (n < 4) return 0;
    gg_rng r;
    rng_seed(&r, seed);
    int32_t *mark = (int32_t *)calloc(n, sizeof(int32_t));   /* stamp: 2*try = blocked, 2*try+1 = seen */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t added = 0, tries = 0;
    while (added < r_edges && tries < max_tries) {
        ++tries;
        int32_t u = (int32_t)rng_below(&r, (uint64_t)n);
        int32_t v = (int32_t)rng_below(&r, (uint64_t)n);
        if (u == v || csr_adjacent(rp, col, u, v, pairs_out, added)) continue;
        int32_t blk = 2 * tries, seenv = 2 * tries + 1;
        /* blocked = N(u) ∩ N(v) */
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t z = col[e];
            if (csr_adjacent(rp, col, v, z, pairs_out, added)) mark[z] = blk;
        }
        for (int32_t j = 0; j < added; ++j) {
            int32_t a = pairs_out[2 * j], b = pairs_out[2 * j + 1];
            int32_t z = a == u ? b : (b == u ? a : -1);
            if (z >= 0 && csr_adjacent(rp, col, v, z, pairs_out, added)) mark[z] = blk;
        }
        int found = 0, head = 0, tail = 0;
        mark[u] = seenv;
        queue[tail++] = u;
        while (head < tail && !found) {
            int32_t a = queue[head++];
            int64_t deg = rp[a + 1] - rp[a];
            for (int64_t e = 0; e < deg + added && !found; ++e) {
                int32_t b;
                if (e < deg) {
                    b = col[rp[a] + e];
                } else {
                    int32_t pa = pairs_out[2 * (e - deg)], pb = pairs_out[2 * (e - deg) + 1];
                    b = pa == a ? pb : (pb == a ? pa : -1);
                    if (b < 0) continue;
                }
                if (b == v) { found = 1; break; }
                if (mark[b] == blk || mark[b] == seenv) continue;
                mark[b] = seenv;
                queue[tail++] = b;
            }
        }
        if (!found) continue;
        pairs_out[2 * added] = u;
        pairs_out[2 * added + 1] = v;
        ++added;
    }
    free(queue); free(mark);
    return added;
}

/* CSR of a dense bit-row graph: pass 1 (col == NULL) fills row_ptr and returns
 * nnz; pass 2 fills col (ascending per row). */
int64_t gg_dense_to_csr(int32_t n, int32_t words, const uint32_t *rows, int64_t *row_ptr, int32_t *col) {
    if (!col) {
        row_ptr[0] = 0;
        for (int32_t v = 0; v < n; ++v) {
            int64_t c = 0;
            for (int32_t w = 0; w < words; ++w) c += __builtin_popcount(rows[(int64_t)v * words + w]);
            row_ptr[v + 1] = row_ptr[v] + c;
        }
        return row_ptr[n];
    }
    for (int32_t v = 0; v < n; ++v) {
        int64_t k = row_ptr[v];
        for (int32_t w = 0; w < words; ++w) {
            uint32_t bits = rows[(int64_t)v * words + w];
            while (bits) {
                col[k++] = (w << 5) + __builtin_ctz(bits);
                bits &= bits - 1;
            }
        }
    }
    return row_ptr[n];
}
