/*
 * oracle.c -- CPU oracle for dynamic single-source shortest paths.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (paper, Section 3 "Example to Illustrate Dynamic SSSP" and
 * the DynSSSP/staticSSSP listings of Appendix "SSSP"): after each update batch
 * is applied to the edge set -- all deletions first, then all insertions, the
 * order of the DynSSSP driver -- dist[v] is the shortest-path distance from
 * the source in the directed, positively weighted graph.  The method reaches
 * this value incrementally; the oracle uses the plain definition instead and
 * recomputes from scratch after every batch with binary-heap Dijkstra over
 * int64 path lengths.  It never updates distances incrementally.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - Unreachable vertices hold INT_MAX/2, the value the appendix listing
 *     stores on deletion (Decremental and OnDelete).  A finite distance at or
 *     above that value is reported as a range error (ORACLE_ERANGE).
 *   - Weights are integers 1 <= w <= 2^20 (propEdge<int>; zero weights would
 *     allow parent cycles).
 *   - Deleting an absent edge is a counted no-op; a repeated deletion of the
 *     same edge finds it absent the second time.
 *   - Insertions are taken in (src, dst, w) order; inserting an edge that is
 *     present after the deletions is a counted no-op that keeps the old
 *     weight, so among repeated insertions of one edge the smallest w wins.
 *   - An edge deleted and inserted in one batch ends up present with the
 *     inserted weight (deletions come first).
 *
 * Parents are not computed: several parent arrays are correct, so they are
 * checked by invariants (oracle/invariants.py) instead.
 *
 * Graph model: one growable array per row, sorted by destination, with
 * binary search for lookups and memmove for updates.  Slow and obvious.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ERANGE (-3)

/* INT_MAX/2: the "infinite" distance of the appendix's SSSP listing. */
static const int64_t ORACLE_INF = 2147483647 / 2;
static const int32_t ORACLE_WMAX = 1 << 20;

typedef struct {
    int32_t dst;
    int32_t w;
} or_edge;

typedef struct {
    int32_t n;
    int32_t *deg;
    int32_t *cap;
    or_edge **row;
} or_graph;

/* ---- row primitives ---------------------------------------------------- */

/* First index in row u whose destination is >= v. */
static int32_t row_lower_bound(const or_graph *g, int32_t u, int32_t v) {
    int32_t lo = 0, hi = g->deg[u];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (g->row[u][mid].dst < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int row_reserve(or_graph *g, int32_t u, int32_t need) {
    if (need <= g->cap[u]) return ORACLE_OK;
    int32_t c = g->cap[u] ? g->cap[u] : 4;
    while (c < need) c *= 2;
    or_edge *p = (or_edge *)realloc(g->row[u], (size_t)c * sizeof(or_edge));
    if (!p) return ORACLE_ENOMEM;
    g->row[u] = p;
    g->cap[u] = c;
    return ORACLE_OK;
}

/* Insert (u -> v, w) if absent.  Returns 1 if inserted, 0 if present. */
static int row_insert(or_graph *g, int32_t u, int32_t v, int32_t w, int *err) {
    int32_t i = row_lower_bound(g, u, v);
    if (i < g->deg[u] && g->row[u][i].dst == v) return 0;
    if (row_reserve(g, u, g->deg[u] + 1) != ORACLE_OK) { *err = ORACLE_ENOMEM; return 0; }
    memmove(&g->row[u][i + 1], &g->row[u][i],
            (size_t)(g->deg[u] - i) * sizeof(or_edge));
    g->row[u][i].dst = v;
    g->row[u][i].w = w;
    g->deg[u] += 1;
    return 1;
}

/* Delete (u -> v) if present.  Returns 1 if deleted, 0 if absent. */
static int row_delete(or_graph *g, int32_t u, int32_t v) {
    int32_t i = row_lower_bound(g, u, v);
    if (i >= g->deg[u] || g->row[u][i].dst != v) return 0;
    memmove(&g->row[u][i], &g->row[u][i + 1],
            (size_t)(g->deg[u] - i - 1) * sizeof(or_edge));
    g->deg[u] -= 1;
    return 1;
}

/* ---- graph lifetime ---------------------------------------------------- */

void or_graph_free(or_graph *g) {
    if (!g) return;
    if (g->row) {
        for (int32_t u = 0; u < g->n; ++u) free(g->row[u]);
    }
    free(g->row);
    free(g->deg);
    free(g->cap);
    free(g);
}

/*
 * Build the model from a CSR (row_off[n+1], col[m], w[m]); rows need not be
 * sorted.  Returns NULL on a bad argument, a duplicate edge, an id out of
 * range or a weight outside [1, 2^20]; *status receives the reason.
 * Self-loops are accepted: with w >= 1 they never shorten a path.
 */
or_graph *or_graph_new(int32_t n, const int64_t *row_off, const int32_t *col,
                       const int32_t *w, int *status) {
    *status = ORACLE_EINVAL;
    if (n <= 0 || !row_off) return NULL;
    if (row_off[0] != 0) return NULL;
    for (int32_t u = 0; u < n; ++u)
        if (row_off[u + 1] < row_off[u]) return NULL;
    or_graph *g = (or_graph *)calloc(1, sizeof(or_graph));
    if (!g) { *status = ORACLE_ENOMEM; return NULL; }
    g->n = n;
    g->deg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    g->cap = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    g->row = (or_edge **)calloc((size_t)n, sizeof(or_edge *));
    if (!g->deg || !g->cap || !g->row) { or_graph_free(g); *status = ORACLE_ENOMEM; return NULL; }
    int err = ORACLE_OK;
    for (int32_t u = 0; u < n; ++u) {
        for (int64_t e = row_off[u]; e < row_off[u + 1]; ++e) {
            int32_t v = col[e], wt = w[e];
            if (v < 0 || v >= n || wt < 1 || wt > ORACLE_WMAX) {
                or_graph_free(g); *status = ORACLE_EINVAL; return NULL;
            }
            if (!row_insert(g, u, v, wt, &err)) {
                or_graph_free(g);
                *status = err ? err : ORACLE_EINVAL;   /* duplicate edge */
                return NULL;
            }
        }
    }
    *status = ORACLE_OK;
    return g;
}

int64_t or_num_edges(const or_graph *g) {
    int64_t m = 0;
    for (int32_t u = 0; u < g->n; ++u) m += g->deg[u];
    return m;
}

/* Export the current edge set as a row-sorted CSR (arrays sized by caller:
 * row_off[n+1], col[m], w[m] with m = or_num_edges). */
void or_export_csr(const or_graph *g, int64_t *row_off, int32_t *col, int32_t *w) {
    int64_t e = 0;
    row_off[0] = 0;
    for (int32_t u = 0; u < g->n; ++u) {
        for (int32_t i = 0; i < g->deg[u]; ++i) {
            col[e] = g->row[u][i].dst;
            w[e] = g->row[u][i].w;
            ++e;
        }
        row_off[u + 1] = e;
    }
}

/* ---- batch application ------------------------------------------------- */

typedef struct { int32_t u, v, w; } or_triple;

static int cmp_triple(const void *a, const void *b) {
    const or_triple *x = (const or_triple *)a, *y = (const or_triple *)b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return 0;
}

/*
 * Apply one batch: every deletion, then every insertion (DynSSSP driver:
 * OnDelete/updateCSRDel/Decremental before OnAdd/updateCSRAdd/Incremental).
 * The whole batch is validated before the graph changes; on ORACLE_EINVAL
 * the graph is untouched.  counters[4] receives
 * {deletions applied, deletions of absent edges, insertions applied,
 *  insertions of present edges}.
 */
int or_apply_batch(or_graph *g,
                   int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                   int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                   const int32_t *add_w, int64_t *counters) {
    const int32_t n = g->n;
    for (int64_t i = 0; i < n_del; ++i)
        if (del_src[i] < 0 || del_src[i] >= n || del_dst[i] < 0 || del_dst[i] >= n)
            return ORACLE_EINVAL;
    for (int64_t i = 0; i < n_add; ++i)
        if (add_src[i] < 0 || add_src[i] >= n || add_dst[i] < 0 || add_dst[i] >= n ||
            add_w[i] < 1 || add_w[i] > ORACLE_WMAX)
            return ORACLE_EINVAL;

    int64_t del_ok = 0, del_absent = 0, add_ok = 0, add_present = 0;
    for (int64_t i = 0; i < n_del; ++i) {
        if (row_delete(g, del_src[i], del_dst[i])) ++del_ok; else ++del_absent;
    }
    or_triple *t = NULL;
    if (n_add > 0) {
        t = (or_triple *)malloc((size_t)n_add * sizeof(or_triple));
        if (!t) return ORACLE_ENOMEM;
        for (int64_t i = 0; i < n_add; ++i) {
            t[i].u = add_src[i]; t[i].v = add_dst[i]; t[i].w = add_w[i];
        }
        qsort(t, (size_t)n_add, sizeof(or_triple), cmp_triple);
    }
    int err = ORACLE_OK;
    for (int64_t i = 0; i < n_add; ++i) {
        if (row_insert(g, t[i].u, t[i].v, t[i].w, &err)) ++add_ok;
        else if (err) { free(t); return err; }
        else ++add_present;
    }
    free(t);
    if (counters) {
        counters[0] = del_ok; counters[1] = del_absent;
        counters[2] = add_ok; counters[3] = add_present;
    }
    return ORACLE_OK;
}

/* ---- Dijkstra ---------------------------------------------------------- */

typedef struct { int64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *size, heap_item x) {
    int64_t i = (*size)++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
    heap_item top = h[0];
    heap_item last = h[--(*size)];
    int64_t i = 0, n = *size;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= n) break;
        if (c + 1 < n && h[c + 1].d < h[c].d) ++c;
        if (last.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    if (n > 0) h[i] = last;
    return top;
}

/*
 * Single-source shortest paths from src by Dijkstra with a binary heap and
 * lazy deletion, path lengths in int64.  dist_out[v] = length, or INT_MAX/2
 * if v is unreachable.  Returns ORACLE_ERANGE if a finite length does not
 * fit below INT_MAX/2 (dist_out is still filled, clamped to INT_MAX/2).
 */
int or_dijkstra(const or_graph *g, int32_t src, int32_t *dist_out) {
    const int32_t n = g->n;
    if (src < 0 || src >= n) return ORACLE_EINVAL;
    int64_t *d = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    int64_t m = or_num_edges(g);
    heap_item *h = (heap_item *)malloc((size_t)(m + 1) * sizeof(heap_item));
    if (!d || !done || !h) { free(d); free(done); free(h); return ORACLE_ENOMEM; }
    for (int32_t v = 0; v < n; ++v) d[v] = INT64_MAX;
    int64_t hs = 0;
    d[src] = 0;
    heap_item s0 = {0, src};
    heap_push(h, &hs, s0);
    while (hs > 0) {
        heap_item it = heap_pop(h, &hs);
        int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (int32_t i = 0; i < g->deg[u]; ++i) {
            int32_t v = g->row[u][i].dst;
            int64_t nd = d[u] + g->row[u][i].w;
            if (nd < d[v]) {
                d[v] = nd;
                heap_item x = {nd, v};
                heap_push(h, &hs, x);
            }
        }
    }
    int rc = ORACLE_OK;
    for (int32_t v = 0; v < n; ++v) {
        if (d[v] == INT64_MAX) {
            dist_out[v] = (int32_t)ORACLE_INF;
        } else if (d[v] >= ORACLE_INF) {
            dist_out[v] = (int32_t)ORACLE_INF;
            rc = ORACLE_ERANGE;
        } else {
            dist_out[v] = (int32_t)d[v];
        }
    }
    free(d); free(done); free(h);
    return rc;
}

/* ------------------------------------------------------------------------
 * PageRank (paper, appendix listing "Dynamic PR coded in StarPlat DSL":
 * staticPR, Incremental, Decremental, DynPR).  Single precision, as the
 * listing's propNode<float>.
 *
 * One Jacobi step over a vertex set S, with N = number of vertices and d
 * the damping factor:
 *     pr'[v] = (1 - d) / N + d * sum_{u -> v} pr[u] / outdeg(u)   (v in S)
 * in-neighbours u in increasing id order, each term pr[u] / outdeg(u)
 * rounded to float and added to a float sum.  Vertices without out-edges
 * pass no rank on (the listing divides by count_outNbrs of in-neighbours
 * only).  Steps repeat until sum_{v in S} |pr'[v] - pr[v]| <= beta or
 * max_iter steps have run; the listing accumulates the signed difference,
 * read here as its absolute value (a signed sum can stop on cancellation).
 *
 * staticPR: S = all vertices, pr = 1/N at the start.
 * DynPR, per batch: (1) the destinations of the deletions are flagged and
 * the flags spread along out-edges to every reachable vertex of the current
 * graph (propagateNodeFlags, read as forward reachability); (2) the
 * deletions are applied (updateCSRDel); (3) Jacobi steps over the flagged
 * vertices from their current ranks (Decremental); then the same three
 * steps for the insertions (propagateNodeFlags on the graph after the
 * deletions, updateCSRAdd, Incremental).  Unflagged vertices keep their
 * ranks.
 * ---------------------------------------------------------------------- */

/* In-neighbour lists of the current graph, sorted by source id. */
typedef struct {
    int64_t *off;
    int32_t *src;
    int32_t *outdeg;
} or_rev;

static void rev_free(or_rev *r) {
    free(r->off);
    free(r->src);
    free(r->outdeg);
}

static int rev_build(const or_graph *g, or_rev *r) {
    const int32_t n = g->n;
    int64_t m = or_num_edges(g);
    r->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    r->src = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    r->outdeg = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!r->off || !r->src || !r->outdeg) {
        rev_free(r);
        return ORACLE_ENOMEM;
    }
    for (int32_t u = 0; u < n; ++u) {
        r->outdeg[u] = g->deg[u];
        for (int32_t j = 0; j < g->deg[u]; ++j) r->off[g->row[u][j].dst + 1] += 1;
    }
    for (int32_t v = 0; v < n; ++v) r->off[v + 1] += r->off[v];
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!fill) {
        rev_free(r);
        return ORACLE_ENOMEM;
    }
    for (int32_t v = 0; v < n; ++v) fill[v] = r->off[v];
    /* sources visited in increasing order, so every list comes out sorted */
    for (int32_t u = 0; u < n; ++u)
        for (int32_t j = 0; j < g->deg[u]; ++j) r->src[fill[g->row[u][j].dst]++] = u;
    free(fill);
    return ORACLE_OK;
}

/* Jacobi steps over the vertices with flag[v] != 0 (all if flag == NULL). */
static int pr_iterate(const or_graph *g, const unsigned char *flag, float d, float beta,
                      int32_t max_iter, float *pr, int32_t *iters) {
    const int32_t n = g->n;
    or_rev r;
    int st = rev_build(g, &r);
    if (st != ORACLE_OK) return st;
    float *nxt = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
    if (!nxt) {
        rev_free(&r);
        return ORACLE_ENOMEM;
    }
    const float base = (1.0f - d) / (float)n;
    int32_t it = 0;
    double diff;
    do {
        diff = 0.0;
        for (int32_t v = 0; v < n; ++v) {
            if (flag && !flag[v]) continue;
            float sum = 0.0f;
            for (int64_t e = r.off[v]; e < r.off[v + 1]; ++e) {
                const int32_t u = r.src[e];
                const float term = pr[u] / (float)r.outdeg[u];
                sum = sum + term;
            }
            const float prod = d * sum;
            const float val = base + prod;
            diff += fabs((double)val - (double)pr[v]);
            nxt[v] = val;
        }
        for (int32_t v = 0; v < n; ++v)
            if (!flag || flag[v]) pr[v] = nxt[v];
        ++it;
    } while (diff > (double)beta && it < max_iter);
    *iters = it;
    free(nxt);
    rev_free(&r);
    return ORACLE_OK;
}

/* Flag the given destinations and every vertex reachable from them. */
static int64_t propagate_flags(const or_graph *g, const int32_t *dst, int64_t k,
                               unsigned char *flag) {
    const int32_t n = g->n;
    int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!queue) return -1;
    int64_t head = 0, tail = 0;
    memset(flag, 0, (size_t)n);
    for (int64_t i = 0; i < k; ++i) {
        const int32_t v = dst[i];
        if (!flag[v]) {
            flag[v] = 1;
            queue[tail++] = v;
        }
    }
    while (head < tail) {
        const int32_t v = queue[head++];
        for (int32_t j = 0; j < g->deg[v]; ++j) {
            const int32_t x = g->row[v][j].dst;
            if (!flag[x]) {
                flag[x] = 1;
                queue[tail++] = x;
            }
        }
    }
    free(queue);
    return tail;
}

int or_pr_static(const or_graph *g, float d, float beta, int32_t max_iter, float *pr,
                 int32_t *iters) {
    if (!g || !pr || !iters || max_iter < 1 || !(d >= 0.0f && d <= 1.0f) || !(beta >= 0.0f))
        return ORACLE_EINVAL;
    for (int32_t v = 0; v < g->n; ++v) pr[v] = 1.0f / (float)g->n;
    return pr_iterate(g, NULL, d, beta, max_iter, pr, iters);
}

/* counters: [0..3] as or_apply_batch, [4] flagged for the deletions, [5]
 * flagged for the insertions, [6] Jacobi steps of Decremental, [7] of
 * Incremental. */
int or_pr_batch(or_graph *g, int64_t n_del, const int32_t *del_src, const int32_t *del_dst,
                int64_t n_add, const int32_t *add_src, const int32_t *add_dst,
                const int32_t *add_w, float d, float beta, int32_t max_iter, float *pr,
                int64_t *counters) {
    if (!g || !pr || !counters || n_del < 0 || n_add < 0 || max_iter < 1) return ORACLE_EINVAL;
    for (int64_t i = 0; i < n_del; ++i)
        if (del_src[i] < 0 || del_src[i] >= g->n || del_dst[i] < 0 || del_dst[i] >= g->n)
            return ORACLE_EINVAL;
    for (int64_t i = 0; i < n_add; ++i)
        if (add_src[i] < 0 || add_src[i] >= g->n || add_dst[i] < 0 || add_dst[i] >= g->n ||
            add_w[i] < 1 || add_w[i] > ORACLE_WMAX)
            return ORACLE_EINVAL;
    unsigned char *flag = (unsigned char *)malloc((size_t)(g->n > 0 ? g->n : 1));
    if (!flag) return ORACLE_ENOMEM;
    int64_t c1[4] = {0, 0, 0, 0}, c2[4] = {0, 0, 0, 0};
    int32_t it1 = 0, it2 = 0;
    int st = ORACLE_OK;
    /* deletions: OnDelete flags, propagateNodeFlags, updateCSRDel, Decremental */
    int64_t f1 = propagate_flags(g, del_dst, n_del, flag);
    if (f1 < 0) st = ORACLE_ENOMEM;
    if (st == ORACLE_OK) st = or_apply_batch(g, n_del, del_src, del_dst, 0, NULL, NULL, NULL, c1);
    if (st == ORACLE_OK && f1 > 0) st = pr_iterate(g, flag, d, beta, max_iter, pr, &it1);
    /* insertions: OnAdd flags, propagateNodeFlags, updateCSRAdd, Incremental */
    int64_t f2 = 0;
    if (st == ORACLE_OK) {
        f2 = propagate_flags(g, add_dst, n_add, flag);
        if (f2 < 0) st = ORACLE_ENOMEM;
    }
    if (st == ORACLE_OK) st = or_apply_batch(g, 0, NULL, NULL, n_add, add_src, add_dst, add_w, c2);
    if (st == ORACLE_OK && f2 > 0) st = pr_iterate(g, flag, d, beta, max_iter, pr, &it2);
    free(flag);
    if (st != ORACLE_OK) return st;
    counters[0] = c1[0];
    counters[1] = c1[1];
    counters[2] = c2[2];
    counters[3] = c2[3];
    counters[4] = f1;
    counters[5] = f2;
    counters[6] = it1;
    counters[7] = it2;
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------
 * Triangle count (paper, appendix listing "Dynamic TC coded in StarPlat
 * DSL", staticTC): for every vertex v, every neighbour u < v and every
 * neighbour w > v of v such that u -> w is an edge, count one.  On a
 * symmetric graph (every edge stored in both directions) this counts every
 * triangle once, at its middle vertex.  The dynamic form of the listing
 * (Decremental / Incremental corrections) reaches the same number for the
 * graph after the batch; the oracle recounts from scratch.
 * ---------------------------------------------------------------------- */
int or_tc_static(const or_graph *g, int64_t *count) {
    if (!g || !count) return ORACLE_EINVAL;
    int64_t c = 0;
    for (int32_t v = 0; v < g->n; ++v) {
        const or_edge *r = g->row[v];
        for (int32_t a = 0; a < g->deg[v]; ++a) {
            const int32_t u = r[a].dst;
            if (u >= v) continue;
            for (int32_t b = 0; b < g->deg[v]; ++b) {
                const int32_t w = r[b].dst;
                if (w <= v) continue;
                const int32_t j = row_lower_bound(g, u, w);
                if (j < g->deg[u] && g->row[u][j].dst == w) ++c;
            }
        }
    }
    *count = c;
    return ORACLE_OK;
}
