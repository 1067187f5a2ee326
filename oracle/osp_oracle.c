/*
 * FP64 CPU oracle for offset score propagation (OSP / OSP-T).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header, table or helper with the CUDA
 * engine: it is a plain, slow, single-threaded restatement of the paper
 * (Yoon, Jin, Kang, "Fast and Accurate Random Walk with Restart on Dynamic
 * Graphs with Guarantees", WWW 2018) written so that it can be checked
 * against the text by eye. Every floating-point quantity is a double.
 *
 * Readings of the paper taken here (each is pinned by a test):
 *  - Graph (Sec. 2.1, Eq. 1): a simple directed graph with unit weights;
 *    duplicate edges collapse, self-loops are kept. A~ has 1/d_u at each
 *    out-neighbour of u; a dead-end row (d_u = 0) is all zero.
 *  - CPI (Sec. 2.2): x(0) = q_CPI = c * e_s, x(i) = (1-c) A~^T x(i-1),
 *    r = sum_i x(i). The sum includes x(0).
 *  - OSP (Sec. 3.1, Algorithm 1): q_offset = (1-c)(B~^T - A~^T) r_old;
 *    r_offset starts at q_offset (the sum over i >= 0 of the Sec. 3.1
 *    equations and Theorem 2 include i = 0), then x(i) = (1-c) B~^T x(i-1) is
 *    added for i = 1, 2, ...; r_new = r_old + r_offset.
 *  - Stopping rule (Algorithm 1, Sec. 3.2): the loop is a do-while. It
 *    computes x(i), adds it, and stops once ||x(i)||_1 <= eps, so at least one
 *    propagation step always runs (Table 2: OSP-T with ||q_offset||_1 below
 *    eps still reports one iteration; CPI at eps = 1e-9 reports 116).
 *  - Node insertion (Sec. 3.4.1): a new node gets the next id, an empty row
 *    and column, and a zero score. Node deletion removes the node's out-edges
 *    (its row of B~ becomes zero) and also its in-edges; its id is never
 *    reused. Op 4 is the literal form of that sentence: only the node's row
 *    becomes zero (all its out-edges go); its in-edges stay and the node
 *    stays live.
 *  - Update batches: operations apply in order; Delta A is the difference
 *    between the rows after the whole batch and the rows before it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t u, v, op; /* op: 0 insert edge, 1 delete edge, 2 add node, 3 delete node,
                         4 zero the node's row (remove its out-edges only) */
} orc_update;

typedef struct {
    int32_t iterations;     /* propagation steps x(1)..x(k) performed */
    double q_l1;            /* ||x(0)||_1 (||q_offset||_1 for OSP, c for CPI) */
    double last_l1;         /* ||x(k)||_1 */
    int64_t visited_edges;  /* sum over steps of out-edges of nodes with x != 0 */
} orc_stats;

/* ------------------------------------------------------------------------ */
/* Sorted integer lists (one per node and direction)                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t *a;
    int32_t len, cap;
} ivec;

/* index of x in the sorted list, or -(insertion point)-1 */
static int64_t ivec_find(const ivec *s, int32_t x) {
    int64_t lo = 0, hi = s->len;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (s->a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    if (lo < s->len && s->a[lo] == x) return lo;
    return -lo - 1;
}

static int ivec_reserve(ivec *s, int32_t need) {
    if (need <= s->cap) return 0;
    int32_t cap = s->cap ? s->cap : 4;
    while (cap < need) cap *= 2;
    int32_t *p = (int32_t *)realloc(s->a, (size_t)cap * sizeof(int32_t));
    if (!p) return -1;
    s->a = p;
    s->cap = cap;
    return 0;
}

/* insert x keeping the list sorted; returns 1 if inserted, 0 if present */
static int ivec_insert(ivec *s, int32_t x) {
    int64_t f = ivec_find(s, x);
    if (f >= 0) return 0;
    int64_t at = -f - 1;
    if (ivec_reserve(s, s->len + 1)) return -1;
    memmove(s->a + at + 1, s->a + at, (size_t)(s->len - at) * sizeof(int32_t));
    s->a[at] = x;
    s->len++;
    return 1;
}

/* remove x; returns 1 if removed, 0 if absent */
static int ivec_remove(ivec *s, int32_t x) {
    int64_t f = ivec_find(s, x);
    if (f < 0) return 0;
    memmove(s->a + f, s->a + f + 1, (size_t)(s->len - f - 1) * sizeof(int32_t));
    s->len--;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Dynamic graph: the edge set, kept as sorted out- and in-lists             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, cap, m;
    ivec *out, *in;
    uint8_t *dead;
} orc_graph;

static int graph_grow(orc_graph *g, int64_t need) {
    if (need <= g->cap) return 0;
    int64_t cap = g->cap ? g->cap : 16;
    while (cap < need) cap *= 2;
    ivec *o = (ivec *)realloc(g->out, (size_t)cap * sizeof(ivec));
    if (!o) return -1;
    g->out = o;
    ivec *i = (ivec *)realloc(g->in, (size_t)cap * sizeof(ivec));
    if (!i) return -1;
    g->in = i;
    uint8_t *d = (uint8_t *)realloc(g->dead, (size_t)cap);
    if (!d) return -1;
    g->dead = d;
    memset(g->out + g->cap, 0, (size_t)(cap - g->cap) * sizeof(ivec));
    memset(g->in + g->cap, 0, (size_t)(cap - g->cap) * sizeof(ivec));
    memset(g->dead + g->cap, 0, (size_t)(cap - g->cap));
    g->cap = cap;
    return 0;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Fill sorted lists from a list of (first << 32 | second) keys sorted ascending. */
static int fill_lists(ivec *lists, const uint64_t *keys, int64_t k) {
    int64_t i = 0;
    while (i < k) {
        int64_t j = i;
        int32_t head = (int32_t)(keys[i] >> 32);
        while (j < k && (int32_t)(keys[j] >> 32) == head) j++;
        ivec *s = &lists[head];
        if (ivec_reserve(s, (int32_t)(j - i))) return -1;
        for (int64_t t = i; t < j; t++) s->a[t - i] = (int32_t)(keys[t] & 0xffffffffu);
        s->len = (int32_t)(j - i);
        i = j;
    }
    return 0;
}

void orc_graph_free(orc_graph *g);

/* Build the edge set of a graph with n nodes from m (src, dst) pairs.
 * Duplicates collapse; self-loops are kept; undirected != 0 stores both
 * directions of every pair (Sec. 4.1: an undirected edge is two directed
 * edges). Returns NULL on a bad id or out of memory. */
orc_graph *orc_graph_new(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                         int undirected) {
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    if (!g) return NULL;
    if (graph_grow(g, n > 0 ? n : 1)) goto fail;
    g->n = n;
    int64_t k = undirected ? 2 * m : m;
    uint64_t *keys = (uint64_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(uint64_t));
    if (!keys) goto fail;
    for (int64_t e = 0; e < m; e++) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) {
            free(keys);
            goto fail;
        }
        keys[e] = ((uint64_t)(uint32_t)src[e] << 32) | (uint32_t)dst[e];
        if (undirected) keys[m + e] = ((uint64_t)(uint32_t)dst[e] << 32) | (uint32_t)src[e];
    }
    /* sorted, de-duplicated (src, dst) set -> out-lists */
    qsort(keys, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t u = 0;
    for (int64_t e = 0; e < k; e++)
        if (e == 0 || keys[e] != keys[e - 1]) keys[u++] = keys[e];
    g->m = u;
    if (fill_lists(g->out, keys, u)) {
        free(keys);
        goto fail;
    }
    /* the same set keyed (dst, src) -> in-lists */
    for (int64_t e = 0; e < u; e++) keys[e] = (keys[e] << 32) | (keys[e] >> 32);
    qsort(keys, (size_t)u, sizeof(uint64_t), cmp_u64);
    if (fill_lists(g->in, keys, u)) {
        free(keys);
        goto fail;
    }
    free(keys);
    return g;
fail:
    orc_graph_free(g);
    return NULL;
}

void orc_graph_free(orc_graph *g) {
    if (!g) return;
    for (int64_t i = 0; i < g->cap; i++) {
        free(g->out ? g->out[i].a : NULL);
        free(g->in ? g->in[i].a : NULL);
    }
    free(g->out);
    free(g->in);
    free(g->dead);
    free(g);
}

int64_t orc_graph_n(const orc_graph *g) { return g->n; }
int64_t orc_graph_m(const orc_graph *g) { return g->m; }

/* Check a batch against the sequential rules without changing the graph.
 * Returns -1 if valid, else the index of the first invalid operation.
 * Rules: op codes 0..4; every id named must exist at that point of the batch
 * (nodes added earlier in the batch count) and must not have been deleted
 * before (earlier batches or earlier in this batch); a node is deleted at
 * most once and never if it is in protect[0..n_protect). */
int64_t orc_graph_validate(const orc_graph *g, const orc_update *ops, int64_t U,
                           const int32_t *protect, int32_t n_protect) {
    int64_t n = g->n;
    int64_t adds = 0;
    for (int64_t p = 0; p < U; p++) adds += ops[p].op == 2;
    uint8_t *dead = (uint8_t *)calloc((size_t)(n + adds + 1), 1);
    if (!dead) return 0;
    memcpy(dead, g->dead, (size_t)n);
    int64_t bad = -1;
    for (int64_t p = 0; p < U && bad < 0; p++) {
        int32_t op = ops[p].op, u = ops[p].u, v = ops[p].v;
        if (op == 0 || op == 1) {
            if (u < 0 || u >= n || v < 0 || v >= n || dead[u] || dead[v]) bad = p;
        } else if (op == 2) {
            n++;
        } else if (op == 3) {
            if (u < 0 || u >= n || dead[u]) bad = p;
            for (int32_t s = 0; s < n_protect && bad < 0; s++)
                if (protect[s] == u) bad = p;
            if (bad < 0) dead[u] = 1;
        } else if (op == 4) {
            if (u < 0 || u >= n || dead[u]) bad = p;
        } else {
            bad = p;
        }
    }
    free(dead);
    return bad;
}

/* Apply a batch in order. Returns -1 on success, or the index of the first
 * invalid operation (then the graph is unchanged). */
int64_t orc_graph_apply(orc_graph *g, const orc_update *ops, int64_t U, const int32_t *protect,
                        int32_t n_protect) {
    int64_t bad = orc_graph_validate(g, ops, U, protect, n_protect);
    if (bad >= 0) return bad;
    for (int64_t p = 0; p < U; p++) {
        int32_t op = ops[p].op, u = ops[p].u, v = ops[p].v;
        if (op == 0) { /* insert edge (no-op if present) */
            int r = ivec_insert(&g->out[u], v);
            if (r < 0) return -2;
            if (r == 1) {
                if (ivec_insert(&g->in[v], u) < 0) return -2;
                g->m++;
            }
        } else if (op == 1) { /* delete edge (no-op if absent) */
            if (ivec_remove(&g->out[u], v)) {
                ivec_remove(&g->in[v], u);
                g->m--;
            }
        } else if (op == 2) { /* add node: next id, empty row and column */
            if (graph_grow(g, g->n + 1)) return -2;
            g->n++;
        } else if (op == 4) { /* zero row u: its out-edges go, nothing else changes */
            ivec *o = &g->out[u];
            for (int32_t t = 0; t < o->len; t++) {
                ivec_remove(&g->in[o->a[t]], u);
                g->m--;
            }
            o->len = 0;
        } else { /* delete node u: all out- and in-edges go, the id stays dead */
            ivec *o = &g->out[u];
            for (int32_t t = 0; t < o->len; t++) {
                if (o->a[t] != u) ivec_remove(&g->in[o->a[t]], u);
                g->m--;
            }
            o->len = 0;
            ivec *in = &g->in[u];
            for (int32_t t = 0; t < in->len; t++) {
                if (in->a[t] == u) continue; /* the self-loop was counted above */
                ivec_remove(&g->out[in->a[t]], u);
                g->m--;
            }
            in->len = 0;
            g->dead[u] = 1;
        }
    }
    return -1;
}

/* Out-edges as CSR: row_ptr[n+1], col[m], each row ascending. */
void orc_graph_csr(const orc_graph *g, int64_t *row_ptr, int32_t *col) {
    int64_t e = 0;
    for (int64_t u = 0; u < g->n; u++) {
        row_ptr[u] = e;
        memcpy(col + e, g->out[u].a, (size_t)g->out[u].len * sizeof(int32_t));
        e += g->out[u].len;
    }
    row_ptr[g->n] = e;
}

/* In-edges as CSC: col_ptr[n+1], row[m], each column ascending. */
void orc_graph_csc(const orc_graph *g, int64_t *col_ptr, int32_t *row) {
    int64_t e = 0;
    for (int64_t v = 0; v < g->n; v++) {
        col_ptr[v] = e;
        memcpy(row + e, g->in[v].a, (size_t)g->in[v].len * sizeof(int32_t));
        e += g->in[v].len;
    }
    col_ptr[g->n] = e;
}

void orc_graph_dead(const orc_graph *g, uint8_t *out) { memcpy(out, g->dead, (size_t)g->n); }

/* ------------------------------------------------------------------------ */
/* Propagation (Sec. 2.2 CPI and Algorithm 1)                                */
/* ------------------------------------------------------------------------ */

/* y = A~^T x for the row-normalised adjacency A~ of a CSR graph (Eq. 1):
 * y[v] = sum over edges (u, v) of x[u] / d_u. Dead-end rows contribute
 * nothing. Returns the number of edges visited (rows with x[u] != 0). */
static int64_t spmv_transposed(int64_t n, const int64_t *row_ptr, const int32_t *col,
                               const double *x, double *y) {
    int64_t visited = 0;
    for (int64_t v = 0; v < n; v++) y[v] = 0.0;
    for (int64_t u = 0; u < n; u++) {
        int64_t d = row_ptr[u + 1] - row_ptr[u];
        if (d == 0 || x[u] == 0.0) continue;
        double w = x[u] / (double)d;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) y[col[e]] += w;
        visited += d;
    }
    return visited;
}

static double l1(int64_t n, const double *x) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += fabs(x[i]);
    return s;
}

/* Cumulative power iteration from a start vector x0 (Sec. 2.2):
 *   r = x(0) + x(1) + ... + x(k),  x(i) = (1-c) A~^T x(i-1),
 * as a do-while loop that stops after the first i with ||x(i)||_1 <= eps
 * (Algorithm 1 loop), or after exactly force_iters steps when force_iters > 0
 * (used to replay an iteration count chosen elsewhere). l1_hist, if given,
 * receives ||x(0)||_1 .. ||x(k)||_1 (max_iter + 1 entries). Returns 0, or 1
 * if max_iter steps ran without meeting the rule. */
int orc_propagate(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *x0,
                  double c, double eps, int32_t force_iters, int32_t max_iter, double *r,
                  double *l1_hist, orc_stats *st) {
    double *x = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *y = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!x || !y) {
        free(x);
        free(y);
        return -1;
    }
    for (int64_t i = 0; i < n; i++) {
        x[i] = x0[i];
        r[i] = x0[i];
    }
    orc_stats s;
    s.q_l1 = l1(n, x);
    s.iterations = 0;
    s.visited_edges = 0;
    s.last_l1 = s.q_l1;
    if (l1_hist) l1_hist[0] = s.q_l1;
    int rc = 0;
    for (;;) {
        s.visited_edges += spmv_transposed(n, row_ptr, col, x, y);
        for (int64_t i = 0; i < n; i++) x[i] = (1.0 - c) * y[i];
        for (int64_t i = 0; i < n; i++) r[i] += x[i];
        s.iterations++;
        s.last_l1 = l1(n, x);
        if (l1_hist && s.iterations <= max_iter) l1_hist[s.iterations] = s.last_l1;
        if (force_iters > 0) {
            if (s.iterations >= force_iters) break;
        } else if (s.last_l1 <= eps) {
            break;
        }
        if (s.iterations >= max_iter) {
            rc = 1;
            break;
        }
    }
    free(x);
    free(y);
    if (st) *st = s;
    return rc;
}

/* CPI for seed s (Sec. 2.2): start vector q_CPI = c * e_s. */
int orc_cpi(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t seed, double c,
            double eps, int32_t force_iters, int32_t max_iter, double *r, double *l1_hist,
            orc_stats *st) {
    double *q = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!q) return -1;
    q[seed] = c;
    int rc = orc_propagate(n, row_ptr, col, q, c, eps, force_iters, max_iter, r, l1_hist, st);
    free(q);
    return rc;
}

/* Offset seed vector (Sec. 3.1, Algorithm 1 first step):
 *   q_offset = (1-c) (B~^T - A~^T) r_old,
 * written entry by entry: q[v] = (1-c) sum_u r_old[u] (B~[u][v] - A~[u][v]).
 * The old graph has n_old nodes and the new one n_new >= n_old; nodes added
 * by the batch have an all-zero old row and column and r_old = 0 (Sec. 3.4.1).
 * For each row u the two sorted rows are walked together; an entry present in
 * both rows contributes 1/d'_u - 1/d_u, which is exactly zero for an unchanged
 * row. */
void orc_offset(int64_t n_old, const int64_t *rp_old, const int32_t *col_old, int64_t n_new,
                const int64_t *rp_new, const int32_t *col_new, const double *r_old, double c,
                double *q) {
    for (int64_t v = 0; v < n_new; v++) q[v] = 0.0;
    for (int64_t u = 0; u < n_new; u++) {
        double ru = u < n_old ? r_old[u] : 0.0;
        int64_t a0 = u < n_old ? rp_old[u] : 0, a1 = u < n_old ? rp_old[u + 1] : 0;
        int64_t b0 = rp_new[u], b1 = rp_new[u + 1];
        double wa = a1 > a0 ? 1.0 / (double)(a1 - a0) : 0.0; /* A~[u][.] */
        double wb = b1 > b0 ? 1.0 / (double)(b1 - b0) : 0.0; /* B~[u][.] */
        int64_t i = a0, j = b0;
        while (i < a1 || j < b1) {
            int32_t va = i < a1 ? col_old[i] : INT32_MAX;
            int32_t vb = j < b1 ? col_new[j] : INT32_MAX;
            double diff;
            int32_t v;
            if (va == vb) {
                v = va;
                diff = wb - wa;
                i++;
                j++;
            } else if (va < vb) {
                v = va;
                diff = -wa;
                i++;
            } else {
                v = vb;
                diff = wb;
                j++;
            }
            q[v] += (1.0 - c) * ru * diff;
        }
    }
}

/* OSP / OSP-T (Algorithm 1): r_new = r_old + r_offset, where r_offset is the
 * cumulative propagation of q_offset over the new graph. r_new has n_new
 * entries; q_out (n_new, nullable) receives q_offset. */
int orc_osp(int64_t n_old, const int64_t *rp_old, const int32_t *col_old, int64_t n_new,
            const int64_t *rp_new, const int32_t *col_new, const double *r_old, double c,
            double eps, int32_t force_iters, int32_t max_iter, double *r_new, double *q_out,
            double *l1_hist, orc_stats *st) {
    size_t nb = (size_t)(n_new > 0 ? n_new : 1) * sizeof(double);
    double *q = (double *)malloc(nb);
    double *roff = (double *)malloc(nb);
    if (!q || !roff) {
        free(q);
        free(roff);
        return -1;
    }
    orc_offset(n_old, rp_old, col_old, n_new, rp_new, col_new, r_old, c, q);
    int rc = orc_propagate(n_new, rp_new, col_new, q, c, eps, force_iters, max_iter, roff, l1_hist,
                           st);
    for (int64_t v = 0; v < n_new; v++) r_new[v] = (v < n_old ? r_old[v] : 0.0) + roff[v];
    if (q_out) memcpy(q_out, q, nb);
    free(q);
    free(roff);
    return rc;
}

/* Residual of Eq. 1 for seed s: rho = c e_s - (I - (1-c) B~^T) r. Because
 * every column sum of (1-c) B~^T is at most 1-c, ||(I - (1-c) B~^T)^-1||_1 is
 * at most 1/c, so ||r - r*||_1 <= ||rho||_1 / c. Returns ||rho||_1. */
double orc_residual_l1(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t seed,
                       double c, const double *r) {
    double *y = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!y) return -1.0;
    spmv_transposed(n, row_ptr, col, r, y);
    double s = 0.0;
    for (int64_t v = 0; v < n; v++) {
        double rho = (v == seed ? c : 0.0) - (r[v] - (1.0 - c) * y[v]);
        s += fabs(rho);
    }
    free(y);
    return s;
}
