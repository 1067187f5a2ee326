/*
 * Seeded synthetic inputs at benchmark scale: R-MAT and Chung-Lu edge draws,
 * and the sort / de-duplication of edge keys. This file draws inputs only; it
 * holds none of the RWR / OSP arithmetic, so the CUDA engine and the CPU
 * oracle can both consume what it produces.
 *
 * Random numbers come from a counter-based generator: value j of stream `key`
 * is the SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to
 * key + (j + 1) * 0x9E3779B97F4A7C15. Draw i of a sampler reads a fixed block
 * of counters, so the result does not depend on how many threads run.
 *
 * An edge is the 64-bit key (source << 32) | target; ids stay below 2^25.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ull
#define NO_EDGE 0xFFFFFFFFFFFFFFFFull /* a rejected draw (self-loop) */

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t j) { return mix64(key + (j + 1) * GAMMA); }

/* ------------------------------------------------------------------------ */
/* a tiny fork/join helper                                                   */
/* ------------------------------------------------------------------------ */
typedef void (*range_fn)(void *arg, int64_t lo, int64_t hi, int t);

typedef struct {
    range_fn fn;
    void *arg;
    int64_t lo, hi;
    int t;
} job;

static void *job_run(void *p) {
    job *j = (job *)p;
    j->fn(j->arg, j->lo, j->hi, j->t);
    return NULL;
}

#define MAX_THREADS 64

static void parallel_for(range_fn fn, void *arg, int64_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAX_THREADS) nthreads = MAX_THREADS;
    if (n < 65536) nthreads = 1;
    job jobs[MAX_THREADS];
    pthread_t th[MAX_THREADS];
    int started[MAX_THREADS];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].fn = fn;
        jobs[t].arg = arg;
        jobs[t].lo = n * t / nthreads;
        jobs[t].hi = n * (t + 1) / nthreads;
        jobs[t].t = t;
        started[t] = t > 0 && pthread_create(&th[t], NULL, job_run, &jobs[t]) == 0;
    }
    job_run(&jobs[0]);
    for (int t = 1; t < nthreads; t++) {
        if (started[t]) pthread_join(th[t], NULL);
        else job_run(&jobs[t]); /* no thread: run it here */
    }
}

/* ------------------------------------------------------------------------ */
/* R-MAT: each of `scale` levels picks a quadrant with probabilities a, b, c,  */
/* d = 1 - a - b - c (a: both bits 0, b: target bit 1, c: source bit 1,        */
/* d: both 1), from a 32-bit uniform; draw i uses counters 16 i .. 16 i + 15.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int scale;
    uint64_t ta, tab, tabc;
    int64_t start;
    const int64_t *perm;
    uint64_t *out;
    int keep_loops;
} rmat_arg;

static void rmat_range(void *p, int64_t lo, int64_t hi, int t) {
    (void)t;
    const rmat_arg *A = (const rmat_arg *)p;
    for (int64_t i = lo; i < hi; i++) {
        const uint64_t c0 = (uint64_t)(A->start + i) * 16u;
        uint64_t u = 0, v = 0;
        for (int l = 0; l < A->scale; l += 2) {
            const uint64_t w = draw(A->key, c0 + (uint64_t)(l >> 1));
            for (int h = 0; h < 2 && l + h < A->scale; h++) {
                const uint64_t r = (w >> (32 * h)) & 0xFFFFFFFFull;
                const uint64_t ub = r >= A->tab;
                const uint64_t vb = (r >= A->ta && r < A->tab) || r >= A->tabc;
                u = (u << 1) | ub;
                v = (v << 1) | vb;
            }
        }
        if (u == v && !A->keep_loops) {
            A->out[i] = NO_EDGE;
            continue;
        }
        if (A->perm) {
            u = (uint64_t)A->perm[u];
            v = (uint64_t)A->perm[v];
        }
        A->out[i] = (u << 32) | v;
    }
}

/* Draws start .. start + count - 1 of the R-MAT sampler as edge keys (ids
 * relabelled by perm when not NULL); a self-loop gives NO_EDGE unless
 * keep_loops. */
void gen_rmat(uint64_t key, int32_t scale, double a, double b, double c, int64_t start,
              int64_t count, const int64_t *perm, uint64_t *out, int32_t keep_loops,
              int32_t nthreads) {
    const double s = 4294967296.0;
    rmat_arg A;
    A.key = key;
    A.scale = scale;
    A.ta = (uint64_t)(a * s);
    A.tab = (uint64_t)((a + b) * s);
    A.tabc = (uint64_t)((a + b + c) * s);
    A.start = start;
    A.perm = perm;
    A.out = out;
    A.keep_loops = keep_loops;
    parallel_for(rmat_range, &A, count, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Chung-Lu: both endpoints drawn with probability proportional to a weight,  */
/* by inverse transform on the normalised cumulative weights; draw i uses     */
/* counters 2 i and 2 i + 1. The key is the unordered pair (min, max) of the  */
/* relabelled ids.                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    const double *cdf;
    int64_t n;
    int64_t start;
    const int64_t *perm;
    uint64_t *out;
    int keep_loops;
} cl_arg;

static int64_t upper_bound_d(const double *a, int64_t n, double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static void cl_range(void *p, int64_t lo, int64_t hi, int t) {
    (void)t;
    const cl_arg *A = (const cl_arg *)p;
    for (int64_t i = lo; i < hi; i++) {
        const uint64_t c0 = (uint64_t)(A->start + i) * 2u;
        const double r1 = (double)(draw(A->key, c0) >> 11) * (1.0 / 9007199254740992.0);
        const double r2 = (double)(draw(A->key, c0 + 1) >> 11) * (1.0 / 9007199254740992.0);
        int64_t u = upper_bound_d(A->cdf, A->n, r1);
        int64_t v = upper_bound_d(A->cdf, A->n, r2);
        if (u > A->n - 1) u = A->n - 1;
        if (v > A->n - 1) v = A->n - 1;
        uint64_t pu = (uint64_t)A->perm[u], pv = (uint64_t)A->perm[v];
        if (pu == pv && !A->keep_loops) {
            A->out[i] = NO_EDGE;
            continue;
        }
        if (!A->keep_loops && pu > pv) {
            uint64_t x = pu;
            pu = pv;
            pv = x;
        }
        A->out[i] = (pu << 32) | pv;
    }
}

/* Draws start .. start + count - 1 of the Chung-Lu sampler. Without
 * keep_loops the key is the canonical pair (min, max) and a self-loop gives
 * NO_EDGE; with keep_loops the key is (u, v) in draw order. */
void gen_chunglu(uint64_t key, const double *cdf, int64_t n, int64_t start, int64_t count,
                 const int64_t *perm, uint64_t *out, int32_t keep_loops, int32_t nthreads) {
    cl_arg A;
    A.key = key;
    A.cdf = cdf;
    A.n = n;
    A.start = start;
    A.perm = perm;
    A.out = out;
    A.keep_loops = keep_loops;
    parallel_for(cl_range, &A, count, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Sorting and de-duplication of keys                                         */
/* ------------------------------------------------------------------------ */
#define RADIX_BITS 11
#define RADIX (1 << RADIX_BITS)

typedef struct {
    const uint64_t *src;
    uint64_t *dst;
    int shift;
    int nthreads;
    int64_t *hist; /* [nthreads][RADIX]: counts, then start offsets */
} radix_arg;

static void radix_count(void *p, int64_t lo, int64_t hi, int t) {
    radix_arg *A = (radix_arg *)p;
    int64_t *h = A->hist + (int64_t)t * RADIX;
    memset(h, 0, sizeof(int64_t) * RADIX);
    for (int64_t i = lo; i < hi; i++) h[(A->src[i] >> A->shift) & (RADIX - 1)]++;
}

static void radix_scatter(void *p, int64_t lo, int64_t hi, int t) {
    radix_arg *A = (radix_arg *)p;
    int64_t *h = A->hist + (int64_t)t * RADIX;
    for (int64_t i = lo; i < hi; i++) {
        const uint64_t k = A->src[i];
        A->dst[h[(k >> A->shift) & (RADIX - 1)]++] = k;
    }
}

/* Ascending sort of keys[0 .. n) over their low `bits` bits (the others must
 * be zero), least significant digit first; returns 0, or -1 out of memory. */
static int radix_sort(uint64_t *keys, int64_t n, int bits, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAX_THREADS) nthreads = MAX_THREADS;
    if (n < 65536) nthreads = 1;
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * RADIX * (size_t)nthreads);
    if (!tmp || !hist) {
        free(tmp);
        free(hist);
        return -1;
    }
    uint64_t *a = keys, *b = tmp;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        radix_arg A = {a, b, shift, nthreads, hist};
        parallel_for(radix_count, &A, n, nthreads);
        int64_t run = 0;
        for (int d = 0; d < RADIX; d++)
            for (int t = 0; t < nthreads; t++) {
                const int64_t c = hist[(int64_t)t * RADIX + d];
                hist[(int64_t)t * RADIX + d] = run;
                run += c;
            }
        parallel_for(radix_scatter, &A, n, nthreads);
        uint64_t *x = a;
        a = b;
        b = x;
    }
    if (a != keys) memcpy(keys, a, sizeof(uint64_t) * (size_t)n);
    free(tmp);
    free(hist);
    return 0;
}

/* Drop NO_EDGE entries, sort ascending (keys below 2^bits) and remove
 * duplicates, in place. Returns the number of distinct keys, or -1 out of
 * memory. */
int64_t keys_sort_unique(uint64_t *keys, int64_t n, int32_t bits, int32_t nthreads) {
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (keys[i] != NO_EDGE) keys[k++] = keys[i];
    if (radix_sort(keys, k, bits, nthreads)) return -1;
    int64_t u = 0;
    for (int64_t i = 0; i < k; i++)
        if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
    return u;
}

/* (base minus del) union ins, all three ascending and duplicate-free, into out
 * (room for nb + ni); returns its length. Deletions apply to base only, so a
 * key in both del and ins ends up present. */
int64_t keys_apply(const uint64_t *base, int64_t nb, const uint64_t *ins, int64_t ni,
                   const uint64_t *del, int64_t nd, uint64_t *out) {
    int64_t i = 0, j = 0, d = 0, k = 0;
    while (i < nb || j < ni) {
        if (j >= ni || (i < nb && base[i] < ins[j])) {
            const uint64_t x = base[i++];
            while (d < nd && del[d] < x) d++;
            if (d < nd && del[d] == x) continue;
            out[k++] = x;
        } else if (i >= nb || ins[j] < base[i]) {
            out[k++] = ins[j++];
        } else {
            out[k++] = ins[j++];
            i++;
        }
    }
    return k;
}

/* Union of two ascending duplicate-free key arrays into out (room for
 * na + nb); returns its length. */
int64_t keys_merge_unique(const uint64_t *a, int64_t na, const uint64_t *b, int64_t nb,
                          uint64_t *out) {
    int64_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) out[k++] = a[i++];
        else if (b[j] < a[i]) out[k++] = b[j++];
        else {
            out[k++] = a[i++];
            j++;
        }
    }
    while (i < na) out[k++] = a[i++];
    while (j < nb) out[k++] = b[j++];
    return k;
}
