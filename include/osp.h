/*
 * osp.h - C ABI of the GB300 offset-score-propagation engine.
 *
 * The engine tracks Random Walk with Restart (RWR) scores on a graph that
 * changes by batches of edge and node insertions and deletions, following
 * OSP / OSP-T (Yoon, Jin, Kang, "Fast and Accurate Random Walk with Restart
 * on Dynamic Graphs with Guarantees", WWW 2018, arXiv 1712.00595).
 *
 * Problem statement (Sec. 1): given a time-evolving graph, a seed node s and a
 * restart probability c, keep the RWR vector r of Eq. 1,
 *     r = (1-c) A~^T r + c q,   q = e_s,
 * up to date after every change. A~ is the row-normalised adjacency matrix
 * (1/d_u at every out-neighbour of u; an all-zero row for a dead-end).
 *
 * Every call below runs its arithmetic in CUDA kernels on one GPU. All
 * pointers are plain host pointers unless the name ends in _device, in which
 * case they are device pointers on the context's device, read or written in
 * stream order on the context's stream. Input arrays are copied; the caller
 * keeps ownership of everything it passes in and of every output buffer.
 * Nothing here retains a caller pointer after the call returns.
 *
 * Errors: every call returns an osp_status. On OSP_EINVAL the context state is
 * unchanged (all checks run before any state is written). osp_last_error()
 * describes the last failure. One context must not be used from two threads
 * at once; different contexts are independent.
 */
#ifndef OSP_H
#define OSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osp_ctx osp_ctx; /* opaque; created by osp_create, owned by the library */

typedef enum {
    OSP_OK = 0,
    OSP_EINVAL = -1,   /* bad argument or invalid update batch; state unchanged */
    OSP_ENOMEM = -2,   /* device allocation failed, the HBM budget would be exceeded, or the
                          node or edge capacity reserved at load is exhausted */
    OSP_ECUDA = -3,    /* a CUDA runtime call failed */
    OSP_ETIMEOUT = -4, /* a bounded device wait (grid barrier) gave up */
    OSP_ENOCONV = -5,  /* iteration cap reached before ||x(i)||_1 <= eps; scores hold the
                          truncated sum */
    OSP_ESTATE = -6,   /* call out of order (e.g. apply before load/seed/init) */
    OSP_ENOTSUP = -7   /* valid request this build does not implement */
} osp_status;

/* Arithmetic of the propagation (Sec. 2.2 / Algorithm 1 loop). Running sums and
 * stored scores are always FP64: an FP32 sum with Kahan compensation costs the
 * same 8 bytes per entry and is less exact, so it is not offered.
 * FP64:        gather vector, products and every sum in double.
 * FP32_ACC64:  gather vector and products in float (in-row sums of the pull
 *              step in float); scores r, the offset vector, push-step
 *              accumulation and the ||x||_1 stopping test in double.
 * BF16_ACC64:  batches store the gather vector as bfloat16 (rounded to
 *              nearest), products and in-row sums in float, r / offset /
 *              stopping test in double; osp_init_scores runs as FP32_ACC64.
 *              Each stored value's rounding residual is carried into the
 *              rounding of the same entry at the next step (error feedback),
 *              so the stored values' rounding errors telescope instead of
 *              adding up over the steps. Two or more seeds only
 *              (osp_set_seeds returns OSP_ENOTSUP for one). */
typedef enum {
    OSP_PREC_FP64 = 0,
    OSP_PREC_FP32_ACC64 = 1,
    OSP_PREC_BF16_ACC64 = 2
} osp_precision;

/* One update. Operations of a batch apply in order (Sec. 3.4.1 for nodes).
 *  OSP_OP_INSERT_EDGE (u,v): add edge u->v; no-op if present.
 *  OSP_OP_DELETE_EDGE (u,v): remove edge u->v; no-op if absent.
 *  OSP_OP_ADD_NODE:          new node with the next id (n, n+1, ...), no edges,
 *                            score 0; u and v are ignored.
 *  OSP_OP_DELETE_NODE (u):   remove every out- and in-edge of u; the id stays
 *                            allocated and dead and may not be named again.
 *  OSP_OP_ZERO_ROW (u):      the literal form of the node deletion of Sec. 3.4.1:
 *                            only u's row of B~ becomes zero, i.e. every out-edge
 *                            of u is removed (u turns into a dead-end); its
 *                            in-edges stay, u stays live and later ops may name
 *                            it again (an edge u->v inserted after the op is
 *                            kept). Allowed on a seed. v is ignored.
 * A batch is invalid if an op names an id that does not exist at that point
 * of the batch or is dead, deletes a node twice, deletes a seed, or has an
 * unknown op code. */
enum {
    OSP_OP_INSERT_EDGE = 0,
    OSP_OP_DELETE_EDGE = 1,
    OSP_OP_ADD_NODE = 2,
    OSP_OP_DELETE_NODE = 3,
    OSP_OP_ZERO_ROW = 4
};
typedef struct {
    int32_t u;
    int32_t v;
    int32_t op;
} osp_update; /* 12 bytes, no padding */

typedef struct {
    int32_t precision;  /* osp_precision */
    int32_t device;     /* CUDA device ordinal */
    void *stream;       /* cudaStream_t the engine runs on; NULL = an engine-owned stream */
    int64_t max_nodes;  /* node capacity to reserve (0 = 1.25 x loaded n + 4096) */
    double push_alpha;  /* sparse (push) steps while frontier out-edges <= m / alpha (0 = 14) */
    double push_beta;   /* ... and frontier size <= n / beta (0 = 24) */
    int32_t max_iter;   /* iteration cap; 0 = ceil(log_{1-c}(eps/2)) + 8 (Theorem 3) */
    int32_t node_order; /* internal node order: 0 = the caller's ids, 1 = descending
                           out-degree of the loaded graph. Results are the same up to
                           rounding order; every call uses the caller's ids. */
    int32_t use_graphs; /* != 0: each apply call replays its kernel sequence from CUDA
                           graphs (one pair per batch-size bucket, eps and fixed step counts,
                           captured on first use and rebuilt when device buffers move),
                           which removes most host launch work per batch. */
    int32_t autotune;   /* != 0: osp_init_scores first times the pull-step schedule candidates
                           (task size 512/1024/2048 x long-list threshold, and node weight
                           2/4/8 with several seeds) on the first CPI steps and keeps the
                           fastest for every later call (osp_get_schedule reports it). */
    int32_t seed_gather; /* seed block (two or more seeds), how pull steps read source rows:
                            0 = by row size (2 for rows of at most 256 bytes, i.e. 32 K x the
                            element size, else 1), 1 = each lane loads its columns of up to eight
                            rows into registers, 2 = whole rows are copied into a shared-memory
                            ring by bulk asynchronous copies (cp.async.bulk, mbarrier). Results
                            are the same up to rounding order. */
    int32_t seed_group;  /* seed block: columns per column group of the pull steps (32, 64, 128
                            or 256, at most Sp; 0 = 32 for bf16 gather rows, else Sp, one
                            group). A pull step walks the graph
                            once per group that still has a running column, so groups whose
                            seeds have all stopped cost nothing; inside a group, a lane whose
                            columns have all stopped loads and stores nothing. With bf16 rows
                            in 32-column groups (and more than 32 seeds) each call also orders
                            the columns into groups by offset size, largest first, and once
                            only the first 8 (4) of that order run, steps read compact 8 (4)
                            column rows. Results are the same up to rounding order. */
    int32_t deterministic; /* != 0 (one seed; osp_set_seeds with two or more returns
                              OSP_ENOTSUP): every propagation step pulls (no push steps, so
                              each costs a pass over all edges), warps take their work in a
                              fixed order, long in-lists add their pieces in piece order, and
                              the batch offset q_offset is summed exactly in fixed point
                              (units of 2^-62, |error| <= 2^-63 per term). The same calls on
                              the same device and options then give the same bits in the
                              scores, the per-step norms and the statistics on every run.
                              autotune is ignored (a timed choice would change the bits). */
    int64_t l2_hot_bytes; /* seed block with node_order 1: bytes of L2 given to the gather rows
                             of the highest out-degree nodes (kept in L2 before other lines);
                             0 = 60% of the device's L2, < 0 = none. */
    int64_t hbm_budget_bytes; /* device memory the context may allocate (graph store, score
                                 blocks, query slots together); a call that would exceed it
                                 returns OSP_ENOMEM and allocates nothing more. 0 = no limit. */
} osp_options;

/* Per-call statistics (the columns of Table 2 plus bookkeeping). */
typedef struct {
    int32_t iterations;      /* propagation steps x(1)..x(k) run */
    int32_t push_iterations; /* of those, steps run over a sparse frontier */
    double qoff_l1;          /* ||x(0)||_1: ||q_offset||_1 (OSP) or c (CPI) */
    double last_x_l1;        /* ||x(k)||_1 at the stop */
    int64_t visited_edges;   /* edges read by the propagation steps */
    int64_t n_nodes;         /* node ids in use after the call (dead ones included) */
    int64_t m_edges;         /* live directed edges after the call */
    int64_t net_inserts;     /* edges the batch actually added */
    int64_t net_deletes;     /* edges the batch actually removed (node deletions and row
                                zeroings included); a batch above osp_max_batch() sums
                                both counts over its sub-batches */
    int64_t changed_rows;    /* rows u with B~[u] != A~[u] (candidates) */
    int64_t bad_op;          /* OSP_EINVAL from a batch: index of the first invalid op; else -1 */
    int64_t push_frontier;   /* sum over push steps of the frontier size |F(i-1)| */
    int64_t push_reached;    /* sum over push steps of the nodes reached |F(i)| */
    float ms_update;         /* device time of ingest + graph merge + offset (CUDA events) */
    float ms_propagate;      /* device time of the propagation kernel (CUDA events) */
    int32_t kernel_launches; /* kernels this call launched */
    int32_t reserved;
    int64_t pull_dst_nodes;  /* nodes with a nonempty in-list (destinations of a pull step) */
    int64_t pull_src_nodes;  /* nodes with a nonempty out-list (sources a pull step gathers) */
    double residual_bound;   /* bound on ||rho||_1, rho = c q - (I - (1-c) B~^T) r, of the scores
                                stored after the call (exact arithmetic; the max over seeds when
                                S > 1). Each call adds its untaken tail's residual x(k+1),
                                ||x(k+1)||_1 <= (1-c) ||x(k)||_1 (Algorithm 1 stopping rule,
                                Theorem 4); osp_init_scores restarts it. Then
                                ||r - r*||_1 <= residual_bound / c. */
} osp_batch_stats;

/* Fill *opt with defaults (FP32_ACC64, device 0, engine-owned stream). */
void osp_default_options(osp_options *opt);

/* Create a context on opt->device (opt may be NULL for defaults). */
osp_status osp_create(osp_ctx **out, const osp_options *opt);

/* Free every resource of the context. NULL is accepted. */
void osp_destroy(osp_ctx *ctx);

/* Load the initial graph G (Sec. 2.1): n nodes, m directed edges src[i]->dst[i]
 * (host arrays). Duplicate edges collapse; self-loops are kept; undirected != 0
 * stores both directions of each pair (Sec. 4.1). Replaces any previous graph
 * and invalidates scores. EINVAL for ids outside [0, n) or n >= 2^25. */
osp_status osp_load_graph(osp_ctx *ctx, int64_t n, int64_t m, const int32_t *src,
                          const int32_t *dst, int undirected);

/* Seed value selecting PageRank mode (osp_set_seeds with S = 1). */
#define OSP_PAGERANK (-1)

/* Set the seed node(s) and the restart probability c in (0, 1) (Eq. 1). Each of
 * the S seeds (1 <= S <= 256, distinct live ids, host array) gets its own RWR
 * vector r_j with q = e_{s_j}; seed_idx j of the query calls selects it.
 * S > 1 keeps the vectors as one n x Sp block (Sp = 32, 64, 128 or 256 columns,
 * the smallest that holds S) and runs every step as a sparse-matrix times
 * dense-block product; each column stops on its own test (Algorithm 1's loop
 * test per seed). Device memory for S > 1: about Sp (16 + 2 b_y) bytes per node
 * slot (b_y = 8 for FP64, 4 otherwise). A seed cannot be
 * deleted by a batch. Invalidates scores.
 * PageRank mode (the paper's commented seed = -1 variant of Algorithm 1):
 * S = 1 and seeds[0] = OSP_PAGERANK make q the uniform vector 1/n0 over the
 * n0 nodes present now; q then stays fixed (OSP assumes a fixed q), so nodes
 * added later have no restart mass and a deleted node keeps its c/n0. */
osp_status osp_set_seeds(osp_ctx *ctx, const int32_t *seeds, int32_t S, double c);

/* Compute scores from scratch by CPI (Sec. 2.2): x(0) = c e_s, stop after the
 * first x(i) with ||x(i)||_1 <= eps (per seed when S > 1). stats may be NULL;
 * with S > 1 its iteration count is the longest seed's and its norms are the
 * maxima over the seeds (osp_get_seed_stats gives each seed's). */
osp_status osp_init_scores(osp_ctx *ctx, double eps, osp_batch_stats *stats);

/* Apply one batch of U updates (host array, U <= 2^22, see osp_max_batch) and update
 * the scores by OSP / OSP-T (Algorithm 1):
 *   q_offset = (1-c)(B~^T - A~^T) r_old,  r_new = r_old + sum_i ((1-c)B~^T)^i q_offset,
 * stopping after the first term with ||x(i)||_1 <= eps. Exact OSP is a small
 * eps (Sec. 3.1 suggests 1e-9); OSP-T is a larger one (Sec. 3.2). The graph
 * update is applied in full even when the scores return ENOCONV. stats may be
 * NULL. Returns EINVAL (stats->bad_op set) for an invalid batch, with the
 * state unchanged when U <= osp_max_batch() (larger batches: see there).
 * Synchronises the context stream before returning. */
osp_status osp_apply_updates(osp_ctx *ctx, const osp_update *ops, int64_t U, double eps,
                             osp_batch_stats *stats);

/* As osp_apply_updates, with ops already in device memory. */
osp_status osp_apply_updates_device(osp_ctx *ctx, const osp_update *ops_device, int64_t U,
                                    double eps, osp_batch_stats *stats);

/* Largest U applied as one unit (16,384): an invalid op leaves the state
 * unchanged. Apply calls accept up to 2^22 ops; a larger batch is ingested
 * and merged in sub-batches of at most osp_max_batch() ops, all against the
 * same r_old (their offsets add up to the whole batch's offset), followed by
 * one propagation. Sub-batches are consecutive runs of the batch, except for
 * a host batch of edge insertions and deletions only, with every id below
 * the node count: its ops are then ordered by source node (ops of one node
 * keep their order; ops of different nodes commute) and each sub-batch takes
 * whole source nodes, so that a node's out-list changes, and its offset terms
 * are formed, once per call. If an op of a later sub-batch is invalid, the
 * sub-batches before it stay applied and propagated, the call returns
 * OSP_EINVAL and stats->bad_op gives the op's index in the caller's batch. */
int64_t osp_max_batch(void);

/* Copy the scores of seed seed_idx to out[0 .. n) (host). normalize != 0 returns
 * r / ||r||_1, the dead-end handled vector of Theorem 5 (Sec. 3.4.2); 0 returns
 * the stored, unnormalised r_temp (||r||_1 is summed in a fixed order, so the
 * same r always gives the same bits). A deleted node keeps its entry; its exact
 * RWR value is 0 and the stored value approaches it like any other entry. */
osp_status osp_query(osp_ctx *ctx, int32_t seed_idx, int normalize, double *out);

/* As osp_query, writing to a device buffer of n doubles. */
osp_status osp_query_device(osp_ctx *ctx, int32_t seed_idx, int normalize, double *out_device);

/* The k highest-scoring nodes of seed seed_idx, ordered by score descending and
 * then id ascending (host outputs of k entries; fewer if n < k, count in *k_out).
 * 1 <= k <= 4096. normalize != 0 divides the returned scores by ||r||_1
 * (Theorem 5); the ranking is the same either way. */
osp_status osp_topk(osp_ctx *ctx, int32_t seed_idx, int32_t k, int normalize, int32_t *ids,
                    double *scores, int32_t *k_out);

/* Largest n accepted by osp_topk_noalloc (the engine's node-id limit, 2^25 - 1). */
#define OSP_TOPK_NOALLOC_MAX_N 33554431

/* Top-k of a score vector that is already on the device, for callers that
 * cannot allocate device memory when they query: a process whose device memory
 * all belongs to its own pool allocator, or a latency-bound loop that cannot
 * take the device-wide synchronisation cudaMalloc/cudaFree may cause. The paper
 * has no counterpart; it ranks the vector exactly like osp_topk ranks a
 * context's scores (score descending, then index ascending).
 *
 * Arguments, all device pointers on the CURRENT device: scores_device holds n
 * doubles (read only), ids_device receives k int32 indices, out_scores_device
 * k doubles and k_out_device one int32, the number written (min(k, n)).
 * normalize != 0 divides the returned scores by the vector's L1 norm, which
 * leaves the ranking unchanged. The caller owns every
 * buffer. The call is asynchronous on `stream` (a cudaStream_t; NULL is the
 * default stream): results are ready when the stream reaches that point.
 *
 * Memory: the call allocates nothing. Its scratch is one fixed array of about
 * 180 KB in the library's own device memory, one per device. The first call on
 * each device is the set-up: with that device current it looks the array up
 * (under CUDA's default lazy module loading this loads the library module that
 * holds it, which takes device memory once) and sets the sort kernel's
 * shared-memory limit; make that first call before any stream capture begins.
 * The set-up is kept for the life of the process: a cudaDeviceReset between
 * calls is not supported (the array's address and the limit would be stale). Calls that could run at the same time on the GPU (different
 * streams, different host threads) share the array and race; order them.
 *
 * Errors: OSP_EINVAL when n < 0, n > OSP_TOPK_NOALLOC_MAX_N, k is outside
 * [1, 4096], a needed pointer is NULL, or the current device ordinal is above
 * 63 (nothing is launched then); OSP_ECUDA when a CUDA call or launch fails. */
osp_status osp_topk_noalloc(const double *scores_device, int64_t n, int32_t k, int normalize,
                            int32_t *ids_device, double *out_scores_device,
                            int32_t *k_out_device, void *stream);

/* Query slots for serving: queries that overlap on the device with the next
 * update batch. Allocates nslots (0 <= nslots <= 64; 0 frees them) slots, each
 * with its own top-k scratch and an n-double column buffer (about 8 bytes per
 * node slot plus 130 KB of device memory, so the HBM budget for queries sets
 * nslots; plus 48 KB of host-mapped pinned memory for the result), and a
 * second CUDA stream for them. A query enqueued with osp_topk_async reads the
 * scores as of the last completed init/apply call; the ingest, merge and
 * offset kernels of the next apply run alongside it, and that call's
 * propagation kernel (the only kernel that changes the scores) waits for
 * every query enqueued before it. */
osp_status osp_query_slots(osp_ctx *ctx, int32_t nslots);

/* Enqueue the top-k of seed seed_idx (as osp_topk) in a free slot and return
 * without waiting. OSP_ESTATE if the slot still holds a query. */
osp_status osp_topk_async(osp_ctx *ctx, int32_t slot, int32_t seed_idx, int32_t k, int normalize);

/* Enqueue the top-k of m seeds (1 <= m <= 32; seed seed_idx[i] in slot
 * slots[i], slots distinct and free) as one launch sequence on the query
 * stream and return without waiting; collect each slot with osp_topk_wait.
 * Same results as m calls of osp_topk_async. OSP_EINVAL on a bad slot, seed,
 * k or count, OSP_ESTATE if a slot still holds a query; nothing is enqueued
 * then. */
osp_status osp_topk_async_many(osp_ctx *ctx, const int32_t *slots, const int32_t *seed_idx,
                               int32_t m, int32_t k, int normalize);

/* Wait for the slot's query and copy its result (host arrays of k entries,
 * count in *k_out); the slot is free again afterwards. The kernels write the
 * result to host-mapped memory of the slot, so this is a wait and a host
 * copy. */
osp_status osp_topk_wait(osp_ctx *ctx, int32_t slot, int32_t *ids, double *scores, int32_t *k_out);

/* Copy the current graph as sorted adjacency (host arrays): direction 0 gives
 * out-edges (CSR of A~'s pattern), 1 gives in-edges (CSC). ptr has n+1 entries,
 * idx has m; each list ascending. */
osp_status osp_export_graph(osp_ctx *ctx, int direction, int64_t *ptr, int32_t *idx);

/* Current node count (ids in use, dead ones included) and live edge count. */
osp_status osp_get_size(osp_ctx *ctx, int64_t *n, int64_t *m);

/* Current node count (ids in use, dead ones included); -1 for a NULL context. */
int64_t osp_num_nodes(const osp_ctx *ctx);

/* Per seed, the residual bound of osp_batch_stats.residual_bound (host array of up to
 * cap entries, count in *count = min(S, cap)): ||rho_j||_1 of seed j's stored scores
 * is at most out[j] in exact arithmetic, so ||r_j - r_j*||_1 <= out[j] / c. */
osp_status osp_get_residual_bounds(osp_ctx *ctx, double *out, int32_t cap, int32_t *count);

/* Device memory the context holds now (bytes of its own allocations). */
int64_t osp_device_bytes(const osp_ctx *ctx);

/* Per seed of the last init/apply call (host arrays of up to cap entries, any of
 * them NULL to skip): the steps the seed ran, ||x(0)||_1 (its ||q_offset||_1)
 * and ||x(k)||_1 at its stop. *count = min(S, cap). */
osp_status osp_get_seed_stats(osp_ctx *ctx, int32_t *iterations, double *qoff_l1,
                              double *last_l1, int32_t cap, int32_t *count);

/* The pull-step schedule in force (host array of 4): items per warp task,
 * in-list length above which lists are summed in pieces, the piece length, and
 * the items a node counts for in task planning. */
osp_status osp_get_schedule(osp_ctx *ctx, int32_t *out);

/* Fix each seed's number of propagation steps for the following init/apply
 * calls (k[j] > 0: seed j runs exactly k[j] steps; 0: its eps rule), to
 * compare precisions step for step; k = NULL clears. S must equal the number of
 * seeds. osp_set_fixed_iterations, when nonzero, takes precedence. */
osp_status osp_set_seed_iterations(osp_ctx *ctx, const int32_t *k, int32_t S);

/* ||x(0)||_1 .. ||x(k)||_1 of the last init/apply call (host, up to cap entries;
 * with several seeds each entry is the maximum over the seeds that ran the step). */
osp_status osp_get_l1_history(osp_ctx *ctx, double *out, int32_t cap, int32_t *count);

/* Device time in microseconds of the parts of the last init/apply propagation
 * (device clock): entry 0 is the x(0) pass, entry i the step computing x(i).
 * Up to cap entries; the count in *count. */
osp_status osp_get_step_times(osp_ctx *ctx, double *us, int32_t cap, int32_t *count);

/* Run the next propagations for exactly k steps regardless of eps (k > 0), or
 * go back to the eps rule (k = 0). Used to compare precisions step for step. */
osp_status osp_set_fixed_iterations(osp_ctx *ctx, int32_t k);

/* Description of the last error on this context ("" if none). Valid until the
 * next call on the context. */
const char *osp_last_error(const osp_ctx *ctx);

/* Static name of a status code. */
const char *osp_status_string(osp_status s);

/* Failure-detection self-test on `device` (no context needed). Every wait of
 * the engine's persistent kernels is bounded (2 s of device time); this runs
 * one of those waits on scratch memory of its own:
 *   which 0: the grid barrier, 4 CTAs;
 *   which 1: the mbarrier of a staged-row batch (two 128-byte rows announced).
 * lose = 0: every CTA arrives / both rows land; returns OSP_OK.
 * lose = 1: one CTA never arrives / the second row is never copied; the wait
 * runs out, the kernel returns and OSP_ETIMEOUT is returned (about 2 s for
 * the barrier, 4 s for the mbarrier, which waits once more for its copies).
 * The device stays usable. OSP_EINVAL for a bad which; OSP_ECUDA on a CUDA
 * error. */
osp_status osp_selftest_wait(int32_t device, int32_t which, int32_t lose);

#ifdef __cplusplus
}
#endif
#endif /* OSP_H */
