/*
 * maxflow.h -- C ABI of the GB300 dynamic max-flow library.
 *
 * The library computes the maximum s-t flow of a directed graph with int32
 * capacities and keeps it up to date under batches of capacity updates,
 * following "Scalable Maxflow Processing for Dynamic Graphs" (Kannappan,
 * Kumar, Nasre):
 *   - the problem statement: Sec. 2.1 (flow network, capacity and
 *     conservation constraints) and Sec. 4.1 (a batch is a set of edges with
 *     new capacities, higher or lower than before);
 *   - the residual graph: the Bi-CSR of Sec. 5.1 (every pair (u,v) with an
 *     edge in either direction has a slot at u and a slot at v, plus the
 *     index of the reverse slot);
 *   - the static solve: Alg. 1 (initialisation, source saturation, loop of
 *     backward BFS Alg. 4, push-relabel Alg. 2, remove-invalid-edges Alg. 3);
 *   - the incremental re-solve: Alg. 5 (apply the batch, send back flow that
 *     no longer fits, recompute excess, saturate the source edges again, loop
 *     of backward BFS Alg. 6 rooted at t and every deficient vertex,
 *     Alg. 2, Alg. 3) and its value formula;
 *   - the certificate: the cut A = {h = n}, B = {h < n} (Sec. 3.1 Theorem 3.4
 *     and the note after Theorem 3.6; Sec. 4.3).
 *
 * Every entry point returns an int status (MAXFLOW_OK = 0 or an error code
 * below); maxflow_strerror() names it.  No entry point throws, aborts or
 * faults the GPU on bad input: arguments are checked first and an error is
 * returned with the state unchanged.
 *
 * Memory: the library copies every input it is given and owns its device
 * state; output buffers belong to the caller.  Device memory comes from the
 * allocator callbacks in maxflow_opts (e.g. PyTorch's caching allocator) or,
 * when those are NULL, from cudaMalloc.  All GPU work of a context is issued
 * on the context's stream.  Host pointers may be pageable or pinned; pinned
 * memory makes the copies asynchronous with the host.
 *
 * Threads: a context must not be used from two host threads at once.
 * Different contexts are independent.
 */
#ifndef MAXFLOW_GB300_H
#define MAXFLOW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MAXFLOW_OK                0
#define MAXFLOW_ERR_INVALID       1  /* bad argument: s == t, id out of range, negative capacity, n < 2, NULL */
#define MAXFLOW_ERR_OOM           2  /* device or host allocation failed */
#define MAXFLOW_ERR_CUDA          3  /* a CUDA runtime call failed (no usable GPU, launch error, ...) */
#define MAXFLOW_ERR_NOT_CONVERGED 4  /* the iteration or time cap was hit; the state stays a valid preflow */
#define MAXFLOW_ERR_STATE         5  /* call out of order (e.g. query before a solve) */
#define MAXFLOW_ERR_INTERNAL      6  /* a self-check failed (certificate, device wait gave up) */
#define MAXFLOW_ERR_TOO_LARGE     7  /* more slots than int32 indexing allows, or a capacity sum overflows int32 */

typedef struct maxflow_ctx maxflow_ctx;   /* opaque, library-owned */

/* A graph as host COO arrays (caller-owned; copied by maxflow_init).
 * Self-loops are dropped and parallel edges are summed (their total must fit
 * in int32).  Capacities must be >= 0. */
typedef struct {
    int32_t n;              /* vertices 0 .. n-1, n >= 2 */
    int64_t m;              /* number of COO entries */
    const int32_t *src;
    const int32_t *dst;
    const int32_t *cap;
} maxflow_graph;

/* A batch of capacity updates (Sec. 4.1): each (u, v, new_cap) SETS
 * cap(u, v) = new_cap.  new_cap = 0 deletes the edge (its slots remain, with
 * capacity 0).  If no slot exists for the pair {u, v} the update inserts one
 * (into the per-vertex slack; a full row triggers a rebuild inside the call).
 * Within one batch the last update of a directed pair wins; u == v is
 * ignored.  The batch is validated whole before any state changes. */
typedef struct {
    int64_t count;
    const int32_t *u;
    const int32_t *v;
    const int32_t *new_cap;
    int32_t on_device;      /* 0: host arrays; 1: device arrays on the context's GPU */
} maxflow_batch;

typedef void *(*maxflow_alloc_fn)(size_t bytes, void *user, void *stream);
typedef void (*maxflow_free_fn)(void *ptr, size_t bytes, void *user, void *stream);

typedef struct {
    int32_t kernel_cycles;      /* push/relabel cycles per vertex per discharge (Alg. 2's KERNEL_CYCLES);
                                   0 = max(1, ceil(m / n)), the paper's average-degree heuristic (Sec. 6.1) */
    int32_t data_driven;        /* 1: worklist of active vertices (Sec. 5.2.1 O1); 0: topology-driven */
    int32_t fix_steep;          /* 1: run remove-invalid-edges (Alg. 3) after each iteration's discharge;
                                   0 (the default): skip it -- every iteration starts with an exact global
                                   relabel, which restores h(u) <= h(v) + 1 on every residual edge, and
                                   Alg. 3's whole-residual pushes create deficits that cost iterations */
    int32_t grid_blocks;        /* cooperative grid size; 0 = sized from the graph and the GPU */
    int64_t max_iters;          /* outer-iteration cap per solve; 0 = 4n + 1000 */
    double  time_limit_s;       /* device wall-clock cap per solve; 0 = 120 s */
    double  wait_limit_s;       /* cap on any single device-side wait (grid barrier); 0 = 1 s */
    float   slack_factor;       /* spare slots per vertex for insertions: max(slack_min, ceil(deg * factor)),
                                   rounded up so that every row's size is a multiple of 4 slots */
    int32_t slack_min;
    int32_t device;             /* CUDA device ordinal; -1 = the current device */
    void   *stream;             /* cudaStream_t for all work of the context; NULL = legacy default stream */
    maxflow_alloc_fn alloc;     /* optional device allocator (NULL: cudaMalloc) */
    maxflow_free_fn  free;
    void   *alloc_user;
} maxflow_opts;

typedef struct {
    int64_t n, m_edges;             /* vertices; directed edges with a slot (merged, incl. zero capacity) */
    int64_t slots, slot_capacity;   /* used and reserved Bi-CSR slots */
    int32_t kernel_cycles, grid_blocks, block_threads, blocks_per_sm;
    int64_t solves, updates, rebuilds;
    /* last solve (static, incremental or extraction run) */
    int64_t iterations, bfs_levels, pushes, relabels, steep_fixes;
    int64_t active_first, active_total;     /* active vertices in the first / all iterations */
    int64_t bytes_bfs, bytes_discharge, bytes_fix, bytes_worklist, bytes_apply;  /* algorithmic bytes, per solve */
    double  ms_last;                /* device time of the last solve kernel (CUDA events) */
    double  ms_bfs, ms_discharge, ms_fix, ms_worklist, ms_apply;  /* device wall time per phase (globaltimer) */
    int64_t value;                  /* value of the last solve */
    double  ms_kernel;              /* device clock from kernel entry to its last grid barrier */
    int64_t barriers;               /* grid barriers the last solve kernel passed */
    int64_t discharge_rounds;       /* discharge rounds the last solve ran (all iterations) */
    int32_t rounds;                 /* current setting of maxflow_set_rounds (0: adaptive) */
    int32_t reserved0;
    double  ms_update;              /* device time of every launch of the last update or solve call */
    /* where the last solve's discharge rounds spent their time, summed over all
       warps (microseconds): on rows above warp_max_slots (CTAs and 4-warp groups),
       on rows up to it (one warp each), on the thread-per-vertex rows */
    double  us_discharge_cta_rows;
    double  us_discharge_warp_rows;
    double  us_discharge_thread_rows;
} maxflow_stats_t;

/* Fill o with the defaults documented above. */
void maxflow_default_opts(maxflow_opts *o);

/* Build the residual Bi-CSR of g (Sec. 5.1) on the GPU and run the static
 * solve (Alg. 1 with Alg. 4/6 heights, Alg. 2, Alg. 3).  s != t, both in
 * [0, n).  opt may be NULL (defaults).  On success *out is a new context;
 * on error *out is NULL.  MAXFLOW_ERR_TOO_LARGE when the merged capacities
 * of a pair, c(u,v) + c(v,u), exceed INT32_MAX (residual capacities are
 * int32 and c_f(u,v) + c_f(v,u) stays equal to that sum). */
int maxflow_init(maxflow_ctx **out, const maxflow_graph *g, int32_t s, int32_t t, const maxflow_opts *opt);

/* Apply a batch and re-solve incrementally (Alg. 5 and Alg. 6): apply the
 * capacity changes to the residual capacities, send back flow that exceeds
 * a new capacity, update the excess, saturate the source edges, then resume
 * push-relabel from the current heights and excesses.  Returns when the
 * re-solve is done (the value is then available to maxflow_query).
 * Errors: MAXFLOW_ERR_INVALID for an endpoint out of [0, n) or a negative
 * capacity; MAXFLOW_ERR_TOO_LARGE when the batch would leave a pair with
 * c(u,v) + c(v,u) > INT32_MAX (the final capacity of both directions counts,
 * including the batch's own update of the reverse direction), the limit
 * maxflow_init also enforces.  Both are detected on the whole batch before
 * any capacity, slot or excess changes: a refused batch leaves the state as
 * it was. */
int maxflow_update(maxflow_ctx *c, const maxflow_batch *b);

/* The current maximum-flow value (value formula of Alg. 5: the sum of e(v)
 * over v != s with h(v) < n, which equals e(t) plus the deficits).
 * side (NULL or n host bytes): 1 for the source side A = {h = n} of the
 * minimum cut (Sec. 3.1 note), 0 otherwise.  cut_cap (NULL ok): total capacity
 * of edges from A to V \ A, equal to the value.  Synchronises the stream. */
int maxflow_query(maxflow_ctx *c, int64_t *value, uint8_t *side, int64_t *cut_cap);

/* The comparator of Sec. 6.2: re-solve the current graph from zero flow
 * (Alg. 1) instead of incrementally. */
int maxflow_resolve_static(maxflow_ctx *c);

/* A feasible maximum flow (Sec. 3.1 Theorem 3.3, Lemma 3.5, Sec. 4.3 Claim):
 * the excess left in A is returned to s and the deficits in B are filled
 * from t, on a copy of the state (the solver state is not changed).
 * On input *count is the capacity of the output arrays; on output it is the
 * number of directed edges with capacity > 0.  If the capacity is too small
 * (or the arrays are NULL) nothing is written and MAXFLOW_OK is returned with
 * the needed count.  Outputs are host arrays: edge (u[i], v[i]) with
 * capacity cap[i] carries flow[i], 0 <= flow[i] <= cap[i]. */
int maxflow_get_flow(maxflow_ctx *c, int64_t *count, int32_t *u, int32_t *v, int32_t *cap, int32_t *flow);

/* Set KERNEL_CYCLES (Alg. 2) for the following solves: k >= 1, or 0 for the
 * average-degree heuristic of Sec. 6.1.  The global-relabel frequency of the
 * paper follows from it (Sec. 6.1: too low means many BFS, too high sends flow
 * the wrong way). */
int maxflow_set_kernel_cycles(maxflow_ctx *c, int32_t k);

/* Discharge rounds per global relabel.  1 is the paper's data-driven kernel
 * (Sec. 5.2.1 O1): the vertices active right after the backward BFS get
 * KERNEL_CYCLES cycles each.  With r > 1, vertices that become active while a
 * round runs (they receive flow) are discharged in the next round, up to r
 * rounds, before the next BFS -- as in the paper's kernel, where every vertex
 * checks e(u) > 0 on each of its cycles.  0 (the default) is adaptive, not in
 * the paper: at least 2 rounds, then more while the discharge of the current
 * iteration has taken less than half the time of its BFS, at most 1024, so
 * that a global relabel that costs much (a deep BFS, as on grids) is spread
 * over more discharge work.  MAXFLOW_ERR_INVALID below 0. */
int maxflow_set_rounds(maxflow_ctx *c, int32_t rounds);

/* With on = 1 (the default), a vertex that still has excess and a height
 * below n after its KERNEL_CYCLES cycles in a discharge round is discharged
 * again in the next round of the same iteration (when one follows), instead of
 * waiting for the next global relabel; on = 0 keeps only the vertices that
 * became active during the round.  Not in the paper (it steers work only: the
 * value and the certificate do not depend on it).  MAXFLOW_ERR_INVALID unless
 * on is 0 or 1. */
int maxflow_set_requeue(maxflow_ctx *c, int32_t on);

/* Cycles by row length: with div > 0, a vertex whose row has d slots gets
 * max(KERNEL_CYCLES, d / div) cycles per discharge call, so a long row (whose
 * first scan costs most of its discharge) makes more pushes per scan; 0 (the
 * default) gives every vertex KERNEL_CYCLES.  Not in the paper (it steers
 * work only).  MAXFLOW_ERR_INVALID below 0. */
int maxflow_set_cycle_div(maxflow_ctx *c, int32_t div);

/* Small BFS levels on one CTA: a top-down level whose frontier holds at most
 * `slots` slots (and at most as many vertices) runs in the first CTA alone,
 * level after level, without a grid barrier between levels (the labels are
 * those of Alg. 4 / Alg. 6 either way); the grid meets again when a frontier
 * grows past the limit, the BFS ends, or after 256 such levels.  0 (the
 * default) turns it off: measured on R-MAT, grids and the batched instances it
 * did not pay (a level of a few hundred slots costs about as much in one CTA as
 * the grid's barrier does).  Not in the paper.  MAXFLOW_ERR_INVALID below 0. */
int maxflow_set_bfs_tail(maxflow_ctx *c, int32_t slots);

/* Run remove-invalid-edges (Alg. 3) after each iteration's discharge rounds
 * (on = 1) or not (on = 0) from the next solve on; the same switch as
 * maxflow_opts.fix_steep.  MAXFLOW_ERR_INVALID unless on is 0 or 1. */
int maxflow_set_fix_steep(maxflow_ctx *c, int32_t on);

/* ---- learned schedule (an addition to the paper's fixed KERNEL_CYCLES) ----
 *
 * A schedule (action) is a mode -- 0: incremental re-solve (Alg. 5), 1: apply
 * the batch then re-solve from zero flow (Alg. 1) -- with a number of
 * discharge rounds (0: adaptive), of KERNEL_CYCLES (0: the average-degree
 * heuristic of Sec. 6.1), a row-length divisor for the cycles
 * (maxflow_set_cycle_div) and whether remove-invalid-edges (Alg. 3) runs.
 * Action 0 is the library's default schedule, action 5 the paper's fixed
 * one.  The action table is fixed; maxflow_sched_actions returns it (host
 * arrays of cap entries; pass all NULL to get only the count).  A schedule
 * never changes the result, only the work. */
int maxflow_sched_actions(int32_t *mode, int32_t *rounds, int32_t *cycles, int32_t *cycle_div, int32_t *fix,
                          int32_t cap, int32_t *count);

/* The 16 scheduler features of a batch for this context (host array of 16
 * floats): batch size and fraction of the graph, graph size and degree, the
 * fractions of updates touching s, touching t and deleting, the mean new
 * capacity over the graph's mean, the last incremental solve's iterations,
 * time, first active count and BFS levels (the initial solve's until the first
 * update; a static re-solve leaves them), the initial static solve's
 * iterations and time, and a constant 1.  Reads the batch only (no change to
 * the state).  Sec. 6.1
 * ties the choice of KERNEL_CYCLES to the graph, which these features describe.
 * MAXFLOW_ERR_INVALID for NULL c or out, MAXFLOW_ERR_STATE while evicted,
 * MAXFLOW_ERR_CUDA. */
int maxflow_features(maxflow_ctx *c, const maxflow_batch *b, float *out);

/* Apply the batch and re-solve with the given action (index into the table):
 * maxflow_update (Alg. 5) with that action's rounds and KERNEL_CYCLES, or the
 * batch then a static re-solve (Alg. 1).  Errors as maxflow_update, plus
 * MAXFLOW_ERR_INVALID for an action outside the table. */
int maxflow_run_action(maxflow_ctx *c, const maxflow_batch *b, int32_t action);

/* A fully connected network x (n_in) -> ReLU(H) -> ReLU(H) -> y (n_out) in
 * fp32 on the device, trained with Adam on masked squared error; used to
 * predict the log device time of each action from the features.  No
 * counterpart in the paper.  The network owns its device memory (destroy
 * releases it; NULL is a no-op); every array argument below is a host array
 * owned by the caller, row-major.  create: MAXFLOW_ERR_INVALID for NULL out or
 * sizes outside 1..64 inputs, 1..256 hidden units, 1..64 outputs; every other
 * call: MAXFLOW_ERR_INVALID for NULL pointers, rows < 1 or a parameter count
 * other than the network's; MAXFLOW_ERR_CUDA / MAXFLOW_ERR_OOM from the
 * device. */
typedef struct maxflow_mlp maxflow_mlp;
int maxflow_mlp_create(maxflow_mlp **out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream);
void maxflow_mlp_destroy(maxflow_mlp *m);
int maxflow_mlp_shape(maxflow_mlp *m, int32_t *n_in, int32_t *n_hidden, int32_t *n_out, int64_t *n_params);
/* Flat parameters [W1 (H x n_in) | b1 | W2 (H x H) | b2 | W3 (n_out x H) | b3], host arrays. */
int maxflow_mlp_get_params(maxflow_mlp *m, float *host, int64_t count);
int maxflow_mlp_set_params(maxflow_mlp *m, const float *host, int64_t count);
/* y (rows x n_out) from x (rows x n_in); host arrays. */
int maxflow_mlp_forward(maxflow_mlp *m, const float *x, int32_t rows, float *y);
/* Gradient of L = sum(mask * (y - target)^2) / sum(mask) with respect to the
 * flat parameters, and L; host arrays (grad has n_params entries). */
int maxflow_mlp_grad(maxflow_mlp *m, const float *x, const float *target, const float *mask, int32_t rows,
                     float *grad, float *loss);
/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8) at learning rate lr. */
int maxflow_mlp_train(maxflow_mlp *m, const float *x, const float *target, const float *mask, int32_t rows,
                      int32_t steps, float lr, float *loss_last);

/* Compute the batch's features, let the network predict each action's log
 * time, and run the action with the smallest prediction (written to
 * *action_out, may be NULL).  The network must have 16 inputs and one output
 * per action (else MAXFLOW_ERR_INVALID).  Every action gives the same maximum
 * flow; errors as maxflow_run_action. */
int maxflow_update_scheduled(maxflow_ctx *c, const maxflow_batch *b, maxflow_mlp *m, int32_t *action_out);

/* Work split thresholds (by used slots of a vertex's row): the discharge gives
 * rows of at most thread_max_slots one thread, rows of at most warp_max_slots
 * one warp, longer rows a 4-warp group up to a quarter of the CTA's snapshot
 * buffer (about 7.2 K slots) and the longest a whole CTA (remove-invalid-edges:
 * a warp up to warp_max_slots, then a CTA); the BFS splits rows longer than
 * bfs_item_min_slots into 256-slot work items.  All three 0: the defaults,
 * thread_max_slots 8, or 4 on a graph of at most 8 merged directed edges per
 * vertex (grids, geometric and layered graphs: many short discharge rounds,
 * where a warp's parallel scan of a short row beats one thread's), then 512
 * and 256.  Not in the paper (it steers work only).  MAXFLOW_ERR_INVALID for
 * NULL c, a zero or negative threshold (unless all three are 0) or
 * warp_max_slots < thread_max_slots. */
int maxflow_set_tuning(maxflow_ctx *c, int32_t thread_max_slots, int32_t warp_max_slots, int32_t bfs_item_min_slots);

/* Test of the bounded waits (no counterpart in the paper): one BFS-only launch
 * in which CTA `cta` (0 <= cta < the context's grid) never arrives at its
 * first grid barrier.  The other CTAs give up after maxflow_opts.wait_limit_s,
 * record the wait error and leave the kernel, so the call returns
 * MAXFLOW_ERR_INTERNAL instead of hanging; the barrier words are reset and the
 * context stays usable (heights may be stale until the next solve).
 * MAXFLOW_ERR_INVALID for cta out of range. */
int maxflow_test_stalled_barrier(maxflow_ctx *c, int32_t cta);

/* Direction of the global-relabel BFS levels (direction-optimising BFS, not
 * in the paper, which sweeps top-down).  A level runs bottom-up -- each
 * unlabelled vertex looks through its own row for a neighbour of the current
 * level with residual towards it, stopping at the first -- once the frontier's
 * slots exceed 1/alpha of the still unexplored slots, and top-down again once
 * the frontier holds fewer than n/beta vertices.  The labels are the same
 * either way.  alpha = 0 keeps every level top-down.  Defaults 14 and 24.
 * MAXFLOW_ERR_INVALID for alpha < 0 or beta < 1. */
int maxflow_set_bfs_switch(maxflow_ctx *c, int32_t alpha, int32_t beta);

/* Solve many instances in ONE persistent cooperative launch (on the first
 * context's device and stream): the grid is cut into groups of group_blocks
 * CTAs, and each group takes the next instance (largest first) and runs its
 * whole solve.  batches == NULL: a static re-solve of every instance (Alg. 1);
 * otherwise batches[i] is applied to ctxs[i] and the flow repaired
 * incrementally (Alg. 5).  Instances whose insertions overflow their rows are
 * grown and re-run alone.  *ms_out (may be NULL): device time of the launch.
 * Returns the first error of any instance; every instance's value is then
 * available through maxflow_query. */
int maxflow_solve_batched(maxflow_ctx *const *ctxs, int32_t count, const maxflow_batch *batches, int32_t group_blocks,
                          double *ms_out);

/* Make `stream` (a cudaStream_t on the context's device; NULL = the legacy
 * default stream) the stream of every later call on this context.  Every
 * call of this library returns with its own device work finished, so the
 * switch waits for nothing (in particular not for other work queued on the
 * old stream); after a call that failed, synchronise the old stream first.
 * maxflow_solve_batched issues on the stream of its first context.  No
 * counterpart in the paper. */
int maxflow_set_stream(maxflow_ctx *c, void *stream);

/* Grow the batch scratch (dedup hash tables, staging) to hold batches of up to
 * `count` updates now rather than inside the next update, so that
 * maxflow_device_bytes accounts for it beforehand.  It never shrinks.
 * MAXFLOW_ERR_TOO_LARGE past 2^29 updates.  No counterpart in the paper. */
int maxflow_reserve_batch(maxflow_ctx *c, int64_t count);

/* ---- Sec. 5.2.2 (O2): push and pull ----------------------------------------
 * maxflow_resolve_static_pp: the static push-pull.  Re-solve from scratch with
 * the edges out of s and the edges into t both saturated; the deficient
 * vertices this leaves act as sinks of the push-relabel loop.  The value is the
 * max flow and the final heights give the min cut, as for
 * maxflow_resolve_static.
 *
 * maxflow_resolve_static_pull: the pull-relabel of the same section on its own.
 * Only the edges into t are saturated; every deficient vertex pulls from its
 * lowest residual in-neighbour, with heights measured from s (and from any
 * overflowing vertex) along residual edges; the value is the flow that leaves
 * s.  A push-height BFS follows so that the cut, queries and later updates
 * see the same labels as after a push solve.
 *
 * maxflow_update_pp: the dynamic push-pull ("dyn-pp-str").  Needs a solved
 * context (otherwise it runs maxflow_update).  Three steps:
 *   1 apply the batch (as maxflow_update), take the sides of the last min cut
 *     from the heights the previous solve ended with (side 1: the vertex
 *     reached t or a deficit), and send the whole residual of every edge from
 *     side 0 to side 1, so that no residual path leads from side 0 to side 1;
 *   2 one launch whose grid is split in two groups of CTAs: push-relabel on
 *     side 1 (roots t and the deficient vertices of side 1) and pull-relabel
 *     on side 0 (roots s and the overflowing vertices of side 0).  The two
 *     parts touch disjoint vertices and edges (the paper runs them on two
 *     streams);
 *   3 a push solve over the whole graph for what is left (an overflowing
 *     vertex of side 1 that reaches a deficient vertex of side 0).
 * stop_after in {1, 2} returns after that step (for inspection; the context
 * is then unsolved until the next update); 0 or 3 runs all.  The value equals
 * maxflow_update's.  maxflow_stats reports the last launch; ms_update the
 * three launches together.  No counterpart in the ABI of the paper. */
int maxflow_resolve_static_pp(maxflow_ctx *c);
int maxflow_resolve_static_pull(maxflow_ctx *c);
int maxflow_update_pp(maxflow_ctx *c, const maxflow_batch *b, int32_t stop_after);

/* Device memory the context holds, in bytes (graph, vertex state, scratch).
 * No counterpart in the paper; serving uses it to admit contexts by memory. */
int maxflow_device_bytes(maxflow_ctx *c, int64_t *bytes);

/* maxflow_evict parks the context's whole state (Bi-CSR slot arrays, residual
 * capacities, heights, excesses) in one pinned host block and releases every
 * device allocation; maxflow_restore allocates again and copies the state
 * back (the per-slot pair sums c(u,v) + c(v,u) are not parked: the restore
 * rebuilds them on the device from the capacities and the reverse index).
 * The pinned block is kept after a restore for the next eviction and
 * freed by maxflow_destroy.  While evicted, every call that needs the device
 * returns MAXFLOW_ERR_STATE (maxflow_query without side/cut_cap still returns
 * the last value; stats, trace and the setters work).  Since the dynamic
 * algorithm resumes from any valid preflow and labelling (Sec. 4.2), a
 * restored context continues exactly where it stopped.  Both are no-ops when
 * already in the requested state; both synchronise the context's stream.
 * On failure of maxflow_restore the context stays evicted.  No counterpart in
 * the paper. */
int maxflow_evict(maxflow_ctx *c);
int maxflow_restore(maxflow_ctx *c);

/* Sizes in bytes of the device allocations an evicted context held, in
 * allocation order: an upper bound of what maxflow_restore allocates (for an
 * admission check with maxflow_arena_fits).  *count receives their number;
 * sizes is filled when cap >= *count.  MAXFLOW_ERR_STATE when not evicted. */
int maxflow_evicted_sizes(maxflow_ctx *c, int64_t *sizes, int32_t cap, int32_t *count);

/* ---- device-memory arena (serving many contexts under one budget) -------
 * No counterpart in the paper.  maxflow_arena_create reserves `bytes` of
 * device memory with one cudaMalloc on `device` (base NULL), or manages the
 * caller's region [base, base + bytes) (base 256-byte aligned; the caller
 * keeps ownership and the arena never dereferences it); contexts created with
 *     opts.alloc = maxflow_arena_alloc, opts.free = maxflow_arena_free,
 *     opts.alloc_user = arena
 * take their device memory from it, so that later allocations (restores,
 * batch scratch) make no CUDA allocation call and the budget is a physical
 * bound.  Placement is best fit with coalescing; requests of 1 MiB or more
 * take the head of the smallest free block that fits, smaller ones the tail
 * of the highest free block.  When nothing fits: with allow_overflow the
 * request falls back to cudaMalloc (counted in fallbacks / overflow_*),
 * otherwise it fails and the library call returns MAXFLOW_ERR_OOM.  Thread
 * safe.  Frees return memory at once: the library's calls finish their
 * device work before returning, so a freed block has no work in flight.
 * maxflow_arena_destroy synchronises the device and frees what the arena
 * allocated; every context using the arena must be destroyed first.
 * MAXFLOW_ERR_INVALID for bytes <= 0 or a misaligned base; MAXFLOW_ERR_OOM
 * when the reservation fails. */
typedef struct maxflow_arena maxflow_arena;
typedef struct {
    int64_t capacity, in_use, peak_in_use, free_total, largest_free, free_blocks;
    int64_t overflow_in_use, overflow_peak, fallbacks, failed;
} maxflow_arena_stats_t;

int maxflow_arena_create(int32_t device, int64_t bytes, int32_t allow_overflow, void *base, maxflow_arena **out);
void maxflow_arena_destroy(maxflow_arena *a);
void *maxflow_arena_alloc(size_t bytes, void *user, void *stream);
void maxflow_arena_free(void *ptr, size_t bytes, void *user, void *stream);
int maxflow_arena_stats(maxflow_arena *a, maxflow_arena_stats_t *out);
/* *fits = 1 when allocations of the given sizes, made in this order now,
 * would all be placed in the arena (same placement policy; nothing is
 * allocated), else 0. */
int maxflow_arena_fits(maxflow_arena *a, const int64_t *sizes, int32_t count, int32_t *fits);

/* A deep copy of the context's state (graph, residual capacities, heights,
 * excesses, value) on the same device and stream, as a new context; used to
 * try several schedules from one state and to checkpoint a dynamic graph
 * (the dynamic algorithm resumes from any saved state, Sec. 4.2). */
int maxflow_clone(maxflow_ctx *c, maxflow_ctx **out);

/* Rollback for a failed re-solve (no counterpart in the paper; recovery around
 * the dynamic algorithm, which can resume from any saved state, Sec. 4.2).
 * maxflow_checkpoint keeps a deep copy of the context's state (as
 * maxflow_clone; it replaces an earlier checkpoint and costs one copy of the
 * device state).  maxflow_rollback makes the context exactly that saved state
 * again -- graph, residual capacities, heights, excesses, value and settings
 * -- and drops the checkpoint; use it when a call since the checkpoint
 * returned an error (MAXFLOW_ERR_NOT_CONVERGED, MAXFLOW_ERR_INTERNAL, ...).
 * Both synchronise the context's stream.  Rollback without a checkpoint:
 * MAXFLOW_ERR_STATE (nothing changes); either while evicted: MAXFLOW_ERR_STATE. */
int maxflow_checkpoint(maxflow_ctx *c);
int maxflow_rollback(maxflow_ctx *c);

/* Counters and timings of the context and of its last solve, into a
 * caller-owned struct.  Host-side copy, no GPU work.  MAXFLOW_ERR_INVALID for
 * NULL c or out. */
int maxflow_stats(maxflow_ctx *c, maxflow_stats_t *out);

/* Timeline of the last solve kernel: for each grid barrier (at most `cap`),
 * the phase boundary it closed and its time in microseconds after kernel
 * entry.  Boundary ids: 0 start, 1 prologue step, 2 batch validated,
 * 3 batch located (and the rows' room for new pairs checked), 4 unused,
 * 5 capacities changed, 6 iteration start,
 * 7 BFS roots set, 8 BFS level done, 9 worklist built, 10 discharge done,
 * 11 end, 12 first pass of a bottom-up BFS level done (its long rows follow),
 * 13 the grid meets again after BFS levels that the first CTA ran alone,
 * 14 the long rows labelled by the last level are split into work items (a
 * top-down level follows).
 * *count receives the number of entries written.  Host arrays. */
int maxflow_trace(maxflow_ctx *c, int32_t *boundary, double *t_us, int32_t cap, int32_t *count);

/* The work of the phases in the same timeline (entry i belongs to boundary i
 * of maxflow_trace): slots[i] = slots scanned by the BFS, discharge and
 * remove-invalid phases from kernel entry up to that barrier (cumulative);
 * info[i] for a BFS level (boundaries 7 and 8): bit 30 set if the level ran
 * bottom-up, bits 20-29 the work items of long rows it expanded (capped at
 * 1023), bits 0-19 the vertices it labelled (capped at 2^20 - 1); for a
 * discharge round (boundary 10): bits 20-29 the vertices of the CTA-per-vertex
 * bin, bits 0-19 all vertices of the round's lists; 0 otherwise.
 * cta_last_us[i] / cta_mean_us[i]: when the last CTA and the average CTA
 * finished the phase that barrier i closed, in microseconds after the release
 * of the barrier before it (0 for phases that do not record it): a last CTA
 * far behind the mean marks a phase bound by a few long rows.  Any array may
 * be NULL.  Host arrays.  No counterpart in the paper (instrumentation). */
int maxflow_trace_work(maxflow_ctx *c, int64_t *slots, int32_t *info, double *cta_last_us, double *cta_mean_us,
                       int32_t cap, int32_t *count);

/* Release every resource of the context (NULL is a no-op). */
void maxflow_destroy(maxflow_ctx *c);

/* A static string naming a status code. */
const char *maxflow_strerror(int code);

/* The residual Bi-CSR of Sec. 5.1 that maxflow_init builds from the graph
 * (self-loops dropped, parallel edges summed, one slot at u and one at v for
 * every pair with an edge in either direction) and the slack options,
 * computed on the host only: no GPU and no context are needed.
 *   *slot_capacity  in: length of the caller's per-slot arrays; out: S, the
 *                   reserved slots (used slots plus each row's slack,
 *                   max(slack_min, ceil(deg * slack_factor))).
 *   off   [n + 1]   reserved start of each row;   deg [n]  used slots of each row
 *   slot_dst, slot_cap, slot_rev, slot_pcap [S]:  per slot, its head v, c(u, v),
 *                   the index of the slot (v, u), and c(u, v) + c(v, u).  The
 *                   used slots of row u are off[u] .. off[u] + deg[u] - 1,
 *                   sorted by head; slack slots hold (u, 0, itself, 0).
 * Every output may be NULL.  With all of them NULL the call only reports S.
 * With any array given and *slot_capacity < S it returns MAXFLOW_ERR_INVALID
 * (and S), writing nothing.  Other errors as maxflow_init for the graph:
 * MAXFLOW_ERR_INVALID (n < 2, an id out of range, a negative capacity, a
 * negative slack option, NULL slot_capacity), MAXFLOW_ERR_TOO_LARGE,
 * MAXFLOW_ERR_OOM.  Host arrays, owned by the caller. */
int maxflow_build_layout(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                         float slack_factor, int32_t slack_min, int64_t *slot_capacity, int32_t *off, int32_t *deg,
                         int32_t *slot_dst, int32_t *slot_cap, int32_t *slot_rev, int32_t *slot_pcap);

/* Number of kernels this library has launched in the calling process, over
 * every context, batched launch, network and no-allocation call since the
 * library was loaded.  Read it before and after a region to count that
 * region's launches (a solve is one cooperative launch; an update whose
 * insertions overflow a row's slack adds the layout rebuild's four kernels
 * and a second solve launch).  A launch counts when it was enqueued
 * without an error.  Needs no GPU and no context; never fails.  Not a
 * passage of the paper: instrumentation of this library. */
int64_t maxflow_kernel_launches(void);

/* ---- step-level entry points (each runs one step of the path) ------------ */

/* Replace the state by the flow assignment f(u[i], v[i]) = f[i] on the listed
 * directed edges (all others 0): c_f(u,v) = c(u,v) - f(u,v) + f(v,u) and
 * e(x) = inflow - outflow (the residual graph of Sec. 2.1 and the excess of
 * Sec. 3).  Each (u, v) must be an edge with 0 <= f <= cap, else
 * MAXFLOW_ERR_INVALID with the state unchanged.  Host arrays, copied.  Heights
 * are left as they are.  MAXFLOW_ERR_STATE while evicted. */
int maxflow_set_flow(maxflow_ctx *c, int64_t count, const int32_t *u, const int32_t *v, const int32_t *f);

/* The batch part of Alg. 5 only (apply, clamp, excess, source saturation); no
 * re-solve.  The batch is checked as in maxflow_update, with the same errors. */
int maxflow_apply(maxflow_ctx *c, const maxflow_batch *b);

/* Alg. 6 only: heights = residual distance to {t} and every deficient vertex,
 * h(s) = n, unreached vertices n.  Leaves flows and excesses unchanged. */
int maxflow_global_relabel(maxflow_ctx *c);

/* Resume the push-relabel loop (the re-solve loop of Alg. 5) on the current state,
 * without applying anything or saturating the source. */
int maxflow_resolve(maxflow_ctx *c);

/* Residual slots, row by row: (u, v, cap(u,v), c_f(u,v)) of the Sec. 5.1
 * Bi-CSR.  *count in/out as in maxflow_get_flow (the number of used slots).
 * Host arrays, owned by the caller.  MAXFLOW_ERR_INVALID for NULL c or count,
 * MAXFLOW_ERR_STATE while evicted, MAXFLOW_ERR_CUDA. */
int maxflow_get_residual(maxflow_ctx *c, int64_t *count, int32_t *u, int32_t *v, int32_t *cap, int32_t *cf);

/* Heights and excesses (n entries each; either may be NULL).  Host arrays,
 * owned by the caller.  MAXFLOW_ERR_INVALID for NULL c, MAXFLOW_ERR_STATE while
 * evicted, MAXFLOW_ERR_CUDA. */
int maxflow_get_vertex_state(maxflow_ctx *c, int32_t *h, int64_t *e);

/* Self-check of the state on the device.  Writes, for the current state:
 * out[0] slots that break c_f(u,v) + c_f(v,u) = c(u,v) + c(v,u) or c_f >= 0
 * (Sec. 3.1 Theorem 3.3); out[1] vertices whose tracked excess differs from
 * the sum of its slots' c_f - c; out[2] residual slots from A = {h = n} into
 * B (Theorem 3.4); out[3] active vertices (e > 0, h < n, not s or t);
 * out[4] the cut capacity C(A, B); out[5] the value formula.  Six entries. */
int maxflow_check(maxflow_ctx *c, int64_t *out);

/* ---- for callers that cannot allocate device memory ---------------------- */

/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory once they are running -- a serving process that
 * reserves its whole device memory pool at start-up, or a plugin inside a host
 * application that owns the GPU allocator -- because an allocation can fail
 * under their fixed budget, block, or synchronise the device.
 *
 * It computes the same heights as maxflow_global_relabel on a residual graph
 * the caller holds in device memory: the residual distance of every vertex to
 * the sink and, when deficit_roots != 0, to every vertex other than s with a
 * negative excess as well (deficit_roots == 0: to the sink only); s gets n, and
 * so does every vertex that reaches none of them.  It allocates nothing: the
 * step's scratch (frontier lists and control block) is a file-scope device
 * array sized for MAXFLOW_NOALLOC_MAX_N vertices and MAXFLOW_NOALLOC_MAX_SLOTS
 * slots (about 14 MB, held on every GPU that loads the library until the
 * process exits).
 *   rows:  slots of vertex u are off[u] .. off[u] + deg[u] - 1 (off: n+1 ints, deg: n ints)
 *   slots: dst[x] = head v of slot (u, v); cf[x] = c_f(u, v); pcap[x] = c(u,v) + c(v,u),
 *          so that c_f(v, u) = pcap[x] - cf[x]
 *   e:     n excesses (int64); h: n heights (output)
 * All pointers are device pointers on the current device; nothing is copied.
 * Preparing a device: the CUDA driver may load the library's device code, and
 * with it the array, only when it is first used, and that load takes device
 * memory.  A call with n = 0 (s, t and the arrays ignored; deficit_roots and
 * stream used) does that loading for the current device and runs the step once
 * on a two-vertex graph kept inside the array: make it once per device at
 * start-up, so that later calls take no device memory.
 * Each call reads off[n] back and waits for its kernel, so it synchronises the
 * stream: it must not be issued while that stream is being captured into a
 * CUDA graph.  Calls share the array: two calls that overlap on the GPU race.
 * The call returns when the heights are written.
 * Errors: MAXFLOW_ERR_TOO_LARGE if n > MAXFLOW_NOALLOC_MAX_N or off[n] >
 * MAXFLOW_NOALLOC_MAX_SLOTS (off[n] is read back first); MAXFLOW_ERR_INVALID
 * for n = 1 or n < 0, s or t out of range, s == t, or a NULL pointer. */
#define MAXFLOW_NOALLOC_MAX_N (1 << 20)
#define MAXFLOW_NOALLOC_MAX_SLOTS (1 << 25)
int maxflow_global_relabel_noalloc(int32_t n, int32_t s, int32_t t, const int32_t *off, const int32_t *deg,
                                   const int32_t *dst, const int32_t *cf, const int32_t *pcap, const int64_t *e,
                                   int32_t *h, int32_t deficit_roots, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MAXFLOW_GB300_H */
