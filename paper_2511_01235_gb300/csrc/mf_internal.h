// Internal structures of the GB300 max-flow library (not part of the ABI).
//
// Device layout of one residual graph (Sec. 5.1 Bi-CSR), structure of arrays:
//   off[n+1]   reserved start of each row (rows are never moved in place)
//   deg[n]     used slots of the row: base slots (sorted by dst) then inserted slots
//   bdeg[n]    number of sorted base slots (binary search range)
//   dst[S]     head v of slot (u, v)
//   cf[S]      residual capacity c_f(u, v)
//   cap[S]     capacity c(u, v) (0 for a reverse-only slot)
//   rev[S]     index of the slot (v, u)
//   pcap[S]    c(u, v) + c(v, u): with the pair-sum invariant (Sec. 3.1
//              Theorem 3.3) c_f(v, u) = pcap - c_f(u, v), so the backward BFS
//              reads the reverse residual without a gather through rev.
//   h[n]       heights (int32), e[n] excesses (int64)
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#define MF_BLOCK 512          // threads per CTA of the persistent kernel
#define MF_WARPS (MF_BLOCK / 32)
#define MF_SMALL_DEG 8        // discharge: rows up to this many slots get one thread
#define MF_SMALL_DEG_SPARSE 4 // ... on a graph of at most MF_SPARSE_DEG merged directed edges per vertex
#define MF_SPARSE_DEG 8
#define MF_HUB_DEG 512        // discharge: rows above this many slots get a 4-warp group (or a whole CTA)
#define MF_NBIN 4             // discharge row kinds: thread, warp, 4-warp group, CTA
#define MF_GROUP_WARPS 4      // warps of a group; a group keeps rows up to a quarter of the snapshot
#define MF_BFS_HUB 256        // BFS: rows above this many slots enter the frontier as work items
#define MF_BFS_CHUNK 256      // BFS: slots per work item
#define MF_ACTIVE_HIST 64
#define MF_DEFAULT_ROUNDS 2   // adaptive discharge rounds: the minimum per iteration
#define MF_MAX_ROUNDS 1024    // adaptive rounds: upper bound per iteration
#define MF_TRACE 256          // hook timeline entries kept per launch
#define MF_BU_ALPHA 14        // BFS default: go bottom-up when the frontier's slots exceed the unexplored slots / alpha
#define MF_BU_BETA 24         // BFS default: back to top-down when the frontier holds fewer than n / beta vertices
#define MF_WARP_STAGE 512     // discharge: largest row a warp keeps on chip (per-warp slice of the snapshot)
#define MF_ROW_ALIGN 4        // rows start on multiples of this many slots (16-byte loads of slot fields)
#define MF_BU_SCAN 256        // bottom-up BFS: slots of a row its warp scans before deferring the rest
#define MF_BU_CHUNK 256       // bottom-up BFS: slots per deferred work item (one warp, 8 per lane)
#define MF_TAIL_SLOTS 2048    // BFS default: frontiers up to this many slots run in one CTA
#define MF_TAIL_RUN 256       // BFS: levels CTA 0 runs alone before the grid meets once (bounds the others' wait)

// Solve-kernel status (ctrl->status)
#define MF_ST_RUNNING 0
#define MF_ST_CONVERGED 1
#define MF_ST_CAP 2           // iteration or time cap
#define MF_ST_ERROR 3         // ctrl->err holds the error

// ctrl->err values
#define MF_E_NONE 0
#define MF_E_INVALID 1        // batch entry out of range / negative capacity
#define MF_E_OVERFLOW 2       // insertion needs more slack than a row has
#define MF_E_WAIT 3           // a grid barrier wait gave up
#define MF_E_INTERNAL 4
#define MF_E_TOO_LARGE 5      // a batch would leave a pair with c(u,v) + c(v,u) > INT32_MAX

// Kernel modes (bit mask)
#define MF_M_STATIC_INIT 1    // c_f = cap, e = 0, h = 0, saturate the source (Alg. 1)
#define MF_M_APPLY 2          // the batch part of Alg. 5
#define MF_M_SOLVE 4          // the push-relabel loop
#define MF_M_BFS_ONLY 8       // one backward BFS, then stop
#define MF_M_NO_DEFICIT_ROOTS 16  // BFS roots: the sink only (flow extraction runs)
#define MF_M_SKIP_SOURCE_SAT 32   // apply without saturating the source again
#define MF_M_SAT_SINK 64          // static init also saturates every edge into the sink (Sec. 5.2.2 static push-pull)
#define MF_M_NO_SRC_SAT 128       // static init leaves the source edges alone (the pull-only static solve)
#define MF_M_CUT 256              // after the batch: record the sides of the last cut, saturate the edges S -> T
#define MF_M_NO_VALUE 512         // skip the value phase (the side-limited push / pull parts)

struct alignas(128) MfLine {
    unsigned int w[32];
};

// Control block in device memory.  Fields that many CTAs update with atomics
// sit on their own 128-byte lines.  Fields marked (hook) are written only by
// the single thread that completes a grid barrier, while every other CTA
// waits, and are read by all CTAs after it: every CTA sees the same value.
// Hook-written values that the phases and the kernel's loop read.  They fill
// one 128-byte line of their own; after every grid barrier one thread of each
// CTA copies them into shared memory with 16-byte loads issued together, so a
// phase pays one round trip to L2 for all of them instead of one per field.
struct alignas(128) MfDesc {
    int status;
    int level;
    int lvl_lo, lvl_hi;
    int hub_lo, hub_hi;
    int bfs_done;
    int wl_sel;           // which worklist buffer the current round reads
    int wl_n[MF_NBIN];
    int ins_n, touch_n;
    int round;            // discharge round within the iteration
    int dis_more;         // another discharge round follows
    int fix_n[2];         // vertices for remove-invalid-edges (warp list, CTA list)
    int qstamp, fstamp;   // dedupe stamps (never reset: they only grow across launches)
    int bu_mode;          // the coming BFS level runs bottom-up
    int bu_split;         // the bottom-up level just scanned deferred long rows: their pass follows
    int bfs_cta_mode;     // the coming top-down level is small: CTA 0 runs it (and the next small ones) alone
    int defer_n;          // work items of that pass
    int need_total;       // the coming BFS initialisation sums the used slots (first BFS of a launch)
    int pad0;
    unsigned long long t_phase;   // when the last barrier's hook ran
    int long_lo, long_hi;         // long-row vertices labelled by the last level (blong)
    int expand;                   // the coming top-down level first splits them into work items
    int pad1;
};
static_assert(sizeof(MfDesc) == 128, "MfDesc is one 128-byte line, copied as 16-byte vectors");

struct MfCtrl {
    MfLine bar_count;     // w[0]: arrivals at the current barrier
    MfLine bar_gen;       // w[0]: barrier generation
    MfLine err;           // w[0]: sticky error (MF_E_*)
    MfLine bfs_tail;      // w[0]: regular frontier append position
    MfLine hub_tail;      // w[0]: frontier work-item append position
    MfLine head0;         // w[0]: dynamic work head
    MfLine head1;
    MfLine head2;
    MfLine head3;
    // each counter that many warps bump at once on a line of its own: returning
    // atomics on one line are served one after another
    MfLine wl_tail[MF_NBIN + 1];   // [0..3]: worklist append positions per bin, [4]: active vertices
    MfLine misc;          // w[0]: insert list tail, w[1]: touched tail, w[2]: overflow flag
    MfLine aux_tail[MF_NBIN + 2];  // [0..3]: next-round worklist tails, [4]/[5]: remove-invalid lists (warp / CTA)
    MfLine defer_tail;    // w[0]: bottom-up work items of long rows deferred to the level's second pass
    MfLine long_tail;     // w[0]: append position of the long-row vertex list (blong)
    MfLine bfs_acc;       // 64-bit words: [0] slots of the vertices labelled in this level, [1] their number,
                          // [2] used slots of the whole graph (summed by the BFS initialisation)
    // ---- (hook) snapshots: what the phases read, copied to shared memory once per barrier ----
    MfDesc d;
    unsigned long long t_bfs0, t_dis0;   // this iteration: BFS start, discharge start (adaptive rounds)
    long long vis_slots;  // slots of the vertices labelled so far in this BFS
    long long iters;
    unsigned long long t_start;
    // ---- results and statistics (atomics, flushed once per CTA per phase) ----
    long long value;
    long long pushes, relabels, steep, bfs_levels, active_total, active_first;
    long long slots_bfs, verts_bfs, slots_dis, cycles_dis, slots_fix, verts_fix, verts_wl, n_apply;
    long long lab_bfs;        // vertices labelled by all BFS levels
    long long hscan_bfs;      // heights read by the passes over all vertices of bottom-up levels
    long long slots_apply;    // slots read by the batch phases (slot search, source row)
    long long clamps_apply;   // slots whose residual went negative and was sent back
    unsigned long long ns_bfs, ns_dis, ns_fix, ns_wl, ns_apply;
    unsigned long long ns_dis_cta, ns_dis_warp, ns_dis_thread;   // discharge time by row kind, summed over workers
    int active_hist[MF_ACTIVE_HIST];
    long long rounds_total;
    // ---- tracing: kernel entry (block 0, before the first barrier), last hook, hook timeline ----
    unsigned long long t_entry, t_exit;
    long long barriers;
    int trace_n;
    int trace_hook[MF_TRACE];
    unsigned long long trace_t[MF_TRACE];
    // work per traced phase: slots scanned so far (BFS + discharge + remove-invalid, cumulative), and
    // BFS: bit 30 = the level ran bottom-up, bits 20..29 = work items, bits 0..19 = vertices labelled;
    // discharge round: bits 20..29 = CTA-bin (hub) vertices, bits 0..19 = vertices in the round's lists
    long long trace_slots[MF_TRACE];
    int trace_info[MF_TRACE];
    // when the CTAs finished the phase that a barrier closes (ns after the previous barrier's release):
    // the last one and the mean, per traced barrier
    unsigned long long fin_max, fin_sum;
    unsigned trace_fin_max[MF_TRACE], trace_fin_mean[MF_TRACE];
};

struct MfGraph {
    int32_t n;
    int64_t slot_cap;
    int32_t *off, *deg, *bdeg;
    int32_t *dst, *cf, *cap, *rev, *pcap;
    int32_t *h;
    long long *e;
};

struct MfScratch {
    int32_t *border;          // [n] BFS order (level segments)
    int2 *bitem;              // [n + slot_cap / MF_BFS_CHUNK + 64] frontier work items (first slot, length)
    int32_t *blong;           // [n] vertices with rows longer than bfs_hub labelled by the BFS, split into
                              // work items only if a top-down level follows; nullptr: items at once
    int2 *bdefer;             // [n + slot_cap / MF_BFS_CHUNK + 64] bottom-up deferred chunks (vertex, first slot);
                              // nullptr: bottom-up threads scan whole rows themselves
    int32_t *wl[2][MF_NBIN];  // [n] worklists (two buffers for discharge rounds) per row kind: thread, warp,
                              // 4-warp group, CTA
    int32_t *vmark;           // [n] round stamp of the last time a vertex was queued
    int32_t *fixmark;         // [n] iteration stamp of the last time a vertex was listed for Alg. 3
    int32_t *fixl[2];         // [n] vertices relabelled this iteration: rows <= MF_HUB_DEG, rows above
    // batch apply
    int64_t batch_cap;
    int32_t hash_bits;
    unsigned long long *hkey; // [1 << hash_bits] directed-pair dedup
    int32_t *hval;
    unsigned long long *pkey; // [1 << hash_bits] new-pair dedup
    int32_t *pval;
    int32_t *bslot;           // [batch_cap] slot of each update (-2: superseded or ignored)
    int32_t *ins_list;        // [batch_cap] new-pair table positions
    int32_t *hused;           // [batch_cap] dedup table positions in use
    int32_t *clamp;           // [batch_cap] updates that lowered a capacity
    int32_t *ins_need;        // [n]
    int32_t *bu, *bv, *bc;    // [batch_cap] staging of a host batch
};

struct MfParams {
    MfGraph g;
    MfScratch sc;
    MfCtrl *ctrl;
    int32_t *cf;              // residual array of this run (g.cf, or a copy for extraction)
    int32_t *h;
    long long *e;
    int32_t sink, source;
    int32_t mode;
    int32_t kernel_cycles;
    int32_t rounds;           // discharge rounds between two global relabels (1 = the paper's O1 worklist);
                              // 0: adaptive (at least MF_DEFAULT_ROUNDS, more while discharging has taken
                              // less than half the time of this iteration's BFS)
    int32_t small_deg;        // discharge: rows up to this many slots get one thread
    int32_t hub_deg;          // discharge / remove-invalid: rows above this many slots get a group (or a CTA)
    int32_t group_deg;        // discharge: rows above this many slots get a whole CTA (<= hub_deg: no groups)
    int32_t bfs_hub;          // BFS: rows above this many slots enter the frontier as work items
    int32_t bu_alpha;         // BFS direction switch (0: top-down only), see MF_BU_ALPHA
    int32_t bu_beta;
    int32_t fix_steep;
    int32_t data_driven;
    int32_t pull;             // 0: push excess toward t and deficits;
                              // 1: pull for deficits from s and excess (Sec. 5.2.2)
    int32_t side_root;        // -1: every deficient (push) / overflowing (pull) vertex is a root;
                              // else only side[v] == side_root
    uint8_t *side;            // [n] sides of the last cut (1: reaches t or a deficit, 0: not); written by MF_M_CUT
    int32_t test_skip_cta;    // >= 0: that CTA never arrives at the first barrier (tests the bounded waits)
    int32_t requeue;          // discharge rounds: a vertex still active after its cycles joins the next round
    int32_t cycle_div;        // > 0: a row of d slots gets max(kernel_cycles, d / cycle_div) cycles
    int32_t tail_slots;       // BFS: a top-down level whose frontier holds at most this many slots (and
                              // vertices) runs in CTA 0 alone, without grid barriers; 0: never
    int32_t stage_slots;      // dynamic shared memory of the launch in ints: the discharge's on-chip row snapshot
                              // (a CTA keeps rows up to this many slots; 0: none)
    long long max_iters;
    unsigned long long time_limit_ns;
    unsigned long long wait_limit_ns;
    // batch
    int64_t bcount;
    const int32_t *bu, *bv, *bc;
};

// Host-built Bi-CSR (graph_build.cpp)
struct MfHostGraph {
    int32_t n = 0;
    int64_t m_merged = 0;     // directed edges with capacity > 0 or explicitly given (merged)
    int64_t slot_cap = 0, slots = 0;
    int32_t *off = nullptr, *deg = nullptr, *bdeg = nullptr;
    int32_t *dst = nullptr, *cap = nullptr, *rev = nullptr, *pcap = nullptr, *cf = nullptr;
    void release();
};

// Build from COO.  Returns MAXFLOW_* status.
int mf_build_host(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                  float slack_factor, int32_t slack_min, MfHostGraph &out);

// solver.cu
int mf_launch(const MfParams &p, int grid, void *stream);
int mf_launch_multi(const MfParams *plist_dev, int count, int gsize, int grid, unsigned *gstate, unsigned *head,
                    unsigned long long wait_ns, int *abort, void *stream, int stage_bytes);
int mf_stage_bytes(int device, int *bytes);
int mf_max_coresident_blocks(int device, int *per_sm, int *num_sms, int dyn_bytes);
int mf_launch_aux(int which, const MfParams &p, void *stream, long long *dev_out, const void *extra);

#define MF_AUX_SET_CF_RESET 1     // cf = cap on all used slots
#define MF_AUX_SET_FLOW 2         // extra = {count, u, v, f} device arrays; validate into dev_out[0] or apply
#define MF_AUX_EXCESS 3           // e = sum(cf - cap) per row
#define MF_AUX_CHECK 4            // dev_out[0..5]
#define MF_AUX_SIDE 5             // extra = uint8_t* side (device)
#define MF_AUX_CUT 6              // dev_out[0] = cut capacity
#define MF_AUX_REVERSE_CF 7       // extra = int32_t* out: out[x] = cf[rev[x]]
#define MF_AUX_CLEAR_SCRATCH 8    // reset hash tables and ins_need
#define MF_AUX_DUMP 9             // extra = int32_t* rowid per slot (u of each slot index)
#define MF_AUX_NEGATE_E 10        // e = -e
#define MF_AUX_PCAP 11            // pcap = cap + cap[rev] on every used slot (after a restore)

// device-side rebuild (rows grow, flows and excesses stay in place); noff holds
// n + 1 row starts followed by the scan's tile totals: mf_rebuild_scratch(n) int64
#define MF_SCAN_TILE 4096
inline long long mf_scan_tiles(long long n) { return n / MF_SCAN_TILE + 1; }
inline long long mf_rebuild_scratch(long long n) { return n + 1 + mf_scan_tiles(n) + 1; }
int mf_rebuild_capacity(const MfParams &p, void *stream, float slack_factor, int slack_min, long long *noff);
// the copy: rows of more than MF_MOVE_PIECE new slots are moved in pieces of that
// size, listed in items[] (mf_move_items(slot_cap) entries) with their count in *nitems
#define MF_MOVE_PIECE 1024
inline long long mf_move_items(long long slot_cap) { return 2 * (slot_cap / MF_MOVE_PIECE) + 64; }
int mf_rebuild_move(const MfParams &p, void *stream, const long long *noff, int32_t *off, int32_t *dst, int32_t *cf,
                    int32_t *cap, int32_t *rev, int32_t *pcap, long long slot_cap, int2 *items, unsigned *nitems);

// scheduler features of a batch (16 floats)
#define MF_FEATURES 16
struct MfFeatIn {
    const int32_t *bu, *bv, *bc;
    long long count;
    int32_t n, s, t;
    long long m;
    float mean_cap;
    float host[6];            // features 9..14, known on the host
};
int mf_features(const MfFeatIn &f, float *out_dev, void *stream);

int mf_set_flow_items(const MfParams &p, void *stream, long long *dev_bad, long long count, const int32_t *du,
                      const int32_t *dv, const int32_t *df, int apply);
