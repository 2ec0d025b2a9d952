// Device code of the GB300 dynamic max-flow library (sm_103a).
//
// One cooperative, persistent kernel runs a whole solve: the optional static
// initialisation (Alg. 1) or batch repair (Alg. 5),
// then the loop { backward BFS (Alg. 4 / Alg. 6), direction-optimising, which
// also builds the active-vertex worklist (Sec. 5.2.1 O1) ; stop if empty ;
// push-relabel discharge (Alg. 2) in one or more rounds ; remove-invalid-edges
// (Alg. 3, when enabled: off by default) }, then the value formula of Alg. 5.
// Phases are separated by a grid barrier instead of kernel launches, so the
// termination test never leaves the device and a small update costs one
// launch.  Every barrier wait is bounded in time: on expiry the CTA records
// MF_E_WAIT and returns, and the host reports MAXFLOW_ERR_INTERNAL.
//
// Readings of the paper used here (the same as the CPU oracle's):
//   - BFS roots are the sink and every vertex other than s, t with e < 0
//     (Alg. 6), in the static solve too, and h(s) = n always;
//   - termination is tested right after a complete BFS;
//   - a relabel with no residual neighbour, or above n, sets h = n;
//   - ties between equal-height neighbours go to the lowest slot index;
//   - the value is the sum of e(v) over v != s with h(v) < n.
// Excess of the sink and the source is accumulated per CTA in shared memory
// and added once per phase (every vertex may push into the sink, and one
// global atomic per push would serialise on that word).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/maxflow.h"
#include "mf_internal.h"

namespace {

constexpr unsigned long long kEmpty = ~0ull;

// The CTAs that run one solve: the whole grid for mf_solve_kernel, one group
// of the grid for mf_multi_kernel.  Every phase distributes its work over
// vb() in [0, vn()), and the grid barrier waits for vn() CTAs.
__shared__ int g_vb, g_vn;

// Dynamic shared memory of the persistent kernels: the on-chip snapshot of a
// row during its discharge (P.stage_slots ints).
extern __shared__ __align__(16) int mf_stage[];
__device__ __forceinline__ int vb() { return g_vb; }
__device__ __forceinline__ int vn() { return g_vn; }

// First work index of this thread in a grid-stride loop (stride vn() *
// blockDim.x) that spreads a short list over the whole grid: consecutive
// indices go to different CTAs, so a batch of a few thousand updates keeps
// every SM's memory pipeline busy instead of crowding onto the first CTAs.
// spread_warp keeps 32 consecutive indices in one warp (warp-uniform loops).
// Row kind of a vertex with d used slots: 0 thread, 1 warp, 2 four-warp group, 3 CTA.
__device__ __forceinline__ int row_bin(const MfParams &P, int d)
{
    return d <= P.small_deg ? 0 : (d <= P.hub_deg ? 1 : (d <= P.group_deg ? 2 : 3));
}

__device__ __forceinline__ long long spread_thread() { return (long long)threadIdx.x * vn() + vb(); }
__device__ __forceinline__ long long spread_warp()
{
    return ((long long)(threadIdx.x >> 5) * vn() + vb()) * 32 + (threadIdx.x & 31);
}

__device__ __forceinline__ int ldg_cg(const int *p) { return __ldcg(p); }
__device__ __forceinline__ long long ldg_cg(const long long *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ long long atomic_add_ll(long long *p, long long v)
{
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned hash_slot(unsigned long long key, int bits)
{
    return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

// Claim k work items from a shared head; returns the first index (>= cnt when
// the work is exhausted).  The head is read first so that idle warps do not
// queue atomics on it once the work is gone.  Call with the whole warp.
__device__ __forceinline__ int warp_grab(unsigned *head, int cnt, unsigned k)
{
    int b = 0;
    if ((threadIdx.x & 31) == 0) {
        unsigned cur = *(volatile unsigned *)head;
        b = (int)(cur >= (unsigned)cnt ? cur : atomicAdd(head, k));
    }
    return __shfl_sync(0xffffffffu, b, 0);
}

// Items [0, cnt) dealt out to nw workers without a rush on one counter: the
// worker of rank w takes chunk [w*k, w*k + k) first, with no atomic; the
// chunks past nw*k are grabbed k at a time from the head (which starts at 0).
// A grab-only scheme sends, when every warp of the grid starts a short phase at
// once, one atomic per warp to the same word; the L2 serialises them, and a
// warp that comes back for more work waits behind all of them.  `first` is the
// caller's flag, true before the first call.  Called by the whole warp.
__device__ __forceinline__ int warp_deal(unsigned *head, int cnt, unsigned k, int w, int nw, bool &first)
{
    if (first) {
        first = false;
        const long long b = (long long)w * k;
        if (b < cnt) return (int)b;
    }
    const long long base = (long long)nw * k;
    if (base >= cnt) return cnt;
    long long b = 0;
    if ((threadIdx.x & 31) == 0) {
        const unsigned cur = *(volatile unsigned *)head;
        b = base + (base + cur >= cnt ? cur : atomicAdd(head, k));
    }
    b = __shfl_sync(0xffffffffu, b, 0);
    return b < cnt ? (int)b : cnt;
}

// Rank of this warp for warp_deal among the warps of nctas CTAs (all of the
// grid, or CTA 0 alone): consecutive ranks sit in different CTAs, so a few
// items spread over many SMs, and the ranks are rotated by `skip`, so that the
// warps that took the first `skip` items of an earlier list come last in this
// one.
__device__ __forceinline__ int warp_rank(int nctas, int skip)
{
    const int nw = nctas * (int)(blockDim.x >> 5);
    const int r = (int)(threadIdx.x >> 5) * nctas + vb();
    const int s = skip % nw;
    return r >= s ? r - s : r - s + nw;
}

// Per-CTA accumulators, flushed to global memory once per phase.
struct Sh {
    long long sink_e, src_e;
    long long pushes, relabels, steep, slots, verts, cycles;
    long long lab_slots, lab_cnt;     // BFS: slots and number of the vertices labelled this level
    unsigned long long dis_cta_ns, dis_warp_ns, dis_thread_ns;   // discharge: time of this CTA's warps by row kind
    unsigned long long red[MF_WARPS];
    long long wsum[MF_WARPS];
    int wcnt[MF_WARPS];
    long long bcast_rem;
    int bcast_k;
    int bcast_i;
    long long tb_e[MF_BLOCK / (32 * MF_GROUP_WARPS)];   // per team (CTA: [0]; 4-warp groups: [g]) broadcasts
    int tb_h[MF_BLOCK / (32 * MF_GROUP_WARPS)];
    int tb_i[MF_BLOCK / (32 * MF_GROUP_WARPS)];
    int bcast_h;
    long long bcast_e;
    int ok;
    unsigned gen;
    MfDesc d;         // the hook's snapshot, copied after every barrier
};

enum Hook {
    H_START = 0,
    H_NONE,
    H_APPLY_VALID,
    H_APPLY_LOCATED,
    H_APPLY_CHECKED,      // unused (the room check runs inside the locate phase); keeps the trace ids
    H_APPLY_DELTA,
    H_ITER,
    H_BFS_START,
    H_BFS_NEXT,
    H_WL,
    H_DIS,
    H_FINAL,
    H_BU_SPLIT,
    H_BFS_JOIN,
    H_EXPANDED,
};

__device__ __forceinline__ int rd(const int &x) { return __ldcg(&x); }
__device__ __forceinline__ unsigned rd(const unsigned &x) { return __ldcg(&x); }
__device__ __forceinline__ long long rd(const long long &x) { return __ldcg(&x); }
__device__ __forceinline__ unsigned long long rd(const unsigned long long &x) { return __ldcg(&x); }

// The termination test of the loop (Alg. 1 / Alg. 5: stop when no active
// vertex remains), taken right after a complete backward BFS.
__device__ __forceinline__ void decide_iteration(const MfParams &P, MfCtrl *c, unsigned long long now,
                                                 const unsigned (&wl)[MF_NBIN + 1], long long iters,
                                                 unsigned long long t_start, int qstamp, int fstamp)
{
    c->d.round = 0;
    for (int i = 0; i < MF_NBIN + 2; ++i) c->aux_tail[i].w[0] = 0;
    c->d.qstamp = qstamp + 1;
    c->d.fstamp = fstamp + 1;
    const int active = (int)wl[MF_NBIN];
    c->t_dis0 = now;
    for (int b = 0; b < MF_NBIN; ++b) c->d.wl_n[b] = (int)wl[b];
    c->head0.w[0] = c->head1.w[0] = c->head2.w[0] = c->head3.w[0] = 0;
    if (iters < MF_ACTIVE_HIST) c->active_hist[iters] = active;
    if (iters == 0) c->active_first = active;
    c->active_total = rd(c->active_total) + active;
    if (active == 0) {
        c->d.status = MF_ST_CONVERGED;
    } else if (iters >= P.max_iters || now - t_start > P.time_limit_ns) {
        c->d.status = MF_ST_CAP;
    } else {
        c->iters = iters + 1;
    }
}

// Hook work that opens an iteration of the loop (its BFS comes next).
__device__ __forceinline__ void begin_iteration(MfCtrl *c, unsigned long long now)
{
    c->t_bfs0 = now;
    c->bfs_tail.w[0] = 0;
    c->hub_tail.w[0] = 0;
    c->long_tail.w[0] = 0;
    // the used-slot total (acc word 2) only changes with insertions, which
    // come before the first BFS: later iterations keep it
    for (int i = 0; i < 4; ++i) c->bfs_acc.w[i] = 0;
    c->d.need_total = rd(c->bfs_acc.w[4]) == 0 && rd(c->bfs_acc.w[5]) == 0;
    c->d.bu_mode = 0;
    for (int i = 0; i <= MF_NBIN; ++i) c->wl_tail[i].w[0] = 0;
    c->head0.w[0] = c->head1.w[0] = c->head2.w[0] = c->head3.w[0] = 0;
}

// Executed by the one thread that completes a grid barrier, while every
// other CTA waits for it.  All fields it needs are loaded first (through L2)
// so the barrier's critical path holds one memory round trip.
__device__ __noinline__ void run_hook(const MfParams &P, int hook)
{
    MfCtrl *c = P.ctrl;
    const unsigned long long now = gtimer();
    if (hook == H_BU_SPLIT) {
        // after the first pass of a bottom-up level: a second pass over the
        // deferred long rows, or (none deferred) the level is complete
        const unsigned dn = rd(c->defer_tail.w[0]);
        if (dn == 0) {
            c->d.bu_split = 0;
            hook = H_BFS_NEXT;
        } else {
            c->d.bu_split = 1;
            c->d.defer_n = (int)dn;
            c->defer_tail.w[0] = 0;
            c->head1.w[0] = 0;
        }
    }
    const unsigned long long t_phase = rd(c->d.t_phase);
    const int trace_n = hook == H_START ? 0 : rd(c->trace_n);
    const long long barriers = hook == H_START ? 0 : rd(c->barriers);
    const unsigned bfs_tail = rd(c->bfs_tail.w[0]), item_tail = rd(c->hub_tail.w[0]);
    const int lvl_hi = rd(c->d.lvl_hi), hub_hi = rd(c->d.hub_hi), level = rd(c->d.level), hub_lo_old = rd(c->d.hub_lo);
    const long long iters = rd(c->iters), bfs_levels = rd(c->bfs_levels);
    const unsigned long long t_start = rd(c->t_start);
    unsigned wl[MF_NBIN + 1], misc[4];
    for (int i = 0; i <= MF_NBIN; ++i) wl[i] = rd(c->wl_tail[i].w[0]);
    for (int i = 0; i < 4; ++i) misc[i] = rd(c->misc.w[i]);
    unsigned aux[MF_NBIN + 2];
    for (int i = 0; i < MF_NBIN + 2; ++i) aux[i] = rd(c->aux_tail[i].w[0]);
    const int sel = rd(c->d.wl_sel), round = rd(c->d.round), qstamp = rd(c->d.qstamp), fstamp = rd(c->d.fstamp);
    const long long rounds_total = rd(c->rounds_total);
    const long long slots_all = rd(c->slots_bfs) + rd(c->slots_dis) + rd(c->slots_fix);
    const unsigned long long fin_max = rd(c->fin_max), fin_sum = rd(c->fin_sum);
    const int bu_prev = rd(c->d.bu_mode);
    int wl_prev[MF_NBIN];
    for (int b = 0; b < MF_NBIN; ++b) wl_prev[b] = rd(c->d.wl_n[b]);
    int tinfo = 0;
    unsigned err = rd(c->err.w[0]);
    const unsigned long long dt = now - t_phase;
    const bool want_wl = P.data_driven && !(P.mode & MF_M_BFS_ONLY);

    c->d.t_phase = now;
    c->barriers = barriers + 1;
    c->t_exit = now;
    c->trace_n = trace_n + 1;
    switch (hook) {
    case H_START:
        err = 0;
        c->err.w[0] = 0;
        c->d.status = MF_ST_RUNNING;
        c->iters = 0;
        c->value = 0;
        c->pushes = c->relabels = c->steep = c->bfs_levels = c->active_total = c->active_first = 0;
        c->slots_bfs = c->verts_bfs = c->slots_dis = c->cycles_dis = c->slots_fix = c->verts_fix = 0;
        c->verts_wl = c->n_apply = 0;
        c->lab_bfs = c->slots_apply = c->clamps_apply = c->hscan_bfs = 0;
        c->fin_max = c->fin_sum = 0;
        c->ns_bfs = c->ns_dis = c->ns_fix = c->ns_wl = c->ns_apply = 0;
        c->ns_dis_cta = c->ns_dis_warp = c->ns_dis_thread = 0;
        c->bfs_tail.w[0] = 0;
        c->hub_tail.w[0] = 0;
        c->long_tail.w[0] = 0;
        c->defer_tail.w[0] = 0;
        c->d.bu_split = 0;
        c->head0.w[0] = c->head1.w[0] = c->head2.w[0] = c->head3.w[0] = 0;
        for (int i = 0; i <= MF_NBIN; ++i) c->wl_tail[i].w[0] = 0;
        for (int i = 0; i < 8; ++i) c->misc.w[i] = 0;
        for (int i = 0; i < MF_ACTIVE_HIST; ++i) c->active_hist[i] = 0;
        for (int i = 0; i < MF_NBIN + 2; ++i) c->aux_tail[i].w[0] = 0;
        for (int i = 0; i < 8; ++i) c->bfs_acc.w[i] = 0;
        c->d.bu_mode = 0;
        c->d.bfs_cta_mode = 0;
        c->d.need_total = 1;
        c->d.round = 0;
        c->d.dis_more = 0;
        c->rounds_total = 0;
        c->t_start = now;
        break;
    case H_APPLY_VALID:
        c->ns_apply = rd(c->ns_apply) + dt;
        break;
    case H_APPLY_LOCATED:
        c->ns_apply = rd(c->ns_apply) + dt;
        c->d.ins_n = (int)misc[0];
        if (misc[2] != 0 && err == 0) {      // a row has no room for its new pairs
            err = MF_E_OVERFLOW;
            c->err.w[0] = err;
        }
        break;
    case H_APPLY_DELTA:
        c->ns_apply = rd(c->ns_apply) + dt;
        c->d.touch_n = (int)misc[1];
        break;
    case H_NONE:
        c->ns_apply = rd(c->ns_apply) + dt;
        break;
    case H_ITER:
        c->ns_fix = rd(c->ns_fix) + dt;
        begin_iteration(c, now);
        break;
    case H_BFS_START:
    case H_BFS_NEXT: {
        c->ns_bfs = rd(c->ns_bfs) + dt;
        const bool first = hook == H_BFS_START;
        const int lo = first ? 0 : lvl_hi, hlo = first ? 0 : hub_hi, llo = first ? 0 : rd(c->d.long_hi);
        const unsigned long_tail = rd(c->long_tail.w[0]);
        const bool done = lo == (int)bfs_tail && hlo == (int)item_tail && llo == (int)long_tail;
        if (!first && !done) c->bfs_levels = bfs_levels + 1;
        c->d.level = first ? 0 : level + 1;
        c->d.lvl_lo = lo;
        c->d.lvl_hi = (int)bfs_tail;
        c->d.hub_lo = hlo;
        c->d.hub_hi = (int)item_tail;
        c->d.long_lo = llo;
        c->d.long_hi = (int)long_tail;
        c->head0.w[0] = c->head1.w[0] = 0;
        c->d.bfs_done = done;
        {
            // direction of the coming level (Beamer's test): bottom-up once the
            // frontier's slots exceed 1/alpha of the unexplored slots, back to
            // top-down once it holds fewer than n/beta vertices
            const unsigned long long *acc = (const unsigned long long *)c->bfs_acc.w;
            const long long fr = (long long)__ldcg(acc + 0), cnt = (long long)__ldcg(acc + 1);
            const long long tot = (long long)__ldcg(acc + 2);
            const long long vis = (first ? 0 : rd(c->vis_slots)) + fr;
            tinfo = ((first ? 0 : bu_prev) << 30) | ((first ? 0 : min(hub_hi - hub_lo_old, 1023)) << 20) |
                    (int)min(cnt, (long long)((1 << 20) - 1));
            int bu = first ? 0 : rd(c->d.bu_mode);
            if (P.bu_alpha <= 0) bu = 0;
            else if (!bu && fr * P.bu_alpha > tot - vis) bu = 1;
            else if (bu && cnt * P.bu_beta < (long long)P.g.n) bu = 0;
            c->d.bu_mode = bu;
            c->vis_slots = vis;
            // a top-down level after one that labelled long rows first splits them
            // into work items (a bottom-up level never reads them)
            const int expand = (!done && !bu && (int)long_tail > llo) ? 1 : 0;
            c->d.expand = expand;
            // a small top-down frontier is expanded by CTA 0 alone: a level of a
            // few hundred slots costs a grid barrier otherwise
            c->d.bfs_cta_mode =
                (!done && !bu && !expand && P.tail_slots > 0 && fr <= P.tail_slots && cnt <= P.tail_slots) ? 1 : 0;
            c->bfs_acc.w[0] = c->bfs_acc.w[1] = c->bfs_acc.w[2] = c->bfs_acc.w[3] = 0;   // per level; [2] stays
        }
        if (done && want_wl) decide_iteration(P, c, now, wl, iters, t_start, qstamp, fstamp);
        break;
    }
    case H_WL:
        c->ns_wl = rd(c->ns_wl) + dt;
        decide_iteration(P, c, now, wl, iters, t_start, qstamp, fstamp);
        break;
    case H_DIS: {
        // after a discharge round: run another one over the vertices that
        // became active during it, or end the discharge of this iteration
        c->ns_dis = rd(c->ns_dis) + dt;
        tinfo = (min(wl_prev[2] + wl_prev[3], 1023) << 20) |
                min(wl_prev[0] + wl_prev[1] + wl_prev[2] + wl_prev[3], (1 << 20) - 1);
        c->head0.w[0] = c->head1.w[0] = c->head2.w[0] = c->head3.w[0] = 0;
        c->rounds_total = rounds_total + 1;
        const unsigned nxt = aux[0] + aux[1] + aux[2] + aux[3];
        // fixed: P.rounds rounds; adaptive (P.rounds == 0): at least
        // MF_DEFAULT_ROUNDS, then more while this iteration's discharge has
        // taken less than half of its BFS -- a global relabel that costs much
        // (deep BFS, e.g. grids) is amortised over more rounds
        bool more = nxt > 0 && err == 0 && round + 1 < MF_MAX_ROUNDS;
        if (more && round + 1 >= (P.rounds > 0 ? P.rounds : MF_DEFAULT_ROUNDS)) {
            if (P.rounds > 0) {
                more = false;
            } else {
                const unsigned long long t_bfs0 = rd(c->t_bfs0), t_dis0 = rd(c->t_dis0);
                more = 2 * (now - t_dis0) < t_dis0 - t_bfs0;
            }
        }
        if (more) {
            c->d.wl_sel = sel ^ 1;
            for (int b = 0; b < MF_NBIN; ++b) {
                c->d.wl_n[b] = (int)aux[b];
                c->aux_tail[b].w[0] = 0;
            }
            c->d.round = round + 1;
            c->d.qstamp = qstamp + 1;
            c->d.dis_more = 1;
        } else {
            c->d.dis_more = 0;
            c->d.fix_n[0] = (int)aux[MF_NBIN];
            c->d.fix_n[1] = (int)aux[MF_NBIN + 1];
            // without Alg. 3 the next iteration's BFS follows at once: this
            // barrier opens it
            if (!P.fix_steep) begin_iteration(c, now);
        }
        break;
    }
    case H_FINAL:
        break;
    case H_BFS_JOIN:
        c->ns_bfs = rd(c->ns_bfs) + dt;
        break;
    case H_EXPANDED:
        // the long rows' work items are written: the level takes them with the rest
        c->ns_bfs = rd(c->ns_bfs) + dt;
        c->d.hub_hi = (int)item_tail;
        c->d.expand = 0;
        c->head0.w[0] = c->head1.w[0] = 0;
        break;
    case H_BU_SPLIT:
        c->ns_bfs = rd(c->ns_bfs) + dt;
        tinfo = (1 << 30) | (int)min((long long)rd(c->d.defer_n), (long long)((1 << 20) - 1));
        break;
    }
    if (trace_n < MF_TRACE) {
        c->trace_hook[trace_n] = hook;
        c->trace_t[trace_n] = now;
        c->trace_slots[trace_n] = slots_all;
        c->trace_info[trace_n] = tinfo;
        c->trace_fin_max[trace_n] = (unsigned)min(fin_max, 0xffffffffull);
        c->trace_fin_mean[trace_n] = (unsigned)min(fin_sum / (unsigned long long)vn(), 0xffffffffull);
    }
    c->fin_max = 0;
    c->fin_sum = 0;
    if (err != 0) c->d.status = MF_ST_ERROR;
}

// The hook's snapshot into shared memory: eight 16-byte loads through L2,
// issued together (one round trip).  Called by one thread, after the barrier's
// acquire (or by the thread that ran the hook itself).
__device__ __forceinline__ void load_desc(const MfCtrl *c, Sh &sh)
{
    constexpr int kN = (int)(sizeof(MfDesc) / sizeof(int4));
    const int4 *src = reinterpret_cast<const int4 *>(&c->d);
    int4 v[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) v[i] = __ldcg(src + i);
    int4 *dst = reinterpret_cast<int4 *>(&sh.d);
#pragma unroll
    for (int i = 0; i < kN; ++i) dst[i] = v[i];
}

// Grid-wide barrier with a hook.  Returns false if this CTA gave up waiting
// (the caller must return from the kernel at once).  Each CTA counts the
// barrier generations it has passed (sh.gen), so arriving needs no read.
__device__ __noinline__ bool grid_sync(const MfParams &P, int hook, Sh &sh)
{
    MfCtrl *c = P.ctrl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = sh.gen;
        __threadfence();
        unsigned arrived = atomicAdd(&c->bar_count.w[0], 1u) + 1u;
        if (arrived == vn()) {
            atomicExch(&c->bar_count.w[0], 0u);
            run_hook(P, hook);
            __threadfence();
            st_release(&c->bar_gen.w[0], gen + 1u);
        } else {
            unsigned long long t0 = 0;
            unsigned spins = 0;
            while (ld_acquire(&c->bar_gen.w[0]) == gen) {
                ++spins;
                if (spins > 64) __nanosleep(spins > 4096 ? 200 : 32);
                if ((spins & 31u) == 0) {
                    unsigned long long now = gtimer();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > P.wait_limit_ns) {
                        atomicCAS(&c->err.w[0], 0u, (unsigned)MF_E_WAIT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        sh.gen = gen + 1u;
        sh.ok = ok;
        if (ok) load_desc(c, sh);
    }
    __syncthreads();
    return sh.ok != 0;
}


// Flush per-CTA accumulators (excess of sink/source and counters).
__device__ void flush_acc(const MfParams &P, Sh &sh, int phase)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        MfCtrl *c = P.ctrl;
        {
            // when this CTA finished the phase, after the release of the barrier that opened it
            const unsigned long long t0 = sh.d.t_phase, now = gtimer();
            const unsigned long long d = now > t0 ? now - t0 : 0;
            atomicMax(&c->fin_max, d);
            atomicAdd(&c->fin_sum, d);
        }
        if (sh.sink_e) atomic_add_ll(P.e + P.sink, sh.sink_e);
        if (sh.src_e) atomic_add_ll(P.e + P.source, sh.src_e);
        if (sh.pushes) atomic_add_ll(&c->pushes, sh.pushes);
        if (sh.relabels) atomic_add_ll(&c->relabels, sh.relabels);
        if (sh.steep) atomic_add_ll(&c->steep, sh.steep);
        if (sh.slots || sh.verts || sh.cycles) {
            if (phase == 0) {
                atomic_add_ll(&c->slots_bfs, sh.slots);
                atomic_add_ll(&c->verts_bfs, sh.verts);
                atomic_add_ll(&c->hscan_bfs, sh.cycles);
            } else if (phase == 1) {
                atomic_add_ll(&c->slots_dis, sh.slots);
                atomic_add_ll(&c->cycles_dis, sh.cycles);
            } else if (phase == 2) {
                atomic_add_ll(&c->slots_fix, sh.slots);
                atomic_add_ll(&c->verts_fix, sh.verts);
            } else if (phase == 3) {
                atomic_add_ll(&c->verts_wl, sh.verts);
            } else {
                atomic_add_ll(&c->n_apply, sh.verts);
                atomic_add_ll(&c->slots_apply, sh.slots);
                atomic_add_ll(&c->clamps_apply, sh.cycles);
            }
        }
        if (sh.dis_cta_ns || sh.dis_warp_ns || sh.dis_thread_ns) {
            atomicAdd(&c->ns_dis_cta, sh.dis_cta_ns);
            atomicAdd(&c->ns_dis_warp, sh.dis_warp_ns);
            atomicAdd(&c->ns_dis_thread, sh.dis_thread_ns);
            sh.dis_cta_ns = sh.dis_warp_ns = sh.dis_thread_ns = 0;
        }
        if (sh.lab_cnt) {
            atomic_add_ll(&c->lab_bfs, sh.lab_cnt);
            unsigned long long *acc = (unsigned long long *)c->bfs_acc.w;
            atomicAdd(acc + 0, (unsigned long long)sh.lab_slots);
            atomicAdd(acc + 1, (unsigned long long)sh.lab_cnt);
        }
        sh.sink_e = sh.src_e = 0;
        sh.pushes = sh.relabels = sh.steep = sh.slots = sh.verts = sh.cycles = 0;
        sh.lab_slots = sh.lab_cnt = 0;
    }
    __syncthreads();
}

// Add d to the excess of z (sink and source go to the CTA accumulators).
__device__ __forceinline__ void add_excess(const MfParams &P, Sh &sh, int z, long long d)
{
    if (z == P.sink)
        atomicAdd((unsigned long long *)&sh.sink_e, (unsigned long long)d);
    else if (z == P.source)
        atomicAdd((unsigned long long *)&sh.src_e, (unsigned long long)d);
    else
        atomic_add_ll(P.e + z, d);
}

// ---------------------------------------------------------------------------
// Static initialisation (Alg. 1)
// ---------------------------------------------------------------------------

// c_f = c on every slot, e = h = 0: a streaming copy, 16-byte vectors with four
// in flight per thread (the slot arrays start on 256-byte boundaries).
__device__ __noinline__ void phase_static_reset(const MfParams &P)
{
    const long long gt = (long long)vb() * blockDim.x + threadIdx.x;
    const long long gs = (long long)vn() * blockDim.x;
    const long long n4 = P.g.slot_cap >> 2;
    const int4 *src = reinterpret_cast<const int4 *>(P.g.cap);
    int4 *dst = reinterpret_cast<int4 *>(P.cf);
    long long x = gt;
    for (; x + 3 * gs < n4; x += 4 * gs) {
        const int4 a = __ldcs(src + x), b = __ldcs(src + x + gs), c = __ldcs(src + x + 2 * gs),
                   d = __ldcs(src + x + 3 * gs);
        __stcg(dst + x, a);
        __stcg(dst + x + gs, b);
        __stcg(dst + x + 2 * gs, c);
        __stcg(dst + x + 3 * gs, d);
    }
    for (; x < n4; x += gs) __stcg(dst + x, __ldcs(src + x));
    for (long long y = (n4 << 2) + gt; y < P.g.slot_cap; y += gs) P.cf[y] = __ldcg(P.g.cap + y);
    for (long long v = gt; v < P.g.n; v += gs) {
        P.e[v] = 0;
        P.h[v] = 0;
    }
}

__device__ __noinline__ void phase_saturate_source(const MfParams &P, Sh &sh)
{
    const int s = P.source;
    const int r0 = P.g.off[s];
    const int d = ldg_cg(P.g.deg + s);
    long long acc = 0;
    for (int j = vb() * blockDim.x + threadIdx.x; j < d; j += vn() * blockDim.x) {
        int x = r0 + j;
        int c = ldg_cg(P.g.cap + x);
        int y = ldg_cg(P.g.rev + x);
        P.cf[x] = 0;
        P.cf[y] = ldg_cg(P.g.pcap + x);
        int z = ldg_cg(P.g.dst + x);
        if (z == P.sink)
            atomicAdd((unsigned long long *)&sh.sink_e, (unsigned long long)(long long)c);
        else
            P.e[z] = c;
        acc -= c;
    }
    if (acc) atomicAdd((unsigned long long *)&sh.src_e, (unsigned long long)acc);
}

// Static push-pull (Sec. 5.2.2): every edge into t is saturated as well; its
// tail keeps the deficit, and the deficient vertices then act as sinks.
__device__ __noinline__ void phase_saturate_sink(const MfParams &P, Sh &sh)
{
    const int t = P.sink;
    const int r0 = P.g.off[t];
    const int d = ldg_cg(P.g.deg + t);
    long long acc = 0;
    for (int j = vb() * blockDim.x + threadIdx.x; j < d; j += vn() * blockDim.x) {
        const int x = r0 + j;                  // slot (t, z)
        const int y = ldg_cg(P.g.rev + x);     // slot (z, t)
        const int c = ldg_cg(P.cf + y);
        if (c > 0) {
            P.cf[y] = 0;
            P.cf[x] = ldg_cg(P.cf + x) + c;
            add_excess(P, sh, ldg_cg(P.g.dst + x), -(long long)c);
            acc += c;
        }
    }
    if (acc) atomicAdd((unsigned long long *)&sh.sink_e, (unsigned long long)acc);
}

// Dynamic push-pull (Sec. 5.2.2): the sides of the last cut, read from the
// heights the previous solve ended with (1: the vertex reached t or a
// deficit, 0: it did not) ...
__device__ __noinline__ void phase_cut_side(const MfParams &P)
{
    const int n = P.g.n;
    const long long gs = (long long)vn() * blockDim.x;
    for (long long v = (long long)vb() * blockDim.x + threadIdx.x; v < n; v += gs) {
        uint8_t sd = ldg_cg(P.h + v) < n ? 1 : 0;
        if (v == P.source) sd = 0;
        if (v == P.sink) sd = 1;
        P.side[v] = sd;
    }
}

// ... then every residual edge from side 0 to side 1 sends all it can, so
// that no residual path leads from side 0 to side 1.  One warp per row.
__device__ __noinline__ void phase_saturate_cut(const MfParams &P, Sh &sh)
{
    const int n = P.g.n;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)vn() * blockDim.x) >> 5;
    for (long long u = ((long long)vb() * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        if (P.side[u] != 0) continue;
        const int r0 = P.g.off[u], d = ldg_cg(P.g.deg + u);
        long long out = 0;
        for (int j = lane; j < d; j += 32) {
            const int x = r0 + j;
            const int c = ldg_cg(P.cf + x);
            if (c <= 0) continue;
            const int z = ldg_cg(P.g.dst + x);
            if (P.side[z] != 1) continue;
            P.cf[x] = 0;
            atomicAdd(P.cf + ldg_cg(P.g.rev + x), c);
            add_excess(P, sh, z, (long long)c);
            out += c;
        }
        out = warp_sum_ll(out);
        if (lane == 0 && out) add_excess(P, sh, (int)u, -out);
    }
}

// Append val to arr for the lanes with take, one atomic per warp.  Called by
// the whole warp.
__device__ __forceinline__ void warp_append(unsigned *tail, int *arr, bool take, int val)
{
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(tail, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (take) arr[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// ---------------------------------------------------------------------------
// Batch apply and repair (Alg. 5)
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool batch_entry(const MfParams &P, long long i, int &u, int &v, int &c)
{
    u = __ldcg(P.bu + i);
    v = __ldcg(P.bv + i);
    c = __ldcg(P.bc + i);
    return u >= 0 && u < P.g.n && v >= 0 && v < P.g.n && c >= 0;
}

// Validate every entry; insert the directed key into the dedup table, where
// the largest batch index (the last update of the pair) wins.
__device__ __noinline__ void phase_apply_validate(const MfParams &P)
{
    MfCtrl *ctl = P.ctrl;
    const int bits = P.sc.hash_bits;
    const unsigned mask = (1u << bits) - 1u;
    const int lane = threadIdx.x & 31;
    // warp-uniform loop: the positions taken in the table are appended with one atomic per warp
    for (long long base = spread_warp() - lane; base < P.bcount; base += (long long)vn() * blockDim.x) {
        const long long i = base + lane;
        bool fresh = false;
        unsigned pos = 0;
        int u, v, c;
        if (i < P.bcount) {
            if (!batch_entry(P, i, u, v, c)) {
                atomicCAS(&ctl->err.w[0], 0u, (unsigned)MF_E_INVALID);
            } else if (u != v) {
                unsigned long long key = ((unsigned long long)(unsigned)u << 32) | (unsigned)v;
                pos = hash_slot(key, bits);
                for (unsigned probe = 0; probe <= mask; ++probe) {
                    unsigned long long prev = atomicCAS(P.sc.hkey + pos, kEmpty, key);
                    if (prev == kEmpty || prev == key) {
                        fresh = prev == kEmpty;
                        atomicMax(P.sc.hval + pos, (int)i);
                        break;
                    }
                    pos = (pos + 1u) & mask;
                }
            }
        }
        warp_append(&ctl->misc.w[3], P.sc.hused, fresh, (int)pos);   // positions to clear afterwards
    }
}

// Slot of (u, v) in u's row, or -1: an 8-way search of the sorted base slots
// (seven pivots loaded together per round, so a row of 2^15 slots takes five
// dependent rounds instead of fifteen), then a scan of the inserted slots.
// *probes counts the dst entries read.
__device__ __forceinline__ int find_slot(const MfParams &P, int u, int v, int *probes = nullptr)
{
    const int r0 = P.g.off[u];
    const int bd = ldg_cg(P.g.bdeg + u);
    int lo = r0, hi = r0 + bd;      // the first base slot with dst >= v lies in [lo, hi]
    int k = 0;
    while (hi - lo > 8) {
        const int step = (hi - lo) >> 3;
        int below = 0;
#pragma unroll
        for (int q = 1; q < 8; ++q) below += ldg_cg(P.g.dst + lo + q * step) < v ? 1 : 0;
        k += 7;
        const int nlo = below > 0 ? lo + below * step + 1 : lo;
        if (below < 7) hi = lo + (below + 1) * step;
        lo = nlo;
    }
    int below = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) below += (lo + q < hi && ldg_cg(P.g.dst + lo + q) < v) ? 1 : 0;
    k += hi - lo;
    int found = -1;
    const int lb = lo + below;
    if (lb < r0 + bd && ldg_cg(P.g.dst + lb) == v) found = lb;
    ++k;
    if (found < 0) {
        const int end = r0 + ldg_cg(P.g.deg + u);
        for (int x = r0 + bd; x < end; ++x) {
            ++k;
            if (ldg_cg(P.g.dst + x) == v) {
                found = x;
                break;
            }
        }
    }
    if (probes) *probes += k;
    return found;
}

__device__ __forceinline__ unsigned hash_find(const unsigned long long *keys, int bits, unsigned long long key)
{
    const unsigned mask = (1u << bits) - 1u;
    unsigned pos = hash_slot(key, bits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long k = __ldcg(keys + pos);
        if (k == key) return pos;
        if (k == kEmpty) return 0xffffffffu;
        pos = (pos + 1u) & mask;
    }
    return 0xffffffffu;
}

// Locate the slot of every surviving update; a missing pair is entered once
// into the new-pair table and counted against both rows' spare slots.  The
// pair sum the batch leaves behind is checked here, before anything changes:
// c' plus the final capacity of the reverse direction -- the batch's own
// update of (v, u) if it has one, else the current c(v, u), else 0 for a new
// pair -- must fit int32 (residual capacities are int32 and c_f(u,v) +
// c_f(v,u) equals that sum).  A batch that breaks it sets MF_E_TOO_LARGE and
// is refused whole.
__device__ __noinline__ void phase_apply_locate(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int bits = P.sc.hash_bits;
    const unsigned mask = (1u << bits) - 1u;
    const int lane = threadIdx.x & 31;
    int probes = 0;
    for (long long base = spread_warp() - lane; base < P.bcount; base += (long long)vn() * blockDim.x) {
        const long long i = base + lane;
        bool fresh = false;
        unsigned pp = 0;
        int u = 0, v = 0, c = 0;
        if (i < P.bcount) batch_entry(P, i, u, v, c);
        unsigned long long key = ((unsigned long long)(unsigned)u << 32) | (unsigned)v;
        const unsigned pos = (i < P.bcount && u != v) ? hash_find(P.sc.hkey, bits, key) : 0xffffffffu;
        if (i >= P.bcount) {
            // past the batch
        } else if (pos == 0xffffffffu || __ldcg(P.sc.hval + pos) != (int)i) {
            P.sc.bslot[i] = -2;     // a self-loop, or a later update of the same pair wins
        } else {
            const int x = find_slot(P, u, v, &probes);
            P.sc.bslot[i] = x;
            {
                const unsigned long long rkey = ((unsigned long long)(unsigned)v << 32) | (unsigned)u;
                const unsigned rp = hash_find(P.sc.hkey, bits, rkey);
                long long crev = 0;
                if (rp != 0xffffffffu) crev = __ldcg(P.bc + __ldcg(P.sc.hval + rp));
                else if (x >= 0) crev = ldg_cg(P.g.cap + ldg_cg(P.g.rev + x));
                if ((long long)c + crev > (long long)INT32_MAX)
                    atomicCAS(&ctl->err.w[0], 0u, (unsigned)MF_E_TOO_LARGE);
            }
            if (x < 0) {
                const int a = min(u, v), b = max(u, v);
                const unsigned long long pk = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
                pp = hash_slot(pk, bits);
                for (unsigned probe = 0; probe <= mask; ++probe) {
                    unsigned long long prev = atomicCAS(P.sc.pkey + pp, kEmpty, pk);
                    if (prev == kEmpty) {
                        // the room check: the increment that reaches a row's final
                        // demand sees it, so a row short of spare slots is flagged
                        fresh = true;
                        const int na = atomicAdd(P.sc.ins_need + a, 1) + 1;
                        const int nb = atomicAdd(P.sc.ins_need + b, 1) + 1;
                        if (na > P.g.off[a + 1] - P.g.off[a] - ldg_cg(P.g.deg + a) ||
                            nb > P.g.off[b + 1] - P.g.off[b] - ldg_cg(P.g.deg + b))
                            atomicExch(&ctl->misc.w[2], 1u);
                        break;
                    }
                    if (prev == pk) break;
                    pp = (pp + 1u) & mask;
                }
            }
        }
        warp_append(&ctl->misc.w[0], P.sc.ins_list, fresh, (int)pp);   // each new pair once
    }
    if (probes) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)probes);
}

// Winning new capacity of the directed pair (a, b) in the batch, or -1 if the
// batch does not set it.
__device__ __forceinline__ int batch_cap_of(const MfParams &P, int a, int b)
{
    const unsigned long long key = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
    const unsigned pos = hash_find(P.sc.hkey, P.sc.hash_bits, key);
    return pos == 0xffffffffu ? -1 : __ldcg(P.bc + __ldcg(P.sc.hval + pos));
}

// Alg. 5, capacity step, in one phase: (1) every new pair gets its two slots,
// with the batch's capacities set directly (no flow runs on a new pair, so
// c_f = c); (2) every located update sets c(u,v) = c', adds c' - c to c_f(u,v)
// and to both pair sums, and when c_f(u,v) drops below zero sends the
// difference back (the clamp step: c_f(v,u) -= d, e(u) += d, e(v) -= d).
// The dedup table gives every directed pair one owner; the only other writer
// of c_f(u,v) is the owner of (v,u), and the two clamps cannot both fire (the
// pair's residuals sum to the new c(u,v) + c(v,u) >= 0), so the order of the
// atomics does not matter.
__device__ __noinline__ void phase_apply_change(const MfParams &P, Sh &sh)
{
    const int nins = sh.d.ins_n;
    long long applied = 0, clamped = 0;
    for (long long k = spread_thread(); k < nins; k += (long long)vn() * blockDim.x) {
        int pp = __ldcg(P.sc.ins_list + k);
        unsigned long long pk = __ldcg(P.sc.pkey + pp);
        int a = (int)(pk >> 32), b = (int)(pk & 0xffffffffu);
        const int ca = batch_cap_of(P, a, b), cb = batch_cap_of(P, b, a);
        const int xa = P.g.off[a] + atomicAdd(P.g.deg + a, 1);
        const int xb = P.g.off[b] + atomicAdd(P.g.deg + b, 1);
        const int va = ca > 0 ? ca : 0, vb2 = cb > 0 ? cb : 0;
        P.g.dst[xa] = b;
        P.g.dst[xb] = a;
        P.g.rev[xa] = xb;
        P.g.rev[xb] = xa;
        P.g.cap[xa] = va;
        P.g.cap[xb] = vb2;
        P.g.pcap[xa] = P.g.pcap[xb] = va + vb2;
        P.cf[xa] = va;
        P.cf[xb] = vb2;
        P.sc.pval[pp] = xa;
        P.sc.ins_need[a] = 0;
        P.sc.ins_need[b] = 0;
        applied += (ca >= 0 ? 1 : 0) + (cb >= 0 ? 1 : 0);
    }
    for (long long i = spread_thread(); i < P.bcount; i += (long long)vn() * blockDim.x) {
        const int x = __ldcg(P.sc.bslot + i);
        if (x < 0) continue;                 // superseded, ignored, or a new pair (set above)
        int u, v, c;
        batch_entry(P, i, u, v, c);
        const int old = ldg_cg(P.g.cap + x);
        const int delta = c - old;
        ++applied;
        if (delta == 0) continue;
        const int y = ldg_cg(P.g.rev + x);
        P.g.cap[x] = c;
        const int cf_new = atomicAdd(P.cf + x, delta) + delta;
        atomicAdd(P.g.pcap + x, delta);
        atomicAdd(P.g.pcap + y, delta);
        if (cf_new < 0) {
            const int d = -cf_new;
            atomicAdd(P.cf + x, d);
            atomicAdd(P.cf + y, -d);
            add_excess(P, sh, u, (long long)d);
            add_excess(P, sh, v, -(long long)d);
            ++clamped;
        }
    }
    if (applied) atomicAdd((unsigned long long *)&sh.verts, (unsigned long long)applied);
    if (clamped) atomicAdd((unsigned long long *)&sh.cycles, (unsigned long long)clamped);
}

// keep_need: leave ins_need[] as it is (the rows' demand of spare slots after
// an overflow; the rebuild that follows reads and clears it).
__device__ __noinline__ void phase_apply_cleanup(const MfParams &P, bool keep_need)
{
    MfCtrl *ctl = P.ctrl;
    const int nused = (int)*(volatile unsigned *)&ctl->misc.w[3];
    const int nins = (int)*(volatile unsigned *)&ctl->misc.w[0];
    for (int k = vb() * blockDim.x + threadIdx.x; k < nused; k += vn() * blockDim.x) {
        int pos = __ldcg(P.sc.hused + k);
        P.sc.hkey[pos] = kEmpty;
        P.sc.hval[pos] = -1;
    }
    for (int k = vb() * blockDim.x + threadIdx.x; k < nins; k += vn() * blockDim.x) {
        int pp = __ldcg(P.sc.ins_list + k);
        unsigned long long pk = __ldcg(P.sc.pkey + pp);
        if (pk != kEmpty && !keep_need) {
            int a = (int)(pk >> 32), b = (int)(pk & 0xffffffffu);
            P.sc.ins_need[a] = 0;
            P.sc.ins_need[b] = 0;
        }
        P.sc.pkey[pp] = kEmpty;
        P.sc.pval[pp] = -1;
    }
}

// The source step of Alg. 5 (reading: push the remaining residual of every edge out
// of the source and add it to the head's excess).
__device__ __noinline__ void phase_resaturate(const MfParams &P, Sh &sh)
{
    const int s = P.source;
    const int r0 = P.g.off[s];
    const int d = ldg_cg(P.g.deg + s);
    long long acc = 0;
    if (vb() == 0 && threadIdx.x == 0) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)d);
    for (int j = vb() * blockDim.x + threadIdx.x; j < d; j += vn() * blockDim.x) {
        int x = r0 + j;
        int c = ldg_cg(P.cf + x);
        if (c > 0) {
            P.cf[x] = 0;
            atomicAdd(P.cf + ldg_cg(P.g.rev + x), c);
            add_excess(P, sh, ldg_cg(P.g.dst + x), (long long)c);
            acc -= c;
        }
    }
    if (acc) atomicAdd((unsigned long long *)&sh.src_e, (unsigned long long)acc);
}

// ---------------------------------------------------------------------------
// Backward BFS (Alg. 4 / Alg. 6)
// ---------------------------------------------------------------------------

template <int R>
__device__ __forceinline__ void write_items(const MfParams &P, const int (&nc)[R], const int (&x0)[R],
                                            const int (&d)[R], unsigned ibase, int cexcl, int ctot);

// Labelled vertices enter the next frontier either as one entry of the
// regular list (rows of at most bfs_hub slots, expanded warp-cooperatively)
// or, for longer rows, as ceil(deg / MF_BFS_CHUNK) work items (first slot,
// length) that any warp can take: no row is ever walked by one warp alone.
// With with_wl, a labelled vertex that has excess (and is neither the sink
// nor the source) also joins the worklist of the coming discharge (Sec. 5.2.1
// O1): it is active exactly when this BFS labels it, so no separate pass over
// all vertices is needed.
//
// Each lane brings R candidates; the six lists (regular frontier, four
// worklist bins, work items) are reserved with one warp scan and one round of
// atomics issued together, so a warp pays one append round trip per R slots.
// Called by the whole warp.
template <int R>
__device__ __forceinline__ void frontier_push(const MfParams &P, Sh &sh, const bool (&take)[R], const int (&z)[R],
                                              const int (&d)[R], const long long (&ev)[R], bool with_wl, int sel,
                                              bool eager = false)
{
    MfCtrl *ctl = P.ctrl;
    const int lane = threadIdx.x & 31;
    // long rows go to the long-row list, to be split into work items only if a
    // top-down level follows (a bottom-up level never reads them); `eager`
    // (the roots: the first level is top-down) or no list: items at once
    const bool lazy = !eager && P.sc.blong != nullptr;
    // per-lane counts packed 8 bits each: [0] regular, [1..MF_NBIN] worklist
    // bins; and this lane's long rows (lazy) or their work items
    unsigned long long packed = 0;
    int nch = 0;
    long long lab_slots = 0;
    int lab_n = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!take[r]) continue;
        lab_slots += d[r];
        ++lab_n;
        if (d[r] > P.bfs_hub) nch += lazy ? 1 : (d[r] + MF_BFS_CHUNK - 1) / MF_BFS_CHUNK;
        else packed += 1ull;
        if (with_wl && ev[r] > 0) packed += 1ull << (8 * (row_bin(P, d[r]) + 1));
    }
    unsigned long long incl = packed;
    int cincl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        const int yc = __shfl_up_sync(0xffffffffu, cincl, o);
        if (lane >= o) {
            incl += y;
            cincl += yc;
        }
    }
    const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
    const int ctot = __shfl_sync(0xffffffffu, cincl, 31);
    const unsigned long long excl = incl - packed;
    // slots and number of the vertices labelled (the BFS direction test reads them)
    lab_slots = warp_sum_ll(lab_slots);
    const long long lab_cnt = warp_sum_ll((long long)lab_n);
    if (lane == 0 && lab_cnt) {      // per CTA in shared memory, flushed with the phase's counters
        atomicAdd((unsigned long long *)&sh.lab_slots, (unsigned long long)lab_slots);
        atomicAdd((unsigned long long *)&sh.lab_cnt, (unsigned long long)lab_cnt);
    }
    if (total == 0 && ctot == 0) return;
    static_assert(MF_NBIN == 4, "one reservation per worklist bin below");
    // One lane reserves room in every list the warp appends to.  The
    // reservations are independent, so they are issued back to back and the
    // warp waits for one round trip, not one per list.
    const unsigned k0 = (unsigned)(total & 0xffull), k1 = (unsigned)((total >> 8) & 0xffull),
                   k2 = (unsigned)((total >> 16) & 0xffull), k3 = (unsigned)((total >> 24) & 0xffull),
                   k4 = (unsigned)((total >> 32) & 0xffull);
    unsigned b0 = 0, b1 = 0, b2 = 0, b3 = 0, b4 = 0, bi = 0;
    if (lane == 0) {
        if (k0) b0 = atomicAdd(&ctl->bfs_tail.w[0], k0);
        if (k1) b1 = atomicAdd(&ctl->wl_tail[0].w[0], k1);
        if (k2) b2 = atomicAdd(&ctl->wl_tail[1].w[0], k2);
        if (k3) b3 = atomicAdd(&ctl->wl_tail[2].w[0], k3);
        if (k4) b4 = atomicAdd(&ctl->wl_tail[3].w[0], k4);
        if (ctot) bi = atomicAdd(lazy ? &ctl->long_tail.w[0] : &ctl->hub_tail.w[0], (unsigned)ctot);
        const unsigned act = k1 + k2 + k3 + k4;
        if (act) atomicAdd(&ctl->wl_tail[MF_NBIN].w[0], act);
    }
    unsigned pos[MF_NBIN + 1];
    pos[0] = __shfl_sync(0xffffffffu, b0, 0) + (unsigned)(excl & 0xffull);
    pos[1] = __shfl_sync(0xffffffffu, b1, 0) + (unsigned)((excl >> 8) & 0xffull);
    pos[2] = __shfl_sync(0xffffffffu, b2, 0) + (unsigned)((excl >> 16) & 0xffull);
    pos[3] = __shfl_sync(0xffffffffu, b3, 0) + (unsigned)((excl >> 24) & 0xffull);
    pos[4] = __shfl_sync(0xffffffffu, b4, 0) + (unsigned)((excl >> 32) & 0xffull);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!take[r]) continue;
        if (d[r] <= P.bfs_hub) P.sc.border[pos[0]++] = z[r];
        if (with_wl && ev[r] > 0) {
            const int bin = row_bin(P, d[r]);
            P.sc.wl[sel][bin][pos[bin + 1]++] = z[r];
        }
    }
    if (ctot == 0) return;
    const unsigned ibase = __shfl_sync(0xffffffffu, bi, 0);
    const int cexcl = cincl - nch;
    if (lazy) {
        unsigned at = ibase + (unsigned)cexcl;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (take[r] && d[r] > P.bfs_hub) P.sc.blong[at++] = z[r];
        return;
    }
    int x0[R], nc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool big = take[r] && d[r] > P.bfs_hub;
        nc[r] = big ? (d[r] + MF_BFS_CHUNK - 1) / MF_BFS_CHUNK : 0;
        x0[r] = big ? P.g.off[z[r]] : 0;
    }
    write_items<R>(P, nc, x0, d, ibase, cexcl, ctot);
}

// Long rows: ceil(deg / MF_BFS_CHUNK) work items each (first slot, length),
// which any warp can take.  A hub of 10^5 slots has hundreds of items, so the
// warp writes all its rows' items together, 32 at a time (each lane finds the
// row that owns its item), at ibase + [0, ctot); lane L's rows own the items
// from cexcl (the exclusive prefix of nc over the lanes).  Called by the whole warp.
template <int R>
__device__ __forceinline__ void write_items(const MfParams &P, const int (&nc)[R], const int (&x0)[R],
                                            const int (&d)[R], unsigned ibase, int cexcl, int ctot)
{
    const int lane = threadIdx.x & 31;
    for (int i0 = 0; i0 < ctot; i0 += 32) {         // the same trip count in every lane
        const int i = i0 + lane;
        int owner = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1) {
            const int cand = owner + st;
            const int ec = __shfl_sync(0xffffffffu, cexcl, cand & 31);
            if (cand < 32 && ec <= i) owner = cand;
        }
        int j = i - __shfl_sync(0xffffffffu, cexcl, owner);
        int ix = 0, idg = 0, ic = -1;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int ncr = __shfl_sync(0xffffffffu, nc[r], owner);
            const int xr = __shfl_sync(0xffffffffu, x0[r], owner);
            const int dr = __shfl_sync(0xffffffffu, d[r], owner);
            if (ic < 0 && j >= 0 && j < ncr) {
                ic = j;
                ix = xr;
                idg = dr;
            }
            j -= ncr;
        }
        if (i < ctot) {
            const int len = idg - ic * MF_BFS_CHUNK;
            P.sc.bitem[ibase + (unsigned)i] = make_int2(ix + ic * MF_BFS_CHUNK, len < MF_BFS_CHUNK ? len : MF_BFS_CHUNK);
        }
    }
}

__device__ __noinline__ void phase_bfs_init(const MfParams &P, Sh &sh)
{
    const int n = P.g.n;
    const bool deficit_roots = (P.mode & MF_M_NO_DEFICIT_ROOTS) == 0;
    const bool pull = P.pull != 0;
    const bool need_total = sh.d.need_total != 0;
    long long total = 0;
    const int lane = threadIdx.x & 31;
    const long long gs = (long long)vn() * blockDim.x;
    if (vb() == 0 && threadIdx.x == 0) sh.verts += n;     // every vertex: e read, h written
    for (long long base = (long long)vb() * blockDim.x + threadIdx.x - lane; base < n; base += gs) {
        const int v = (int)base + lane;
        bool root[1] = {false};
        int zv[1] = {v}, dv[1] = {0};
        long long ev[1] = {0};
        int dall = 0;
        if (v < n) {
            if (need_total) dall = ldg_cg(P.g.deg + v);
            // push: t and the deficient vertices; pull (Sec. 5.2.2): s and the
            // overflowing vertices; with a side given, only that side's
            const bool side_ok = P.side_root < 0 || P.side[v] == P.side_root;
            if (pull)
                root[0] = (v == P.source) || (v != P.sink && side_ok && ldg_cg(P.e + v) > 0);
            else
                root[0] = (v == P.sink) || (deficit_roots && v != P.source && side_ok && ldg_cg(P.e + v) < 0);
            P.h[v] = root[0] ? 0 : n;
            if (root[0]) dv[0] = need_total ? dall : ldg_cg(P.g.deg + v);
        }
        total += dall;
        if (__any_sync(0xffffffffu, root[0])) frontier_push<1>(P, sh, root, zv, dv, ev, false, 0, true);
    }
    if (need_total) {
        // one atomic per CTA for the used-slot total
        total = warp_sum_ll(total);
        if (lane == 0) sh.wsum[threadIdx.x >> 5] = total;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh.wsum[w];
            if (t) atomicAdd((unsigned long long *)P.ctrl->bfs_acc.w + 2, (unsigned long long)t);
        }
        __syncthreads();
    }
}

// Visit BR slots per lane at level L.  Slot x = (u, z): z gets height L+1 if
// it is unlabelled, is not the source, and has a residual edge (z, u), i.e.
// c_f(z, u) = pcap - c_f(u, z) > 0.  Each stage (slot loads, height gathers,
// claims, degree/excess loads) is issued for all BR slots together, so each
// lane keeps BR independent requests in flight.
template <int BR>
__device__ __forceinline__ void bfs_visit(const MfParams &P, Sh &sh, const int (&x)[BR], const bool (&valid)[BR], int L,
                                          int sel)
{
    const bool with_wl = P.data_driven && !(P.mode & MF_M_BFS_ONLY);
    const bool pull = P.pull != 0;
    const int skip = pull ? P.sink : P.source;     // the terminal a BFS never labels
    const int n = P.g.n;
    int z[BR], rc[BR], hz[BR], d[BR];
    bool claim[BR];
    long long ev[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
        z[r] = valid[r] ? ldg_cg(P.g.dst + x[r]) : skip;
        // push heights follow c_f(z, u) (backward); pull heights c_f(u, z) (forward)
        rc[r] = valid[r] ? (pull ? ldg_cg(P.cf + x[r]) : ldg_cg(P.g.pcap + x[r]) - ldg_cg(P.cf + x[r])) : 0;
    }
#pragma unroll
    for (int r = 0; r < BR; ++r) hz[r] = (rc[r] > 0 && z[r] != skip) ? ldg_cg(P.h + z[r]) : 0;
#pragma unroll
    for (int r = 0; r < BR; ++r) claim[r] = hz[r] == n && atomicCAS(P.h + z[r], n, L + 1) == n;
#pragma unroll
    for (int r = 0; r < BR; ++r) {
        d[r] = claim[r] ? ldg_cg(P.g.deg + z[r]) : 0;
        const bool term = z[r] == P.sink || z[r] == P.source;
        ev[r] = (with_wl && claim[r] && !term) ? (pull ? -ldg_cg(P.e + z[r]) : ldg_cg(P.e + z[r])) : 0;
    }
    frontier_push<BR>(P, sh, claim, z, d, ev, with_wl, sel);
}

constexpr int kBR = 4;

// Before a top-down level that follows one which labelled long rows: each
// long row becomes its ceil(deg / MF_BFS_CHUNK) work items.  Warps take the
// long-row vertices 32 at a time and write their items together.
__device__ __noinline__ void phase_bfs_expand(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int lane = threadIdx.x & 31;
    const int lo = sh.d.long_lo, cnt = sh.d.long_hi - lo;
    const int nwarps = vn() * (int)(blockDim.x >> 5);
    const int rank = warp_rank(vn(), 0);
    bool first = true;
    for (;;) {
        const int b = warp_deal(&ctl->head0.w[0], cnt, 32u, rank, nwarps, first);
        if (b >= cnt) break;
        const int k = b + lane;
        const int z = k < cnt ? __ldcg(P.sc.blong + lo + k) : -1;
        int d[1], x0[1], nc[1];
        d[0] = z >= 0 ? ldg_cg(P.g.deg + z) : 0;
        x0[0] = z >= 0 ? P.g.off[z] : 0;
        nc[0] = (d[0] + MF_BFS_CHUNK - 1) / MF_BFS_CHUNK;
        int incl = nc[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned bi = 0;
        if (lane == 0 && tot) bi = atomicAdd(&ctl->hub_tail.w[0], (unsigned)tot);
        bi = __shfl_sync(0xffffffffu, bi, 0);
        write_items<1>(P, nc, x0, d, bi, incl - nc[0], tot);
    }
}

__device__ __noinline__ void phase_bfs_level(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int L = sh.d.level;
    const int sel = sh.d.wl_sel;
    const int lane = threadIdx.x & 31;
    long long slots = 0;
    const int nctas = sh.d.bfs_cta_mode ? 1 : vn();      // CTA 0 alone runs the small levels
    const int nwarps = nctas * (int)(blockDim.x >> 5);
    // chunks of long rows: one warp per item (at most MF_BFS_CHUNK slots)
    const int ilo = sh.d.hub_lo, icnt = sh.d.hub_hi - ilo;
    bool first = true;
    const int rank_i = warp_rank(nctas, 0);
    for (;;) {
        const int i = warp_deal(&ctl->head1.w[0], icnt, 1u, rank_i, nwarps, first);
        if (i >= icnt) break;
        const int2 it = __ldcg(P.sc.bitem + ilo + i);
        if (lane == 0) slots += it.y;
        for (int kb = 0; kb < it.y; kb += 32 * kBR) {
            int xs[kBR];
            bool vs[kBR];
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                int k = kb + r * 32 + lane;
                vs[r] = k < it.y;
                xs[r] = it.x + k;
            }
            bfs_visit<kBR>(P, sh, xs, vs, L, sel);
        }
    }
    // regular frontier: warps take up to 32 vertices at a time and expand their
    // rows together (each lane finds the vertex that owns its slot); a small
    // frontier is dealt out fewer vertices per warp, so that its rows spread
    // over many warps instead of queueing in one
    const int lo = sh.d.lvl_lo, cnt = sh.d.lvl_hi - lo;
    const int take = max(1, min(32, cnt / max(1, nwarps)));
    first = true;
    const int rank_f = warp_rank(nctas, icnt);
    for (;;) {
        const int b = warp_deal(&ctl->head0.w[0], cnt, (unsigned)take, rank_f, nwarps, first);
        if (b >= cnt) break;
        int idx = b + lane;
        int u = (lane < take && idx < cnt) ? __ldcg(P.sc.border + lo + idx) : -1;
        int d = u >= 0 ? ldg_cg(P.g.deg + u) : 0;
        int r0 = u >= 0 ? P.g.off[u] : 0;
        int incl = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - d;
        const int T = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 0) slots += T;
        for (int kb = 0; kb < T; kb += 32 * kBR) {
            int xs[kBR];
            bool vs[kBR];
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                const int k = kb + r * 32 + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    int cand = owner + step;
                    int ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < 32 && ec <= k) owner = cand;
                }
                int rb = __shfl_sync(0xffffffffu, r0, owner);
                int eb = __shfl_sync(0xffffffffu, excl, owner);
                vs[r] = k < T;
                xs[r] = rb + (k - eb);
            }
            bfs_visit<kBR>(P, sh, xs, vs, L, sel);
        }
    }
    if (slots) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)slots);
}

// A BFS level bottom-up (direction-optimising BFS): every unlabelled vertex v
// looks through its own row for a neighbour u of the current level with a
// residual edge towards it -- c_f(v, u) > 0, v's own slot, for the push
// heights; c_f(u, v) = pcap - c_f(v, u) for the pull heights -- and stops at
// the first one.  The labels equal the top-down level's (each vertex is
// labelled L + 1 exactly when it has such a neighbour); the work follows the
// unlabelled vertices' rows up to the first hit instead of the frontier's
// rows, which pays off once the frontier holds most of the graph.
__device__ __noinline__ void phase_bfs_bottom_up(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int n = P.g.n;
    const int L = sh.d.level;
    const int sel = sh.d.wl_sel;
    const bool pull = P.pull != 0;
    const int skip = pull ? P.sink : P.source;
    const bool with_wl = P.data_driven && !(P.mode & MF_M_BFS_ONLY);
    const int lane = threadIdx.x & 31;
    const long long gs = (long long)vn() * blockDim.x;
    // A warp takes 32 vertices.  Each unlabelled one first looks at kA slots of
    // its row alone; the rows still open after that are scanned by the whole
    // warp together, 128 slots per step over their concatenation (each lane
    // finds the row that owns its slot), and a row drops out of the scan as
    // soon as one of its slots finds a neighbour of level L.  Slots past
    // MF_BU_SCAN of a row go to the level's second pass as work items, so no
    // warp walks a very long row alone.
    constexpr int kA = 4;
    const int cap = P.sc.bdefer != nullptr ? MF_BU_SCAN : 0x7fffffff;
    long long slots = 0, unl = 0;
    if (vb() == 0 && threadIdx.x == 0) sh.cycles += n;    // every vertex's height is read
    for (long long base = (long long)vb() * blockDim.x + threadIdx.x - lane; base < n; base += gs) {
        const int v = (int)base + lane;
        const bool ok = v < n && v != skip;
        const int hv = ok ? ldg_cg(P.h + v) : 0;
        const int r0 = ok ? P.g.off[v] : 0;
        const int d = ok ? ldg_cg(P.g.deg + v) : 0;
        const bool open = ok && hv == n;
        bool take[1] = {false};
        int zv[1] = {v}, dv[1] = {d};
        long long ev[1] = {0};
        if (open) {
            ++unl;
            int c[kA], z[kA];
#pragma unroll
            for (int r = 0; r < kA; ++r) {
                const int x = r0 + r;
                const bool in = r < d;
                c[r] = in ? (pull ? ldg_cg(P.g.pcap + x) - ldg_cg(P.cf + x) : ldg_cg(P.cf + x)) : 0;
                z[r] = in ? ldg_cg(P.g.dst + x) : 0;
            }
#pragma unroll
            for (int r = 0; r < kA; ++r) take[0] |= c[r] > 0 && ldg_cg(P.h + z[r]) == L;
            slots += d < kA ? d : kA;
        }
        // the warp-cooperative scan of the rows still open
        const int lim = d < cap ? d : cap;
        const int rem = (open && !take[0] && lim > kA) ? lim - kA : 0;
        int incl = rem;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - rem;
        const int T = __shfl_sync(0xffffffffu, incl, 31);
        const unsigned pend = __ballot_sync(0xffffffffu, rem > 0);
        unsigned hit = 0;
        for (int kb = 0; kb < T && (pend & ~hit) != 0; kb += 32 * kA) {
            int c[kA], z[kA], ow[kA];
#pragma unroll
            for (int r = 0; r < kA; ++r) {
                const int k = kb + r * 32 + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int cand = owner + step;
                    const int ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < 32 && ec <= k) owner = cand;
                }
                const int rb = __shfl_sync(0xffffffffu, r0, owner);
                const int eb = __shfl_sync(0xffffffffu, excl, owner);
                const bool live = k < T && !((hit >> owner) & 1u);
                const int x = rb + kA + (k - eb);
                ow[r] = owner;
                c[r] = live ? (pull ? ldg_cg(P.g.pcap + x) - ldg_cg(P.cf + x) : ldg_cg(P.cf + x)) : 0;
                z[r] = live ? ldg_cg(P.g.dst + x) : 0;
                slots += live ? 1 : 0;
            }
            unsigned mine = 0;
#pragma unroll
            for (int r = 0; r < kA; ++r)
                if (c[r] > 0 && ldg_cg(P.h + z[r]) == L) mine |= 1u << ow[r];
            hit |= __reduce_or_sync(0xffffffffu, mine);
        }
        if ((hit >> lane) & 1u) take[0] = true;
        int nitem = 0, x0 = 0;
        if (take[0]) {
            P.h[v] = L + 1;
            if (with_wl && v != P.sink && v != P.source) ev[0] = pull ? -ldg_cg(P.e + v) : ldg_cg(P.e + v);
        } else if (open && d > lim) {
            nitem = (d - lim + MF_BU_CHUNK - 1) / MF_BU_CHUNK;
            x0 = r0 + lim;
        }
        if (__any_sync(0xffffffffu, take[0])) frontier_push<1>(P, sh, take, zv, dv, ev, with_wl, sel);
        if (__any_sync(0xffffffffu, nitem > 0)) {
            int ic = nitem;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ic, o);
                if (lane >= o) ic += y;
            }
            const int tot = __shfl_sync(0xffffffffu, ic, 31);
            unsigned at = 0;
            if (lane == 0) at = atomicAdd(&ctl->defer_tail.w[0], (unsigned)tot);
            at = __shfl_sync(0xffffffffu, at, 0) + (unsigned)(ic - nitem);
            for (int cc = 0; cc < nitem; ++cc) P.sc.bdefer[at + cc] = make_int2(v, x0 + cc * MF_BU_CHUNK);
        }
    }
    if (slots) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)slots);
    if (unl) atomicAdd((unsigned long long *)&sh.verts, (unsigned long long)unl);
}

// Second pass of a bottom-up level: the deferred chunks of long rows whose
// first MF_BU_SCAN slots held no neighbour of level L with a residual edge
// towards it.  One warp per chunk of MF_BU_CHUNK slots, 8 per lane; the first
// chunk of a row that finds one labels the vertex (a claim by CAS, as other
// chunks of the same row may find one too).
__device__ __noinline__ void phase_bfs_bottom_up_long(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int n = P.g.n;
    const int L = sh.d.level;
    const int sel = sh.d.wl_sel;
    const bool pull = P.pull != 0;
    const bool with_wl = P.data_driven && !(P.mode & MF_M_BFS_ONLY);
    const int lane = threadIdx.x & 31;
    const int cnt = sh.d.defer_n;
    constexpr int kR = MF_BU_CHUNK / 32;
    long long slots = 0;
    const int nwarps = vn() * (int)(blockDim.x >> 5);
    const int rank = warp_rank(vn(), 0);
    bool first = true;
    for (;;) {
        const int i = warp_deal(&ctl->head1.w[0], cnt, 1u, rank, nwarps, first);
        if (i >= cnt) break;
        const int2 it = __ldcg(P.sc.bdefer + i);
        const int v = it.x;
        if (ldg_cg(P.h + v) != n) continue;       // another chunk of the row labelled it (same value in every lane)
        const int d = ldg_cg(P.g.deg + v);
        const int end = P.g.off[v] + d;
        const int len = end - it.y < MF_BU_CHUNK ? end - it.y : MF_BU_CHUNK;
        int c[kR], z[kR];
        bool hit = false;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int j = r * 32 + lane;
            const int x = it.y + j;
            const bool ok = j < len;
            c[r] = ok ? (pull ? ldg_cg(P.g.pcap + x) - ldg_cg(P.cf + x) : ldg_cg(P.cf + x)) : 0;
            z[r] = ok ? ldg_cg(P.g.dst + x) : 0;
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) hit |= c[r] > 0 && ldg_cg(P.h + z[r]) == L;
        if (lane == 0) slots += len;
        bool won[1] = {false};
        int zv[1] = {v}, dv[1] = {d};
        long long ev[1] = {0};
        if (__any_sync(0xffffffffu, hit)) {
            if (lane == 0) {
                won[0] = atomicCAS(P.h + v, n, L + 1) == n;
                if (won[0] && with_wl && v != P.sink && v != P.source)
                    ev[0] = pull ? -ldg_cg(P.e + v) : ldg_cg(P.e + v);
            }
            if (__any_sync(0xffffffffu, won[0])) frontier_push<1>(P, sh, won, zv, dv, ev, with_wl, sel);
        }
    }
    if (slots) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)slots);
}

// ---------------------------------------------------------------------------
// Worklist of active vertices (Sec. 5.2.1 O1) with the termination count
// ---------------------------------------------------------------------------

__device__ __noinline__ void phase_worklist(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int sel = sh.d.wl_sel;
    const int n = P.g.n;
    const int lane = threadIdx.x & 31;
    const long long gs = (long long)vn() * blockDim.x;
    for (long long base = (long long)vb() * blockDim.x + threadIdx.x - lane; base < n; base += gs) {
        int v = (int)base + lane;
        bool cand = v < n && v != P.sink && v != P.source;
        const long long ev = cand ? ldg_cg(P.e + v) : 0;
        bool act = cand && ldg_cg(P.h + v) < n && (P.pull ? ev < 0 : ev > 0);
        bool listed = P.data_driven ? act : cand;
        int bin = 0;
        if (listed) bin = row_bin(P, ldg_cg(P.g.deg + v));
        unsigned am = __ballot_sync(0xffffffffu, act);
        if (lane == 0 && am) atomicAdd(&ctl->wl_tail[MF_NBIN].w[0], (unsigned)__popc(am));
#pragma unroll
        for (int b = 0; b < MF_NBIN; ++b) warp_append(&ctl->wl_tail[b].w[0], P.sc.wl[sel][b], listed && bin == b, v);
    }
}

// ---------------------------------------------------------------------------
// Discharge (Alg. 2)
// ---------------------------------------------------------------------------

// What a discharge round needs besides the graph: where vertices that become
// active are queued for the next round, and the stamps that keep each vertex
// at most once per round in that queue and once per iteration in the lists
// of remove-invalid-edges.
struct DisCtx {
    int nsel;        // worklist buffer of the next round
    int qstamp;      // stamp of this round's queue
    int fstamp;      // stamp of this iteration's remove-invalid lists
    bool queue;      // a next round follows, so queue newly active vertices
};

// z just became active (its excess went from <= 0 to > 0 during this round):
// give it to the next round (Alg. 2's kernel checks e(u) > 0 on every cycle,
// so a vertex that receives flow while the kernel runs is discharged too).
__device__ __forceinline__ void enqueue_active(const MfParams &P, int z, const DisCtx &dc)
{
    const int dz = ldg_cg(P.g.deg + z);      // in flight together with the stamp exchange
    if (atomicExch(P.sc.vmark + z, dc.qstamp) == dc.qstamp) return;
    const int bin = row_bin(P, dz);
    const unsigned pos = atomicAdd(&P.ctrl->aux_tail[bin].w[0], 1u);
    P.sc.wl[dc.nsel][bin][pos] = z;
}

// u still has something to move after its KERNEL_CYCLES cycles (excess for a
// push, a deficit for a pull) and a height below n: with P.requeue it joins the
// next round's queue too, instead of waiting for the next global relabel.
template <bool PULL>
__device__ __forceinline__ void requeue_if_active(const MfParams &P, int u, const DisCtx &dc)
{
    if (!P.requeue || !dc.queue) return;
    const long long eu = ldg_cg(P.e + u);
    if ((PULL ? eu < 0 : eu > 0) && ldg_cg(P.h + u) < P.g.n) enqueue_active(P, u, dc);
}

// u was relabelled: list it (once per iteration) for remove-invalid-edges;
// only relabelled vertices can have steep residual edges.
__device__ __forceinline__ void note_relabel(const MfParams &P, int u, const DisCtx &dc)
{
    if (atomicExch(P.sc.fixmark + u, dc.fstamp) == dc.fstamp) return;
    const int d = ldg_cg(P.g.deg + u);
    const int li = d > P.hub_deg ? 1 : 0;
    const unsigned pos = atomicAdd(&P.ctrl->aux_tail[MF_NBIN + li].w[0], 1u);
    P.sc.fixl[li][pos] = u;
}

// Move amt > 0 along slot x = (u, z) of u, y = rev[x]: a push lowers c_f(u, z)
// (slot x), a pull (Sec. 5.2.2) lowers c_f(z, u) (slot y); e(z) changes by
// -/+ amt and z joins the next round's queue if that makes it active.  The
// caller updates e(u).  Only u's owner lowers the slot it moves through, so
// an amount read from that slot can always be moved.
template <bool PULL>
__device__ __forceinline__ void move_flow(const MfParams &P, Sh &sh, int x, int y, int z, long long amt,
                                          const DisCtx &dc)
{
    if (PULL) {
        atomicSub(P.cf + y, (int)amt);
        atomicAdd(P.cf + x, (int)amt);
    } else {
        atomicSub(P.cf + x, (int)amt);
        atomicAdd(P.cf + y, (int)amt);
    }
    const long long dz = PULL ? -amt : amt;
    if (z == P.sink) {
        atomicAdd((unsigned long long *)&sh.sink_e, (unsigned long long)dz);
    } else if (z == P.source) {
        atomicAdd((unsigned long long *)&sh.src_e, (unsigned long long)dz);
    } else {
        const long long old = atomic_add_ll(P.e + z, dz);
        const bool became = PULL ? (old >= 0 && old + dz < 0) : (old <= 0 && old + dz > 0);
        if (dc.queue && became) enqueue_active(P, z, dc);
    }
}

// Residual of slot x in the direction of the move, from the slot's own row:
// c_f(u, z) for a push, c_f(z, u) = pcap - c_f(u, z) for a pull.
template <bool PULL>
__device__ __forceinline__ int residual_dir(const MfParams &P, int x)
{
    return PULL ? ldg_cg(P.g.pcap + x) - ldg_cg(P.cf + x) : ldg_cg(P.cf + x);
}

// The amount slot x of u can move now (exact): c_f(u, z) for a push, c_f(z, u) for a pull.
template <bool PULL>
__device__ __forceinline__ int movable(const MfParams &P, int x, int y)
{
    return PULL ? ldg_cg(P.cf + y) : ldg_cg(P.cf + x);
}

// Lowest residual neighbour over slots j = j0, j0 + step, ... (j < d) of the
// row at r0, as a key (h(v) << 32 | j) so the minimum also breaks ties by the
// lowest slot index.  Slots are read kU at a time with their loads issued
// together.
template <int kU, bool PULL>
__device__ __forceinline__ unsigned long long scan_lowest(const MfParams &P, int r0, int d, int j0, int step)
{
    unsigned long long best = kEmpty;
    for (int jb = j0; jb < d; jb += step * kU) {
        int c[kU], z[kU], hz[kU];
#pragma unroll
        for (int r = 0; r < kU; ++r) {
            int j = jb + r * step;
            // push: out-residual c_f(u, z); pull: in-residual c_f(z, u) = pcap - c_f(u, z)
            c[r] = j < d ? (PULL ? ldg_cg(P.g.pcap + r0 + j) - ldg_cg(P.cf + r0 + j) : ldg_cg(P.cf + r0 + j)) : 0;
            z[r] = j < d ? ldg_cg(P.g.dst + r0 + j) : 0;
        }
#pragma unroll
        for (int r = 0; r < kU; ++r) hz[r] = c[r] > 0 ? ldg_cg(P.h + z[r]) : 0;
#pragma unroll
        for (int r = 0; r < kU; ++r) {
            if (c[r] > 0) {
                unsigned long long key = ((unsigned long long)(unsigned)hz[r] << 32) | (unsigned)(jb + r * step);
                best = key < best ? key : best;
            }
        }
    }
    return best;
}

// Heights of a row's heads kept on chip for the cycles after the first scan:
// stg[j] = h(head of slot j) for a slot with residual capacity in the move's
// direction, kNoRes for the others.  A snapshot: heights only rise while the
// discharge runs and residuals of u's own slots only rise except through u's
// own moves (which update stg), so every candidate is checked against global
// memory before flow moves through it.  Slots that gain residual capacity
// meanwhile wait for the next discharge call.
constexpr int kNoRes = 0x7fffffff;

// KERNEL_CYCLES of Alg. 2 for a row of d slots: P.kernel_cycles, or with
// P.cycle_div > 0 at least d / P.cycle_div, so that a long row, whose first
// scan dominates its discharge, makes more of its pushes per scan.
__device__ __forceinline__ int cycles_for(const MfParams &P, int d)
{
    if (P.cycle_div <= 0) return P.kernel_cycles;
    const int k = d / P.cycle_div;
    return k > P.kernel_cycles ? k : P.kernel_cycles;
}
// push passes of one discharge call that may find only stale snapshot entries
// without using up a cycle (each such pass corrects at least one entry upward)
constexpr int kStaleMax = 8;

// The first scan of a row: the lowest residual height as scan_lowest does, and
// the snapshot of every slot of the row in stg.
template <int kU, bool PULL>
__device__ __forceinline__ unsigned long long scan_and_stage(const MfParams &P, int r0, int d, int j0, int step,
                                                             int *stg)
{
    unsigned long long best = kEmpty;
    for (int jb = j0; jb < d; jb += step * kU) {
        int c[kU], z[kU], hz[kU];
#pragma unroll
        for (int r = 0; r < kU; ++r) {
            const int j = jb + r * step;
            c[r] = j < d ? (PULL ? ldg_cg(P.g.pcap + r0 + j) - ldg_cg(P.cf + r0 + j) : ldg_cg(P.cf + r0 + j)) : 0;
            z[r] = j < d ? ldg_cg(P.g.dst + r0 + j) : 0;
        }
#pragma unroll
        for (int r = 0; r < kU; ++r) hz[r] = c[r] > 0 ? ldg_cg(P.h + z[r]) : kNoRes;
#pragma unroll
        for (int r = 0; r < kU; ++r) {
            const int j = jb + r * step;
            if (j < d) stg[j] = hz[r];
            if (c[r] > 0) {
                const unsigned long long key = ((unsigned long long)(unsigned)hz[r] << 32) | (unsigned)j;
                best = key < best ? key : best;
            }
        }
    }
    return best;
}

__device__ __forceinline__ int comp4(const int4 &a, int e)
{
    return e == 0 ? a.x : (e == 1 ? a.y : (e == 2 ? a.z : a.w));
}

// The first scan of a row with 16-byte loads: rows start on multiples of four
// slots (MF_ROW_ALIGN), so slot group g (slots 4g .. 4g+3) is one int4 of
// each slot array.  Thread t of nt takes groups t, t + nt, ... two at a time
// (eight slots in flight).  Same result as scan_and_stage.
template <bool PULL>
__device__ __forceinline__ unsigned long long scan_and_stage_v4(const MfParams &P, int r0, int d, int t, int nt,
                                                                int *stg)
{
    unsigned long long best = kEmpty;
    const int ng = (d + 3) >> 2;
    const int4 *cf4 = reinterpret_cast<const int4 *>(P.cf + r0);
    const int4 *dst4 = reinterpret_cast<const int4 *>(P.g.dst + r0);
    const int4 *pc4 = reinterpret_cast<const int4 *>(P.g.pcap + r0);
    for (int g0 = t; g0 < ng; g0 += 2 * nt) {
        int4 c[2], z[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int g = g0 + q * nt;
            if (g < ng) {
                c[q] = __ldcg(cf4 + g);
                z[q] = __ldcg(dst4 + g);
                if (PULL) {
                    const int4 pc = __ldcg(pc4 + g);
                    c[q] = make_int4(pc.x - c[q].x, pc.y - c[q].y, pc.z - c[q].z, pc.w - c[q].w);
                }
            } else {
                c[q] = make_int4(0, 0, 0, 0);
                z[q] = make_int4(0, 0, 0, 0);
            }
        }
        int hz[8], res[8];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * (g0 + q * nt) + e;
                res[4 * q + e] = j < d ? comp4(c[q], e) : 0;
                hz[4 * q + e] = res[4 * q + e] > 0 ? ldg_cg(P.h + comp4(z[q], e)) : kNoRes;
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * (g0 + q * nt) + e;
                if (j < d) stg[j] = hz[4 * q + e];
                if (res[4 * q + e] > 0) {
                    const unsigned long long key = ((unsigned long long)(unsigned)hz[4 * q + e] << 32) | (unsigned)j;
                    best = key < best ? key : best;
                }
            }
        }
    }
    return best;
}

// Later scans: the lowest entry of the snapshot, from shared memory only.
__device__ __forceinline__ unsigned long long scan_staged(const int *stg, int d, int j0, int step)
{
    unsigned long long best = kEmpty;
    for (int j = j0; j < d; j += step) {
        const int hz = stg[j];
        if (hz != kNoRes) {
            const unsigned long long key = ((unsigned long long)(unsigned)hz << 32) | (unsigned)j;
            best = key < best ? key : best;
        }
    }
    return best;
}

// What slot x of u (row position j, snapshot entry *sj) can move now towards
// a head of height want: 0 unless the head still has that height and the slot
// still has residual capacity; the snapshot entry is corrected on the way.
template <bool PULL>
__device__ __forceinline__ int staged_amount(const MfParams &P, int x, int want, int &sj)
{
    const int hz = ldg_cg(P.h + ldg_cg(P.g.dst + x));
    if (hz != want) {
        sj = hz;
        return 0;
    }
    const int c = movable<PULL>(P, x, ldg_cg(P.g.rev + x));
    if (c <= 0) {
        sj = kNoRes;
        return 0;
    }
    return c;
}

// One thread per vertex (rows of at most small_deg slots).  Returns true
// if u was relabelled (only then can it have steep residual edges, Alg. 3).
// PULL: u is deficient and pulls (Sec. 5.2.2); its "excess" is -e(u).
// Rows of at most kTS slots keep the heads' heights in registers after the
// first scan.
template <bool PULL>
__device__ __noinline__ bool discharge_thread(const MfParams &P, Sh &sh, int u, const DisCtx &dc)
{
    constexpr int kTS = 8;
    bool lifted = false;
    const int n = P.g.n;
    const int r0 = P.g.off[u];
    const int d = ldg_cg(P.g.deg + u);
    int hu = ldg_cg(P.h + u);
    long long scans = 0, moves = 0, fused = 0, gscan = 0;
    int cyc = 0;
    if (d <= kTS) {
        int hc[kTS];
        bool have = false;
        int stale = 0;
        while (cyc < P.kernel_cycles) {
            const long long eu = PULL ? -ldg_cg(P.e + u) : ldg_cg(P.e + u);
            if (!(hu < n && eu > 0)) break;
            ++scans;
            unsigned long long best = kEmpty;
            // the snapshot serves the pushes; a relabel is decided on fresh values
            // (a slot that gained residual capacity since the snapshot may be lower)
            for (int pass = 0; pass < 2; ++pass) {
                if (!have || pass == 1) {
                    int c[kTS], z[kTS];
#pragma unroll
                    for (int j = 0; j < kTS; ++j) {
                        c[j] = j < d ? residual_dir<PULL>(P, r0 + j) : 0;
                        z[j] = j < d ? ldg_cg(P.g.dst + r0 + j) : 0;
                    }
#pragma unroll
                    for (int j = 0; j < kTS; ++j) hc[j] = c[j] > 0 ? ldg_cg(P.h + z[j]) : kNoRes;
                    gscan += d;
                }
                const bool fresh = !have || pass == 1;
                have = true;
                best = kEmpty;
#pragma unroll
                for (int j = 0; j < kTS; ++j) {
                    if (hc[j] != kNoRes) {
                        const unsigned long long key = ((unsigned long long)(unsigned)hc[j] << 32) | (unsigned)j;
                        best = key < best ? key : best;
                    }
                }
                const int bh = best == kEmpty ? 0x7fffffff : (int)(best >> 32);
                if (fresh || !(best == kEmpty || hu <= bh)) break;
            }
            const int best_h = best == kEmpty ? 0x7fffffff : (int)(best >> 32);
            if (best == kEmpty || hu <= best_h) {
                // relabel (the relabel step of Alg. 2), then on to the pushes it makes admissible
                hu = (best == kEmpty || best_h >= n - 1) ? n : best_h + 1;
                P.h[u] = hu;
                lifted = true;
                atomicAdd((unsigned long long *)&sh.relabels, 1ull);
                ++cyc;
                if (hu >= n || cyc >= P.kernel_cycles) continue;
            }
            // the cycles Alg. 2 would run next: the slots of height best_h in slot
            // order, each taking min(residual, what is left)
            long long rem = eu, sent = 0;
            int k = 0;
            const int jstart = (int)(best & 0xffffffffu);
#pragma unroll
            for (int j = 0; j < kTS; ++j) {
                if (j < jstart || j >= d || rem <= 0 || cyc + k >= P.kernel_cycles || hc[j] != best_h) continue;
                const int x = r0 + j;
                int sj = hc[j];
                const int c = staged_amount<PULL>(P, x, best_h, sj);
                hc[j] = sj;
                ++fused;
                if (c <= 0) continue;
                const long long a = rem < (long long)c ? rem : (long long)c;
                move_flow<PULL>(P, sh, x, ldg_cg(P.g.rev + x), ldg_cg(P.g.dst + x), a, dc);
                if (a == c) hc[j] = kNoRes;
                rem -= a;
                sent += a;
                ++k;
            }
            if (sent) atomic_add_ll(P.e + u, PULL ? sent : -sent);
            moves += k;
            // a pass that found only stale entries corrected them and costs no cycle (bounded)
            if (k > 0) cyc += k;
            else if (++stale > kStaleMax) cyc += 1;
        }
    } else {
        while (cyc < P.kernel_cycles) {
            const long long eu = PULL ? -ldg_cg(P.e + u) : ldg_cg(P.e + u);
            if (!(hu < n && eu > 0)) break;
            ++scans;
            gscan += d;
            unsigned long long best = scan_lowest<4, PULL>(P, r0, d, 0, 1);
            int best_h = best == kEmpty ? 0x7fffffff : (int)(best >> 32);
            if (best == kEmpty || hu <= best_h) {
                hu = (best == kEmpty || best_h >= n - 1) ? n : best_h + 1;
                P.h[u] = hu;
                lifted = true;
                atomicAdd((unsigned long long *)&sh.relabels, 1ull);
                ++cyc;
                if (hu >= n || cyc >= P.kernel_cycles) continue;
            }
            long long rem = eu, sent = 0;
            int k = 0;
            int j = (int)(best & 0xffffffffu);
            const int jstart = j;
            for (; j < d && rem > 0 && cyc + k < P.kernel_cycles; ++j) {
                const int x = r0 + j;
                if (residual_dir<PULL>(P, x) <= 0) continue;
                const int z = ldg_cg(P.g.dst + x);
                if (ldg_cg(P.h + z) != best_h) continue;
                const int y = ldg_cg(P.g.rev + x);
                const int c = movable<PULL>(P, x, y);
                if (c <= 0) continue;
                const long long a = rem < (long long)c ? rem : (long long)c;
                move_flow<PULL>(P, sh, x, y, z, a, dc);
                rem -= a;
                sent += a;
                ++k;
            }
            if (sent) atomic_add_ll(P.e + u, PULL ? sent : -sent);
            moves += k;
            fused += j - jstart;
            cyc += k > 0 ? k : 1;
        }
    }
    if (scans) {
        atomicAdd((unsigned long long *)&sh.cycles, (unsigned long long)scans);
        atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)(gscan + fused));
    }
    if (moves) atomicAdd((unsigned long long *)&sh.pushes, (unsigned long long)moves);
    return lifted;
}

// One warp per vertex; ST: the row's heads are kept in stg (this warp's slice
// of the on-chip snapshot) after the first scan.
template <bool PULL, bool ST>
__device__ __noinline__ bool discharge_warp_rows(const MfParams &P, Sh &sh, int u, int d, const DisCtx &dc, int *stg)
{
    bool lifted = false;
    const int n = P.g.n;
    const int lane = threadIdx.x & 31;
    const int r0 = P.g.off[u];
    const int kcyc = cycles_for(P, d);
    constexpr bool st = ST;
    bool have = false;
    int stale = 0;
    int hu = ldg_cg(P.h + u);
    long long scans = 0, moves = 0, fused = 0, gscan = 0;
    int cyc = 0;
    while (cyc < kcyc) {
        const long long eu = PULL ? -ldg_cg(P.e + u) : ldg_cg(P.e + u);
        if (!(hu < n && eu > 0)) break;
        ++scans;
        unsigned long long best;
        if (!st) {
            best = warp_min_u64(scan_lowest<8, PULL>(P, r0, d, lane, 32));
            gscan += d;
        } else if (!have) {
            best = warp_min_u64(scan_and_stage_v4<PULL>(P, r0, d, lane, 32, stg));
            have = true;
            gscan += d;
            __syncwarp();
        } else {
            best = warp_min_u64(scan_staged(stg, d, lane, 32));
            const int bh = best == kEmpty ? 0x7fffffff : (int)(best >> 32);
            if (best == kEmpty || hu <= bh) {
                // a relabel is decided on fresh values: refresh the snapshot first
                __syncwarp();
                best = warp_min_u64(scan_and_stage_v4<PULL>(P, r0, d, lane, 32, stg));
                gscan += d;
                __syncwarp();
            }
        }
        int best_h = best == kEmpty ? 0x7fffffff : (int)(best >> 32);
        if (best == kEmpty || hu <= best_h) {
            // relabel, then straight on to the pushes it makes admissible
            hu = (best == kEmpty || best_h >= n - 1) ? n : best_h + 1;
            lifted = true;
            if (lane == 0) {
                P.h[u] = hu;
                atomicAdd((unsigned long long *)&sh.relabels, 1ull);
            }
            ++cyc;
            if (hu >= n || cyc >= kcyc) {
                __syncwarp();
                continue;
            }
        }
        {
            // Alg. 2's next cycles, fused: the slots of height best_h in slot
            // order take min(residual, what is left); each step covers 8 * 32
            // slots, every lane 8 contiguous ones, with a warp prefix sum over
            // the lanes' totals.
            constexpr int kSeg = 8;
            const int j0 = (int)(best & 0xffffffffu);
            long long rem = eu, sent = 0;
            int k = 0;
            int seg = 1;    // one slot per lane first, kSeg after
            for (int jb = j0; jb < d && rem > 0 && cyc + k < kcyc; jb += seg * 32, seg = kSeg) {
                const int js = jb + lane * seg;
                int a[kSeg];
                long long tsum = 0;
                int tcnt = 0;
                if (st) {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        const int j = js + r;
                        a[r] = (r < seg && j < d && stg[j] == best_h) ? 1 : 0;
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            int sj = stg[js + r];
                            a[r] = staged_amount<PULL>(P, r0 + js + r, best_h, sj);
                            stg[js + r] = sj;
                            ++fused;
                            tsum += a[r];
                            tcnt += a[r] > 0 ? 1 : 0;
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        a[r] = 0;
                        const int j = js + r;
                        if (r < seg && j < d && residual_dir<PULL>(P, r0 + j) > 0) a[r] = 1;
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            const int x = r0 + js + r;
                            a[r] = ldg_cg(P.h + ldg_cg(P.g.dst + x)) == best_h ? 1 : 0;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            const int x = r0 + js + r;
                            const int c = movable<PULL>(P, x, ldg_cg(P.g.rev + x));
                            a[r] = c > 0 ? c : 0;
                            tsum += a[r];
                            tcnt += a[r] > 0 ? 1 : 0;
                        }
                    }
                    fused += seg;
                }
                long long incl = tsum;
                int cincl = tcnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
                    const int tc = __shfl_up_sync(0xffffffffu, cincl, o);
                    if (lane >= o) {
                        incl += t;
                        cincl += tc;
                    }
                }
                long long off = incl - tsum;
                int coff = cincl - tcnt;
                long long mine = 0;
                int mk = 0;
                if (tcnt > 0 && off < rem && cyc + k + coff < kcyc) {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r] <= 0) continue;
                        if (off < rem && cyc + k + coff < kcyc) {
                            const long long g = a[r] < rem - off ? a[r] : rem - off;
                            const int x = r0 + js + r;
                            move_flow<PULL>(P, sh, x, ldg_cg(P.g.rev + x), ldg_cg(P.g.dst + x), g, dc);
                            if (st && g == a[r]) stg[js + r] = kNoRes;
                            mine += g;
                            ++mk;
                        }
                        off += a[r];
                        ++coff;
                    }
                }
                const long long tot = warp_sum_ll(mine);
                const int kk = (int)warp_sum_ll((long long)mk);
                rem -= tot;
                sent += tot;
                k += kk;
                __syncwarp();              // snapshot entries written above are read by other lanes next
            }
            if (lane == 0 && sent) atomic_add_ll(P.e + u, PULL ? sent : -sent);
            moves += k;
            // staged: a pass that found only stale entries corrected them and costs no cycle (bounded)
            if (k > 0) cyc += k;
            else if (!st || ++stale > kStaleMax) cyc += 1;
        }
        __syncwarp();
    }
    fused = warp_sum_ll(fused);
    if (lane == 0) {
        if (scans) {
            atomicAdd((unsigned long long *)&sh.cycles, (unsigned long long)scans);
            atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)(gscan + fused));
        }
        if (moves) atomicAdd((unsigned long long *)&sh.pushes, (unsigned long long)moves);
    }
    return lifted;
}

// One warp per vertex (returns the same value in every lane).  stg: this
// warp's slice of the on-chip snapshot (wcap entries), used when the row fits.
template <bool PULL>
__device__ __forceinline__ bool discharge_warp(const MfParams &P, Sh &sh, int u, const DisCtx &dc, int *stg, int wcap)
{
    const int d = ldg_cg(P.g.deg + u);
    if (stg != nullptr && d <= wcap) return discharge_warp_rows<PULL, true>(P, sh, u, d, dc, stg);
    return discharge_warp_rows<PULL, false>(P, sh, u, d, dc, nullptr);
}

// The threads that discharge one long row together: the whole CTA, or a group
// of MF_GROUP_WARPS warps (a quarter of the CTA, with its own named barrier and
// its own quarter of the snapshot), so that four rows of moderate length are
// discharged side by side.  tid: thread index in the team, n: its threads,
// w0 / nw: its first warp and warp count in the CTA, g: its broadcast slot.
struct CtaTeam {
    int tid, n, w0, nw, g;
    __device__ CtaTeam() : tid((int)threadIdx.x), n((int)blockDim.x), w0(0), nw((int)(blockDim.x >> 5)), g(0) {}
    __device__ void sync() const { __syncthreads(); }
};

struct GroupTeam {
    int tid, n, w0, nw, g;
    __device__ GroupTeam()
        : tid((int)threadIdx.x & (32 * MF_GROUP_WARPS - 1)), n(32 * MF_GROUP_WARPS),
          w0((int)(threadIdx.x >> 5) & ~(MF_GROUP_WARPS - 1)), nw(MF_GROUP_WARPS),
          g((int)threadIdx.x / (32 * MF_GROUP_WARPS))
    {
    }
    __device__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(n) : "memory"); }
};

// One team per vertex; ST: the row's heads are kept in stg (the team's share of
// the on-chip snapshot) after the first scan.
template <bool PULL, bool ST, class Team>
__device__ __noinline__ bool discharge_team_rows(const MfParams &P, Sh &sh, int u, int d, const DisCtx &dc, int *stg)
{
    const Team T;
    bool lifted = false;
    const int n = P.g.n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int r0 = P.g.off[u];
    const int kcyc = cycles_for(P, d);
    constexpr bool st = ST;
    bool have = false;
    int stale = 0;
    long long cand = 0;
    int cyc = 0;
    while (cyc < kcyc) {
        if (T.tid == 0) {
            sh.tb_e[T.g] = PULL ? -ldg_cg(P.e + u) : ldg_cg(P.e + u);
            sh.tb_h[T.g] = ldg_cg(P.h + u);
        }
        T.sync();
        const long long eu = sh.tb_e[T.g];
        const int hu = sh.tb_h[T.g];
        if (!(hu < n && eu > 0)) {
            T.sync();
            break;
        }
        unsigned long long best;
        bool global_scan = !st || !have;
        if (!st) best = scan_lowest<8, PULL>(P, r0, d, T.tid, T.n);
        else if (!have) best = scan_and_stage_v4<PULL>(P, r0, d, T.tid, T.n, stg);
        else best = scan_staged(stg, d, T.tid, T.n);
        have = true;
        best = warp_min_u64(best);
        if (lane == 0) sh.red[wid] = best;
        T.sync();
        unsigned long long b = kEmpty;
        for (int w = T.w0; w < T.w0 + T.nw; ++w) b = sh.red[w] < b ? sh.red[w] : b;
        if (!global_scan && (b == kEmpty || hu <= (int)(b >> 32))) {
            // a relabel is decided on fresh values: refresh the snapshot first
            T.sync();               // every warp has read sh.red
            best = warp_min_u64(scan_and_stage_v4<PULL>(P, r0, d, T.tid, T.n, stg));
            if (lane == 0) sh.red[wid] = best;
            T.sync();
            b = kEmpty;
            for (int w = T.w0; w < T.w0 + T.nw; ++w) b = sh.red[w] < b ? sh.red[w] : b;
            global_scan = true;
        }
        const int best_h = b == kEmpty ? 0x7fffffff : (int)(b >> 32);
        if (T.tid == 0) {
            atomicAdd((unsigned long long *)&sh.cycles, 1ull);
            if (global_scan) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)d);
        }
        bool go = b != kEmpty && hu > best_h;
        if (!go) {
            // relabel, then straight on to the pushes it makes admissible
            const int nh = (b == kEmpty || best_h >= n - 1) ? n : best_h + 1;
            if (T.tid == 0) {
                P.h[u] = nh;
                atomicAdd((unsigned long long *)&sh.relabels, 1ull);
            }
            lifted = true;
            ++cyc;
            go = nh < n && cyc < kcyc;
        }
        if (go) {
            // Alg. 2's next cycles, fused (as in discharge_warp): a step covers
            // seg * T.n slots, every thread seg contiguous ones, so slot
            // order is thread order and one team prefix sum over the threads'
            // totals orders all the amounts of the step.  The first step takes
            // one slot per thread (the excess often runs out there), later
            // ones kSeg.
            constexpr int kSeg = 8;
            const int j0 = (int)(b & 0xffffffffu);
            long long rem = eu;
            int k = 0;
            long long sent = 0;
            int seg = 1;
            for (int jb = j0; jb < d && rem > 0 && cyc + k < kcyc; jb += seg * T.n, seg = kSeg) {
                const int js = jb + T.tid * seg;
                int a[kSeg];
                long long tsum = 0;
                int tcnt = 0;
                if (st) {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        const int j = js + r;
                        a[r] = (r < seg && j < d && stg[j] == best_h) ? 1 : 0;
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            int sj = stg[js + r];
                            a[r] = staged_amount<PULL>(P, r0 + js + r, best_h, sj);
                            stg[js + r] = sj;
                            ++cand;
                            tsum += a[r];
                            tcnt += a[r] > 0 ? 1 : 0;
                        }
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        a[r] = 0;
                        const int j = js + r;
                        if (r < seg && j < d && residual_dir<PULL>(P, r0 + j) > 0) a[r] = 1;   // candidate
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            const int x = r0 + js + r;
                            const int z = ldg_cg(P.g.dst + x);
                            a[r] = ldg_cg(P.h + z) == best_h ? 1 : 0;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r]) {
                            const int x = r0 + js + r;
                            const int c = movable<PULL>(P, x, ldg_cg(P.g.rev + x));
                            a[r] = c > 0 ? c : 0;
                            tsum += a[r];
                            tcnt += a[r] > 0 ? 1 : 0;
                        }
                    }
                    if (T.tid == 0)
                        atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)(seg * T.n));
                }
                long long incl = tsum;
                int cincl = tcnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
                    const int tc = __shfl_up_sync(0xffffffffu, cincl, o);
                    if (lane >= o) {
                        incl += t;
                        cincl += tc;
                    }
                }
                if (lane == 31) {
                    sh.wsum[wid] = incl;
                    sh.wcnt[wid] = cincl;
                }
                T.sync();
                long long off = incl - tsum;
                int coff = cincl - tcnt;
                for (int w = T.w0; w < wid; ++w) {
                    off += sh.wsum[w];
                    coff += sh.wcnt[w];
                }
                long long mine = 0;
                int mk = 0;
                if (tcnt > 0 && off < rem && cyc + k + coff < kcyc) {
#pragma unroll
                    for (int r = 0; r < kSeg; ++r) {
                        if (a[r] <= 0) continue;
                        if (off < rem && cyc + k + coff < kcyc) {
                            const long long g = a[r] < rem - off ? a[r] : rem - off;
                            const int x = r0 + js + r;
                            move_flow<PULL>(P, sh, x, ldg_cg(P.g.rev + x), ldg_cg(P.g.dst + x), g, dc);
                            if (st && g == a[r]) stg[js + r] = kNoRes;
                            mine += g;
                            ++mk;
                        }
                        off += a[r];
                        ++coff;
                    }
                }
                const long long wt = warp_sum_ll(mine);
                const int wk = (int)warp_sum_ll((long long)mk);
                T.sync();               // every warp has read the prefix words
                if (lane == 0) {
                    sh.wsum[wid] = wt;
                    sh.wcnt[wid] = wk;
                }
                T.sync();
                long long tot = 0;
                int kk = 0;
                for (int w = T.w0; w < T.w0 + T.nw; ++w) {
                    tot += sh.wsum[w];
                    kk += sh.wcnt[w];
                }
                rem -= tot;
                sent += tot;
                k += kk;
                T.sync();               // before the words are reused
            }
            if (T.tid == 0) {
                if (sent) atomic_add_ll(P.e + u, PULL ? sent : -sent);
                if (k) atomicAdd((unsigned long long *)&sh.pushes, (unsigned long long)k);
            }
            // staged: a pass that found only stale entries corrected them and costs no cycle (bounded)
            if (k > 0) cyc += k;
            else if (!st || ++stale > kStaleMax) cyc += 1;
        }
        T.sync();
    }
    if (cand) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)cand);
    return lifted;
}

// One CTA per vertex (hubs).  All threads of the CTA call this together;
// the return value is meaningful in thread 0.  stg: the CTA's on-chip
// snapshot (ccap entries), used when the row fits.
template <bool PULL>
__device__ __forceinline__ bool discharge_cta(const MfParams &P, Sh &sh, int u, const DisCtx &dc, int *stg, int ccap)
{
    const int d = ldg_cg(P.g.deg + u);
    if (stg != nullptr && d <= ccap) return discharge_team_rows<PULL, true, CtaTeam>(P, sh, u, d, dc, stg);
    return discharge_team_rows<PULL, false, CtaTeam>(P, sh, u, d, dc, nullptr);
}

// One 4-warp group per vertex (rows up to group_deg slots, which fit the
// group's share of the snapshot).  All threads of the group call this
// together; the return value is meaningful in the group's thread 0.
template <bool PULL>
__device__ __forceinline__ bool discharge_group(const MfParams &P, Sh &sh, int u, const DisCtx &dc, int *stg, int gcap)
{
    const int d = ldg_cg(P.g.deg + u);
    if (stg != nullptr && d <= gcap) return discharge_team_rows<PULL, true, GroupTeam>(P, sh, u, d, dc, stg);
    return discharge_team_rows<PULL, false, GroupTeam>(P, sh, u, d, dc, nullptr);
}

template <bool PULL>
__device__ __noinline__ void phase_discharge(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int lane = threadIdx.x & 31;
    const int sel = sh.d.wl_sel;
    DisCtx dc;
    dc.nsel = sel ^ 1;
    dc.qstamp = sh.d.qstamp;
    dc.fstamp = sh.d.fstamp;
    // queue the vertices that become active for a next round if one may follow
    // (adaptive rounds: the hook decides after this round)
    dc.queue = sh.d.round + 1 < (P.rounds > 0 ? P.rounds : MF_MAX_ROUNDS);
    const int *wl0 = P.sc.wl[sel][0], *wl1 = P.sc.wl[sel][1], *wl2 = P.sc.wl[sel][2], *wl3 = P.sc.wl[sel][3];
    int *stage = P.stage_slots > 0 ? mf_stage : nullptr;
    const unsigned long long t_a = gtimer();
    // the longest rows: one CTA each
    const int nh = sh.d.wl_n[3];
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned cur = *(volatile unsigned *)&ctl->head2.w[0];
            sh.bcast_i = (int)(cur >= (unsigned)nh ? cur : atomicAdd(&ctl->head2.w[0], 1u));
        }
        __syncthreads();
        int i = sh.bcast_i;
        __syncthreads();
        if (i >= nh) break;
        const int u = __ldcg(wl3 + i);
        const bool lifted = discharge_cta<PULL>(P, sh, u, dc, stage, P.stage_slots);
        if (threadIdx.x == 0) {
            if (lifted) note_relabel(P, u, dc);
            requeue_if_active<PULL>(P, u, dc);
        }
    }
    // long rows up to group_deg: one 4-warp group each, four side by side per
    // CTA, each group on its own quarter of the snapshot buffer
    {
        const GroupTeam T;
        const int gcap = P.stage_slots / (MF_BLOCK / (32 * MF_GROUP_WARPS));
        int *gstage = stage != nullptr ? stage + T.g * gcap : nullptr;
        const int ng = sh.d.wl_n[2];
        for (;;) {
            if (T.tid == 0) {
                unsigned cur = *(volatile unsigned *)&ctl->head3.w[0];
                sh.tb_i[T.g] = (int)(cur >= (unsigned)ng ? cur : atomicAdd(&ctl->head3.w[0], 1u));
            }
            T.sync();
            const int i = sh.tb_i[T.g];
            T.sync();
            if (i >= ng) break;
            const int u = __ldcg(wl2 + i);
            const bool lifted = discharge_group<PULL>(P, sh, u, dc, gstage, gcap);
            if (T.tid == 0) {
                if (lifted) note_relabel(P, u, dc);
                requeue_if_active<PULL>(P, u, dc);
            }
        }
    }
    const unsigned long long t_b = gtimer();
    if (lane == 0) atomicAdd((unsigned long long *)&sh.dis_cta_ns, t_b - t_a);
    // mid-degree rows: one warp each, on a slice of its own group's quarter of
    // the snapshot buffer (free once the group has left the loop above, while
    // the other groups may still be on their rows)
    const int nm = sh.d.wl_n[1];
    const int gq = P.stage_slots / (MF_BLOCK / (32 * MF_GROUP_WARPS));
    const int wcap = min(MF_WARP_STAGE, gq / MF_GROUP_WARPS);
    const int wid = (int)(threadIdx.x >> 5);
    int *wstage = stage != nullptr && wcap > 0
                      ? stage + (wid / MF_GROUP_WARPS) * gq + (wid % MF_GROUP_WARPS) * wcap : nullptr;
    for (;;) {
        const int i = warp_grab(&ctl->head1.w[0], nm, 1u);
        if (i >= nm) break;
        const int u = __ldcg(wl1 + i);
        const bool lifted = discharge_warp<PULL>(P, sh, u, dc, wstage, wcap);
        if (lane == 0) {
            if (lifted) note_relabel(P, u, dc);
            requeue_if_active<PULL>(P, u, dc);
        }
    }
    const unsigned long long t_c = gtimer();
    // small rows: one thread each, 32 per grab
    const int ns = sh.d.wl_n[0];
    for (;;) {
        const int b = warp_grab(&ctl->head0.w[0], ns, 32u);
        if (b >= ns) break;
        if (b + lane < ns) {
            const int u = __ldcg(wl0 + b + lane);
            if (discharge_thread<PULL>(P, sh, u, dc)) note_relabel(P, u, dc);
            requeue_if_active<PULL>(P, u, dc);
        }
    }
    __syncwarp();
    const unsigned long long t_d = gtimer();
    if (lane == 0) {
        // per warp, into the CTA's accumulators (one global atomic per CTA and phase)
        atomicAdd((unsigned long long *)&sh.dis_warp_ns, t_c - t_b);
        atomicAdd((unsigned long long *)&sh.dis_thread_ns, t_d - t_c);
    }
}

// ---------------------------------------------------------------------------
// Remove invalid edges (Alg. 3)
// ---------------------------------------------------------------------------

// Alg. 3 on slots j = j0, j0 + step, ... of u's row: push the whole residual
// of every steep slot (h(u) > h(v) + 1).  Returns the flow sent out of u.
// Only vertices relabelled in the discharge can have steep slots (heights are
// exact after the BFS and neighbours only rise), so only those are scanned.
// PULL (Sec. 5.2.2): a steep in-residual c_f(v, u) is pulled whole, and the
// return value is minus the flow received.
template <bool PULL>
__device__ __forceinline__ long long fix_scan(const MfParams &P, Sh &sh, int hu, int r0, int d, int j0, int step)
{
    constexpr int kF = 4;
    long long out = 0;
    for (int jb = j0; jb < d; jb += step * kF) {
        int c[kF], z[kF], hz[kF];
#pragma unroll
        for (int r = 0; r < kF; ++r) {
            const int j = jb + r * step;
            c[r] = j < d ? (PULL ? ldg_cg(P.g.pcap + r0 + j) - ldg_cg(P.cf + r0 + j) : ldg_cg(P.cf + r0 + j)) : 0;
            z[r] = j < d ? ldg_cg(P.g.dst + r0 + j) : 0;
        }
#pragma unroll
        for (int r = 0; r < kF; ++r) hz[r] = c[r] > 0 ? ldg_cg(P.h + z[r]) : 0x7fffffff;
#pragma unroll
        for (int r = 0; r < kF; ++r) {
            if (c[r] > 0 && hu > hz[r] + 1) {
                const int x = r0 + jb + r * step;
                if (PULL) {
                    const int y = ldg_cg(P.g.rev + x);
                    const int old = atomicExch(P.cf + y, 0);
                    if (old > 0) {
                        atomicAdd(P.cf + x, old);
                        add_excess(P, sh, z[r], -(long long)old);
                        atomicAdd((unsigned long long *)&sh.steep, 1ull);
                        out -= old;
                    }
                } else {
                    const int old = atomicExch(P.cf + x, 0);
                    if (old > 0) {
                        atomicAdd(P.cf + ldg_cg(P.g.rev + x), old);
                        add_excess(P, sh, z[r], (long long)old);
                        atomicAdd((unsigned long long *)&sh.steep, 1ull);
                        out += old;
                    }
                }
            }
        }
    }
    return out;
}

template <bool PULL>
__device__ __noinline__ void phase_fix(const MfParams &P, Sh &sh)
{
    MfCtrl *ctl = P.ctrl;
    const int lane = threadIdx.x & 31;
    long long slots = 0, verts = 0;
    // rows above hub_deg: one CTA each
    const int nh = sh.d.fix_n[1];
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned cur = *(volatile unsigned *)&ctl->head2.w[0];
            sh.bcast_i = (int)(cur >= (unsigned)nh ? cur : atomicAdd(&ctl->head2.w[0], 1u));
        }
        __syncthreads();
        int i = sh.bcast_i;
        __syncthreads();
        if (i >= nh) break;
        const int u = __ldcg(P.sc.fixl[1] + i);
        const int hu = ldg_cg(P.h + u);
        const int r0 = P.g.off[u], d = ldg_cg(P.g.deg + u);
        long long out = fix_scan<PULL>(P, sh, hu, r0, d, threadIdx.x, blockDim.x);
        if (out) atomic_add_ll(P.e + u, -out);
        if (threadIdx.x == 0) { slots += d; ++verts; }
    }
    // the others: one warp each
    const int nw = sh.d.fix_n[0];
    for (;;) {
        const int i = warp_grab(&ctl->head1.w[0], nw, 1u);
        if (i >= nw) break;
        const int u = __ldcg(P.sc.fixl[0] + i);
        const int hu = ldg_cg(P.h + u);
        const int r0 = P.g.off[u], d = ldg_cg(P.g.deg + u);
        long long out = warp_sum_ll(fix_scan<PULL>(P, sh, hu, r0, d, lane, 32));
        if (lane == 0) {
            if (out) atomic_add_ll(P.e + u, -out);
            slots += d;
            ++verts;
        }
    }
    if (slots) atomicAdd((unsigned long long *)&sh.slots, (unsigned long long)slots);
    if (verts) atomicAdd((unsigned long long *)&sh.verts, (unsigned long long)verts);
}

// ---------------------------------------------------------------------------
// Value (Alg. 5 last lines, reading R3)
// ---------------------------------------------------------------------------

__device__ __noinline__ void phase_value(const MfParams &P)
{
    // push (R3): sum of e(v) over v != s with h(v) < n; pull (Sec. 5.2.2, the
    // mirror): sum of -e(v) over v != t with h(v) < n
    const int n = P.g.n;
    const bool pull = P.pull != 0;
    const int skip = pull ? P.sink : P.source;
    long long acc = 0;
    for (long long v = (long long)vb() * blockDim.x + threadIdx.x; v < n; v += (long long)vn() * blockDim.x)
        if ((int)v != skip && ldg_cg(P.h + v) < n) acc += pull ? -ldg_cg(P.e + v) : ldg_cg(P.e + v);
    acc = warp_sum_ll(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomic_add_ll(&P.ctrl->value, acc);
}

// One whole solve of one instance by the vn() CTAs of the caller: the
// optional static initialisation or batch repair, the push-relabel loop and
// the value.  Returns false only if this CTA gave up waiting at a barrier
// (the caller must then leave the kernel); every other exit is taken by all
// CTAs together.
__device__ __noinline__ bool solve_instance(const MfParams &P, Sh &sh)
{
    if (vb() == 0 && threadIdx.x == 0) P.ctrl->t_entry = gtimer();
    if (threadIdx.x == 0) {
        sh.gen = ld_acquire(&P.ctrl->bar_gen.w[0]);   // nobody can pass the first barrier before all have read it
        sh.sink_e = sh.src_e = 0;
        sh.pushes = sh.relabels = sh.steep = sh.slots = sh.verts = sh.cycles = 0;
        sh.lab_slots = sh.lab_cnt = 0;
        sh.dis_cta_ns = sh.dis_warp_ns = sh.dis_thread_ns = 0;
    }
    // a CTA that never arrives (tests only): the others give up after
    // wait_limit_ns, record MF_E_WAIT and leave the kernel
    if (P.test_skip_cta == vb()) return true;
    if (!grid_sync(P, H_START, sh)) return false;

    if (P.mode & MF_M_STATIC_INIT) {
        phase_static_reset(P);
        if (!grid_sync(P, H_NONE, sh)) return false;
        if (!(P.mode & MF_M_NO_SRC_SAT)) {
            phase_saturate_source(P, sh);
            flush_acc(P, sh, 4);
            if (!grid_sync(P, H_NONE, sh)) return false;
        }
        if (P.mode & MF_M_SAT_SINK) {
            phase_saturate_sink(P, sh);
            flush_acc(P, sh, 4);
            if (!grid_sync(P, H_NONE, sh)) return false;
        }
    }
    if (P.mode & MF_M_APPLY) {
        phase_apply_validate(P);
        if (!grid_sync(P, H_APPLY_VALID, sh)) return false;
        if (sh.d.status != MF_ST_RUNNING) {
            phase_apply_cleanup(P, false);
            return grid_sync(P, H_FINAL, sh);
        }
        phase_apply_locate(P, sh);
        flush_acc(P, sh, 4);
        if (!grid_sync(P, H_APPLY_LOCATED, sh)) return false;
        if (sh.d.status != MF_ST_RUNNING) {
            // a row overflow keeps the rows' demand for the rebuild that follows;
            // a refused batch (pair sum) leaves nothing behind
            phase_apply_cleanup(P, *(volatile unsigned *)&P.ctrl->err.w[0] == MF_E_OVERFLOW);
            return grid_sync(P, H_FINAL, sh);
        }
        phase_apply_change(P, sh);
        flush_acc(P, sh, 4);
        if (!grid_sync(P, H_APPLY_DELTA, sh)) return false;
        // the source step reads the final residuals; the tables are cleared beside it
        phase_apply_cleanup(P, false);
        if (!(P.mode & MF_M_SKIP_SOURCE_SAT)) phase_resaturate(P, sh);
        flush_acc(P, sh, 4);
        // straight on to the loop: this barrier opens its first iteration
        if (!(P.mode & MF_M_CUT) && (P.mode & (MF_M_SOLVE | MF_M_BFS_ONLY))) {
            if (!grid_sync(P, H_ITER, sh)) return false;
            if (sh.d.status != MF_ST_RUNNING) return true;
            goto loop;
        }
        if (!grid_sync(P, H_NONE, sh)) return false;
        if (P.mode & MF_M_CUT) {
            phase_cut_side(P);
            if (!grid_sync(P, H_NONE, sh)) return false;
            phase_saturate_cut(P, sh);
            flush_acc(P, sh, 4);
            if (!grid_sync(P, H_NONE, sh)) return false;
        }
        if (sh.d.status != MF_ST_RUNNING) return true;
    }
    if (!(P.mode & (MF_M_SOLVE | MF_M_BFS_ONLY))) return true;

    if (!grid_sync(P, H_ITER, sh)) return false;
loop:
    for (;;) {
        // backward BFS
        phase_bfs_init(P, sh);
        flush_acc(P, sh, 0);               // the roots' label counters feed the first level's direction
        if (!grid_sync(P, H_BFS_START, sh)) return false;
        while (!sh.d.bfs_done) {
            if (sh.d.bfs_cta_mode) {
                // small levels: CTA 0 alone, its own thread 0 running the level
                // hook; the other CTAs wait at the next grid barrier
                if (vb() == 0) {
                    int run = 0;
                    do {
                        phase_bfs_level(P, sh);
                        flush_acc(P, sh, 0);
                        if (threadIdx.x == 0) {
                            run_hook(P, H_BFS_NEXT);
                            load_desc(P.ctrl, sh);
                        }
                        __syncthreads();
                    } while (++run < MF_TAIL_RUN && !sh.d.bfs_done && sh.d.bfs_cta_mode);
                }
                if (!grid_sync(P, H_BFS_JOIN, sh)) return false;
                continue;
            }
            if (sh.d.bu_mode) {
                phase_bfs_bottom_up(P, sh);
                flush_acc(P, sh, 0);
                if (!grid_sync(P, H_BU_SPLIT, sh)) return false;     // ends the level if nothing was deferred
                if (sh.d.bu_split) {
                    phase_bfs_bottom_up_long(P, sh);
                    flush_acc(P, sh, 0);
                    if (!grid_sync(P, H_BFS_NEXT, sh)) return false;
                }
            } else {
                if (sh.d.expand) {
                    phase_bfs_expand(P, sh);
                    if (!grid_sync(P, H_EXPANDED, sh)) return false;
                }
                phase_bfs_level(P, sh);
                flush_acc(P, sh, 0);
                if (!grid_sync(P, H_BFS_NEXT, sh)) return false;
            }
        }
        if (P.mode & MF_M_BFS_ONLY) return true;
        // worklist and termination test (built during the BFS when data-driven)
        if (!P.data_driven) {
            phase_worklist(P, sh);
            if (!grid_sync(P, H_WL, sh)) return false;
        }
        if (sh.d.status != MF_ST_RUNNING) break;
        // discharge rounds, then remove-invalid-edges
        do {
            if (P.pull) phase_discharge<true>(P, sh);
            else phase_discharge<false>(P, sh);
            flush_acc(P, sh, 1);
            if (!grid_sync(P, H_DIS, sh)) return false;
        } while (sh.d.dis_more);
        if (P.fix_steep) {
            if (P.pull) phase_fix<true>(P, sh);
            else phase_fix<false>(P, sh);
            flush_acc(P, sh, 2);
            if (!grid_sync(P, H_ITER, sh)) return false;
        }
    }
    if (sh.d.status == MF_ST_ERROR) return true;
    if (!(P.mode & MF_M_NO_VALUE)) phase_value(P);
    return grid_sync(P, H_FINAL, sh);
}

__global__ void __launch_bounds__(MF_BLOCK, 2) mf_solve_kernel(MfParams P)
{
    __shared__ Sh sh;
    if (threadIdx.x == 0) {
        g_vb = blockIdx.x;
        g_vn = gridDim.x;
    }
    __syncthreads();
    solve_instance(P, sh);
}

// Barrier of one group of CTAs (no hook): w[0] arrivals, w[1] generation.
__device__ bool group_sync(unsigned *w, unsigned &gen_local, unsigned long long wait_ns, int *abort)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned gen = gen_local;
        __threadfence();
        if (atomicAdd(w, 1u) + 1u == (unsigned)vn()) {
            atomicExch(w, 0u);
            __threadfence();
            st_release(w + 1, gen + 1u);
        } else {
            unsigned long long t0 = 0;
            unsigned spins = 0;
            while (ld_acquire(w + 1) == gen) {
                ++spins;
                if (spins > 64) __nanosleep(spins > 4096 ? 200 : 32);
                if ((spins & 31u) == 0) {
                    unsigned long long now = gtimer();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > wait_ns) {
                        atomicExch(abort, 1);
                        good = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        gen_local = gen + 1u;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Many instances in one persistent launch: the grid is cut into groups of
// gsize CTAs; each group takes the next instance from a shared queue (the host
// orders it largest first) and runs its whole solve, then takes another.
// gstate holds, per group, 32 words: w[0] arrivals, w[1] generation, w[2] the
// instance the group's first CTA took.
__global__ void __launch_bounds__(MF_BLOCK, 2) mf_multi_kernel(const MfParams *__restrict__ plist, int count,
                                                               int gsize, unsigned *gstate, unsigned *head,
                                                               unsigned long long wait_ns, int *abort)
{
    __shared__ Sh sh;
    __shared__ unsigned ggen;
    const int grp = blockIdx.x / gsize;
    unsigned *gw = gstate + 32 * grp;
    if (threadIdx.x == 0) {
        g_vb = blockIdx.x % gsize;
        g_vn = gsize;
        ggen = ld_acquire(gw + 1);
    }
    __syncthreads();
    for (;;) {
        if (vb() == 0 && threadIdx.x == 0) gw[2] = atomicAdd(head, 1u);
        if (!group_sync(gw, ggen, wait_ns, abort)) return;
        const int i = (int)__ldcg(gw + 2);
        if (i >= count) return;
        if (!solve_instance(plist[i], sh)) {
            atomicExch(abort, 1);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// Auxiliary kernels (state load/readback, checks, queries)
// ---------------------------------------------------------------------------

__global__ void k_cf_reset(MfParams P)
{
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < P.g.slot_cap;
         x += (long long)gridDim.x * blockDim.x)
        P.cf[x] = P.g.cap[x];
}

struct FlowItems {
    long long count;
    const int32_t *u, *v, *f;
    int apply;
};

__global__ void k_set_flow(MfParams P, FlowItems F, long long *bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < F.count;
         i += (long long)gridDim.x * blockDim.x) {
        int u = F.u[i], v = F.v[i], f = F.f[i];
        if (u < 0 || u >= P.g.n || v < 0 || v >= P.g.n || u == v) {
            atomicAdd((unsigned long long *)bad, 1ull);
            continue;
        }
        int x = find_slot(P, u, v);
        if (x < 0 || f < 0 || f > P.g.cap[x]) {
            atomicAdd((unsigned long long *)bad, 1ull);
            continue;
        }
        if (F.apply && f > 0) {
            atomicSub(P.cf + x, f);
            atomicAdd(P.cf + P.g.rev[x], f);
        }
    }
}

// K8: e(v) = sum over v's slots of c_f - c.
__global__ void k_excess(MfParams P, long long *mismatch)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < P.g.n;
         v += (long long)gridDim.x * blockDim.x) {
        int r0 = P.g.off[v], d = P.g.deg[v];
        long long s = 0;
        for (int j = 0; j < d; ++j) s += (long long)P.cf[r0 + j] - (long long)P.g.cap[r0 + j];
        if (mismatch) {
            if (s != P.e[v]) atomicAdd((unsigned long long *)mismatch, 1ull);
        } else {
            P.e[v] = s;
        }
    }
}

__global__ void k_check(MfParams P, long long *out)
{
    const int n = P.g.n;
    long long pair_bad = 0, cross = 0, act = 0, cut = 0, val = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int r0 = P.g.off[v], d = P.g.deg[v];
        int hv = P.h[v];
        for (int j = 0; j < d; ++j) {
            int x = r0 + j, y = P.g.rev[x];
            long long lhs = (long long)P.cf[x] + P.cf[y];
            long long rhs = (long long)P.g.cap[x] + P.g.cap[y];
            if (P.cf[x] < 0 || lhs != rhs || P.g.pcap[x] != rhs || P.g.dst[y] != (int)v || P.g.rev[y] != x) ++pair_bad;
            if (hv == n && P.h[P.g.dst[x]] < n) {
                cut += P.g.cap[x];
                if (P.cf[x] > 0) ++cross;
            }
        }
        if ((int)v != P.sink && (int)v != P.source && P.e[v] > 0 && hv < n) ++act;
        if ((int)v != P.source && hv < n) val += P.e[v];
    }
    atomicAdd((unsigned long long *)&out[0], (unsigned long long)pair_bad);
    atomicAdd((unsigned long long *)&out[2], (unsigned long long)cross);
    atomicAdd((unsigned long long *)&out[3], (unsigned long long)act);
    atomicAdd((unsigned long long *)&out[4], (unsigned long long)cut);
    atomicAdd((unsigned long long *)&out[5], (unsigned long long)val);
}

__global__ void k_side(MfParams P, uint8_t *side)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < P.g.n;
         v += (long long)gridDim.x * blockDim.x)
        side[v] = (P.h[v] == P.g.n) ? 1 : 0;
}

__global__ void k_cut(MfParams P, long long *out)
{
    const int n = P.g.n;
    const int lane = threadIdx.x & 31;
    long long cut = 0;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        if (P.h[w] != n) continue;
        int r0 = P.g.off[w], d = P.g.deg[w];
        for (int j = lane; j < d; j += 32)
            if (P.h[P.g.dst[r0 + j]] < n) cut += P.g.cap[r0 + j];
    }
    cut = warp_sum_ll(cut);
    if (lane == 0 && cut) atomicAdd((unsigned long long *)out, (unsigned long long)cut);
}

__global__ void k_reverse_cf(MfParams P, const int32_t *in, int32_t *out)
{
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < P.g.slot_cap;
         x += (long long)gridDim.x * blockDim.x)
        out[x] = in[P.g.rev[x]];
}

// pcap = c(u, v) + c(v, u) on every used slot, from cap and rev (the pair sum
// a parked state does not keep).  One warp per row.
__global__ void k_pcap(MfParams P)
{
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < P.g.n; u += nw) {
        const int r0 = P.g.off[u], d = P.g.deg[u];
        for (int j = lane; j < d; j += 32) {
            const int x = r0 + j;
            P.g.pcap[x] = P.g.cap[x] + P.g.cap[P.g.rev[x]];
        }
    }
}

__global__ void k_rowid(MfParams P, int32_t *rowid)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < P.g.n;
         v += (long long)gridDim.x * blockDim.x) {
        int r0 = P.g.off[v], d = P.g.deg[v], end = P.g.off[v + 1];
        for (int x = r0; x < end; ++x) rowid[x] = x < r0 + d ? (int)v : -1;
    }
}

__global__ void k_negate(long long *e, int n)
{
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
        e[v] = -e[v];
}

// ---- device-side rebuild of the layout (rows grow; nothing moves to the host) ----

// New reserved size of every row: used slots + pending insertions + slack.
__global__ void k_row_capacity(MfParams P, float slack_factor, int slack_min, long long *cap_out)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < P.g.n;
         u += (long long)gridDim.x * blockDim.x) {
        long long need = (long long)P.g.deg[u] + P.sc.ins_need[u];
        double want = (double)need * (double)slack_factor;
        long long sl = (long long)want;
        if ((double)sl < want) ++sl;
        if (sl < slack_min) sl = slack_min;
        if (sl > (1 << 24)) sl = 1 << 24;
        cap_out[u] = (need + sl + MF_ROW_ALIGN - 1) / MF_ROW_ALIGN * MF_ROW_ALIGN;   // rows stay 16-byte aligned
    }
}

// Exclusive scan of n int64 values in place, in three passes: every CTA scans
// its tile of MF_SCAN_TILE values and leaves the tile's total in part[]; one CTA
// scans the totals; every CTA adds its tile's offset.  a[n] gets the total.
constexpr int kScanThreads = 1024, kScanPer = MF_SCAN_TILE / kScanThreads;

__device__ __forceinline__ long long block_exclusive_scan(long long x, long long *warp_sums, long long &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        const long long ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        long long wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_sums[lane] = wi - ws;              // exclusive offset of each warp
        if (lane == 31) warp_sums[32] = wi;     // the CTA's total
    }
    __syncthreads();
    total = warp_sums[32];
    const long long r = warp_sums[w] + incl - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(long long *a, long long n, long long *part)
{
    __shared__ long long ws[33];
    const long long base = (long long)blockIdx.x * MF_SCAN_TILE + (long long)threadIdx.x * kScanPer;
    long long v[kScanPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? a[base + k] : 0;
        sum += v[k];
    }
    long long total;
    long long run = block_exclusive_scan(sum, ws, total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) a[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile totals (any count), total into part[nt].
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(long long *part, long long nt)
{
    __shared__ long long ws[33];
    long long carry = 0;
    for (long long b0 = 0; b0 < nt; b0 += blockDim.x) {
        const long long i = b0 + threadIdx.x;
        const long long x = i < nt ? part[i] : 0;
        long long total;
        const long long r = block_exclusive_scan(x, ws, total);
        if (i < nt) part[i] = carry + r;
        carry += total;
    }
    if (threadIdx.x == 0) part[nt] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(long long *a, long long n, const long long *part,
                                                            long long nt)
{
    const long long off = part[blockIdx.x];
    const long long base = (long long)blockIdx.x * MF_SCAN_TILE;
    for (int k = threadIdx.x; k < MF_SCAN_TILE; k += blockDim.x)
        if (base + k < n) a[base + k] += off;
    if (blockIdx.x == 0 && threadIdx.x == 0) a[n] = part[nt];
}

struct MoveOut {
    const long long *noff;   // new row starts (int64, n + 1)
    int32_t *off, *dst, *cf, *cap, *rev, *pcap;   // new arrays
    long long slot_cap;
    int2 *items;             // pieces of the long rows: (row, first slot of the piece)
    unsigned *nitems;        // their number
};

// New slot y of row u at position j: the old slot's values when j < d (the
// reverse index of slot (u, v) moves with row v: new_rev = new_off[v] + (rev -
// old_off[v])), else an empty slot (dst = u, no capacity, rev = itself).
__device__ __forceinline__ void move_slot(const MfParams &P, const MoveOut &M, int u, int o0, int d, int j,
                                          long long y)
{
    if (j < d) {
        const int x = o0 + j;
        const int v = __ldcs(P.g.dst + x);
        const int cf = __ldcs(P.g.cf + x), cap = __ldcs(P.g.cap + x), pc = __ldcs(P.g.pcap + x);
        const int rv = __ldcs(P.g.rev + x);
        const int rn = (int)__ldg(M.noff + v) + (rv - __ldg(P.g.off + v));
        M.dst[y] = v;
        M.cf[y] = cf;
        M.cap[y] = cap;
        M.pcap[y] = pc;
        M.rev[y] = rn;
    } else {
        M.dst[y] = u;
        M.cf[y] = 0;
        M.cap[y] = 0;
        M.pcap[y] = 0;
        M.rev[y] = (int)y;
    }
}

// Rows longer than MF_MOVE_PIECE slots (new size) become pieces of that many
// slots, listed once the new sizes are known.
__global__ void k_move_items(MfParams P, MoveOut M)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < P.g.n;
         u += (long long)gridDim.x * blockDim.x) {
        const long long S = M.noff[u + 1] - M.noff[u];
        if (S <= MF_MOVE_PIECE) continue;
        const int np = (int)((S + MF_MOVE_PIECE - 1) / MF_MOVE_PIECE);
        const unsigned at = atomicAdd(M.nitems, (unsigned)np);
        for (int k = 0; k < np; ++k) M.items[at + k] = make_int2((int)u, k * MF_MOVE_PIECE);
    }
}

// Copy every row to its new place.  Warps take either 32 consecutive rows, of
// which they copy the rows of at most MF_MOVE_PIECE slots as one concatenated
// range (each lane finds the row that owns its slot), or one piece of a long
// row; each lane moves kMv slots per step, so a step keeps kMv independent
// load chains in flight per lane.
constexpr int kMv = 4;
__global__ void k_move_rows(MfParams P, MoveOut M)
{
    const int lane = threadIdx.x & 31;
    const long long nblk = ((long long)P.g.n + 31) >> 5;
    const long long nw = nblk + *(volatile unsigned *)M.nitems;
    for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw;
         w += ((long long)gridDim.x * blockDim.x) >> 5) {
        if (w >= nblk) {
            const int2 it = M.items[w - nblk];
            const int u = it.x;
            const long long n0 = M.noff[u];
            const int S = (int)(M.noff[u + 1] - n0);
            const int o0 = P.g.off[u], d = P.g.deg[u];
            const int end = it.y + MF_MOVE_PIECE < S ? it.y + MF_MOVE_PIECE : S;
            for (int jb = it.y; jb < end; jb += 32 * kMv) {
#pragma unroll
                for (int r = 0; r < kMv; ++r) {
                    const int j = jb + r * 32 + lane;
                    if (j < end) move_slot(P, M, u, o0, d, j, n0 + j);
                }
            }
            continue;
        }
        const int u0 = (int)(w << 5);
        const int u = u0 + lane;
        const bool ok = u < P.g.n;
        const long long n0 = ok ? M.noff[u] : 0;
        const int S = ok ? (int)(M.noff[u + 1] - n0) : 0;
        const int Ss = S <= MF_MOVE_PIECE ? S : 0;      // long rows go by pieces
        const int o0 = ok ? P.g.off[u] : 0, d = ok ? P.g.deg[u] : 0;
        if (ok) M.off[u] = (int)n0;
        int incl = Ss;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - Ss;
        const int T = __shfl_sync(0xffffffffu, incl, 31);
        for (int kb = 0; kb < T; kb += 32 * kMv) {        // the same trip count in every lane
#pragma unroll
            for (int r = 0; r < kMv; ++r) {
                const int k = kb + r * 32 + lane;
                int owner = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const int cand = owner + st;
                    const int ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                    if (cand < 32 && ec <= k) owner = cand;
                }
                const long long rn0 = __shfl_sync(0xffffffffu, n0, owner);
                const int ro = __shfl_sync(0xffffffffu, o0, owner);
                const int rd_ = __shfl_sync(0xffffffffu, d, owner);
                const int re = __shfl_sync(0xffffffffu, excl, owner);
                if (k < T) move_slot(P, M, u0 + owner, ro, rd_, k - re, rn0 + (k - re));
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) M.off[P.g.n] = (int)M.noff[P.g.n];
}

__global__ void k_clear_need(MfParams P)
{
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < P.g.n;
         u += (long long)gridDim.x * blockDim.x)
        P.sc.ins_need[u] = 0;
}

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? MAXFLOW_OK : MAXFLOW_ERR_CUDA; }

}  // namespace

// Dynamic shared memory per CTA of the persistent kernels: as much as still
// lets two CTAs share an SM (the register budget allows two).  Computed once per
// device, with that device current; the kernels' attributes are set to allow it.
int mf_stage_bytes(int device, int *bytes)
{
    static std::mutex mu;
    static int cache[64];
    static bool init = false;
    std::lock_guard<std::mutex> lock(mu);
    if (!init) {
        for (int &x : cache) x = -1;
        init = true;
    }
    if (device < 0 || device >= 64) return MAXFLOW_ERR_INVALID;
    if (cache[device] < 0) {
        cudaFuncAttributes a1{}, a2{};
        int smem_sm = 0, reserved = 0, optin = 0;
        if (cudaFuncGetAttributes(&a1, mf_solve_kernel) != cudaSuccess ||
            cudaFuncGetAttributes(&a2, mf_multi_kernel) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
            return MAXFLOW_ERR_CUDA;
        const long long stat = (long long)(a1.sharedSizeBytes > a2.sharedSizeBytes ? a1.sharedSizeBytes
                                                                                   : a2.sharedSizeBytes);
        long long b = (long long)smem_sm / 2 - reserved - stat;
        if (b > (long long)optin - stat) b = (long long)optin - stat;
        b &= ~255ll;
        if (b < 0) b = 0;
        if (cudaFuncSetAttribute(mf_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) != cudaSuccess ||
            cudaFuncSetAttribute(mf_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) != cudaSuccess)
            return MAXFLOW_ERR_CUDA;
        cudaFuncSetAttribute(mf_solve_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(mf_multi_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaGetLastError();
        cache[device] = (int)b;
    }
    *bytes = cache[device];
    return MAXFLOW_OK;
}

int mf_max_coresident_blocks(int device, int *per_sm, int *num_sms, int dyn_bytes)
{
    int k = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, mf_solve_kernel, MF_BLOCK, (size_t)dyn_bytes) != cudaSuccess)
        return MAXFLOW_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    *per_sm = k;
    *num_sms = sms;
    return k > 0 ? MAXFLOW_OK : MAXFLOW_ERR_CUDA;
}

int mf_launch_multi(const MfParams *plist_dev, int count, int gsize, int grid, unsigned *gstate, unsigned *head,
                    unsigned long long wait_ns, int *abort, void *stream, int stage_bytes)
{
    void *args[] = {(void *)&plist_dev, &count, &gsize, &gstate, &head, &wait_ns, &abort};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)mf_multi_kernel, dim3(grid), dim3(MF_BLOCK), args,
                                                (size_t)stage_bytes, (cudaStream_t)stream);
    return cuda_rc(e);
}

int mf_launch(const MfParams &p, int grid, void *stream)
{
    MfParams q = p;
    void *args[] = {&q};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)mf_solve_kernel, dim3(grid), dim3(MF_BLOCK), args,
                                                (size_t)p.stage_slots * sizeof(int), (cudaStream_t)stream);
    return cuda_rc(e);
}

int mf_launch_aux(int which, const MfParams &p, void *stream, long long *dev_out, const void *extra)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int B = 256;
    long long nv = p.g.n, ns = p.g.slot_cap;
    int gv = (int)((nv + B - 1) / B);
    int gs = (int)((ns + B - 1) / B);
    if (gv > 65535) gv = 65535;
    if (gs > 65535) gs = 65535;
    if (gv < 1) gv = 1;
    if (gs < 1) gs = 1;
    switch (which) {
    case MF_AUX_SET_CF_RESET:
        k_cf_reset<<<gs, B, 0, st>>>(p);
        break;
    case MF_AUX_SET_FLOW: {
        const FlowItems *f = (const FlowItems *)extra;
        int g = (int)((f->count + B - 1) / B);
        if (g < 1) g = 1;
        if (g > 65535) g = 65535;
        k_set_flow<<<g, B, 0, st>>>(p, *f, dev_out);
        break;
    }
    case MF_AUX_EXCESS:
        k_excess<<<gv, B, 0, st>>>(p, dev_out);
        break;
    case MF_AUX_CHECK:
        k_check<<<gv, B, 0, st>>>(p, dev_out);
        if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
        k_excess<<<gv, B, 0, st>>>(p, dev_out + 1);
        break;
    case MF_AUX_SIDE:
        k_side<<<gv, B, 0, st>>>(p, (uint8_t *)extra);
        break;
    case MF_AUX_CUT: {
        int g = (int)((nv * 32 + B - 1) / B);
        if (g > 65535) g = 65535;
        if (g < 1) g = 1;
        k_cut<<<g, B, 0, st>>>(p, dev_out);
        break;
    }
    case MF_AUX_REVERSE_CF: {
        const int32_t *const *io = (const int32_t *const *)extra;
        k_reverse_cf<<<gs, B, 0, st>>>(p, io[0], (int32_t *)io[1]);
        break;
    }
    case MF_AUX_DUMP:
        k_rowid<<<gv, B, 0, st>>>(p, (int32_t *)extra);
        break;
    case MF_AUX_NEGATE_E:
        k_negate<<<gv, B, 0, st>>>(p.e, p.g.n);
        break;
    case MF_AUX_PCAP: {
        long long g = (nv * 32 + B - 1) / B;
        k_pcap<<<(int)(g > 65535 ? 65535 : (g < 1 ? 1 : g)), B, 0, st>>>(p);
        break;
    }
    default:
        return MAXFLOW_ERR_INVALID;
    }
    return cuda_rc(cudaGetLastError());
}

int mf_set_flow_items(const MfParams &p, void *stream, long long *dev_bad, long long count,
                                  const int32_t *du, const int32_t *dv, const int32_t *df, int apply)
{
    FlowItems f{count, du, dv, df, apply};
    return mf_launch_aux(MF_AUX_SET_FLOW, p, stream, dev_bad, &f);
}

int mf_rebuild_capacity(const MfParams &p, void *stream, float slack_factor, int slack_min, long long *noff)
{
    cudaStream_t st = (cudaStream_t)stream;
    int g = (int)((p.g.n + 255) / 256);
    if (g > 65535) g = 65535;
    if (g < 1) g = 1;
    k_row_capacity<<<g, 256, 0, st>>>(p, slack_factor, slack_min, noff);
    if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
    // the tile totals sit behind the n + 1 row starts (mf_rebuild_scratch)
    const long long nt = mf_scan_tiles(p.g.n);
    long long *part = noff + p.g.n + 1;
    k_scan_tiles<<<(int)nt, kScanThreads, 0, st>>>(noff, p.g.n, part);
    if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
    k_scan_parts<<<1, kScanThreads, 0, st>>>(part, nt);
    if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
    k_scan_add<<<(int)nt, kScanThreads, 0, st>>>(noff, p.g.n, part, nt);
    return cuda_rc(cudaGetLastError());
}

int mf_rebuild_move(const MfParams &p, void *stream, const long long *noff, int32_t *off, int32_t *dst, int32_t *cf,
                    int32_t *cap, int32_t *rev, int32_t *pcap, long long slot_cap, int2 *items, unsigned *nitems)
{
    cudaStream_t st = (cudaStream_t)stream;
    MoveOut M{noff, off, dst, cf, cap, rev, pcap, slot_cap, items, nitems};
    if (cudaMemsetAsync(nitems, 0, sizeof(unsigned), st) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    int gi = (int)((p.g.n + 255) / 256);
    if (gi > 65535) gi = 65535;
    if (gi < 1) gi = 1;
    k_move_items<<<gi, 256, 0, st>>>(p, M);
    if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
    // a persistent grid: warps stride over the blocks of 32 rows, then the pieces
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MAXFLOW_ERR_CUDA;
    k_move_rows<<<sms * 8, 256, 0, st>>>(p, M);
    if (cudaGetLastError() != cudaSuccess) return MAXFLOW_ERR_CUDA;
    int gv = (int)((p.g.n + 255) / 256);
    if (gv > 65535) gv = 65535;
    if (gv < 1) gv = 1;
    k_clear_need<<<gv, 256, 0, st>>>(p);
    return cuda_rc(cudaGetLastError());
}

// ---- scheduler features of a batch (one CTA) ----
__global__ void __launch_bounds__(256) k_features(MfFeatIn F, float *out)
{
    __shared__ float red[4][8];
    float ts = 0.f, tt = 0.f, zero = 0.f, capsum = 0.f;
    for (long long i = threadIdx.x; i < F.count; i += blockDim.x) {
        const int u = F.bu[i], v = F.bv[i], c = F.bc[i];
        ts += (u == F.s || v == F.s) ? 1.f : 0.f;
        tt += (u == F.t || v == F.t) ? 1.f : 0.f;
        zero += c == 0 ? 1.f : 0.f;
        capsum += (float)c;
    }
    float vals[4] = {ts, tt, zero, capsum};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float x = vals[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[k][w] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < 4; ++k)
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot[k] += red[k][q];
        const float B = (float)F.count, m = (float)(F.m > 0 ? F.m : 1), n = (float)F.n;
        const float inv = F.count > 0 ? 1.f / B : 0.f;
        out[0] = log2f(1.f + B) / 20.f;
        out[1] = fminf(B / m, 1.f);
        out[2] = log2f(n) / 24.f;
        out[3] = log2f(1.f + m) / 28.f;
        out[4] = (m / n) / 16.f;
        out[5] = tot[0] * inv;
        out[6] = tot[1] * inv;
        out[7] = tot[2] * inv;
        out[8] = F.count > 0 && F.mean_cap > 0.f ? fminf(tot[3] * inv / F.mean_cap, 4.f) / 4.f : 0.f;
        for (int k = 0; k < 6; ++k) out[9 + k] = F.host[k];
        out[15] = 1.f;
    }
}

int mf_features(const MfFeatIn &f, float *out_dev, void *stream)
{
    k_features<<<1, 256, 0, (cudaStream_t)stream>>>(f, out_dev);
    return cuda_rc(cudaGetLastError());
}
