// C ABI of the GB300 dynamic max-flow library (see include/maxflow.h).
//
// A context owns one residual Bi-CSR in device memory and runs every solve
// as one cooperative launch of the persistent kernel in solver.cu.  The host
// side only validates arguments, moves inputs and outputs, sizes scratch
// buffers and, when an insertion finds a row without spare slots, rebuilds
// the layout (keeping flows and excesses) and repeats the update.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/maxflow.h"
#include "mf_internal.h"

// Kernels this library has launched in the process (maxflow_kernel_launches).
static std::atomic<long long> g_kernel_launches{0};

// Also called by noalloc.cu and mlp.cu for their own launches.
void mf_note_launches(int kernels) { g_kernel_launches.fetch_add(kernels, std::memory_order_relaxed); }

// The status of a launch helper that starts `kernels` kernels, counted when it succeeded.
static inline int counted(int rc, int kernels)
{
    if (rc == MAXFLOW_OK) mf_note_launches(kernels);
    return rc;
}

struct maxflow_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    maxflow_ctx *ckpt = nullptr;      // maxflow_checkpoint's saved copy (a clone), or none
    maxflow_opts opt{};
    int32_t n = 0, s = 0, t = 0;
    int32_t kernel_cycles = 1;
    int32_t rounds = 1;
    int32_t small_deg = MF_SMALL_DEG, hub_deg = MF_HUB_DEG, bfs_hub = MF_BFS_HUB;
    int32_t group_deg = MF_HUB_DEG;   // rows above this get a CTA: a quarter of the snapshot buffer
    int32_t bu_alpha = MF_BU_ALPHA, bu_beta = MF_BU_BETA;
    // batched launches started from this context (parameter list, group state)
    MfParams *multi_plist = nullptr;
    unsigned *multi_gstate = nullptr;
    int multi_cap = 0;
    int grid = 1, per_sm = 1, sms = 1;
    int32_t stage_slots = 0;      // dynamic shared memory of the solve launches, in ints
    int32_t requeue = 1;          // discharge rounds re-queue vertices still active after their cycles
    int32_t cycle_div = 0;        // > 0: long rows get max(kernel_cycles, deg / cycle_div) cycles
    int32_t tail_slots = 0;       // BFS frontiers of at most this many slots run in one CTA (0: off)
    MfGraph g{};
    MfScratch sc{};
    MfCtrl *ctrl = nullptr;
    MfCtrl *hctrl = nullptr;      // pinned
    long long *dbuf = nullptr;    // device scratch for aux outputs (16 entries)
    long long *hbuf = nullptr;    // pinned mirror
    int32_t *x_cf = nullptr, *x_cf2 = nullptr, *x_h = nullptr;
    long long *x_e = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;
    bool solved = false;
    int64_t value = 0;
    maxflow_stats_t st{};
    double acc_ms = 0;            // device time of all launches of the current update
    float mean_cap = 0.f;         // mean capacity of the initial edges (scheduler feature)
    double init_ms = 0;           // static solve at init (scheduler feature)
    int64_t init_iters = 0;
    // the last incremental solve (scheduler features): a static re-solve leaves
    // them as they were, so what the features describe does not depend on
    // which kind of action ran last
    int64_t inc_iters = 0, inc_active_first = 0, inc_levels = 0;
    double inc_ms = 0;
    float *feat = nullptr;        // [MF_FEATURES] device
    float *sched_y = nullptr;     // [64] device
    // eviction: the state parked in host memory while the device memory is released
    // (one pinned block, kept after a restore so that the next eviction reuses it)
    bool evicted = false;
    char *park = nullptr;
    size_t park_bytes = 0;
    void *park_map = nullptr;          // the mapping behind `park` when it is huge-page backed
    size_t park_map_bytes = 0;
    int64_t park_slots = 0;
    std::vector<int64_t> park_sizes;   // the device allocations held when evicted
    // the pull part of the dynamic push-pull (its own control block, labels and
    // solve scratch) and the sides of the last cut; allocated on first use
    struct {
        MfCtrl *ctrl = nullptr;
        MfCtrl *hctrl = nullptr;       // pinned
        MfScratch sc{};
        int32_t *h = nullptr;
        uint8_t *side = nullptr;
        int64_t items_for = -1;        // slot capacity sc.bitem was sized for
    } pp;
};

// exported by mlp.cu (C linkage)
extern "C" {
int mlp_forward_device(maxflow_mlp *m, const float *x_dev, int32_t rows, float *y_dev, cudaStream_t st);
int mlp_n_out(const maxflow_mlp *m);
int mlp_n_in(const maxflow_mlp *m);
}

namespace {

struct DeviceGuard {
    int old = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&old) != cudaSuccess) old = -1;
        if (dev >= 0 && dev != old) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (old >= 0) cudaSetDevice(old);
    }
};

void *dalloc(maxflow_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->opt.alloc_user, (void *)c->stream);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) c->allocs.emplace_back(p, bytes);
    return p;
}

void dfree(maxflow_ctx *c, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i) {
        if (c->allocs[i].first == p) {
            size_t b = c->allocs[i].second;
            if (c->opt.free) c->opt.free(p, b, c->opt.alloc_user, (void *)c->stream);
            else cudaFree(p);
            c->allocs.erase(c->allocs.begin() + (long)i);
            return;
        }
    }
}

template <class T>
T *dalloc_n(maxflow_ctx *c, int64_t count)
{
    return (T *)dalloc(c, sizeof(T) * (size_t)(count > 0 ? count : 1));
}

int rc_cuda(cudaError_t e) { return e == cudaSuccess ? MAXFLOW_OK : MAXFLOW_ERR_CUDA; }

#define MF_TRY(expr)                          \
    do {                                      \
        int _rc = (expr);                     \
        if (_rc != MAXFLOW_OK) return _rc;    \
    } while (0)

MfParams base_params(maxflow_ctx *c)
{
    MfParams p{};
    p.g = c->g;
    p.sc = c->sc;
    p.ctrl = c->ctrl;
    p.cf = c->g.cf;
    p.h = c->g.h;
    p.e = c->g.e;
    p.sink = c->t;
    p.source = c->s;
    p.kernel_cycles = c->kernel_cycles;
    p.rounds = c->rounds;
    p.small_deg = c->small_deg;
    p.hub_deg = c->hub_deg;
    p.group_deg = c->group_deg;
    p.bfs_hub = c->bfs_hub;
    p.bu_alpha = c->bu_alpha;
    p.bu_beta = c->bu_beta;
    p.fix_steep = c->opt.fix_steep ? 1 : 0;
    p.data_driven = c->opt.data_driven ? 1 : 0;
    p.pull = 0;
    p.side_root = -1;
    p.test_skip_cta = -1;
    p.stage_slots = c->stage_slots;
    p.requeue = c->requeue;
    p.cycle_div = c->cycle_div;
    p.tail_slots = c->tail_slots;
    p.side = c->pp.side;
    p.max_iters = c->opt.max_iters > 0 ? c->opt.max_iters : 4LL * c->n + 1000;
    double tl = c->opt.time_limit_s > 0 ? c->opt.time_limit_s : 120.0;
    double wl = c->opt.wait_limit_s > 0 ? c->opt.wait_limit_s : 1.0;
    p.time_limit_ns = (unsigned long long)(tl * 1e9);
    p.wait_limit_ns = (unsigned long long)(wl * 1e9);
    return p;
}

// Size the batch scratch for at least `count` updates.
int ensure_batch(maxflow_ctx *c, int64_t count)
{
    if (count <= c->sc.batch_cap && c->sc.hkey) return MAXFLOW_OK;
    int64_t cap = std::max<int64_t>(1024, c->sc.batch_cap);
    while (cap < count) cap *= 2;
    if (cap > (1LL << 29)) return MAXFLOW_ERR_TOO_LARGE;
    int bits = 1;
    while ((1LL << bits) < 2 * cap) ++bits;
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    void *olds[] = {c->sc.hkey, c->sc.hval, c->sc.pkey, c->sc.pval, c->sc.bslot, c->sc.ins_list,
                    c->sc.hused, c->sc.clamp, c->sc.bu, c->sc.bv, c->sc.bc};
    for (void *p : olds) dfree(c, p);
    int64_t hs = 1LL << bits;
    c->sc.hkey = dalloc_n<unsigned long long>(c, hs);
    c->sc.hval = dalloc_n<int32_t>(c, hs);
    c->sc.pkey = dalloc_n<unsigned long long>(c, hs);
    c->sc.pval = dalloc_n<int32_t>(c, hs);
    c->sc.bslot = dalloc_n<int32_t>(c, cap);
    c->sc.ins_list = dalloc_n<int32_t>(c, cap);
    c->sc.hused = dalloc_n<int32_t>(c, cap);
    c->sc.clamp = dalloc_n<int32_t>(c, cap);
    c->sc.bu = dalloc_n<int32_t>(c, cap);
    c->sc.bv = dalloc_n<int32_t>(c, cap);
    c->sc.bc = dalloc_n<int32_t>(c, cap);
    if (!c->sc.hkey || !c->sc.hval || !c->sc.pkey || !c->sc.pval || !c->sc.bslot || !c->sc.ins_list ||
        !c->sc.hused || !c->sc.clamp || !c->sc.bu || !c->sc.bv || !c->sc.bc)
        return MAXFLOW_ERR_OOM;
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.hkey, 0xff, sizeof(unsigned long long) * hs, c->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.hval, 0xff, sizeof(int32_t) * hs, c->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.pkey, 0xff, sizeof(unsigned long long) * hs, c->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.pval, 0xff, sizeof(int32_t) * hs, c->stream)));
    c->sc.batch_cap = cap;
    c->sc.hash_bits = bits;
    return MAXFLOW_OK;
}

void free_graph(maxflow_ctx *c)
{
    void *ps[] = {c->g.off, c->g.deg, c->g.bdeg, c->g.dst, c->g.cf, c->g.cap, c->g.rev, c->g.pcap};
    for (void *p : ps) dfree(c, p);
    c->g.off = c->g.deg = c->g.bdeg = c->g.dst = c->g.cf = c->g.cap = c->g.rev = c->g.pcap = nullptr;
    dfree(c, c->x_cf);
    dfree(c, c->x_cf2);
    c->x_cf = c->x_cf2 = nullptr;
}

// Upload a host layout into freshly allocated slot arrays (vertex arrays kept).
int upload_graph(maxflow_ctx *c, const MfHostGraph &hg)
{
    free_graph(c);
    int64_t S = hg.slot_cap;
    int32_t n = hg.n;
    c->g.n = n;
    c->g.slot_cap = S;
    c->g.off = dalloc_n<int32_t>(c, n + 1);
    c->g.deg = dalloc_n<int32_t>(c, n);
    c->g.bdeg = dalloc_n<int32_t>(c, n);
    c->g.dst = dalloc_n<int32_t>(c, S);
    c->g.cf = dalloc_n<int32_t>(c, S);
    c->g.cap = dalloc_n<int32_t>(c, S);
    c->g.rev = dalloc_n<int32_t>(c, S);
    c->g.pcap = dalloc_n<int32_t>(c, S);
    if (!c->g.off || !c->g.deg || !c->g.bdeg || !c->g.dst || !c->g.cf || !c->g.cap || !c->g.rev || !c->g.pcap)
        return MAXFLOW_ERR_OOM;
    cudaStream_t st = c->stream;
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.off, hg.off, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.deg, hg.deg, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.bdeg, hg.bdeg, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.dst, hg.dst, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.cf, hg.cf, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.cap, hg.cap, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.rev, hg.rev, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st)));
    if (hg.pcap) MF_TRY(rc_cuda(cudaMemcpyAsync(c->g.pcap, hg.pcap, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st)));
    // the host arrays must stay valid until the copies complete
    MF_TRY(rc_cuda(cudaStreamSynchronize(st)));
    dfree(c, c->sc.bitem);
    dfree(c, c->sc.bdefer);
    c->sc.bitem = dalloc_n<int2>(c, (int64_t)n + S / MF_BFS_CHUNK + 64);
    c->sc.bdefer = dalloc_n<int2>(c, (int64_t)n + S / MF_BFS_CHUNK + 64);
    if (!c->sc.bitem || !c->sc.bdefer) return MAXFLOW_ERR_OOM;
    c->st.slot_capacity = S;
    c->st.slots = hg.slots;
    c->st.m_edges = hg.m_merged;
    return MAXFLOW_OK;
}

// Vertex-sized scratch of the solve kernel (frontier, worklists, stamps, lists).
int alloc_vertex_scratch(maxflow_ctx *c)
{
    const int32_t n = c->n;
    c->sc.border = dalloc_n<int32_t>(c, n);
    for (int q = 0; q < 2; ++q)
        for (int b = 0; b < MF_NBIN; ++b) c->sc.wl[q][b] = dalloc_n<int32_t>(c, n);
    c->sc.vmark = dalloc_n<int32_t>(c, n);
    c->sc.fixmark = dalloc_n<int32_t>(c, n);
    c->sc.fixl[0] = dalloc_n<int32_t>(c, n);
    c->sc.fixl[1] = dalloc_n<int32_t>(c, n);
    c->sc.ins_need = dalloc_n<int32_t>(c, n);
    c->sc.blong = dalloc_n<int32_t>(c, n);
    if (!c->sc.border || !c->sc.vmark || !c->sc.fixmark || !c->sc.fixl[0] || !c->sc.fixl[1] || !c->sc.ins_need ||
        !c->sc.blong)
        return MAXFLOW_ERR_OOM;
    for (int q = 0; q < 2; ++q)
        for (int b = 0; b < MF_NBIN; ++b)
            if (!c->sc.wl[q][b]) return MAXFLOW_ERR_OOM;
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.vmark, 0xff, sizeof(int32_t) * n, c->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(c->sc.fixmark, 0xff, sizeof(int32_t) * n, c->stream)));
    return rc_cuda(cudaMemsetAsync(c->sc.ins_need, 0, sizeof(int32_t) * n, c->stream));
}

void choose_grid(maxflow_ctx *c)
{
    int maxg = c->per_sm * c->sms;
    int g = c->opt.grid_blocks;
    if (g <= 0) {
        double want = std::ceil((double)c->g.slot_cap / 8192.0);
        g = (int)std::min<double>(maxg, std::max(2.0, want));
    }
    c->grid = std::max(1, std::min(g, maxg));
    c->st.grid_blocks = c->grid;
    c->st.block_threads = MF_BLOCK;
    c->st.blocks_per_sm = c->per_sm;
}

// The default work split: rows of up to 8 slots get a thread, or up to 4 on a
// sparse graph (at most 8 merged directed edges per vertex: grids, geometric
// and layered graphs), where the rounds are many and short and a warp's
// parallel scan of a 5-8 slot row beats one thread's; then warps up to 512
// slots, 4-warp groups up to a quarter of the snapshot buffer, CTAs above; BFS
// work items for rows of more than 256 slots.
void default_split(maxflow_ctx *c)
{
    const int64_t m = c->st.m_edges;
    c->small_deg = m <= (int64_t)MF_SPARSE_DEG * c->n ? MF_SMALL_DEG_SPARSE : MF_SMALL_DEG;
    c->hub_deg = MF_HUB_DEG;
    c->bfs_hub = MF_BFS_HUB;
    c->group_deg = std::max<int32_t>(c->hub_deg, c->stage_slots / (MF_BLOCK / (32 * MF_GROUP_WARPS)));
}

// The statistics of the solve that just ended become the scheduler's view of
// the last incremental solve.
void note_incremental(maxflow_ctx *c)
{
    c->inc_iters = c->st.iterations;
    c->inc_active_first = c->st.active_first;
    c->inc_levels = c->st.bfs_levels;
    c->inc_ms = c->st.ms_last;
}

void fill_stats(maxflow_ctx *c, const MfCtrl &h, float ms)
{
    maxflow_stats_t &s = c->st;
    s.iterations = h.iters;
    s.bfs_levels = h.bfs_levels;
    s.pushes = h.pushes;
    s.relabels = h.relabels;
    s.steep_fixes = h.steep;
    s.active_first = h.active_first;
    s.active_total = h.active_total;
    // algorithmic bytes of the paper's Bi-CSR (int32 per slot field, int64 excess), counted by the kernel:
    //   BFS: per scanned slot dst + cf + pcap + h[dst] = 16 B; per vertex record read (roots pass: e + h;
    //        bottom-up, unlabelled vertex: h + off + deg) 12 B; per height read in a bottom-up pass 4 B;
    //        per labelled vertex h claim + deg + e + append = 20 B
    //   discharge: per scanned slot in a cycle dst + cf + h[dst] = 12 B; per cycle off + deg + h + e = 20 B;
    //        per push two c_f and two excess read-modify-writes = 48 B
    //   remove-invalid: per slot 12 B; per vertex 20 B; per steep push 48 B
    //   worklist (only when it is a pass of its own, data_driven = 0): e + h + deg per vertex = 16 B
    //   apply: per applied update the record, the slot's cap, cf, pcap and its reverse's pcap
    //        (read-modify-write), rev and the dedup entry = 12 + 8 + 8 + 8 + 8 + 4 + 12 = 60 B;
    //        per slot read by the search or the source row 4 B; per clamp two c_f and two excess RMWs 48 B
    s.bytes_bfs = 16 * h.slots_bfs + 12 * h.verts_bfs + 4 * h.hscan_bfs + 20 * h.lab_bfs;
    s.bytes_discharge = 12 * h.slots_dis + 20 * h.cycles_dis + 48 * h.pushes;
    s.bytes_fix = 12 * h.slots_fix + 20 * h.verts_fix + 48 * h.steep;
    s.bytes_worklist = c->opt.data_driven ? 0 : 16LL * c->n * (h.iters + 1);
    s.bytes_apply = 60 * h.n_apply + 4 * h.slots_apply + 48 * h.clamps_apply;
    s.ms_last = ms;
    s.ms_bfs = h.ns_bfs * 1e-6;
    s.ms_discharge = h.ns_dis * 1e-6;
    s.ms_fix = h.ns_fix * 1e-6;
    s.ms_worklist = h.ns_wl * 1e-6;
    s.ms_apply = h.ns_apply * 1e-6;
    s.ms_kernel = (h.t_exit - h.t_entry) * 1e-6;
    s.ms_update = c->acc_ms;   // run_kernel has added this launch already
    s.us_discharge_cta_rows = h.ns_dis_cta * 1e-3;
    s.us_discharge_warp_rows = h.ns_dis_warp * 1e-3;
    s.us_discharge_thread_rows = h.ns_dis_thread * 1e-3;
    s.discharge_rounds = h.rounds_total;
    s.barriers = h.barriers;
    s.kernel_cycles = c->kernel_cycles;
}

// Launch one solve-kernel run and wait for it.  Returns the kernel's error
// (MF_E_*) in *kerr and its status in *kstatus.
int run_kernel(maxflow_ctx *c, const MfParams &p, int *kerr, int *kstatus)
{
    MF_TRY(rc_cuda(cudaEventRecord(c->ev0, c->stream)));
    MF_TRY(counted(mf_launch(p, c->grid, (void *)c->stream), 1));
    MF_TRY(rc_cuda(cudaEventRecord(c->ev1, c->stream)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->hctrl, c->ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->acc_ms += ms;
    *kerr = (int)c->hctrl->err.w[0];
    *kstatus = c->hctrl->d.status;
    fill_stats(c, *c->hctrl, ms);
    if (*kerr != MF_E_NONE) {
        // a barrier may have been left half-way: reset it for the next launch
        MF_TRY(rc_cuda(cudaMemsetAsync(c->ctrl, 0, 2 * sizeof(MfLine), c->stream)));
        MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    }
    return MAXFLOW_OK;
}

int status_to_rc(int kerr, int kstatus)
{
    if (kerr == MF_E_INVALID) return MAXFLOW_ERR_INVALID;
    if (kerr == MF_E_TOO_LARGE) return MAXFLOW_ERR_TOO_LARGE;
    if (kerr == MF_E_WAIT || kerr == MF_E_INTERNAL) return MAXFLOW_ERR_INTERNAL;
    if (kerr != MF_E_NONE) return MAXFLOW_ERR_INTERNAL;
    if (kstatus == MF_ST_CAP) return MAXFLOW_ERR_NOT_CONVERGED;
    return MAXFLOW_OK;
}

// Run a solve that ends with the value phase; record the value.
int run_solve(maxflow_ctx *c, MfParams p)
{
    c->acc_ms = 0;
    int kerr = 0, kst = 0;
    MF_TRY(run_kernel(c, p, &kerr, &kst));
    int rc = status_to_rc(kerr, kst);
    c->st.solves++;
    if (rc == MAXFLOW_OK || rc == MAXFLOW_ERR_NOT_CONVERGED) {
        c->value = c->hctrl->value;
        c->st.value = c->value;
        c->solved = (rc == MAXFLOW_OK);
    }
    return rc;
}

// Download the used slots as (u, v, cap, cf).
int dump_slots(maxflow_ctx *c, std::vector<int32_t> &su, std::vector<int32_t> &sv, std::vector<int32_t> &scap,
               std::vector<int32_t> &scf, const int32_t *cf_dev)
{
    int64_t S = c->g.slot_cap;
    int32_t *rowid = dalloc_n<int32_t>(c, S);
    if (!rowid) return MAXFLOW_ERR_OOM;
    MfParams p = base_params(c);
    int rc = counted(mf_launch_aux(MF_AUX_DUMP, p, (void *)c->stream, nullptr, rowid), 1);
    std::vector<int32_t> hr((size_t)S), hd((size_t)S), hc((size_t)S), hf((size_t)S);
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(hr.data(), rowid, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(hd.data(), c->g.dst, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(hc.data(), c->g.cap, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(hf.data(), cf_dev, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    dfree(c, rowid);
    if (rc != MAXFLOW_OK) return rc;
    su.clear(); sv.clear(); scap.clear(); scf.clear();
    for (int64_t x = 0; x < S; ++x) {
        if (hr[(size_t)x] < 0) continue;
        su.push_back(hr[(size_t)x]);
        sv.push_back(hd[(size_t)x]);
        scap.push_back(hc[(size_t)x]);
        scf.push_back(hf[(size_t)x]);
    }
    return MAXFLOW_OK;
}

// Grow the rows on the device so that every row has room for its pending
// insertions (ins_need[], left by the kernel that reported the overflow) plus
// fresh slack; flows, capacities and excesses keep their values and the slot
// order inside each row is kept.
int rebuild_device(maxflow_ctx *c)
{
    const int32_t n = c->n;
    MfParams p = base_params(c);
    long long *noff = dalloc_n<long long>(c, mf_rebuild_scratch(n));
    if (!noff) return MAXFLOW_ERR_OOM;
    int rc =
        counted(mf_rebuild_capacity(p, (void *)c->stream, c->opt.slack_factor, c->opt.slack_min, noff), 4);
    long long total = 0;
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(&total, noff + n, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    if (rc == MAXFLOW_OK && total >= (long long)INT32_MAX - 1) rc = MAXFLOW_ERR_TOO_LARGE;
    int32_t *off = nullptr, *dst = nullptr, *cf = nullptr, *cap = nullptr, *rev = nullptr, *pcap = nullptr;
    int2 *items = nullptr;     // pieces of the long rows for the copy; the last entry holds their count
    if (rc == MAXFLOW_OK) {
        items = dalloc_n<int2>(c, mf_move_items(total) + 1);
        off = dalloc_n<int32_t>(c, (int64_t)n + 1);
        dst = dalloc_n<int32_t>(c, total);
        cf = dalloc_n<int32_t>(c, total);
        cap = dalloc_n<int32_t>(c, total);
        rev = dalloc_n<int32_t>(c, total);
        pcap = dalloc_n<int32_t>(c, total);
        if (!items || !off || !dst || !cf || !cap || !rev || !pcap) rc = MAXFLOW_ERR_OOM;
    }
    if (rc == MAXFLOW_OK)
        rc = counted(mf_rebuild_move(p, (void *)c->stream, noff, off, dst, cf, cap, rev, pcap, total, items,
                                     reinterpret_cast<unsigned *>(items + mf_move_items(total))),
                     3);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    dfree(c, items);
    if (rc != MAXFLOW_OK) {
        int32_t *tmp[] = {off, dst, cf, cap, rev, pcap};
        for (int32_t *q : tmp) dfree(c, q);
        dfree(c, noff);
        return rc;
    }
    int32_t *old[] = {c->g.off, c->g.dst, c->g.cf, c->g.cap, c->g.rev, c->g.pcap};
    for (int32_t *q : old) dfree(c, q);
    dfree(c, noff);
    c->g.off = off;
    c->g.dst = dst;
    c->g.cf = cf;
    c->g.cap = cap;
    c->g.rev = rev;
    c->g.pcap = pcap;
    c->g.slot_cap = total;
    dfree(c, c->x_cf);
    dfree(c, c->x_cf2);
    c->x_cf = c->x_cf2 = nullptr;
    dfree(c, c->sc.bitem);
    dfree(c, c->sc.bdefer);
    c->sc.bitem = dalloc_n<int2>(c, (int64_t)n + total / MF_BFS_CHUNK + 64);
    c->sc.bdefer = dalloc_n<int2>(c, (int64_t)n + total / MF_BFS_CHUNK + 64);
    if (!c->sc.bitem || !c->sc.bdefer) return MAXFLOW_ERR_OOM;
    c->st.slot_capacity = total;
    c->st.rebuilds++;
    choose_grid(c);
    return MAXFLOW_OK;
}

int check_host_batch(maxflow_ctx *c, const maxflow_batch *b)
{
    for (int64_t i = 0; i < b->count; ++i) {
        int32_t u = b->u[i], v = b->v[i], w = b->new_cap[i];
        if (u < 0 || u >= c->n || v < 0 || v >= c->n || w < 0) return MAXFLOW_ERR_INVALID;
    }
    return MAXFLOW_OK;
}

// Apply (and optionally solve) a batch.
int do_batch(maxflow_ctx *c, const maxflow_batch *b, int mode)
{
    c->acc_ms = 0;
    if (!b || b->count < 0) return MAXFLOW_ERR_INVALID;
    if (b->count > 0 && (!b->u || !b->v || !b->new_cap)) return MAXFLOW_ERR_INVALID;
    if (!b->on_device) MF_TRY(check_host_batch(c, b));
    MF_TRY(ensure_batch(c, b->count));
    MfParams p = base_params(c);
    p.mode = mode;
    p.bcount = b->count;
    if (b->count > 0) {
        if (b->on_device) {
            p.bu = b->u;
            p.bv = b->v;
            p.bc = b->new_cap;
        } else {
            size_t bytes = sizeof(int32_t) * (size_t)b->count;
            MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bu, b->u, bytes, cudaMemcpyHostToDevice, c->stream)));
            MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bv, b->v, bytes, cudaMemcpyHostToDevice, c->stream)));
            MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bc, b->new_cap, bytes, cudaMemcpyHostToDevice, c->stream)));
            p.bu = c->sc.bu;
            p.bv = c->sc.bv;
            p.bc = c->sc.bc;
        }
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        int kerr = 0, kst = 0;
        MF_TRY(run_kernel(c, p, &kerr, &kst));
        if (kerr == MF_E_OVERFLOW) {
            if (attempt == 1) return MAXFLOW_ERR_INTERNAL;
            MF_TRY(rebuild_device(c));
            p.g = c->g;
            p.sc = c->sc;
            p.cf = c->g.cf;
            continue;
        }
        int rc = status_to_rc(kerr, kst);
        if (mode & MF_M_SOLVE) {
            c->st.solves++;
            if (rc == MAXFLOW_OK || rc == MAXFLOW_ERR_NOT_CONVERGED) {
                c->value = c->hctrl->value;
                c->st.value = c->value;
                c->solved = (rc == MAXFLOW_OK);
            }
        } else if (rc == MAXFLOW_OK) {
            c->solved = false;
        }
        if (rc == MAXFLOW_OK || rc == MAXFLOW_ERR_NOT_CONVERGED) c->st.updates++;
        return rc;
    }
    return MAXFLOW_ERR_INTERNAL;
}

// Parameter list and barrier words of a multi-instance launch, for `count` instances.
int ensure_multi(maxflow_ctx *c, int32_t count)
{
    const int maxg = c->per_sm * c->sms;
    if (c->multi_cap < count || !c->multi_plist) {
        dfree(c, c->multi_plist);
        dfree(c, c->multi_gstate);
        c->multi_cap = std::max(count, 64);
        c->multi_plist = (MfParams *)dalloc(c, sizeof(MfParams) * (size_t)c->multi_cap);
        c->multi_gstate = dalloc_n<unsigned>(c, 32 * (int64_t)(maxg + 2));
        if (!c->multi_plist || !c->multi_gstate) return MAXFLOW_ERR_OOM;
    }
    return MAXFLOW_OK;
}

// The pull part's control block, labels, solve scratch and the cut sides.
int ensure_pp(maxflow_ctx *c)
{
    auto &q = c->pp;
    const int32_t n = c->n;
    if (!q.hctrl) MF_TRY(rc_cuda(cudaMallocHost((void **)&q.hctrl, sizeof(MfCtrl))));
    if (!q.ctrl) {
        q.ctrl = (MfCtrl *)dalloc(c, sizeof(MfCtrl));
        q.h = dalloc_n<int32_t>(c, n);
        q.side = (uint8_t *)dalloc(c, (size_t)n);
        q.sc.border = dalloc_n<int32_t>(c, n);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < MF_NBIN; ++b) q.sc.wl[a][b] = dalloc_n<int32_t>(c, n);
        q.sc.vmark = dalloc_n<int32_t>(c, n);
        q.sc.fixmark = dalloc_n<int32_t>(c, n);
        q.sc.fixl[0] = dalloc_n<int32_t>(c, n);
        q.sc.fixl[1] = dalloc_n<int32_t>(c, n);
        bool ok = q.ctrl && q.h && q.side && q.sc.border && q.sc.vmark && q.sc.fixmark && q.sc.fixl[0] && q.sc.fixl[1];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < MF_NBIN; ++b) ok = ok && q.sc.wl[a][b];
        if (!ok) return MAXFLOW_ERR_OOM;
        MF_TRY(rc_cuda(cudaMemsetAsync(q.ctrl, 0, sizeof(MfCtrl), c->stream)));
        MF_TRY(rc_cuda(cudaMemsetAsync(q.sc.vmark, 0xff, sizeof(int32_t) * (size_t)n, c->stream)));
        MF_TRY(rc_cuda(cudaMemsetAsync(q.sc.fixmark, 0xff, sizeof(int32_t) * (size_t)n, c->stream)));
    }
    if (q.items_for != c->g.slot_cap) {
        dfree(c, q.sc.bitem);
        dfree(c, q.sc.bdefer);
        q.sc.bitem = dalloc_n<int2>(c, (int64_t)n + c->g.slot_cap / MF_BFS_CHUNK + 64);
        q.sc.bdefer = dalloc_n<int2>(c, (int64_t)n + c->g.slot_cap / MF_BFS_CHUNK + 64);
        if (!q.sc.bitem || !q.sc.bdefer) return MAXFLOW_ERR_OOM;
        q.items_for = c->g.slot_cap;
    }
    return rc_cuda(cudaStreamSynchronize(c->stream));
}

int count_slots(maxflow_ctx *c, int64_t *used, int64_t *capped)
{
    std::vector<int32_t> su, sv, scap, scf;
    MF_TRY(dump_slots(c, su, sv, scap, scf, c->g.cf));
    *used = (int64_t)su.size();
    int64_t k = 0;
    for (int32_t x : scap) k += x > 0;
    *capped = k;
    return MAXFLOW_OK;
}

}  // namespace

extern "C" {

void maxflow_default_opts(maxflow_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->kernel_cycles = 0;
    o->data_driven = 1;
    o->fix_steep = 0;        // Alg. 3 off by default: the exact global relabel opens every iteration
    o->grid_blocks = 0;
    o->max_iters = 0;
    o->time_limit_s = 0;
    o->wait_limit_s = 0;
    o->slack_factor = 0.25f;
    o->slack_min = 4;
    o->device = -1;
    o->stream = nullptr;
}

int maxflow_build_layout(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                         float slack_factor, int32_t slack_min, int64_t *slot_capacity, int32_t *off, int32_t *deg,
                         int32_t *slot_dst, int32_t *slot_cap, int32_t *slot_rev, int32_t *slot_pcap)
{
    if (!slot_capacity || !(slack_factor >= 0.f) || slack_min < 0) return MAXFLOW_ERR_INVALID;
    MfHostGraph hg;
    int rc = mf_build_host(n, m, src, dst, cap, slack_factor, slack_min, hg);
    if (rc != MAXFLOW_OK) return rc;
    const int64_t S = hg.slot_cap;
    const bool any = off || deg || slot_dst || slot_cap || slot_rev || slot_pcap;
    if (any && *slot_capacity < S) rc = MAXFLOW_ERR_INVALID;
    if (any && rc == MAXFLOW_OK) {
        if (off) memcpy(off, hg.off, sizeof(int32_t) * ((size_t)n + 1));
        if (deg) memcpy(deg, hg.deg, sizeof(int32_t) * (size_t)n);
        if (slot_dst) memcpy(slot_dst, hg.dst, sizeof(int32_t) * (size_t)S);
        if (slot_cap) memcpy(slot_cap, hg.cap, sizeof(int32_t) * (size_t)S);
        if (slot_rev) memcpy(slot_rev, hg.rev, sizeof(int32_t) * (size_t)S);
        if (slot_pcap) memcpy(slot_pcap, hg.pcap, sizeof(int32_t) * (size_t)S);
    }
    *slot_capacity = S;
    hg.release();
    return rc;
}

int64_t maxflow_kernel_launches(void) { return (int64_t)g_kernel_launches.load(std::memory_order_relaxed); }

const char *maxflow_strerror(int code)
{
    switch (code) {
    case MAXFLOW_OK: return "ok";
    case MAXFLOW_ERR_INVALID: return "invalid argument";
    case MAXFLOW_ERR_OOM: return "out of memory";
    case MAXFLOW_ERR_CUDA: return "CUDA runtime error (no usable GPU or launch failure)";
    case MAXFLOW_ERR_NOT_CONVERGED: return "iteration or time cap reached before convergence";
    case MAXFLOW_ERR_STATE: return "call out of order";
    case MAXFLOW_ERR_INTERNAL: return "internal self-check failed";
    case MAXFLOW_ERR_TOO_LARGE: return "graph too large for int32 slot indexing or capacity sums";
    default: return "unknown status";
    }
}

static void park_free(maxflow_ctx *c);

void maxflow_destroy(maxflow_ctx *c)
{
    if (!c) return;
    if (c->ckpt) {
        maxflow_destroy(c->ckpt);
        c->ckpt = nullptr;
    }
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        while (!c->allocs.empty()) dfree(c, c->allocs.back().first);
        park_free(c);
        if (c->pp.hctrl) cudaFreeHost(c->pp.hctrl);
        if (c->hctrl) cudaFreeHost(c->hctrl);
        if (c->hbuf) cudaFreeHost(c->hbuf);
        if (c->ev0) cudaEventDestroy(c->ev0);
        if (c->ev1) cudaEventDestroy(c->ev1);
    }
    delete c;
}

int maxflow_init(maxflow_ctx **out, const maxflow_graph *g, int32_t s, int32_t t, const maxflow_opts *opt)
{
    if (!out) return MAXFLOW_ERR_INVALID;
    *out = nullptr;
    if (!g || g->n < 2 || g->m < 0 || s < 0 || t < 0 || s >= g->n || t >= g->n || s == t) return MAXFLOW_ERR_INVALID;
    if (g->m > 0 && (!g->src || !g->dst || !g->cap)) return MAXFLOW_ERR_INVALID;
    maxflow_opts o;
    maxflow_default_opts(&o);
    if (opt) o = *opt;
    if (o.slack_factor < 0 || o.slack_min < 0 || o.kernel_cycles < 0) return MAXFLOW_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return MAXFLOW_ERR_CUDA;
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    if (dev >= ndev) return MAXFLOW_ERR_INVALID;

    MfHostGraph hg;
    int rc = mf_build_host(g->n, g->m, g->src, g->dst, g->cap, o.slack_factor, o.slack_min, hg);
    if (rc != MAXFLOW_OK) return rc;

    maxflow_ctx *c = new (std::nothrow) maxflow_ctx();
    if (!c) {
        hg.release();
        return MAXFLOW_ERR_OOM;
    }
    c->opt = o;
    c->device = dev;
    c->stream = (cudaStream_t)o.stream;
    c->n = g->n;
    c->s = s;
    c->t = t;
    c->st.n = g->n;
    {
        double sum = 0;
        for (int64_t i = 0; i < g->m; ++i) sum += g->cap[i];
        c->mean_cap = g->m > 0 ? (float)(sum / (double)g->m) : 0.f;
    }
    DeviceGuard dg(dev);
    rc = dg.ok ? MAXFLOW_OK : MAXFLOW_ERR_CUDA;
    int stage_bytes = 0;
    if (rc == MAXFLOW_OK) rc = mf_stage_bytes(dev, &stage_bytes);
    if (rc == MAXFLOW_OK) rc = mf_max_coresident_blocks(dev, &c->per_sm, &c->sms, stage_bytes);
    c->stage_slots = stage_bytes / (int)sizeof(int);
    c->group_deg = std::max<int32_t>(c->hub_deg, c->stage_slots / (MF_BLOCK / (32 * MF_GROUP_WARPS)));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaEventCreate(&c->ev0));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaEventCreate(&c->ev1));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMallocHost((void **)&c->hctrl, sizeof(MfCtrl)));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMallocHost((void **)&c->hbuf, 16 * sizeof(long long)));
    if (rc == MAXFLOW_OK) rc = upload_graph(c, hg);
    hg.release();
    if (rc == MAXFLOW_OK) {
        int32_t n = c->n;
        c->g.h = dalloc_n<int32_t>(c, n);
        c->g.e = dalloc_n<long long>(c, n);
        c->ctrl = (MfCtrl *)dalloc(c, sizeof(MfCtrl));
        c->dbuf = dalloc_n<long long>(c, 16);
        if (!c->g.h || !c->g.e || !c->sc.bitem || !c->ctrl || !c->dbuf) rc = MAXFLOW_ERR_OOM;
    }
    if (rc == MAXFLOW_OK) rc = alloc_vertex_scratch(c);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->ctrl, 0, sizeof(MfCtrl), c->stream));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->g.h, 0, sizeof(int32_t) * c->n, c->stream));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->g.e, 0, sizeof(long long) * c->n, c->stream));
    if (rc == MAXFLOW_OK) rc = ensure_batch(c, 1024);
    if (rc == MAXFLOW_OK) {
        int64_t m = c->st.m_edges;
        c->kernel_cycles = o.kernel_cycles > 0 ? o.kernel_cycles : (int32_t)std::max<int64_t>(1, (m + c->n - 1) / c->n);
        default_split(c);
        c->rounds = 0;   // adaptive
        c->st.rounds = c->rounds;
        choose_grid(c);
        MfParams p = base_params(c);
        p.mode = MF_M_STATIC_INIT | MF_M_SOLVE;
        rc = run_solve(c, p);
        c->init_ms = c->st.ms_last;
        c->init_iters = c->st.iterations;
        note_incremental(c);
    }
    if (rc == MAXFLOW_OK) {
        c->feat = dalloc_n<float>(c, MF_FEATURES);
        c->sched_y = dalloc_n<float>(c, 64);
        if (!c->feat || !c->sched_y) rc = MAXFLOW_ERR_OOM;
    }
    if (rc != MAXFLOW_OK) {
        maxflow_destroy(c);
        return rc;
    }
    *out = c;
    return MAXFLOW_OK;
}

int maxflow_update(maxflow_ctx *c, const maxflow_batch *b)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    const int rc = do_batch(c, b, MF_M_APPLY | MF_M_SOLVE);
    if (rc == MAXFLOW_OK) note_incremental(c);
    return rc;
}

int maxflow_apply(maxflow_ctx *c, const maxflow_batch *b)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    return do_batch(c, b, MF_M_APPLY);
}

int maxflow_resolve_static(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_STATIC_INIT | MF_M_SOLVE;
    return run_solve(c, p);
}

int maxflow_resolve(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_SOLVE;
    return run_solve(c, p);
}

int maxflow_global_relabel(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_BFS_ONLY;
    int kerr = 0, kst = 0;
    MF_TRY(run_kernel(c, p, &kerr, &kst));
    return kerr == MF_E_NONE ? MAXFLOW_OK : MAXFLOW_ERR_INTERNAL;
}

int maxflow_query(maxflow_ctx *c, int64_t *value, uint8_t *side, int64_t *cut_cap)
{
    if (!c) return MAXFLOW_ERR_STATE;
    if (!c->solved) return MAXFLOW_ERR_STATE;
    if (c->evicted && (side || cut_cap)) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    if (side) {
        uint8_t *ds = (uint8_t *)dalloc(c, (size_t)c->n);
        if (!ds) return MAXFLOW_ERR_OOM;
        int rc = counted(mf_launch_aux(MF_AUX_SIDE, p, (void *)c->stream, nullptr, ds), 1);
        if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemcpyAsync(side, ds, (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
        if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
        dfree(c, ds);
        MF_TRY(rc);
    }
    if (cut_cap) {
        MF_TRY(rc_cuda(cudaMemsetAsync(c->dbuf, 0, sizeof(long long), c->stream)));
        MF_TRY(counted(mf_launch_aux(MF_AUX_CUT, p, (void *)c->stream, c->dbuf, nullptr), 1));
        MF_TRY(rc_cuda(cudaMemcpyAsync(c->hbuf, c->dbuf, sizeof(long long), cudaMemcpyDeviceToHost, c->stream)));
        MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
        *cut_cap = c->hbuf[0];
    }
    if (value) *value = c->value;
    return MAXFLOW_OK;
}

int maxflow_trace(maxflow_ctx *c, int32_t *boundary, double *t_us, int32_t cap, int32_t *count)
{
    if (!c || !count || cap < 0) return MAXFLOW_ERR_INVALID;
    const MfCtrl &h = *c->hctrl;
    int k = std::min<int>(h.trace_n, std::min<int>(cap, MF_TRACE));
    for (int i = 0; i < k; ++i) {
        if (boundary) boundary[i] = h.trace_hook[i];
        if (t_us) t_us[i] = (double)(h.trace_t[i] - h.t_entry) * 1e-3;
    }
    *count = k;
    return MAXFLOW_OK;
}

int maxflow_trace_work(maxflow_ctx *c, int64_t *slots, int32_t *info, double *cta_last_us, double *cta_mean_us,
                       int32_t cap, int32_t *count)
{
    if (!c || !count || cap < 0) return MAXFLOW_ERR_INVALID;
    const MfCtrl &h = *c->hctrl;
    int k = std::min<int>(h.trace_n, std::min<int>(cap, MF_TRACE));
    for (int i = 0; i < k; ++i) {
        if (slots) slots[i] = h.trace_slots[i];
        if (info) info[i] = h.trace_info[i];
        if (cta_last_us) cta_last_us[i] = h.trace_fin_max[i] * 1e-3;
        if (cta_mean_us) cta_mean_us[i] = h.trace_fin_mean[i] * 1e-3;
    }
    *count = k;
    return MAXFLOW_OK;
}

int maxflow_set_kernel_cycles(maxflow_ctx *c, int32_t k)
{
    if (!c || k < 0) return MAXFLOW_ERR_INVALID;
    int64_t m = c->st.m_edges;
    c->kernel_cycles = k > 0 ? k : (int32_t)std::max<int64_t>(1, (m + c->n - 1) / c->n);
    c->st.kernel_cycles = c->kernel_cycles;
    return MAXFLOW_OK;
}

// ---- schedules chosen per update -----------------------------------------------

namespace {

struct SchedAction {
    int32_t mode;      // 0: incremental (Alg. 5), 1: apply the batch, then re-solve from zero flow (Alg. 1)
    int32_t rounds;    // discharge rounds per global relabel (0: adaptive)
    int32_t cycles;    // KERNEL_CYCLES (0: the average-degree heuristic of Sec. 6.1)
    int32_t cycle_div; // > 0: rows of d slots get max(cycles, d / cycle_div) cycles
    int32_t fix;       // 1: remove-invalid-edges (Alg. 3) after each iteration's discharge
};

// Index 0 is the library's default schedule, 5 the paper's fixed one (one
// round, KERNEL_CYCLES = average degree, Alg. 3 after every discharge) and 18
// the paper's static re-solve.
const SchedAction kActions[] = {
    {0, 0, 0, 0, 0},   {0, 0, 0, 256, 0}, {0, 0, 4, 0, 0},   {0, 0, 64, 0, 0},  {0, 0, 64, 256, 0},
    {0, 1, 0, 0, 1},   {0, 1, 16, 0, 0},  {0, 1, 64, 0, 0},  {0, 4, 4, 0, 0},   {0, 4, 16, 0, 0},
    {0, 4, 64, 0, 0},  {0, 16, 4, 0, 0},  {0, 16, 16, 0, 0}, {0, 16, 64, 0, 0}, {0, 64, 16, 0, 0},
    {0, 64, 64, 0, 0}, {1, 0, 0, 0, 0},   {1, 0, 64, 0, 0},  {1, 1, 0, 0, 1},   {1, 16, 16, 0, 0},
};
constexpr int kNumActions = (int)(sizeof(kActions) / sizeof(kActions[0]));

float lg(double x) { return (float)std::log2(1.0 + (x > 0 ? x : 0)); }

// Stage the batch on the device (copying a host batch) and compute its features.
int stage_and_features(maxflow_ctx *c, const maxflow_batch *b, maxflow_batch *dev_view)
{
    if (!b || b->count < 0) return MAXFLOW_ERR_INVALID;
    if (b->count > 0 && (!b->u || !b->v || !b->new_cap)) return MAXFLOW_ERR_INVALID;
    if (!b->on_device) MF_TRY(check_host_batch(c, b));
    MF_TRY(ensure_batch(c, b->count));
    *dev_view = *b;
    if (!b->on_device && b->count > 0) {
        size_t bytes = sizeof(int32_t) * (size_t)b->count;
        MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bu, b->u, bytes, cudaMemcpyHostToDevice, c->stream)));
        MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bv, b->v, bytes, cudaMemcpyHostToDevice, c->stream)));
        MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bc, b->new_cap, bytes, cudaMemcpyHostToDevice, c->stream)));
        dev_view->u = c->sc.bu;
        dev_view->v = c->sc.bv;
        dev_view->new_cap = c->sc.bc;
        dev_view->on_device = 1;
    }
    MfFeatIn f{};
    f.bu = dev_view->u;
    f.bv = dev_view->v;
    f.bc = dev_view->new_cap;
    f.count = b->count;
    f.n = c->n;
    f.s = c->s;
    f.t = c->t;
    f.m = c->st.m_edges;
    f.mean_cap = c->mean_cap;
    f.host[0] = lg((double)c->inc_iters) / 8.f;
    f.host[1] = lg(c->inc_ms * 1000.0) / 16.f;
    f.host[2] = lg((double)c->inc_active_first) / 20.f;
    f.host[3] = lg((double)c->init_iters) / 8.f;
    f.host[4] = lg(c->init_ms * 1000.0) / 16.f;
    f.host[5] = lg((double)c->inc_levels) / 12.f;
    return counted(mf_features(f, c->feat, (void *)c->stream), 1);
}

int run_action(maxflow_ctx *c, const maxflow_batch *dev_batch, int a)
{
    const SchedAction &A = kActions[a];
    const int32_t keep_k = c->kernel_cycles, keep_r = c->rounds, keep_div = c->cycle_div, keep_fix = c->opt.fix_steep;
    int64_t m = c->st.m_edges;
    c->kernel_cycles = A.cycles > 0 ? A.cycles : (int32_t)std::max<int64_t>(1, (m + c->n - 1) / c->n);
    c->rounds = A.rounds;
    c->cycle_div = A.cycle_div;
    c->opt.fix_steep = A.fix;
    int rc;
    if (A.mode == 0) {
        rc = do_batch(c, dev_batch, MF_M_APPLY | MF_M_SOLVE);
        if (rc == MAXFLOW_OK) note_incremental(c);
    } else {
        rc = do_batch(c, dev_batch, MF_M_APPLY | MF_M_SKIP_SOURCE_SAT);
        double ms = c->acc_ms;
        if (rc == MAXFLOW_OK) {
            MfParams p = base_params(c);
            p.mode = MF_M_STATIC_INIT | MF_M_SOLVE;
            rc = run_solve(c, p);
            c->acc_ms += ms;
            c->st.ms_update = c->acc_ms;
        }
    }
    c->kernel_cycles = keep_k;
    c->rounds = keep_r;
    c->cycle_div = keep_div;
    c->opt.fix_steep = keep_fix;
    return rc;
}

}  // namespace

int maxflow_sched_actions(int32_t *mode, int32_t *rounds, int32_t *cycles, int32_t *cycle_div, int32_t *fix,
                          int32_t cap, int32_t *count)
{
    if (!count || cap < 0) return MAXFLOW_ERR_INVALID;
    int k = std::min(cap, kNumActions);
    for (int i = 0; i < k; ++i) {
        if (mode) mode[i] = kActions[i].mode;
        if (rounds) rounds[i] = kActions[i].rounds;
        if (cycles) cycles[i] = kActions[i].cycles;
        if (cycle_div) cycle_div[i] = kActions[i].cycle_div;
        if (fix) fix[i] = kActions[i].fix;
    }
    *count = (mode || rounds || cycles || cycle_div || fix) ? k : kNumActions;
    return MAXFLOW_OK;
}

int maxflow_features(maxflow_ctx *c, const maxflow_batch *b, float *out)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || !out) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    maxflow_batch view;
    MF_TRY(stage_and_features(c, b, &view));
    MF_TRY(rc_cuda(cudaMemcpyAsync(out, c->feat, sizeof(float) * MF_FEATURES, cudaMemcpyDeviceToHost, c->stream)));
    return rc_cuda(cudaStreamSynchronize(c->stream));
}

int maxflow_run_action(maxflow_ctx *c, const maxflow_batch *b, int32_t action)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || action < 0 || action >= kNumActions) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    return run_action(c, b, action);
}

int maxflow_update_scheduled(maxflow_ctx *c, const maxflow_batch *b, maxflow_mlp *m, int32_t *action_out)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || !m) return MAXFLOW_ERR_INVALID;
    if (mlp_n_in(m) != MF_FEATURES || mlp_n_out(m) != kNumActions) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    maxflow_batch view;
    MF_TRY(stage_and_features(c, b, &view));
    MF_TRY(mlp_forward_device(m, c->feat, 1, c->sched_y, c->stream));
    float y[64];
    MF_TRY(rc_cuda(cudaMemcpyAsync(y, c->sched_y, sizeof(float) * kNumActions, cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    int best = 0;
    for (int i = 1; i < kNumActions; ++i)
        if (y[i] < y[best]) best = i;
    if (action_out) *action_out = best;
    return run_action(c, &view, best);
}

int maxflow_set_tuning(maxflow_ctx *c, int32_t thread_max_slots, int32_t warp_max_slots, int32_t bfs_item_min_slots)
{
    if (!c) return MAXFLOW_ERR_INVALID;
    if (thread_max_slots == 0 && warp_max_slots == 0 && bfs_item_min_slots == 0) {
        default_split(c);
        return MAXFLOW_OK;
    }
    if (thread_max_slots < 1 || warp_max_slots < thread_max_slots || bfs_item_min_slots < 1)
        return MAXFLOW_ERR_INVALID;
    c->small_deg = thread_max_slots;
    c->hub_deg = warp_max_slots;
    c->bfs_hub = bfs_item_min_slots;
    c->group_deg = std::max<int32_t>(c->hub_deg, c->stage_slots / (MF_BLOCK / (32 * MF_GROUP_WARPS)));
    return MAXFLOW_OK;
}

int maxflow_test_stalled_barrier(maxflow_ctx *c, int32_t cta)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || cta < 0 || cta >= c->grid) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_BFS_ONLY;
    p.test_skip_cta = cta;
    int kerr = 0, kst = 0;
    MF_TRY(run_kernel(c, p, &kerr, &kst));   // resets the barrier words after an error
    return kerr == MF_E_NONE ? MAXFLOW_OK : status_to_rc(kerr, kst);
}

int maxflow_set_bfs_switch(maxflow_ctx *c, int32_t alpha, int32_t beta)
{
    if (!c || alpha < 0 || beta < 1) return MAXFLOW_ERR_INVALID;
    c->bu_alpha = alpha;
    c->bu_beta = beta;
    return MAXFLOW_OK;
}

int maxflow_solve_batched(maxflow_ctx *const *ctxs, int32_t count, const maxflow_batch *batches, int32_t group_blocks,
                          double *ms_out)
{
    if (!ctxs || count < 1 || group_blocks < 1) return MAXFLOW_ERR_INVALID;
    for (int32_t i = 0; i < count; ++i) {
        if (!ctxs[i] || ctxs[i]->device != ctxs[0]->device) return MAXFLOW_ERR_INVALID;
        if (ctxs[i]->evicted) return MAXFLOW_ERR_STATE;
    }
    maxflow_ctx *c0 = ctxs[0];
    DeviceGuard dg(c0->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    // per-instance parameters, largest instance first in the queue
    std::vector<int32_t> order((size_t)count);
    for (int32_t i = 0; i < count; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(),
              [&](int32_t a, int32_t b) { return ctxs[a]->g.slot_cap > ctxs[b]->g.slot_cap; });
    std::vector<MfParams> plist((size_t)count);
    for (int32_t k = 0; k < count; ++k) {
        maxflow_ctx *c = ctxs[order[(size_t)k]];
        MfParams p = base_params(c);
        if (batches) {
            const maxflow_batch *b = &batches[order[(size_t)k]];
            if (b->count < 0 || (b->count > 0 && (!b->u || !b->v || !b->new_cap))) return MAXFLOW_ERR_INVALID;
            if (!b->on_device) MF_TRY(check_host_batch(c, b));
            MF_TRY(ensure_batch(c, b->count));
            p = base_params(c);
            p.bcount = b->count;
            if (b->count > 0 && !b->on_device) {
                size_t bytes = sizeof(int32_t) * (size_t)b->count;
                MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bu, b->u, bytes, cudaMemcpyHostToDevice, c0->stream)));
                MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bv, b->v, bytes, cudaMemcpyHostToDevice, c0->stream)));
                MF_TRY(rc_cuda(cudaMemcpyAsync(c->sc.bc, b->new_cap, bytes, cudaMemcpyHostToDevice, c0->stream)));
                p.bu = c->sc.bu;
                p.bv = c->sc.bv;
                p.bc = c->sc.bc;
            } else {
                p.bu = b->u;
                p.bv = b->v;
                p.bc = b->new_cap;
            }
            p.mode = MF_M_APPLY | MF_M_SOLVE;
        } else {
            p.mode = MF_M_STATIC_INIT | MF_M_SOLVE;
        }
        plist[(size_t)k] = p;
    }
    const int maxg = c0->per_sm * c0->sms;
    const int gsize = std::min<int>(group_blocks, maxg);
    const int ngroups = std::max(1, std::min<int>(maxg / gsize, count));
    MF_TRY(ensure_multi(c0, count));
    unsigned *gstate = c0->multi_gstate;
    unsigned *head = gstate + 32 * maxg;
    int *abort_flag = (int *)(head + 1);
    MF_TRY(rc_cuda(cudaMemcpyAsync(c0->multi_plist, plist.data(), sizeof(MfParams) * (size_t)count,
                                   cudaMemcpyHostToDevice, c0->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(gstate, 0, sizeof(unsigned) * 32 * (size_t)(maxg + 2), c0->stream)));
    unsigned long long wait_ns = plist[0].wait_limit_ns;
    MF_TRY(rc_cuda(cudaEventRecord(c0->ev0, c0->stream)));
    MF_TRY(counted(mf_launch_multi(c0->multi_plist, count, gsize, ngroups * gsize, gstate, head, wait_ns, abort_flag,
                           (void *)c0->stream, c0->stage_slots * (int)sizeof(int)), 1));
    MF_TRY(rc_cuda(cudaEventRecord(c0->ev1, c0->stream)));
    int abort_h = 0;
    MF_TRY(rc_cuda(cudaMemcpyAsync(&abort_h, abort_flag, sizeof(int), cudaMemcpyDeviceToHost, c0->stream)));
    for (int32_t i = 0; i < count; ++i)
        MF_TRY(rc_cuda(cudaMemcpyAsync(ctxs[i]->hctrl, ctxs[i]->ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost,
                                       c0->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c0->stream)));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c0->ev0, c0->ev1);
    if (ms_out) *ms_out = ms;
    int first_rc = MAXFLOW_OK;
    for (int32_t i = 0; i < count; ++i) {
        maxflow_ctx *c = ctxs[i];
        const int kerr = (int)c->hctrl->err.w[0], kst = c->hctrl->d.status;
        c->acc_ms = ms;
        fill_stats(c, *c->hctrl, ms);
        if (abort_h || kerr != MF_E_NONE) {
            MF_TRY(rc_cuda(cudaMemsetAsync(c->ctrl, 0, 2 * sizeof(MfLine), c->stream)));
            MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
        }
        int rc;
        if (kerr == MF_E_OVERFLOW && batches) {
            rc = do_batch(c, &batches[i], MF_M_APPLY | MF_M_SOLVE);   // grows the rows, then runs alone
        } else {
            rc = abort_h ? MAXFLOW_ERR_INTERNAL : status_to_rc(kerr, kst);
            c->st.solves++;
            if (rc == MAXFLOW_OK || rc == MAXFLOW_ERR_NOT_CONVERGED) {
                c->value = c->hctrl->value;
                c->st.value = c->value;
                c->solved = (rc == MAXFLOW_OK);
                if (batches) c->st.updates++;
            }
        }
        if (rc != MAXFLOW_OK && first_rc == MAXFLOW_OK) first_rc = rc;
    }
    return first_rc;
}

int maxflow_set_stream(maxflow_ctx *c, void *stream)
{
    if (!c) return MAXFLOW_ERR_INVALID;
    c->stream = (cudaStream_t)stream;
    return MAXFLOW_OK;
}

int maxflow_reserve_batch(maxflow_ctx *c, int64_t count)
{
    if (!c || count < 0) return MAXFLOW_ERR_INVALID;
    if (c->evicted) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MF_TRY(ensure_batch(c, count));
    return rc_cuda(cudaStreamSynchronize(c->stream));
}

int maxflow_evicted_sizes(maxflow_ctx *c, int64_t *sizes, int32_t cap, int32_t *count)
{
    if (!c || !count) return MAXFLOW_ERR_INVALID;
    if (!c->evicted) return MAXFLOW_ERR_STATE;
    const int32_t k = (int32_t)c->park_sizes.size();
    *count = k;
    if (sizes && cap >= k) std::memcpy(sizes, c->park_sizes.data(), sizeof(int64_t) * (size_t)k);
    return MAXFLOW_OK;
}

int maxflow_device_bytes(maxflow_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return MAXFLOW_ERR_INVALID;
    int64_t b = 0;
    for (const auto &a : c->allocs) b += (int64_t)a.second;
    *bytes = b;
    return MAXFLOW_OK;
}

// Host memory for a parked state.  Blocks of 64 MiB and more are anonymous
// mappings advised to transparent huge pages and registered with the driver;
// smaller ones (and any failure on that path) come from cudaMallocHost.  With
// small base pages, device-to-host copies into long-lived pinned blocks were
// measured to slow down by up to 20x after unrelated host memory activity in
// the process (the device re-translates the host pages), while huge-page
// blocks kept full speed (about 193 GB/s device-to-host on a GB300 host).
static size_t huge_page_bytes()
{
    static size_t hp = 0;
    if (!hp) {
        hp = 2u << 20;
        if (FILE *f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
            unsigned long long v = 0;
            if (std::fscanf(f, "%llu", &v) == 1 && v >= 4096 && v <= (1ull << 31)) hp = (size_t)v;
            std::fclose(f);
        }
    }
    return hp;
}

static void park_free(maxflow_ctx *c)
{
    if (c->park_map) {
        cudaHostUnregister(c->park);
        munmap(c->park_map, c->park_map_bytes);
    } else if (c->park) {
        cudaFreeHost(c->park);
    }
    c->park = nullptr;
    c->park_map = nullptr;
    c->park_bytes = c->park_map_bytes = 0;
}

static int park_alloc(maxflow_ctx *c, size_t bytes)
{
    park_free(c);
    if (bytes >= (64u << 20)) {
        const size_t hp = huge_page_bytes();
        const size_t sz = (bytes + hp - 1) / hp * hp;
        void *m = mmap(nullptr, sz + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
        if (m != MAP_FAILED) {
            char *a = (char *)(((uintptr_t)m + hp - 1) / hp * hp);
            madvise(a, sz, MADV_HUGEPAGE);
            if (cudaHostRegister(a, sz, cudaHostRegisterDefault) == cudaSuccess) {
                c->park = a;
                c->park_bytes = sz;
                c->park_map = m;
                c->park_map_bytes = sz + hp;
                return MAXFLOW_OK;
            }
            cudaGetLastError();
            munmap(m, sz + hp);
        }
    }
    MF_TRY(rc_cuda(cudaMallocHost((void **)&c->park, bytes)));
    c->park_bytes = bytes;
    return MAXFLOW_OK;
}

// Host view of the parked state: slot arrays, vertex arrays, heights and excesses
// in one pinned block (each part 256-byte aligned).
struct ParkView {
    MfHostGraph g;
    int32_t *h = nullptr;
    long long *e = nullptr;
    size_t bytes = 0;
};

static ParkView park_view(char *base, int32_t n, int64_t S)
{
    ParkView v;
    size_t o = 0;
    auto take = [&](size_t b) {
        char *p = base ? base + o : nullptr;
        o += (b + 255) & ~(size_t)255;
        return p;
    };
    v.g.n = n;
    v.g.slot_cap = S;
    v.g.off = (int32_t *)take(sizeof(int32_t) * ((size_t)n + 1));
    v.g.deg = (int32_t *)take(sizeof(int32_t) * (size_t)n);
    v.g.bdeg = (int32_t *)take(sizeof(int32_t) * (size_t)n);
    v.g.dst = (int32_t *)take(sizeof(int32_t) * (size_t)S);
    v.g.cap = (int32_t *)take(sizeof(int32_t) * (size_t)S);
    v.g.cf = (int32_t *)take(sizeof(int32_t) * (size_t)S);
    v.g.rev = (int32_t *)take(sizeof(int32_t) * (size_t)S);
    v.g.pcap = nullptr;                   // rebuilt from cap and rev on restore
    v.h = (int32_t *)take(sizeof(int32_t) * (size_t)n);
    v.e = (long long *)take(sizeof(long long) * (size_t)n);
    v.bytes = o;
    return v;
}

static void release_device(maxflow_ctx *c)
{
    while (!c->allocs.empty()) dfree(c, c->allocs.back().first);
    c->g = MfGraph{};
    c->sc = MfScratch{};
    c->ctrl = nullptr;
    c->dbuf = nullptr;
    c->feat = c->sched_y = nullptr;
    c->x_cf = c->x_cf2 = c->x_h = nullptr;
    c->x_e = nullptr;
    c->multi_plist = nullptr;
    c->multi_gstate = nullptr;
    c->multi_cap = 0;
    c->pp.ctrl = nullptr;
    c->pp.sc = MfScratch{};
    c->pp.h = nullptr;
    c->pp.side = nullptr;
    c->pp.items_for = -1;
}

int maxflow_evict(maxflow_ctx *c)
{
    if (!c) return MAXFLOW_ERR_INVALID;
    if (c->evicted) return MAXFLOW_OK;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    const int32_t n = c->n;
    const int64_t S = c->g.slot_cap;
    const size_t need = park_view(nullptr, n, S).bytes;
    if (c->park_bytes < need) MF_TRY(park_alloc(c, need));
    ParkView v = park_view(c->park, n, S);
    struct Cp { void *h; const void *d; size_t b; };
    const Cp cps[] = {{v.g.off, c->g.off, sizeof(int32_t) * ((size_t)n + 1)},
                      {v.g.deg, c->g.deg, sizeof(int32_t) * (size_t)n},
                      {v.g.bdeg, c->g.bdeg, sizeof(int32_t) * (size_t)n},
                      {v.g.dst, c->g.dst, sizeof(int32_t) * (size_t)S},
                      {v.g.cap, c->g.cap, sizeof(int32_t) * (size_t)S},
                      {v.g.cf, c->g.cf, sizeof(int32_t) * (size_t)S},
                      {v.g.rev, c->g.rev, sizeof(int32_t) * (size_t)S},
                      {v.h, c->g.h, sizeof(int32_t) * (size_t)n},
                      {v.e, c->g.e, sizeof(long long) * (size_t)n}};
    for (const Cp &cp : cps) MF_TRY(rc_cuda(cudaMemcpyAsync(cp.h, cp.d, cp.b, cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    c->park_slots = S;
    c->park_sizes.clear();
    for (const auto &a : c->allocs) c->park_sizes.push_back((int64_t)a.second);
    release_device(c);
    c->evicted = true;
    return MAXFLOW_OK;
}

int maxflow_restore(maxflow_ctx *c)
{
    if (!c) return MAXFLOW_ERR_INVALID;
    if (!c->evicted) return MAXFLOW_OK;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    const int32_t n = c->n;
    ParkView v = park_view(c->park, n, c->park_slots);
    v.g.slots = c->st.slots;
    v.g.m_merged = c->st.m_edges;
    int rc = upload_graph(c, v.g);
    if (rc == MAXFLOW_OK) {
        c->g.h = dalloc_n<int32_t>(c, n);
        c->g.e = dalloc_n<long long>(c, n);
        c->ctrl = (MfCtrl *)dalloc(c, sizeof(MfCtrl));
        c->dbuf = dalloc_n<long long>(c, 16);
        c->feat = dalloc_n<float>(c, MF_FEATURES);
        c->sched_y = dalloc_n<float>(c, 64);
        if (!c->g.h || !c->g.e || !c->ctrl || !c->dbuf || !c->feat || !c->sched_y) rc = MAXFLOW_ERR_OOM;
    }
    if (rc == MAXFLOW_OK)
        rc = counted(mf_launch_aux(MF_AUX_PCAP, base_params(c), (void *)c->stream, nullptr, nullptr), 1);
    if (rc == MAXFLOW_OK) rc = alloc_vertex_scratch(c);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->ctrl, 0, sizeof(MfCtrl), c->stream));
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(c->g.h, v.h, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(c->g.e, v.e, sizeof(long long) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    if (rc == MAXFLOW_OK) rc = ensure_batch(c, 1024);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    if (rc != MAXFLOW_OK) {
        cudaStreamSynchronize(c->stream);
        release_device(c);
        return rc;
    }
    c->evicted = false;
    choose_grid(c);
    return MAXFLOW_OK;
}

int maxflow_resolve_static_pp(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_STATIC_INIT | MF_M_SAT_SINK | MF_M_SOLVE;
    int rc = run_solve(c, p);
    c->st.ms_update = c->acc_ms;
    return rc;
}

int maxflow_resolve_static_pull(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    p.mode = MF_M_STATIC_INIT | MF_M_NO_SRC_SAT | MF_M_SAT_SINK | MF_M_SOLVE;
    p.pull = 1;
    int rc = run_solve(c, p);
    double ms = c->acc_ms;
    if (rc == MAXFLOW_OK) {
        // leave push heights behind (the cut, queries and later updates read them)
        MfParams q = base_params(c);
        q.mode = MF_M_BFS_ONLY;
        int kerr = 0, kst = 0;
        MF_TRY(run_kernel(c, q, &kerr, &kst));
        if (kerr != MF_E_NONE) rc = status_to_rc(kerr, kst);
        ms = c->acc_ms;
    }
    c->st.ms_update = ms;
    return rc;
}

int maxflow_update_pp(maxflow_ctx *c, const maxflow_batch *b, int32_t stop_after)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_STATE;
    if (stop_after < 0 || stop_after > 3) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    if (!c->solved) return do_batch(c, b, MF_M_APPLY | MF_M_SOLVE);   // no cut to start from
    MF_TRY(ensure_pp(c));
    // 1: the batch (Alg. 5), the sides of the last cut, saturation across it
    int rc = do_batch(c, b, MF_M_APPLY | MF_M_CUT);
    double ms = c->acc_ms;
    if (rc != MAXFLOW_OK || stop_after == 1) {
        c->st.ms_update = ms;
        return rc;
    }
    // 2: push on side 1 and pull on side 0, two CTA groups of one launch
    MF_TRY(ensure_multi(c, 2));
    MfParams pl[2];
    pl[0] = base_params(c);
    pl[0].mode = MF_M_SOLVE | MF_M_NO_VALUE;
    pl[0].side_root = 1;
    pl[1] = base_params(c);
    pl[1].mode = MF_M_SOLVE | MF_M_NO_VALUE;
    pl[1].pull = 1;
    pl[1].side_root = 0;
    pl[1].h = c->pp.h;
    pl[1].ctrl = c->pp.ctrl;
    pl[1].sc = c->pp.sc;
    const int maxg = c->per_sm * c->sms;
    const int gsize = std::max(1, std::min(c->grid, maxg) / 2);
    unsigned *gstate = c->multi_gstate;
    unsigned *head = gstate + 32 * maxg;
    int *abort_flag = (int *)(head + 1);
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->multi_plist, pl, sizeof(pl), cudaMemcpyHostToDevice, c->stream)));
    MF_TRY(rc_cuda(cudaMemsetAsync(gstate, 0, sizeof(unsigned) * 32 * (size_t)(maxg + 2), c->stream)));
    MF_TRY(rc_cuda(cudaEventRecord(c->ev0, c->stream)));
    MF_TRY(counted(mf_launch_multi(c->multi_plist, 2, gsize, 2 * gsize, gstate, head, pl[0].wait_limit_ns, abort_flag,
                           (void *)c->stream, c->stage_slots * (int)sizeof(int)), 1));
    MF_TRY(rc_cuda(cudaEventRecord(c->ev1, c->stream)));
    int abort_h = 0;
    MF_TRY(rc_cuda(cudaMemcpyAsync(&abort_h, abort_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->hctrl, c->ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->pp.hctrl, c->pp.ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    float ms2 = 0.f;
    cudaEventElapsedTime(&ms2, c->ev0, c->ev1);
    ms += ms2;
    const int e0 = (int)c->hctrl->err.w[0], e1 = (int)c->pp.hctrl->err.w[0];
    if (abort_h || e0 != MF_E_NONE || e1 != MF_E_NONE) {
        MF_TRY(rc_cuda(cudaMemsetAsync(c->ctrl, 0, 2 * sizeof(MfLine), c->stream)));
        MF_TRY(rc_cuda(cudaMemsetAsync(c->pp.ctrl, 0, 2 * sizeof(MfLine), c->stream)));
        MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
        c->st.ms_update = ms;
        if (abort_h) return MAXFLOW_ERR_INTERNAL;
        return status_to_rc(e0 != MF_E_NONE ? e0 : e1, MF_ST_ERROR);
    }
    if (stop_after == 2) {
        c->st.ms_update = ms;
        return status_to_rc(MF_E_NONE, c->hctrl->d.status == MF_ST_CAP || c->pp.hctrl->d.status == MF_ST_CAP
                                           ? MF_ST_CAP : MF_ST_CONVERGED);
    }
    // 3: a push solve over the whole graph finishes what the two parts left
    MfParams p = base_params(c);
    p.mode = MF_M_SOLVE;
    rc = run_solve(c, p);
    ms += c->acc_ms;
    c->acc_ms = ms;
    c->st.ms_update = ms;
    return rc;
}

int maxflow_set_requeue(maxflow_ctx *c, int32_t on)
{
    if (!c || on < 0 || on > 1) return MAXFLOW_ERR_INVALID;
    c->requeue = on;
    return MAXFLOW_OK;
}

int maxflow_set_cycle_div(maxflow_ctx *c, int32_t div)
{
    if (!c || div < 0) return MAXFLOW_ERR_INVALID;
    c->cycle_div = div;
    return MAXFLOW_OK;
}

int maxflow_set_bfs_tail(maxflow_ctx *c, int32_t slots)
{
    if (!c || slots < 0) return MAXFLOW_ERR_INVALID;
    c->tail_slots = slots;
    return MAXFLOW_OK;
}

int maxflow_set_fix_steep(maxflow_ctx *c, int32_t on)
{
    if (!c || on < 0 || on > 1) return MAXFLOW_ERR_INVALID;
    c->opt.fix_steep = on;
    return MAXFLOW_OK;
}

int maxflow_set_rounds(maxflow_ctx *c, int32_t rounds)
{
    if (!c || rounds < 0 || rounds > (1 << 20)) return MAXFLOW_ERR_INVALID;
    c->rounds = rounds;
    c->st.rounds = rounds;
    return MAXFLOW_OK;
}

int maxflow_clone(maxflow_ctx *src, maxflow_ctx **out)
{
    if (src && src->evicted) return MAXFLOW_ERR_STATE;
    if (!src || !out) return MAXFLOW_ERR_INVALID;
    *out = nullptr;
    DeviceGuard dg(src->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    maxflow_ctx *c = new (std::nothrow) maxflow_ctx();
    if (!c) return MAXFLOW_ERR_OOM;
    c->opt = src->opt;
    c->device = src->device;
    c->stream = src->stream;
    c->n = src->n;
    c->s = src->s;
    c->t = src->t;
    c->kernel_cycles = src->kernel_cycles;
    c->rounds = src->rounds;
    c->small_deg = src->small_deg;
    c->bu_alpha = src->bu_alpha;
    c->bu_beta = src->bu_beta;
    c->hub_deg = src->hub_deg;
    c->group_deg = src->group_deg;
    c->bfs_hub = src->bfs_hub;
    c->per_sm = src->per_sm;
    c->stage_slots = src->stage_slots;
    c->requeue = src->requeue;
    c->cycle_div = src->cycle_div;
    c->tail_slots = src->tail_slots;
    c->sms = src->sms;
    c->st = src->st;
    c->solved = src->solved;
    c->value = src->value;
    c->mean_cap = src->mean_cap;
    c->init_ms = src->init_ms;
    c->init_iters = src->init_iters;
    c->inc_iters = src->inc_iters;
    c->inc_active_first = src->inc_active_first;
    c->inc_levels = src->inc_levels;
    c->inc_ms = src->inc_ms;
    const int32_t n = c->n;
    const int64_t S = src->g.slot_cap;
    int rc = rc_cuda(cudaEventCreate(&c->ev0));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaEventCreate(&c->ev1));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMallocHost((void **)&c->hctrl, sizeof(MfCtrl)));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMallocHost((void **)&c->hbuf, 16 * sizeof(long long)));
    if (rc == MAXFLOW_OK) {
        c->g.n = n;
        c->g.slot_cap = S;
        c->g.off = dalloc_n<int32_t>(c, n + 1);
        c->g.deg = dalloc_n<int32_t>(c, n);
        c->g.bdeg = dalloc_n<int32_t>(c, n);
        c->g.dst = dalloc_n<int32_t>(c, S);
        c->g.cf = dalloc_n<int32_t>(c, S);
        c->g.cap = dalloc_n<int32_t>(c, S);
        c->g.rev = dalloc_n<int32_t>(c, S);
        c->g.pcap = dalloc_n<int32_t>(c, S);
        c->g.h = dalloc_n<int32_t>(c, n);
        c->g.e = dalloc_n<long long>(c, n);
        c->sc.bitem = dalloc_n<int2>(c, (int64_t)n + S / MF_BFS_CHUNK + 64);
        c->sc.bdefer = dalloc_n<int2>(c, (int64_t)n + S / MF_BFS_CHUNK + 64);
        c->ctrl = (MfCtrl *)dalloc(c, sizeof(MfCtrl));
        c->dbuf = dalloc_n<long long>(c, 16);
        c->feat = dalloc_n<float>(c, MF_FEATURES);
        c->sched_y = dalloc_n<float>(c, 64);
        if (!c->g.off || !c->g.deg || !c->g.bdeg || !c->g.dst || !c->g.cf || !c->g.cap || !c->g.rev || !c->g.pcap ||
            !c->g.h || !c->g.e || !c->sc.bitem || !c->sc.bdefer || !c->ctrl || !c->dbuf || !c->feat || !c->sched_y)
            rc = MAXFLOW_ERR_OOM;
    }
    if (rc == MAXFLOW_OK) rc = alloc_vertex_scratch(c);
    struct Cp { void *d; const void *s; size_t b; };
    if (rc == MAXFLOW_OK) {
        const Cp cps[] = {{c->g.off, src->g.off, sizeof(int32_t) * (size_t)(n + 1)},
                          {c->g.deg, src->g.deg, sizeof(int32_t) * (size_t)n},
                          {c->g.bdeg, src->g.bdeg, sizeof(int32_t) * (size_t)n},
                          {c->g.dst, src->g.dst, sizeof(int32_t) * (size_t)S},
                          {c->g.cf, src->g.cf, sizeof(int32_t) * (size_t)S},
                          {c->g.cap, src->g.cap, sizeof(int32_t) * (size_t)S},
                          {c->g.rev, src->g.rev, sizeof(int32_t) * (size_t)S},
                          {c->g.pcap, src->g.pcap, sizeof(int32_t) * (size_t)S},
                          {c->g.h, src->g.h, sizeof(int32_t) * (size_t)n},
                          {c->g.e, src->g.e, sizeof(long long) * (size_t)n}};
        for (const Cp &cp : cps)
            if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemcpyAsync(cp.d, cp.s, cp.b, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->ctrl, 0, sizeof(MfCtrl), c->stream));
    if (rc == MAXFLOW_OK) rc = ensure_batch(c, std::max<int64_t>(1024, src->sc.batch_cap));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    if (rc != MAXFLOW_OK) {
        maxflow_destroy(c);
        return rc;
    }
    c->grid = src->grid;
    *out = c;
    return MAXFLOW_OK;
}

int maxflow_checkpoint(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_INVALID;
    maxflow_ctx *copy = nullptr;
    MF_TRY(maxflow_clone(c, &copy));
    if (c->ckpt) maxflow_destroy(c->ckpt);
    c->ckpt = copy;
    return MAXFLOW_OK;
}

int maxflow_rollback(maxflow_ctx *c)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_INVALID;
    if (!c->ckpt) return MAXFLOW_ERR_STATE;
    maxflow_ctx *saved = c->ckpt;
    c->ckpt = nullptr;
    {
        DeviceGuard dg(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);      // nothing of the failed call is still running
    }
    std::swap(*c, *saved);           // c takes the saved state (and its device buffers); saved the old one
    c->ckpt = nullptr;
    saved->ckpt = nullptr;
    maxflow_destroy(saved);
    return MAXFLOW_OK;
}

int maxflow_stats(maxflow_ctx *c, maxflow_stats_t *out)
{
    if (!c || !out) return MAXFLOW_ERR_INVALID;
    *out = c->st;
    return MAXFLOW_OK;
}

int maxflow_set_flow(maxflow_ctx *c, int64_t count, const int32_t *u, const int32_t *v, const int32_t *f)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || count < 0) return MAXFLOW_ERR_INVALID;
    if (count > 0 && (!u || !v || !f)) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    int32_t *du = dalloc_n<int32_t>(c, count), *dv = dalloc_n<int32_t>(c, count), *df = dalloc_n<int32_t>(c, count);
    int rc = (du && dv && df) ? MAXFLOW_OK : MAXFLOW_ERR_OOM;
    size_t bytes = sizeof(int32_t) * (size_t)count;
    if (rc == MAXFLOW_OK && count > 0) {
        rc = rc_cuda(cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, c->stream));
        if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, c->stream));
        if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemcpyAsync(df, f, bytes, cudaMemcpyHostToDevice, c->stream));
    }
    MfParams p = base_params(c);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaMemsetAsync(c->dbuf, 0, sizeof(long long), c->stream));
    if (rc == MAXFLOW_OK && count > 0)
        rc = counted(mf_set_flow_items(p, (void *)c->stream, c->dbuf, count, du, dv, df, 0), 1);
    if (rc == MAXFLOW_OK)
        rc = rc_cuda(cudaMemcpyAsync(c->hbuf, c->dbuf, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    if (rc == MAXFLOW_OK && c->hbuf[0] != 0) rc = MAXFLOW_ERR_INVALID;
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_SET_CF_RESET, p, (void *)c->stream, nullptr, nullptr), 1);
    if (rc == MAXFLOW_OK && count > 0)
        rc = counted(mf_set_flow_items(p, (void *)c->stream, c->dbuf, count, du, dv, df, 1), 1);
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_EXCESS, p, (void *)c->stream, nullptr, nullptr), 1);
    if (rc == MAXFLOW_OK) rc = rc_cuda(cudaStreamSynchronize(c->stream));
    dfree(c, du);
    dfree(c, dv);
    dfree(c, df);
    if (rc == MAXFLOW_OK) c->solved = false;
    return rc;
}

int maxflow_get_residual(maxflow_ctx *c, int64_t *count, int32_t *u, int32_t *v, int32_t *cap, int32_t *cf)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || !count) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    std::vector<int32_t> su, sv, scap, scf;
    MF_TRY(dump_slots(c, su, sv, scap, scf, c->g.cf));
    int64_t k = (int64_t)su.size();
    if (!u || !v || !cap || !cf || *count < k) {
        *count = k;
        return MAXFLOW_OK;
    }
    std::memcpy(u, su.data(), sizeof(int32_t) * k);
    std::memcpy(v, sv.data(), sizeof(int32_t) * k);
    std::memcpy(cap, scap.data(), sizeof(int32_t) * k);
    std::memcpy(cf, scf.data(), sizeof(int32_t) * k);
    *count = k;
    return MAXFLOW_OK;
}

int maxflow_get_vertex_state(maxflow_ctx *c, int32_t *h, int64_t *e)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    if (h) MF_TRY(rc_cuda(cudaMemcpyAsync(h, c->g.h, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream)));
    if (e) MF_TRY(rc_cuda(cudaMemcpyAsync(e, c->g.e, sizeof(long long) * c->n, cudaMemcpyDeviceToHost, c->stream)));
    return rc_cuda(cudaStreamSynchronize(c->stream));
}

int maxflow_check(maxflow_ctx *c, int64_t *out)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || !out) return MAXFLOW_ERR_INVALID;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    MfParams p = base_params(c);
    MF_TRY(rc_cuda(cudaMemsetAsync(c->dbuf, 0, 8 * sizeof(long long), c->stream)));
    MF_TRY(counted(mf_launch_aux(MF_AUX_CHECK, p, (void *)c->stream, c->dbuf, nullptr), 2));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->hbuf, c->dbuf, 6 * sizeof(long long), cudaMemcpyDeviceToHost, c->stream)));
    MF_TRY(rc_cuda(cudaStreamSynchronize(c->stream)));
    for (int i = 0; i < 6; ++i) out[i] = c->hbuf[i];
    return MAXFLOW_OK;
}

int maxflow_get_flow(maxflow_ctx *c, int64_t *count, int32_t *u, int32_t *v, int32_t *cap, int32_t *flow)
{
    if (c && c->evicted) return MAXFLOW_ERR_STATE;
    if (!c || !count) return MAXFLOW_ERR_INVALID;
    if (!c->solved) return MAXFLOW_ERR_STATE;
    DeviceGuard dg(c->device);
    if (!dg.ok) return MAXFLOW_ERR_CUDA;
    int64_t used = 0, capped = 0;
    MF_TRY(count_slots(c, &used, &capped));
    if (!u || !v || !cap || !flow || *count < capped) {
        *count = capped;
        return MAXFLOW_OK;
    }
    int64_t S = c->g.slot_cap;
    if (!c->x_cf) c->x_cf = dalloc_n<int32_t>(c, S);
    if (!c->x_cf2) c->x_cf2 = dalloc_n<int32_t>(c, S);
    if (!c->x_h) c->x_h = dalloc_n<int32_t>(c, c->n);
    if (!c->x_e) c->x_e = dalloc_n<long long>(c, c->n);
    if (!c->x_cf || !c->x_cf2 || !c->x_h || !c->x_e) return MAXFLOW_ERR_OOM;
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->x_cf, c->g.cf, sizeof(int32_t) * S, cudaMemcpyDeviceToDevice, c->stream)));
    MF_TRY(rc_cuda(cudaMemcpyAsync(c->x_e, c->g.e, sizeof(long long) * c->n, cudaMemcpyDeviceToDevice, c->stream)));
    maxflow_stats_t keep = c->st;
    // (a) return the excess left on the source side to s (Lemma 3.5): a
    //     push-relabel run whose sink is s, with t excluded.
    MfParams p = base_params(c);
    p.cf = c->x_cf;
    p.h = c->x_h;
    p.e = c->x_e;
    p.sink = c->s;
    p.source = c->t;
    p.mode = MF_M_SOLVE | MF_M_NO_DEFICIT_ROOTS;
    // No Alg. 3 here: it moves whole residuals and can leave a deficit, which
    // these runs do not take as a root; a deficit left in A would then be
    // filled from t in (b) and lower the flow.  The loop's termination test
    // after a full backward BFS does not depend on Alg. 3.
    p.fix_steep = 0;
    int kerr = 0, kst = 0;
    MF_TRY(run_kernel(c, p, &kerr, &kst));
    int rc = status_to_rc(kerr, kst);
    // (b) fill the deficits on the sink side from t (Sec. 4.3 Claim): the
    //     same run on the reversed residual graph with negated excess.
    const int32_t *io1[2] = {c->x_cf, c->x_cf2};
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_REVERSE_CF, p, (void *)c->stream, nullptr, io1), 1);
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_NEGATE_E, p, (void *)c->stream, nullptr, nullptr), 1);
    if (rc == MAXFLOW_OK) {
        MfParams q = p;
        q.cf = c->x_cf2;
        q.sink = c->t;
        q.source = c->s;
        MF_TRY(run_kernel(c, q, &kerr, &kst));
        rc = status_to_rc(kerr, kst);
    }
    const int32_t *io2[2] = {c->x_cf2, c->x_cf};
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_REVERSE_CF, p, (void *)c->stream, nullptr, io2), 1);
    if (rc == MAXFLOW_OK) rc = counted(mf_launch_aux(MF_AUX_NEGATE_E, p, (void *)c->stream, nullptr, nullptr), 1);
    c->st = keep;
    MF_TRY(rc);
    std::vector<int32_t> su, sv, scap, scf;
    MF_TRY(dump_slots(c, su, sv, scap, scf, c->x_cf));
    int64_t k = 0;
    for (size_t i = 0; i < su.size(); ++i) {
        if (scap[i] <= 0) continue;
        u[k] = su[i];
        v[k] = sv[i];
        cap[k] = scap[i];
        int64_t f = (int64_t)scap[i] - scf[i];
        flow[k] = (int32_t)(f > 0 ? f : 0);
        ++k;
    }
    *count = k;
    return MAXFLOW_OK;
}

}  // extern "C"
