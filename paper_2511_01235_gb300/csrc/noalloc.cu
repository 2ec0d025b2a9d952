// Backward-BFS heights on caller-owned device arrays, without allocating.
//
// Some callers cannot allocate device memory on their request path: a serving
// process that reserves its whole device memory pool at start-up, or a plugin
// living inside a host application that owns the GPU allocator, must not call
// cudaMalloc later, because an allocation can fail under their fixed budget,
// can block, or can synchronise the device behind their back.  This entry
// point serves them: the caller passes the residual graph, the excesses and the
// output heights; the only scratch the step needs (the BFS frontier lists and
// the kernel's control block) lives in the file-scope device array below.
//
// The array has a fixed maximum size (MAXFLOW_NOALLOC_MAX_N vertices and
// MAXFLOW_NOALLOC_MAX_SLOTS slots), so every GPU that loads this library holds
// about 14 MB for it until the process exits.
// Every call uses the same array and it keeps the contents of the last call:
// the barrier words of the control block are cleared before each launch, and
// the kernel resets the rest itself.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/maxflow.h"
#include "mf_internal.h"

void mf_note_launches(int kernels);   // the library's launch counter (api.cu)

namespace {

// control block + frontier list (one int per vertex) + work items of long rows
// (at most one per vertex plus one per MF_BFS_CHUNK slots)
constexpr size_t kCtrlBytes = (sizeof(MfCtrl) + 255) & ~(size_t)255;
constexpr size_t kListBytes = (sizeof(int32_t) * (size_t)MAXFLOW_NOALLOC_MAX_N + 255) & ~(size_t)255;
constexpr size_t kItemBytes =
    sizeof(int2) * ((size_t)MAXFLOW_NOALLOC_MAX_N + (size_t)MAXFLOW_NOALLOC_MAX_SLOTS / MF_BFS_CHUNK + 64);
// a two-vertex graph with no slots (off, deg, e, h), for the prepare call
constexpr size_t kPrepBytes = 256;
constexpr size_t kScratchBytes = kCtrlBytes + kListBytes + kItemBytes + kPrepBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
    bool ready = false;
    int per_sm = 0, sms = 0;        // co-resident CTAs of the solve kernel (a property of the device)
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// With the device current: the device address of the scratch array (host
// code cannot use the symbol itself as a device pointer), looked up on every
// call -- after a cudaDeviceReset the module is loaded again at another
// address -- and the occupancy of the solve kernel, queried once per device.
// Both lookups make the driver load the modules that hold the array and the
// kernel if it has not yet (lazy loading), which is what the n = 0 call is for.
int setup_device(int dev, DeviceSetup **out, unsigned char **base)
{
    if (dev < 0 || dev >= kMaxDevices) return MAXFLOW_ERR_INVALID;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return MAXFLOW_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        int rc = mf_max_coresident_blocks(dev, &d.per_sm, &d.sms, 0);
        if (rc != MAXFLOW_OK) return rc;
        d.ready = true;
    }
    *out = &d;
    *base = (unsigned char *)ptr;
    return MAXFLOW_OK;
}

}  // namespace

extern "C" int maxflow_global_relabel_noalloc(int32_t n, int32_t s, int32_t t, const int32_t *off,
                                              const int32_t *deg, const int32_t *dst, const int32_t *cf,
                                              const int32_t *pcap, const int64_t *e, int32_t *h,
                                              int32_t deficit_roots, void *stream)
{
    if (n > MAXFLOW_NOALLOC_MAX_N) return MAXFLOW_ERR_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    DeviceSetup *ds = nullptr;
    unsigned char *base = nullptr;
    if (n == 0) {
        // prepare the device: load the modules (setup_device), then run the step
        // once on a two-vertex graph without slots held in the array itself, so
        // that nothing the driver sets up at a first launch is left for later calls
        int rc = setup_device(dev, &ds, &base);
        if (rc != MAXFLOW_OK) return rc;
        unsigned char *g2 = base + kCtrlBytes + kListBytes + kItemBytes;
        if (cudaMemsetAsync(g2, 0, kPrepBytes, (cudaStream_t)stream) != cudaSuccess) return MAXFLOW_ERR_CUDA;
        int32_t *o = (int32_t *)g2;                       // off[3] = 0, deg[2] = 0
        int64_t *e2 = (int64_t *)(g2 + 64);               // e[2] = 0
        int32_t *h2 = (int32_t *)(g2 + 128);
        return maxflow_global_relabel_noalloc(2, 0, 1, o, o + 4, o, o, o, e2, h2, deficit_roots, stream);
    }
    if (n < 2 || s < 0 || t < 0 || s >= n || t >= n || s == t) return MAXFLOW_ERR_INVALID;
    if (!off || !deg || !dst || !cf || !pcap || !e || !h) return MAXFLOW_ERR_INVALID;
    int rc = setup_device(dev, &ds, &base);
    if (rc != MAXFLOW_OK) return rc;

    MfCtrl *ctrl = (MfCtrl *)base;
    MfParams p;
    std::memset(&p, 0, sizeof(p));
    p.g.n = n;
    p.g.off = const_cast<int32_t *>(off);
    p.g.deg = const_cast<int32_t *>(deg);
    p.g.dst = const_cast<int32_t *>(dst);
    p.g.pcap = const_cast<int32_t *>(pcap);
    p.g.cf = const_cast<int32_t *>(cf);
    p.g.h = h;
    p.g.e = (long long *)const_cast<int64_t *>(e);
    p.sc.border = (int32_t *)(base + kCtrlBytes);
    p.sc.bitem = (int2 *)(base + kCtrlBytes + kListBytes);
    p.sc.bdefer = nullptr;          // bottom-up threads scan whole rows (no deferred chunks: no room for them)
    p.ctrl = ctrl;
    p.cf = p.g.cf;
    p.h = h;
    p.e = p.g.e;
    p.sink = t;
    p.source = s;
    p.mode = MF_M_BFS_ONLY | (deficit_roots ? 0 : MF_M_NO_DEFICIT_ROOTS);
    p.side_root = -1;
    p.test_skip_cta = -1;
    p.kernel_cycles = 1;
    p.rounds = 1;
    p.small_deg = MF_SMALL_DEG;
    p.hub_deg = MF_HUB_DEG;
    p.bfs_hub = MF_BFS_HUB;
    p.bu_alpha = MF_BU_ALPHA;
    p.bu_beta = MF_BU_BETA;
    p.max_iters = 1;
    p.time_limit_ns = 60ull * 1000000000ull;
    p.wait_limit_ns = 1000000000ull;

    cudaStream_t st = (cudaStream_t)stream;
    int32_t nslots = 0;
    if (cudaMemcpyAsync(&nslots, off + n, sizeof(nslots), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MAXFLOW_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    if (nslots < 0) return MAXFLOW_ERR_INVALID;
    if (nslots > MAXFLOW_NOALLOC_MAX_SLOTS) return MAXFLOW_ERR_TOO_LARGE;
    // barrier words must start at zero (a previous call may have ended early)
    if (cudaMemsetAsync(ctrl, 0, 2 * sizeof(MfLine), st) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    int maxg = ds->per_sm * ds->sms;
    int grid = (int)((n + 2047) / 2048);
    if (grid < 2) grid = 2;
    if (grid > maxg) grid = maxg;
    rc = mf_launch(p, grid, stream);
    if (rc != MAXFLOW_OK) return rc;
    mf_note_launches(1);
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, &ctrl->err.w[0], sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return MAXFLOW_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MAXFLOW_ERR_CUDA;
    return err == MF_E_NONE ? MAXFLOW_OK : MAXFLOW_ERR_INTERNAL;
}
