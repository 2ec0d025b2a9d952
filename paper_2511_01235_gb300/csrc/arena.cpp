// Device-memory arena for many resident contexts (serving).
//
// One cudaMalloc of the whole budget at creation (or a region the caller
// owns); contexts allocate from it
// through the maxflow_opts alloc/free callbacks.  No device allocation or free
// happens afterwards, so restoring a context never breaks the concurrency of a
// launch running on another stream (a device allocation is one of the host
// calls that serialises streams), and the budget is a physical bound.
//
// Placement: best fit over an address-ordered free list that coalesces on
// free.  Large requests (>= 1 MiB: slot arrays, vertex arrays) take the head of
// the smallest block that fits; small ones (batch and control scratch) take the
// tail of the highest-addressed block that fits, which keeps small pieces away
// from the large runs that evicted states leave behind.  When nothing fits and
// overflow is allowed, the request falls back to cudaMalloc and is counted;
// otherwise it fails (the library then returns MAXFLOW_ERR_OOM).
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <set>
#include <unordered_map>
#include <utility>

#include "maxflow.h"

struct maxflow_arena {
    int device = 0;
    char *base = nullptr;
    size_t capacity = 0;
    bool allow_overflow = true;
    bool owns = true;                                     // base came from cudaMalloc here
    std::mutex mu;
    std::map<size_t, size_t> free_by_off;                 // offset -> size
    std::set<std::pair<size_t, size_t>> free_by_size;     // (size, offset)
    std::unordered_map<size_t, size_t> used;              // offset -> size
    std::unordered_map<void *, size_t> overflow;          // cudaMalloc fallbacks
    int64_t in_use = 0, peak = 0, ov_in_use = 0, ov_peak = 0, fallbacks = 0, failed = 0;
};

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kLarge = 1u << 20;

void insert_free(maxflow_arena *a, size_t off, size_t size)
{
    // coalesce with the neighbours
    auto nx = a->free_by_off.lower_bound(off);
    if (nx != a->free_by_off.end() && off + size == nx->first) {
        a->free_by_size.erase({nx->second, nx->first});
        size += nx->second;
        nx = a->free_by_off.erase(nx);
    }
    if (nx != a->free_by_off.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            a->free_by_size.erase({pv->second, pv->first});
            off = pv->first;
            size += pv->second;
            a->free_by_off.erase(pv);
        }
    }
    a->free_by_off.emplace(off, size);
    a->free_by_size.emplace(size, off);
}

void take(maxflow_arena *a, size_t block_off, size_t block_size, size_t off, size_t size)
{
    a->free_by_off.erase(block_off);
    a->free_by_size.erase({block_size, block_off});
    if (off > block_off) {
        a->free_by_off.emplace(block_off, off - block_off);
        a->free_by_size.emplace(off - block_off, block_off);
    }
    const size_t end = off + size, bend = block_off + block_size;
    if (bend > end) {
        a->free_by_off.emplace(end, bend - end);
        a->free_by_size.emplace(bend - end, end);
    }
    a->used.emplace(off, size);
    a->in_use += (int64_t)size;
    if (a->in_use > a->peak) a->peak = a->in_use;
}

}  // namespace

extern "C" {

int maxflow_arena_create(int32_t device, int64_t bytes, int32_t allow_overflow, void *base, maxflow_arena **out)
{
    if (!out || bytes <= 0) return MAXFLOW_ERR_INVALID;
    *out = nullptr;
    if (base && ((uintptr_t)base & (kAlign - 1))) return MAXFLOW_ERR_INVALID;
    maxflow_arena *a = new maxflow_arena();
    a->device = device;
    a->allow_overflow = allow_overflow != 0;
    if (base) {
        a->base = (char *)base;
        a->capacity = (size_t)bytes & ~(kAlign - 1);
        a->owns = false;
    } else {
        a->capacity = ((size_t)bytes + kAlign - 1) & ~(kAlign - 1);
        int prev = 0;
        if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
            cudaGetLastError();
            delete a;
            return MAXFLOW_ERR_CUDA;
        }
        cudaError_t e = cudaMalloc((void **)&a->base, a->capacity);
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete a;
            return MAXFLOW_ERR_OOM;
        }
    }
    if (a->capacity == 0) {
        delete a;
        return MAXFLOW_ERR_INVALID;
    }
    insert_free(a, 0, a->capacity);
    *out = a;
    return MAXFLOW_OK;
}

void maxflow_arena_destroy(maxflow_arena *a)
{
    if (!a) return;
    if (a->owns || !a->overflow.empty()) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(a->device);
        cudaDeviceSynchronize();
        for (auto &kv : a->overflow) cudaFree(kv.first);
        if (a->owns) cudaFree(a->base);
        cudaSetDevice(prev);
    }
    delete a;
}

void *maxflow_arena_alloc(size_t bytes, void *user, void * /*stream*/)
{
    maxflow_arena *a = (maxflow_arena *)user;
    if (!a) return nullptr;
    const size_t size = ((bytes ? bytes : 1) + kAlign - 1) & ~(kAlign - 1);
    {
        std::lock_guard<std::mutex> lk(a->mu);
        if (size >= kLarge) {
            auto it = a->free_by_size.lower_bound({size, 0});
            if (it != a->free_by_size.end()) {
                const size_t bs = it->first, bo = it->second;
                take(a, bo, bs, bo, size);
                return a->base + bo;
            }
        } else {
            for (auto it = a->free_by_off.rbegin(); it != a->free_by_off.rend(); ++it) {
                if (it->second >= size) {
                    const size_t bo = it->first, bs = it->second;
                    take(a, bo, bs, bo + bs - size, size);
                    return a->base + bo + bs - size;
                }
            }
        }
        if (!a->allow_overflow) {
            a->failed++;
            return nullptr;
        }
    }
    void *p = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(a->device);
    cudaError_t e = cudaMalloc(&p, size);
    cudaSetDevice(prev);
    std::lock_guard<std::mutex> lk(a->mu);
    if (e != cudaSuccess) {
        cudaGetLastError();
        a->failed++;
        return nullptr;
    }
    a->overflow.emplace(p, size);
    a->fallbacks++;
    a->ov_in_use += (int64_t)size;
    if (a->ov_in_use > a->ov_peak) a->ov_peak = a->ov_in_use;
    return p;
}

void maxflow_arena_free(void *ptr, size_t /*bytes*/, void *user, void * /*stream*/)
{
    maxflow_arena *a = (maxflow_arena *)user;
    if (!a || !ptr) return;
    std::unique_lock<std::mutex> lk(a->mu);
    char *p = (char *)ptr;
    if (p >= a->base && p < a->base + a->capacity) {
        auto it = a->used.find((size_t)(p - a->base));
        if (it == a->used.end()) return;            // not ours: ignore
        const size_t off = it->first, size = it->second;
        a->used.erase(it);
        a->in_use -= (int64_t)size;
        insert_free(a, off, size);
        return;
    }
    auto ov = a->overflow.find(ptr);
    if (ov == a->overflow.end()) return;
    a->ov_in_use -= (int64_t)ov->second;
    a->overflow.erase(ov);
    lk.unlock();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(a->device);
    cudaFree(ptr);
    cudaSetDevice(prev);
}

int maxflow_arena_fits(maxflow_arena *a, const int64_t *sizes, int32_t count, int32_t *fits)
{
    if (!a || !fits || count < 0 || (count > 0 && !sizes)) return MAXFLOW_ERR_INVALID;
    std::lock_guard<std::mutex> lk(a->mu);
    // the placement policy of maxflow_arena_alloc, on a copy of the free list
    std::map<size_t, size_t> by_off = a->free_by_off;
    std::set<std::pair<size_t, size_t>> by_size = a->free_by_size;
    auto take_copy = [&](size_t bo, size_t bs, size_t off, size_t size) {
        by_off.erase(bo);
        by_size.erase({bs, bo});
        if (off > bo) {
            by_off.emplace(bo, off - bo);
            by_size.emplace(off - bo, bo);
        }
        if (bo + bs > off + size) {
            by_off.emplace(off + size, bo + bs - off - size);
            by_size.emplace(bo + bs - off - size, off + size);
        }
    };
    *fits = 1;
    for (int32_t i = 0; i < count; ++i) {
        const size_t size = (((size_t)(sizes[i] > 0 ? sizes[i] : 1)) + kAlign - 1) & ~(kAlign - 1);
        bool ok = false;
        if (size >= kLarge) {
            auto it = by_size.lower_bound({size, 0});
            if (it != by_size.end()) {
                const size_t bs = it->first, bo = it->second;
                take_copy(bo, bs, bo, size);
                ok = true;
            }
        } else {
            for (auto it = by_off.rbegin(); it != by_off.rend(); ++it) {
                if (it->second >= size) {
                    const size_t bo = it->first, bs = it->second;
                    take_copy(bo, bs, bo + bs - size, size);
                    ok = true;
                    break;
                }
            }
        }
        if (!ok) {
            *fits = 0;
            break;
        }
    }
    return MAXFLOW_OK;
}

int maxflow_arena_stats(maxflow_arena *a, maxflow_arena_stats_t *out)
{
    if (!a || !out) return MAXFLOW_ERR_INVALID;
    std::lock_guard<std::mutex> lk(a->mu);
    out->capacity = (int64_t)a->capacity;
    out->in_use = a->in_use;
    out->peak_in_use = a->peak;
    out->free_total = (int64_t)a->capacity - a->in_use;
    out->largest_free = a->free_by_size.empty() ? 0 : (int64_t)a->free_by_size.rbegin()->first;
    out->free_blocks = (int64_t)a->free_by_off.size();
    out->overflow_in_use = a->ov_in_use;
    out->overflow_peak = a->ov_peak;
    out->fallbacks = a->fallbacks;
    out->failed = a->failed;
    return MAXFLOW_OK;
}

}  // extern "C"
