// Host construction of the residual Bi-CSR (Sec. 5.1).
//
// The paper's Bi-CSR stores, for every vertex, both its outgoing and its
// incoming edges, adds a zero-capacity entry wherever a reverse edge is
// missing, and keeps the index of each entry's reverse so that a push touches
// a constant number of words.  Here every unordered pair {u, v} with an edge
// in either direction becomes two slots, (u, v) in row u and (v, u) in row v,
// each with its own capacity (0 if that direction has no edge) and the index
// of the other.  Rows are sorted by head so an update can find its slot by
// binary search, and each row reserves spare slots after its used ones so an
// update can insert a new pair without moving other rows.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/maxflow.h"
#include "mf_internal.h"

namespace {

struct SlotRec {
    int32_t v;
    int32_t cap;   // -1: placeholder for the reverse of an edge (capacity 0 unless that edge exists)
    int32_t cf;
};

template <class F>
void parallel_rows(int32_t n, F fn)
{
    unsigned T = std::thread::hardware_concurrency();
    if (T == 0) T = 1;
    if (T > 32) T = 32;
    if (n < 65536 || T == 1) {
        fn(0, n);
        return;
    }
    std::vector<std::thread> th;
    int32_t per = (n + (int32_t)T - 1) / (int32_t)T;
    for (unsigned k = 0; k < T; ++k) {
        int32_t lo = (int32_t)k * per, hi = std::min<int32_t>(n, lo + per);
        if (lo >= hi) break;
        th.emplace_back([=] { fn(lo, hi); });
    }
    for (auto &x : th) x.join();
}

int32_t slack_of(int64_t deg, float factor, int32_t smin)
{
    double want = (double)deg * (double)factor;
    int64_t s = (int64_t)want;
    if ((double)s < want) ++s;
    if (s < smin) s = smin;
    if (s > (1 << 24)) s = 1 << 24;
    return (int32_t)s;
}

// rows[u] holds (v, cap, cf) records; entries are unique per (u, v) after
// merge_row.  Builds the device layout.
int layout(int32_t n, std::vector<int64_t> &rstart, std::vector<SlotRec> &recs, float slack_factor,
           int32_t slack_min, MfHostGraph &out)
{
    out.n = n;
    // every row starts on a multiple of MF_ROW_ALIGN slots (16 bytes), so the
    // kernels can read a row's slot fields four at a time with 16-byte loads
    std::vector<int64_t> offs((size_t)n + 1, 0);
    for (int32_t u = 0; u < n; ++u) {
        int64_t d = rstart[u + 1] - rstart[u];
        int64_t r = d + slack_of(d, slack_factor, slack_min);
        r = (r + MF_ROW_ALIGN - 1) / MF_ROW_ALIGN * MF_ROW_ALIGN;
        offs[u + 1] = offs[u] + r;
    }
    if (offs[n] >= (int64_t)INT32_MAX - 1) return MAXFLOW_ERR_TOO_LARGE;
    out.slot_cap = offs[n];
    out.slots = rstart[n];
    size_t S = (size_t)out.slot_cap;
    out.off = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    out.deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    out.bdeg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    out.dst = (int32_t *)calloc(S + 1, sizeof(int32_t));
    out.cap = (int32_t *)calloc(S + 1, sizeof(int32_t));
    out.cf = (int32_t *)calloc(S + 1, sizeof(int32_t));
    out.rev = (int32_t *)calloc(S + 1, sizeof(int32_t));
    out.pcap = (int32_t *)calloc(S + 1, sizeof(int32_t));
    if (!out.off || !out.deg || !out.bdeg || !out.dst || !out.cap || !out.cf || !out.rev || !out.pcap) {
        out.release();
        return MAXFLOW_ERR_OOM;
    }
    for (int32_t u = 0; u <= n; ++u) out.off[u] = (int32_t)offs[u];
    int64_t m_real = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t d = rstart[u + 1] - rstart[u];
        out.deg[u] = (int32_t)d;
        out.bdeg[u] = (int32_t)d;
        int32_t base = out.off[u];
        for (int64_t j = 0; j < d; ++j) {
            const SlotRec &r = recs[(size_t)(rstart[u] + j)];
            out.dst[base + j] = r.v;
            out.cap[base + j] = r.cap;
            out.cf[base + j] = r.cf;
            if (r.cap > 0) ++m_real;
        }
        // unused slack: a self-reference with zero capacity (never read by the kernels)
        for (int32_t x = base + (int32_t)d; x < out.off[u + 1]; ++x) {
            out.dst[x] = u;
            out.rev[x] = x;
        }
    }
    out.m_merged = m_real;
    bool bad = false;
    parallel_rows(n, [&](int32_t lo, int32_t hi) {
        for (int32_t u = lo; u < hi; ++u) {
            int32_t base = out.off[u];
            for (int32_t j = 0; j < out.deg[u]; ++j) {
                int32_t v = out.dst[base + j];
                const int32_t *b = out.dst + out.off[v];
                const int32_t *e = b + out.bdeg[v];
                const int32_t *p = std::lower_bound(b, e, u);
                if (p == e || *p != u) { bad = true; continue; }
                int32_t x = base + j, y = (int32_t)(p - out.dst);
                out.rev[x] = y;
                int64_t pc = (int64_t)out.cap[x] + (int64_t)out.cap[y];
                if (pc > INT32_MAX) { bad = true; continue; }
                out.pcap[x] = (int32_t)pc;
            }
        }
    });
    if (bad) {
        out.release();
        return MAXFLOW_ERR_TOO_LARGE;   // only a pair-capacity overflow can get here
    }
    return MAXFLOW_OK;
}

// Counting sort of (u, rec) by u, then per row sort by v and merge equal v.
// merge: caps of real entries are summed (placeholders add nothing); cf is
// summed over real entries too (the caller sets it consistently).
int group_rows(int32_t n, const std::vector<int32_t> &ru, std::vector<SlotRec> &rr, std::vector<int64_t> &rstart,
               std::vector<SlotRec> &out)
{
    size_t K = ru.size();
    rstart.assign((size_t)n + 1, 0);
    for (size_t i = 0; i < K; ++i) rstart[(size_t)ru[i] + 1]++;
    for (int32_t u = 0; u < n; ++u) rstart[u + 1] += rstart[u];
    std::vector<int64_t> fill(rstart.begin(), rstart.end() - 1);
    out.resize(K);
    for (size_t i = 0; i < K; ++i) out[(size_t)fill[ru[i]]++] = rr[i];
    std::vector<int64_t> newlen((size_t)n, 0);
    bool overflow = false;
    parallel_rows(n, [&](int32_t lo, int32_t hi) {
        for (int32_t u = lo; u < hi; ++u) {
            SlotRec *b = out.data() + rstart[u], *e = out.data() + rstart[u + 1];
            std::sort(b, e, [](const SlotRec &a, const SlotRec &c) { return a.v < c.v; });
            int64_t w = 0;
            for (SlotRec *p = b; p < e; ++p) {
                if (w > 0 && b[w - 1].v == p->v) {
                    SlotRec &q = b[w - 1];
                    if (p->cap >= 0) {
                        int64_t c = (int64_t)(q.cap < 0 ? 0 : q.cap) + p->cap;
                        int64_t f = (int64_t)(q.cap < 0 ? 0 : q.cf) + p->cf;
                        if (c > INT32_MAX || f > INT32_MAX) overflow = true;
                        q.cap = (int32_t)c;
                        q.cf = (int32_t)f;
                    }
                } else {
                    b[w++] = *p;
                }
            }
            for (int64_t j = 0; j < w; ++j)
                if (b[j].cap < 0) { b[j].cap = 0; b[j].cf = 0; }
            newlen[u] = w;
        }
    });
    if (overflow) return MAXFLOW_ERR_TOO_LARGE;
    // compact rows
    int64_t pos = 0;
    for (int32_t u = 0; u < n; ++u) {
        int64_t b = rstart[u];
        if (pos != b)
            std::memmove(out.data() + pos, out.data() + b, sizeof(SlotRec) * (size_t)newlen[u]);
        rstart[u] = pos;
        pos += newlen[u];
    }
    rstart[n] = pos;
    out.resize((size_t)pos);
    return MAXFLOW_OK;
}

}  // namespace

void MfHostGraph::release()
{
    free(off); free(deg); free(bdeg); free(dst); free(cap); free(rev); free(pcap); free(cf);
    off = deg = bdeg = dst = cap = rev = pcap = cf = nullptr;
}

int mf_build_host(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                  float slack_factor, int32_t slack_min, MfHostGraph &out)
{
    if (n < 2 || m < 0) return MAXFLOW_ERR_INVALID;
    if (m > 0 && (!src || !dst || !cap)) return MAXFLOW_ERR_INVALID;
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0) return MAXFLOW_ERR_INVALID;
        if (src[i] != dst[i]) ++k;
    }
    // Step 1: merge parallel edges per (u, v).
    std::vector<int32_t> ru;
    std::vector<SlotRec> rr;
    ru.reserve((size_t)k);
    rr.reserve((size_t)k);
    for (int64_t i = 0; i < m; ++i) {
        if (src[i] == dst[i]) continue;
        ru.push_back(src[i]);
        rr.push_back(SlotRec{dst[i], cap[i], cap[i]});
    }
    std::vector<int64_t> rstart;
    std::vector<SlotRec> merged;
    int rc = group_rows(n, ru, rr, rstart, merged);
    if (rc != MAXFLOW_OK) return rc;
    // Step 2: both directions of every pair; a reverse without an edge is a placeholder.
    size_t M = merged.size();
    ru.clear();
    rr.clear();
    ru.reserve(2 * M);
    rr.reserve(2 * M);
    for (int32_t u = 0; u < n; ++u)
        for (int64_t j = rstart[u]; j < rstart[u + 1]; ++j) {
            const SlotRec &e = merged[(size_t)j];
            ru.push_back(u);
            rr.push_back(SlotRec{e.v, e.cap, e.cap});
            ru.push_back(e.v);
            rr.push_back(SlotRec{u, -1, 0});
        }
    std::vector<SlotRec>().swap(merged);
    std::vector<SlotRec> slots;
    rc = group_rows(n, ru, rr, rstart, slots);
    if (rc != MAXFLOW_OK) return rc;
    std::vector<int32_t>().swap(ru);
    std::vector<SlotRec>().swap(rr);
    return layout(n, rstart, slots, slack_factor, slack_min, out);
}
