/*
 * Plain CPU oracle for dynamic max-flow.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load or call this code.  The product path (the CUDA library) never links,
 * imports or runs it, and this file shares no code, header or table with it.
 *
 * Everything is written for clarity, not speed: 64-bit integers throughout,
 * no blocking, no fusion, sequential loops in the order the definitions or the
 * paper's algorithms state them.  Section numbers refer to the paper
 * "Scalable Maxflow Processing for Dynamic Graphs" (Kannappan, Kumar, Nasre).
 *
 * Contents
 *   1. The current graph: self-loops dropped, parallel edges summed.
 *   2. Maximum flow by Dinic's algorithm (Sec. 2.2: layered graphs and
 *      blocking flows) with the minimum cuts S_min / S_max and the cut
 *      capacity (max-flow = min-cut, Sec. 3.1 Theorem 3.4 and Ford-Fulkerson).
 *   3. Maximum flow by Edmonds-Karp on a residual matrix (Sec. 2.2),
 *      an independent second algorithm for small graphs.
 *   4. The paper's residual state (Sec. 5.1 Bi-CSR in abstract form): one
 *      directed slot (u,v) for every pair that has an edge in either
 *      direction, with cap(u,v), c_f(u,v), and the excess e(v).
 *        - flow load and the excess definition e(v) = sum_w (c_f(v,w) - c(v,w))
 *        - Alg. 1, initialisation (static initialisation and source saturation)
 *        - Alg. 4 / Alg. 6 (backward BFS heights = residual distance to the
 *          root set), written as a plain BFS
 *        - Alg. 5, batch part (apply a batch, clamp negative residuals,
 *          recompute excess, saturate the source edges again)
 *        - Alg. 2 on one vertex and Alg. 3, each callable as a single step
 *          from heights the caller sets, and both inside the Alg. 1 /
 *          Alg. 5 loop, run sequentially (one vertex at a time), and the
 *          value formula of Alg. 5.
 *   5. Sec. 5.2.2 (O2) push and pull: saturating the edges into t, the pull
 *      heights (distance from s and the overflowing vertices), pull-relabel
 *      (the mirror of Alg. 2 / Alg. 3 for deficient vertices), the sides of
 *      the last min cut, saturating the edges across it, and pushes / pulls
 *      restricted to one side's roots.
 *
 * Readings of the paper that this oracle takes where the text is ambiguous:
 *   R1 the dynamic loop of Alg. 5 runs until no active vertex remains;
 *   R2 Alg. 5's source step pushes the remaining residual c_f(s,u) and adds
 *      it to e(u) (it does not overwrite e(u));
 *   R3 the value is the sum of e(v) over v != s with h(v) < n, taken right
 *      after a backward BFS that finds no active vertex;
 *   R4 the BFS roots are t and every v not in {s,t} with e(v) < 0 (Alg. 6),
 *      in both the static and the dynamic solve; h(s) = n always;
 *   R5 a relabel with no residual neighbour sets h(u) = n, and every relabel
 *      is clamped to n;
 *   R6 ties among equal-height neighbours go to the first slot in row order
 *      (strict '<' of Alg. 2);
 *   R7 an update sets cap(u,v); a missing pair is inserted with capacity 0
 *      in both directions first; the last update of a pair in a batch wins;
 *      u == v is ignored.
 *   R8 (O2) pull heights: h(v) = residual distance from the root set
 *      {s} + {v not in {s,t}: e(v) > 0} to v; t is never labelled; a
 *      deficient vertex u (e(u) < 0, h(u) < n) pulls min(-e(u), c_f(z,u))
 *      from its lowest residual in-neighbour z when h(u) > h(z), else is
 *      relabelled to 1 + that lowest height (clamped to n); the pull value
 *      is the sum of -e(v) over v != t with h(v) < n;
 *   R9 (O2) the old min cut is T = {h < n} of the push heights the last
 *      solve ended with, S the rest; saturating the edges across it sends
 *      all of c_f(u, v) for u in S, v in T; the push part then takes as roots
 *      t and the deficient vertices of T only, the pull part s and the
 *      overflowing vertices of S only, and a final unrestricted push solve
 *      follows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOMEM 2
#define ORC_ERR_NOT_CONVERGED 3

static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* 1. The current graph                                                     */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t u, v; int64_t c; } orc_edge;

static int cmp_edge(const void *pa, const void *pb)
{
    const orc_edge *a = (const orc_edge *)pa, *b = (const orc_edge *)pb;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

/* Drop self-loops and sum parallel edges; output sorted by (u, v).
 * Returns the number of merged edges written to (mu, mv, mc), each of
 * capacity >= m, or -1 on invalid input. */
int64_t orc_merge(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                  int32_t *mu, int32_t *mv, int64_t *mc)
{
    orc_edge *E = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(m > 0 ? m : 1));
    int64_t k = 0, i, out = 0;
    if (!E) return -1;
    for (i = 0; i < m; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0) { free(E); return -1; }
        if (src[i] == dst[i]) continue;
        E[k].u = src[i]; E[k].v = dst[i]; E[k].c = cap[i]; k++;
    }
    qsort(E, (size_t)k, sizeof(orc_edge), cmp_edge);
    for (i = 0; i < k; i++) {
        if (out > 0 && mu[out - 1] == E[i].u && mv[out - 1] == E[i].v) {
            mc[out - 1] += E[i].c;
        } else {
            mu[out] = E[i].u; mv[out] = E[i].v; mc[out] = E[i].c; out++;
        }
    }
    free(E);
    return out;
}

/* ------------------------------------------------------------------------ */
/* 2. Dinic                                                                 */
/* ------------------------------------------------------------------------ */

/* Arc 2i is input edge i (u -> v, capacity c_i); arc 2i+1 is its reverse
 * (v -> u, capacity 0).  Self-loops get no usable arcs (both capacities 0). */
typedef struct {
    int32_t n;
    int64_t narcs;
    int32_t *to;      /* head of each arc */
    int64_t *res;     /* residual capacity of each arc */
    int64_t *first;   /* CSR over tails: arcs of vertex x are order[first[x] .. first[x+1]) */
    int64_t *order;
} dn_graph;

static void dn_free(dn_graph *g)
{
    free(g->to); free(g->res); free(g->first); free(g->order);
}

static int dn_build(dn_graph *g, int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap)
{
    int64_t i, a;
    int64_t *fill;
    g->n = n;
    g->narcs = 2 * m;
    g->to = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->res = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    g->first = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    fill = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g->to || !g->res || !g->first || !g->order || !fill) { free(fill); dn_free(g); return ORC_ERR_NOMEM; }
    for (i = 0; i < m; i++) {
        int loop = src[i] == dst[i];
        g->to[2 * i] = dst[i];
        g->res[2 * i] = loop ? 0 : cap[i];
        g->to[2 * i + 1] = src[i];
        g->res[2 * i + 1] = 0;
        g->first[src[i] + 1]++;
        g->first[dst[i] + 1]++;
    }
    for (i = 0; i < n; i++) g->first[i + 1] += g->first[i];
    for (i = 0; i < n; i++) fill[i] = g->first[i];
    for (a = 0; a < 2 * m; a++) {
        int32_t tail = g->to[a ^ 1];
        g->order[fill[tail]++] = a;
    }
    free(fill);
    return ORC_OK;
}

/* BFS levels from s over arcs with positive residual; returns 1 if t is reached. */
static int dn_levels(dn_graph *g, int32_t s, int32_t t, int32_t *level, int32_t *queue)
{
    int64_t head = 0, tail = 0, k;
    int32_t x;
    for (x = 0; x < g->n; x++) level[x] = -1;
    level[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t y = queue[head++];
        for (k = g->first[y]; k < g->first[y + 1]; k++) {
            int64_t a = g->order[k];
            int32_t z = g->to[a];
            if (g->res[a] > 0 && level[z] < 0) {
                level[z] = level[y] + 1;
                queue[tail++] = z;
            }
        }
    }
    return level[t] >= 0;
}

/* One blocking flow in the level graph, by depth-first search with
 * current-arc pointers (iterative, so long paths do not overflow the stack). */
static int64_t dn_blocking(dn_graph *g, int32_t s, int32_t t, const int32_t *level, int64_t *cur, int64_t *path)
{
    int64_t total = 0, top = 0, i;
    int32_t x = s;
    for (i = 0; i < g->n; i++) cur[i] = g->first[i];
    for (;;) {
        if (x == t) {
            int64_t b = INT64_MAX, cut_at = 0;
            for (i = 0; i < top; i++) b = min64(b, g->res[path[i]]);
            for (i = 0; i < top; i++) {
                g->res[path[i]] -= b;
                g->res[path[i] ^ 1] += b;
            }
            total += b;
            for (i = 0; i < top; i++) if (g->res[path[i]] == 0) { cut_at = i; break; }
            top = cut_at;
            x = (top == 0) ? s : g->to[path[top - 1]];
            continue;
        }
        {
            int advanced = 0;
            while (cur[x] < g->first[x + 1]) {
                int64_t a = g->order[cur[x]];
                int32_t z = g->to[a];
                if (g->res[a] > 0 && level[z] == level[x] + 1) {
                    path[top++] = a;
                    x = z;
                    advanced = 1;
                    break;
                }
                cur[x]++;
            }
            if (!advanced) {
                if (x == s) break;
                top--;
                x = (top == 0) ? s : g->to[path[top - 1]];
                cur[x]++;   /* the arc we came through leads to a dead end */
            }
        }
    }
    return total;
}

/* Maximum s-t flow of the COO multigraph (src, dst, cap), n vertices.
 *   flow_out (m entries, may be NULL): flow on each input edge, 0 <= f <= cap
 *   smin_out (n bytes, may be NULL): 1 for vertices reachable from s in the
 *             final residual graph (the smallest min-cut source side)
 *   smax_out (n bytes, may be NULL): 1 for vertices that cannot reach t in the
 *             final residual graph (the largest min-cut source side)
 *   cut_out (may be NULL): total capacity of input edges from S_min to V\S_min
 * Returns the value, or -1 on invalid input / no memory. */
int64_t orc_dinic(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                  int32_t s, int32_t t, int32_t *flow_out, uint8_t *smin_out, uint8_t *smax_out,
                  int64_t *cut_out, int64_t *phases_out)
{
    dn_graph g;
    int32_t *level, *queue;
    int64_t *cur, *path, value = 0, phases = 0, i;
    uint8_t *smin, *reach_t;
    if (n < 2 || s < 0 || s >= n || t < 0 || t >= n || s == t) return -1;
    for (i = 0; i < m; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0) return -1;
    if (dn_build(&g, n, m, src, dst, cap) != ORC_OK) return -1;
    level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    path = (int64_t *)malloc(sizeof(int64_t) * (size_t)n + 8);
    smin = (uint8_t *)calloc((size_t)n, 1);
    reach_t = (uint8_t *)calloc((size_t)n, 1);
    if (!level || !queue || !cur || !path || !smin || !reach_t) { value = -1; goto done; }

    while (dn_levels(&g, s, t, level, queue)) {
        value += dn_blocking(&g, s, t, level, cur, path);
        phases++;
    }

    /* S_min: reachable from s through positive residual arcs. */
    {
        int64_t head = 0, tail = 0, k;
        smin[s] = 1; queue[tail++] = s;
        while (head < tail) {
            int32_t y = queue[head++];
            for (k = g.first[y]; k < g.first[y + 1]; k++) {
                int64_t a = g.order[k];
                if (g.res[a] > 0 && !smin[g.to[a]]) { smin[g.to[a]] = 1; queue[tail++] = g.to[a]; }
            }
        }
    }
    /* Vertices that reach t: walk arcs backwards from t.  Arc a^1 leaves y, so
     * arc a enters y from to[a^1]... i.e. for an arc b out of y, arc b^1 goes
     * from to[b] into y. */
    {
        int64_t head = 0, tail = 0, k;
        reach_t[t] = 1; queue[tail++] = t;
        while (head < tail) {
            int32_t y = queue[head++];
            for (k = g.first[y]; k < g.first[y + 1]; k++) {
                int64_t b = g.order[k];
                int32_t x = g.to[b];
                if (g.res[b ^ 1] > 0 && !reach_t[x]) { reach_t[x] = 1; queue[tail++] = x; }
            }
        }
    }
    if (smin_out) memcpy(smin_out, smin, (size_t)n);
    if (smax_out) for (i = 0; i < n; i++) smax_out[i] = (uint8_t)!reach_t[i];
    if (flow_out)
        for (i = 0; i < m; i++) flow_out[i] = (src[i] == dst[i]) ? 0 : (int32_t)(cap[i] - g.res[2 * i]);
    if (cut_out) {
        int64_t c = 0;
        for (i = 0; i < m; i++) if (smin[src[i]] && !smin[dst[i]]) c += cap[i];
        *cut_out = c;
    }
    if (phases_out) *phases_out = phases;
done:
    free(level); free(queue); free(cur); free(path); free(smin); free(reach_t);
    dn_free(&g);
    return value;
}

/* ------------------------------------------------------------------------ */
/* 3. Edmonds-Karp on a dense residual matrix (small n only)                */
/* ------------------------------------------------------------------------ */

int64_t orc_edmonds_karp(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap,
                         int32_t s, int32_t t)
{
    int64_t *r, value = 0, i;
    int32_t *parent, *queue;
    if (n < 2 || n > 4096 || s < 0 || s >= n || t < 0 || t >= n || s == t) return -1;
    r = (int64_t *)calloc((size_t)n * (size_t)n, sizeof(int64_t));
    parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!r || !parent || !queue) { free(r); free(parent); free(queue); return -1; }
    for (i = 0; i < m; i++) {
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || cap[i] < 0) { value = -1; goto done; }
        if (src[i] != dst[i]) r[(size_t)src[i] * n + dst[i]] += cap[i];
    }
    for (;;) {
        int32_t head = 0, tail = 0, x;
        int64_t b;
        for (x = 0; x < n; x++) parent[x] = -1;
        parent[s] = s;
        queue[tail++] = s;
        while (head < tail && parent[t] < 0) {
            int32_t y = queue[head++], z;
            for (z = 0; z < n; z++)
                if (parent[z] < 0 && r[(size_t)y * n + z] > 0) { parent[z] = y; queue[tail++] = z; }
        }
        if (parent[t] < 0) break;
        b = INT64_MAX;
        for (x = t; x != s; x = parent[x]) b = min64(b, r[(size_t)parent[x] * n + x]);
        for (x = t; x != s; x = parent[x]) {
            r[(size_t)parent[x] * n + x] -= b;
            r[(size_t)x * n + parent[x]] += b;
        }
        value += b;
    }
done:
    free(r); free(parent); free(queue);
    return value;
}

/* ------------------------------------------------------------------------ */
/* 4. The paper's residual state                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n;
    int64_t K;          /* number of directed slots */
    int64_t *row;       /* slots of x: row[x] .. row[x+1], sorted by head */
    int32_t *head;      /* v of slot (u, v) */
    int64_t *cap;       /* c(u, v) (0 for a reverse-only slot) */
    int64_t *cf;        /* c_f(u, v) */
    int64_t *rev;       /* slot index of (v, u) */
    int64_t *e;         /* excess */
    int32_t *h;         /* heights of the last BFS / relabels */
} orc_rstate;

void orc_rs_free(orc_rstate *r)
{
    if (!r) return;
    free(r->row); free(r->head); free(r->cap); free(r->cf); free(r->rev); free(r->e); free(r->h);
    free(r);
}

/* Slot index of (u, v), or -1. */
static int64_t rs_find(const orc_rstate *r, int32_t u, int32_t v)
{
    int64_t lo = r->row[u], hi = r->row[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (r->head[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < r->row[u + 1] && r->head[lo] == v) ? lo : -1;
}

/* Build slots from merged edges (mu, mv, mc) plus the given cf per slot pair
 * (NULL: c_f = cap).  Every edge (u, v) gets a slot at u and one at v. */
static orc_rstate *rs_from_edges(int32_t n, int64_t m, const int32_t *mu, const int32_t *mv, const int64_t *mc)
{
    orc_rstate *r = (orc_rstate *)calloc(1, sizeof(orc_rstate));
    orc_edge *S;
    int64_t i, k = 0, K = 0, x;
    if (!r) return NULL;
    S = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(2 * m + 1));
    if (!S) { free(r); return NULL; }
    for (i = 0; i < m; i++) {
        S[k].u = mu[i]; S[k].v = mv[i]; S[k].c = mc[i]; k++;       /* forward slot with its capacity */
        S[k].u = mv[i]; S[k].v = mu[i]; S[k].c = -1; k++;          /* reverse slot, capacity unknown yet */
    }
    qsort(S, (size_t)k, sizeof(orc_edge), cmp_edge);
    /* unique (u, v): a real capacity (>= 0) beats the -1 placeholder */
    for (i = 0; i < k; i++) {
        if (K > 0 && S[K - 1].u == S[i].u && S[K - 1].v == S[i].v) {
            if (S[i].c >= 0) S[K - 1].c = (S[K - 1].c < 0 ? 0 : S[K - 1].c) + S[i].c;
        } else {
            S[K++] = S[i];
        }
    }
    r->n = n;
    r->K = K;
    r->row = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    r->head = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K + 1));
    r->cap = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
    r->cf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
    r->rev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
    r->e = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    r->h = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!r->row || !r->head || !r->cap || !r->cf || !r->rev || !r->e || !r->h) { free(S); orc_rs_free(r); return NULL; }
    for (i = 0; i < K; i++) {
        r->row[S[i].u + 1]++;
        r->head[i] = S[i].v;
        r->cap[i] = S[i].c < 0 ? 0 : S[i].c;
        r->cf[i] = r->cap[i];
    }
    for (x = 0; x < n; x++) r->row[x + 1] += r->row[x];
    free(S);
    for (x = 0; x < n; x++)
        for (i = r->row[x]; i < r->row[x + 1]; i++) r->rev[i] = rs_find(r, r->head[i], (int32_t)x);
    return r;
}

/* The excess definition: e(x) = sum over slots (x, w) of c_f(x, w) - c(x, w),
 * the net flow into x (the excess step of Alg. 5 recomputes it for every vertex). */
void orc_rs_recompute_excess(orc_rstate *r)
{
    int32_t x;
    int64_t i;
    for (x = 0; x < r->n; x++) {
        int64_t e = 0;
        for (i = r->row[x]; i < r->row[x + 1]; i++) e += r->cf[i] - r->cap[i];
        r->e[x] = e;
    }
}

/* A residual state of the current graph with zero flow. */
orc_rstate *orc_rs_new(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, const int32_t *cap)
{
    int32_t *mu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *mv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int64_t *mc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t mm;
    orc_rstate *r = NULL;
    if (mu && mv && mc && n >= 2) {
        mm = orc_merge(n, m, src, dst, cap, mu, mv, mc);
        if (mm >= 0) r = rs_from_edges(n, mm, mu, mv, mc);
    }
    free(mu); free(mv); free(mc);
    return r;
}

/* Load a flow: f(u, v) on each listed edge (u, v) with 0 <= f <= c(u, v);
 * unlisted edges carry 0.  c_f(u, v) = c(u, v) - f(u, v) + f(v, u); then the
 * excess follows from its definition.  Returns ORC_ERR_INVALID (and leaves
 * the state unchanged) if an item names a missing edge or exceeds capacity. */
int orc_rs_set_flow(orc_rstate *r, int64_t k, const int32_t *u, const int32_t *v, const int32_t *f)
{
    int64_t i;
    for (i = 0; i < k; i++) {
        int64_t a;
        if (u[i] < 0 || u[i] >= r->n || v[i] < 0 || v[i] >= r->n) return ORC_ERR_INVALID;
        a = rs_find(r, u[i], v[i]);
        if (a < 0 || f[i] < 0 || f[i] > r->cap[a]) return ORC_ERR_INVALID;
    }
    for (i = 0; i < r->K; i++) r->cf[i] = r->cap[i];
    for (i = 0; i < k; i++) {
        int64_t a = rs_find(r, u[i], v[i]);
        r->cf[a] -= f[i];
        r->cf[r->rev[a]] += f[i];
    }
    orc_rs_recompute_excess(r);
    return ORC_OK;
}

/* Alg. 1, initialisation: e = 0, h = 0, c_f = c, then saturate every edge out of s:
 * c_f(s,u) = 0, c_f(u,s) = c_us + c_su, e(u) = c_su, e(s) -= c_su. */
void orc_rs_static_init(orc_rstate *r, int32_t s)
{
    int64_t i;
    int32_t x;
    for (x = 0; x < r->n; x++) { r->e[x] = 0; r->h[x] = 0; }
    for (i = 0; i < r->K; i++) r->cf[i] = r->cap[i];
    for (i = r->row[s]; i < r->row[s + 1]; i++) {
        int32_t u = r->head[i];
        int64_t j = r->rev[i];
        int64_t c_su = r->cap[i], c_us = r->cap[j];
        r->cf[i] = 0;
        r->cf[j] = c_us + c_su;
        r->e[u] = c_su;
        r->e[s] -= c_su;
    }
}

/* Alg. 4 / Alg. 6: h(v) = number of residual edges on a shortest path from v
 * to the root set, where the roots are t and (if deficit_roots) every
 * v not in {s,t} with e(v) < 0; h(s) = n; vertices that reach no root get n.
 * A residual edge (x, y) has c_f(x, y) > 0. */
void orc_rs_heights(orc_rstate *r, int32_t s, int32_t t, int deficit_roots, int32_t *h_out)
{
    int32_t n = r->n, x;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t head = 0, tail = 0, i;
    for (x = 0; x < n; x++) r->h[x] = n;
    r->h[t] = 0;
    queue[tail++] = t;
    if (deficit_roots)
        for (x = 0; x < n; x++)
            if (x != s && x != t && r->e[x] < 0) { r->h[x] = 0; queue[tail++] = x; }
    while (head < tail) {
        int32_t y = queue[head++];
        for (i = r->row[y]; i < r->row[y + 1]; i++) {
            int32_t z = r->head[i];                 /* candidate predecessor z with edge (z, y) */
            if (z != s && r->h[z] == n && r->cf[r->rev[i]] > 0) {
                r->h[z] = r->h[y] + 1;
                queue[tail++] = z;
            }
        }
    }
    free(queue);
    if (h_out) memcpy(h_out, r->h, sizeof(int32_t) * (size_t)n);
}

/* Alg. 5, batch part, with readings R2 and R7.
 * Returns ORC_ERR_INVALID without changing the state if any update names a
 * vertex out of range or a negative capacity. */
int orc_rs_apply(orc_rstate **pr, int32_t s, int64_t B, const int32_t *bu, const int32_t *bv, const int32_t *bc)
{
    orc_rstate *r = *pr;
    int64_t i, k, nmiss = 0;
    int32_t n = r->n;
    orc_edge *U;
    for (i = 0; i < B; i++)
        if (bu[i] < 0 || bu[i] >= n || bv[i] < 0 || bv[i] >= n || bc[i] < 0) return ORC_ERR_INVALID;

    /* last update of each (u, v) wins: keep the final one, in batch order */
    U = (orc_edge *)malloc(sizeof(orc_edge) * (size_t)(B + 1));
    if (!U) return ORC_ERR_NOMEM;
    k = 0;
    for (i = B - 1; i >= 0; i--) {
        int64_t j, dup = 0;
        if (bu[i] == bv[i]) continue;
        for (j = 0; j < k; j++) if (U[j].u == bu[i] && U[j].v == bv[i]) { dup = 1; break; }
        if (!dup) { U[k].u = bu[i]; U[k].v = bv[i]; U[k].c = bc[i]; k++; }
    }

    /* insert every missing pair with capacity 0 both ways (keeping c_f and e) */
    for (i = 0; i < k; i++) if (rs_find(r, U[i].u, U[i].v) < 0) nmiss++;
    if (nmiss > 0) {
        int64_t m_old = 0, q = 0, x, j;
        int32_t *mu, *mv;
        int64_t *mc, *oldcf;
        orc_rstate *r2;
        for (x = 0; x < n; x++) m_old += r->row[x + 1] - r->row[x];
        mu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m_old + nmiss + 1));
        mv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m_old + nmiss + 1));
        mc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m_old + nmiss + 1));
        for (x = 0; x < n; x++)
            for (j = r->row[x]; j < r->row[x + 1]; j++) {
                mu[q] = (int32_t)x; mv[q] = r->head[j]; mc[q] = r->cap[j]; q++;
            }
        for (i = 0; i < k; i++)
            if (rs_find(r, U[i].u, U[i].v) < 0) { mu[q] = U[i].u; mv[q] = U[i].v; mc[q] = 0; q++; }
        r2 = rs_from_edges(n, q, mu, mv, mc);
        free(mu); free(mv); free(mc);
        if (!r2) { free(U); return ORC_ERR_NOMEM; }
        /* carry c_f, e, h over; new slots start at c_f = 0 */
        oldcf = r2->cf;
        for (j = 0; j < r2->K; j++) oldcf[j] = 0;
        for (x = 0; x < n; x++)
            for (j = r->row[x]; j < r->row[x + 1]; j++) r2->cf[rs_find(r2, (int32_t)x, r->head[j])] = r->cf[j];
        memcpy(r2->e, r->e, sizeof(int64_t) * (size_t)n);
        memcpy(r2->h, r->h, sizeof(int32_t) * (size_t)n);
        orc_rs_free(r);
        r = r2;
        *pr = r;
    }

    /* capacity step: c_f(u, v) += c'_uv - c_uv */
    for (i = 0; i < k; i++) {
        int64_t a = rs_find(r, U[i].u, U[i].v);
        r->cf[a] += U[i].c - r->cap[a];
        r->cap[a] = U[i].c;
    }
    free(U);
    /* clamp step: send back the flow that no longer fits */
    for (i = 0; i < r->K; i++) {
        if (r->cf[i] < 0) {
            r->cf[r->rev[i]] += r->cf[i];
            r->cf[i] = 0;
        }
    }
    /* excess step: excess from its definition */
    orc_rs_recompute_excess(r);
    /* source step (R2): saturate every edge out of s again */
    for (i = r->row[s]; i < r->row[s + 1]; i++) {
        int64_t d = r->cf[i];
        if (d > 0) {
            int32_t u = r->head[i];
            r->cf[i] = 0;
            r->cf[r->rev[i]] += d;
            r->e[u] += d;
            r->e[s] -= d;
        }
    }
    return ORC_OK;
}

/* Value formula (R3): sum of e(v) over v != s with h(v) < n. */
int64_t orc_rs_value(const orc_rstate *r, int32_t s)
{
    int64_t v = 0;
    int32_t x;
    for (x = 0; x < r->n; x++) if (x != s && r->h[x] < r->n) v += r->e[x];
    return v;
}

/* Heights given by the caller (h[v] in [0, n] for every v), for running the
 * single steps below from a state of the test's choosing. */
void orc_rs_set_heights(orc_rstate *r, const int32_t *h)
{
    memcpy(r->h, h, sizeof(int32_t) * (size_t)r->n);
}

/* Alg. 2 on one vertex u: kernel_cycles cycles; a cycle does nothing once u
 * is inactive (h(u) >= n or e(u) <= 0).  A cycle takes the residual slot
 * (u, v) (c_f > 0) whose head has the lowest height, the first slot in row
 * order on ties (R6).  If h(u) is above that height, it pushes
 * min(e(u), c_f(u, v)) along the slot; otherwise it relabels u to that
 * height + 1, or to n when u has no residual slot or the result would
 * exceed n - 1 (R5).  Returns the number of pushes; adds the relabels to
 * *relabels (may be NULL). */
int64_t orc_rs_discharge(orc_rstate *r, int32_t u, int32_t kernel_cycles, int64_t *relabels)
{
    int32_t n = r->n, cnt;
    int64_t pushes = 0;
    for (cnt = 0; cnt < kernel_cycles; cnt++) {
        int64_t best = -1, j;
        int32_t hbest = INT32_MAX;
        if (!(r->h[u] < n && r->e[u] > 0)) continue;
        for (j = r->row[u]; j < r->row[u + 1]; j++)
            if (r->cf[j] > 0 && r->h[r->head[j]] < hbest) { best = j; hbest = r->h[r->head[j]]; }
        if (best >= 0 && r->h[u] > hbest) {
            int64_t d = min64(r->e[u], r->cf[best]);
            int32_t v = r->head[best];
            r->cf[best] -= d;
            r->cf[r->rev[best]] += d;
            r->e[u] -= d;
            r->e[v] += d;
            pushes++;
        } else {
            r->h[u] = (best < 0 || hbest >= n - 1) ? n : hbest + 1;
            if (relabels) (*relabels)++;
        }
    }
    return pushes;
}

/* Alg. 3 on every vertex x not in {s, t}, in increasing id order: every slot
 * (x, v) with c_f(x, v) > 0 and h(x) > h(v) + 1 sends all of c_f(x, v) to v
 * (e(x) falls by it, possibly below 0; e(v) rises by it). */
void orc_rs_remove_invalid(orc_rstate *r, int32_t s, int32_t t)
{
    int32_t x;
    for (x = 0; x < r->n; x++) {
        int64_t j;
        if (x == s || x == t) continue;
        for (j = r->row[x]; j < r->row[x + 1]; j++) {
            int32_t v = r->head[j];
            if (r->cf[j] > 0 && r->h[x] > r->h[v] + 1) {
                int64_t c = r->cf[j];
                r->e[x] -= c;
                r->e[v] += c;
                r->cf[r->rev[j]] += c;
                r->cf[j] = 0;
            }
        }
    }
}

/* The method's loop run sequentially: repeat { Alg. 6 BFS; stop if no active
 * vertex; Alg. 2 on every active vertex in increasing id order; Alg. 3 on
 * every vertex not in {s,t} }.  Returns the value (R3) or -1 when max_iters
 * outer iterations did not reach a state without active vertices. */
int64_t orc_rs_push_relabel(orc_rstate *r, int32_t s, int32_t t, int32_t kernel_cycles, int64_t max_iters,
                            int64_t *iters_out, int64_t *pushes_out, int64_t *relabels_out)
{
    int32_t n = r->n, x;
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t it, pushes = 0, relabels = 0, nact = 0, i;
    for (it = 0; it < max_iters; it++) {
        orc_rs_heights(r, s, t, 1, NULL);
        nact = 0;
        for (x = 0; x < n; x++)
            if (x != s && x != t && r->e[x] > 0 && r->h[x] < n) active[nact++] = x;
        if (nact == 0) break;
        for (i = 0; i < nact; i++) pushes += orc_rs_discharge(r, active[i], kernel_cycles, &relabels);
        orc_rs_remove_invalid(r, s, t);
    }
    free(active);
    if (iters_out) *iters_out = it;
    if (pushes_out) *pushes_out = pushes;
    if (relabels_out) *relabels_out = relabels;
    if (nact != 0) return -1;
    return orc_rs_value(r, s);
}

/* ------------------------------------------------------------------------ */
/* 5. Sec. 5.2.2 (O2): push and pull                                        */
/* ------------------------------------------------------------------------ */

/* Static push-pull initialisation: saturate every edge into t as well:
 * for every pair (z, t), c_f(z, t) = 0, c_f(t, z) += that residual, the
 * residual leaves z (e(z) decreases, possibly below 0) and reaches t. */
void orc_rs_saturate_sink(orc_rstate *r, int32_t t)
{
    int64_t i;
    for (i = r->row[t]; i < r->row[t + 1]; i++) {
        int64_t j = r->rev[i];                 /* slot (z, t) */
        int32_t z = r->head[i];
        int64_t d = r->cf[j];
        if (d > 0) {
            r->cf[j] = 0;
            r->cf[i] += d;
            r->e[z] -= d;
            r->e[t] += d;
        }
    }
}

/* Push heights with the deficit roots limited to one side (R9):
 * roots are t and every v not in {s,t} with e(v) < 0 and side[v] == want
 * (side == NULL: every such v).  Same BFS as orc_rs_heights otherwise. */
void orc_rs_heights_side(orc_rstate *r, int32_t s, int32_t t, const uint8_t *side, int want)
{
    int32_t n = r->n, x;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t head = 0, tail = 0, i;
    for (x = 0; x < n; x++) r->h[x] = n;
    r->h[t] = 0;
    queue[tail++] = t;
    for (x = 0; x < n; x++)
        if (x != s && x != t && r->e[x] < 0 && (!side || side[x] == want)) { r->h[x] = 0; queue[tail++] = x; }
    while (head < tail) {
        int32_t y = queue[head++];
        for (i = r->row[y]; i < r->row[y + 1]; i++) {
            int32_t z = r->head[i];
            if (z != s && r->h[z] == n && r->cf[r->rev[i]] > 0) {
                r->h[z] = r->h[y] + 1;
                queue[tail++] = z;
            }
        }
    }
    free(queue);
}

/* Pull heights (R8): h(v) = residual distance from the roots s and every
 * v not in {s,t} with e(v) > 0 (and side[v] == want when side is given) to
 * v, following residual edges forward: y labelled, c_f(y, z) > 0 labels z. */
void orc_rs_pull_heights(orc_rstate *r, int32_t s, int32_t t, const uint8_t *side, int want, int32_t *h_out)
{
    int32_t n = r->n, x;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t head = 0, tail = 0, i;
    for (x = 0; x < n; x++) r->h[x] = n;
    r->h[s] = 0;
    queue[tail++] = s;
    for (x = 0; x < n; x++)
        if (x != s && x != t && r->e[x] > 0 && (!side || side[x] == want)) { r->h[x] = 0; queue[tail++] = x; }
    while (head < tail) {
        int32_t y = queue[head++];
        for (i = r->row[y]; i < r->row[y + 1]; i++) {
            int32_t z = r->head[i];                 /* residual edge (y, z) */
            if (z != t && r->h[z] == n && r->cf[i] > 0) {
                r->h[z] = r->h[y] + 1;
                queue[tail++] = z;
            }
        }
    }
    free(queue);
    if (h_out) memcpy(h_out, r->h, sizeof(int32_t) * (size_t)n);
}

/* Pull value (R8): sum of -e(v) over v != t with h(v) < n. */
int64_t orc_rs_pull_value(const orc_rstate *r, int32_t t)
{
    int64_t v = 0;
    int32_t x;
    for (x = 0; x < r->n; x++) if (x != t && r->h[x] < r->n) v -= r->e[x];
    return v;
}

/* Push-relabel as orc_rs_push_relabel, with the deficit roots of every BFS
 * limited to side[v] == want.  Returns 0, or -1 when max_iters iterations did
 * not reach a state without active vertices. */
int orc_rs_push_side(orc_rstate *r, int32_t s, int32_t t, const uint8_t *side, int want, int32_t kernel_cycles,
                     int64_t max_iters)
{
    int32_t n = r->n, x;
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t it, nact = 0, i;
    for (it = 0; it < max_iters; it++) {
        orc_rs_heights_side(r, s, t, side, want);
        nact = 0;
        for (x = 0; x < n; x++)
            if (x != s && x != t && r->e[x] > 0 && r->h[x] < n) active[nact++] = x;
        if (nact == 0) break;
        for (i = 0; i < nact; i++) orc_rs_discharge(r, active[i], kernel_cycles, NULL);
        orc_rs_remove_invalid(r, s, t);
    }
    free(active);
    return nact != 0 ? -1 : 0;
}

/* The mirror of Alg. 2 for one deficient vertex u (R8): kernel_cycles
 * cycles; a cycle does nothing once h(u) >= n or e(u) >= 0.  A cycle takes
 * the in-neighbour z with c_f(z, u) > 0 of lowest height (the first slot
 * (u, z) in row order on ties).  If h(u) is above it, u pulls
 * min(-e(u), c_f(z, u)) over (z, u); otherwise u is relabelled as in Alg. 2. */
void orc_rs_pull_discharge(orc_rstate *r, int32_t u, int32_t kernel_cycles)
{
    int32_t n = r->n, cnt;
    for (cnt = 0; cnt < kernel_cycles; cnt++) {
        int64_t best = -1, j;
        int32_t hbest = INT32_MAX;
        if (!(r->h[u] < n && r->e[u] < 0)) continue;
        for (j = r->row[u]; j < r->row[u + 1]; j++)      /* in-residual c_f(z, u) lives at rev[j] */
            if (r->cf[r->rev[j]] > 0 && r->h[r->head[j]] < hbest) { best = j; hbest = r->h[r->head[j]]; }
        if (best >= 0 && r->h[u] > hbest) {
            int64_t in = r->rev[best];
            int64_t d = min64(-r->e[u], r->cf[in]);
            r->cf[in] -= d;
            r->cf[best] += d;
            r->e[u] += d;
            r->e[r->head[best]] -= d;
        } else {
            r->h[u] = (best < 0 || hbest >= n - 1) ? n : hbest + 1;
        }
    }
}

/* The mirror of Alg. 3 (R8), every vertex x not in {s, t} in increasing id
 * order: every in-neighbour z with c_f(z, x) > 0 and h(x) > h(z) + 1 gives
 * all of c_f(z, x) to x (e(z) falls by it, e(x) rises by it). */
void orc_rs_pull_remove_invalid(orc_rstate *r, int32_t s, int32_t t)
{
    int32_t x;
    for (x = 0; x < r->n; x++) {
        int64_t j;
        if (x == s || x == t) continue;
        for (j = r->row[x]; j < r->row[x + 1]; j++) {
            int32_t z = r->head[j];
            int64_t in = r->rev[j];
            if (r->cf[in] > 0 && r->h[x] > r->h[z] + 1) {
                int64_t c = r->cf[in];
                r->e[x] += c;
                r->e[z] -= c;
                r->cf[j] += c;
                r->cf[in] = 0;
            }
        }
    }
}

/* Pull-relabel (R8), the mirror of Alg. 2 / Alg. 3: repeat { pull heights;
 * stop if no deficient vertex v not in {s,t} has h(v) < n; every such u, in
 * increasing id order, up to kernel_cycles times: pull from the lowest
 * residual in-neighbour or relabel; then for every u not in {s,t}, every
 * in-neighbour z with c_f(z, u) > 0 and h(u) > h(z) + 1 gives all of it }.
 * Roots limited to side[v] == want when side is given.  Returns 0 or -1. */
int orc_rs_pull_relabel(orc_rstate *r, int32_t s, int32_t t, const uint8_t *side, int want, int32_t kernel_cycles,
                        int64_t max_iters, int64_t *iters_out)
{
    int32_t n = r->n, x;
    int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t it, nact = 0, i;
    for (it = 0; it < max_iters; it++) {
        orc_rs_pull_heights(r, s, t, side, want, NULL);
        nact = 0;
        for (x = 0; x < n; x++)
            if (x != s && x != t && r->e[x] < 0 && r->h[x] < n) active[nact++] = x;
        if (nact == 0) break;
        for (i = 0; i < nact; i++) orc_rs_pull_discharge(r, active[i], kernel_cycles);
        orc_rs_pull_remove_invalid(r, s, t);
    }
    free(active);
    if (iters_out) *iters_out = it;
    return nact != 0 ? -1 : 0;
}

/* Sides of the last min cut (R9) from the current push heights:
 * side[v] = 1 (T) when h(v) < n, else 0 (S). */
void orc_rs_cut_side(const orc_rstate *r, uint8_t *side)
{
    int32_t x;
    for (x = 0; x < r->n; x++) side[x] = r->h[x] < r->n ? 1 : 0;
}

/* Saturate the edges across the cut (R9): every slot (u, v) with u in S,
 * v in T sends all of c_f(u, v). */
void orc_rs_saturate_cut(orc_rstate *r, const uint8_t *side)
{
    int32_t x;
    int64_t i;
    for (x = 0; x < r->n; x++) {
        if (side[x] != 0) continue;
        for (i = r->row[x]; i < r->row[x + 1]; i++) {
            int32_t v = r->head[i];
            int64_t d = r->cf[i];
            if (side[v] == 1 && d > 0) {
                r->cf[i] = 0;
                r->cf[r->rev[i]] += d;
                r->e[x] -= d;
                r->e[v] += d;
            }
        }
    }
}

/* ---- accessors ---------------------------------------------------------- */

int64_t orc_rs_num_slots(const orc_rstate *r) { return r->K; }
int32_t orc_rs_n(const orc_rstate *r) { return r->n; }

/* Slots in row order: (u, v, c(u,v), c_f(u,v)). */
void orc_rs_get_slots(const orc_rstate *r, int32_t *u, int32_t *v, int64_t *cap, int64_t *cf)
{
    int32_t x;
    int64_t i;
    for (x = 0; x < r->n; x++)
        for (i = r->row[x]; i < r->row[x + 1]; i++) {
            if (u) u[i] = x;
            if (v) v[i] = r->head[i];
            if (cap) cap[i] = r->cap[i];
            if (cf) cf[i] = r->cf[i];
        }
}

void orc_rs_get_vertex(const orc_rstate *r, int64_t *e, int32_t *h)
{
    if (e) memcpy(e, r->e, sizeof(int64_t) * (size_t)r->n);
    if (h) memcpy(h, r->h, sizeof(int32_t) * (size_t)r->n);
}

/* The certificate of Theorem 3.4 on the current state: A = {h == n}; returns
 * the capacity of all edges (u, v) with u in A and v not in A, and stores in
 * *residual_out the number of slots (u, v), u in A, v not in A, with c_f > 0. */
int64_t orc_rs_cut(const orc_rstate *r, int64_t *residual_out)
{
    int64_t c = 0, bad = 0, i;
    int32_t x;
    for (x = 0; x < r->n; x++) {
        if (r->h[x] != r->n) continue;
        for (i = r->row[x]; i < r->row[x + 1]; i++) {
            if (r->h[r->head[i]] == r->n) continue;
            c += r->cap[i];
            if (r->cf[i] > 0) bad++;
        }
    }
    if (residual_out) *residual_out = bad;
    return c;
}
