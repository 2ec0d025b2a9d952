"""Seeded synthetic inputs: graphs and update batches.

This module draws the inputs that both the CUDA path and the CPU oracle are
fed.  It holds none of the max-flow arithmetic (no residual capacities, no
excess, no heights): only random graphs, random capacity assignments and the
bookkeeping of which directed edges currently exist with which capacity
(the "set capacity" semantics of an update batch, Sec. 4.1).

The paper's datasets (Table 1: Pokec, Flickr, StackOverflow, Wikipedia,
LiveJournal; weighted, capacities 1..100) are not available here.  The
generators below stand in for them with the same shape: power-law R-MAT graphs
of 1M-4M vertices and average degree ~16, a segmentation-shaped grid, an
Erdos-Renyi small case and mixes of small instances.  Update batches follow
Sec. 6.2 (existing edges picked at random, capacities raised or lowered), with
insertions and deletions added.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    """A directed graph in COO form with int32 capacities, plus source and sink."""

    n: int
    src: np.ndarray
    dst: np.ndarray
    cap: np.ndarray
    s: int
    t: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _round_half_up(x: float) -> int:
    return int(math.floor(x + 0.5))


# ---------------------------------------------------------------------------
# The current edge set of a dynamic graph
# ---------------------------------------------------------------------------


class EdgeSet:
    """Directed edges (u, v) -> capacity of the current graph, as sorted keys.

    An update (u, v, c') sets the capacity of (u, v) to c' (inserting the edge
    when it is absent); c' = 0 deletes it in the sense that the edge keeps a
    zero capacity.  Within one batch the last update of a pair wins.  The
    initial graph must be a simple digraph (no self-loops, no parallel edges).
    """

    def __init__(self, n: int, src, dst, cap):
        self.n = int(n)
        src = np.asarray(src, dtype=np.int64)
        dst = np.asarray(dst, dtype=np.int64)
        keys = src * self.n + dst
        order = np.argsort(keys, kind="stable")
        self.keys = keys[order]
        if self.keys.size and np.any(self.keys[1:] == self.keys[:-1]):
            raise ValueError("EdgeSet needs distinct (u, v) pairs")
        self.caps = np.asarray(cap, dtype=np.int64)[order].copy()

    @property
    def m(self) -> int:
        return int(self.keys.size)

    def copy(self) -> "EdgeSet":
        e = EdgeSet.__new__(EdgeSet)
        e.n, e.keys, e.caps = self.n, self.keys.copy(), self.caps.copy()
        return e

    def contains(self, u, v) -> np.ndarray:
        k = np.asarray(u, dtype=np.int64) * self.n + np.asarray(v, dtype=np.int64)
        pos = np.searchsorted(self.keys, k)
        pos = np.minimum(pos, max(self.keys.size - 1, 0))
        return (self.keys.size > 0) & (self.keys[pos] == k)

    def cap_of(self, u, v) -> np.ndarray:
        k = np.asarray(u, dtype=np.int64) * self.n + np.asarray(v, dtype=np.int64)
        pos = np.searchsorted(self.keys, k)
        ok = (pos < self.keys.size)
        ok[ok] = self.keys[pos[ok]] == k[ok]
        out = np.zeros(k.shape, dtype=np.int64)
        out[ok] = self.caps[pos[ok]]
        return out

    def apply(self, u, v, c) -> None:
        """Set cap(u, v) = c for every update; last one wins; u == v ignored."""
        u = np.asarray(u, dtype=np.int64)
        v = np.asarray(v, dtype=np.int64)
        c = np.asarray(c, dtype=np.int64)
        keep = u != v
        u, v, c = u[keep], v[keep], c[keep]
        k = u * self.n + v
        # last occurrence of every key
        rk = k[::-1]
        uk, first_in_rev = np.unique(rk, return_index=True)
        ck = c[::-1][first_in_rev]
        pos = np.searchsorted(self.keys, uk)
        hit = pos < self.keys.size
        hit[hit] = self.keys[pos[hit]] == uk[hit]
        self.caps[pos[hit]] = ck[hit]
        if np.any(~hit):
            nk, nc = uk[~hit], ck[~hit]
            ins = np.searchsorted(self.keys, nk)
            self.keys = np.insert(self.keys, ins, nk)
            self.caps = np.insert(self.caps, ins, nc)

    def coo(self):
        u = (self.keys // self.n).astype(np.int32)
        v = (self.keys % self.n).astype(np.int32)
        return u, v, self.caps.astype(np.int32)


# ---------------------------------------------------------------------------
# Update batches (Sec. 6.2 recipe, plus insert / delete)
# ---------------------------------------------------------------------------


@dataclass
class Batch:
    u: np.ndarray
    v: np.ndarray
    cap: np.ndarray

    @property
    def size(self) -> int:
        return int(self.u.shape[0])


def mixed_batch(es: EdgeSet, B: int, rng: np.random.Generator, ins_cap_hi: int,
                inc_hi: int = 50, frac=(0.4, 0.4, 0.1), st_bias=None) -> Batch:
    """A batch of B capacity-set updates: increase / decrease / insert / delete.

    Counts are round(0.4B), round(0.4B), round(0.1B) and the rest.  Increases
    add U[1, inc_hi] to an existing edge, decreases set it to U[0, cap],
    inserts add a pair (u, v) with neither (u, v) nor (v, u) present, capacity
    U[1, ins_cap_hi], and deletes set an existing edge to 0.  Existing edges
    are chosen uniformly without replacement within the batch.  When
    st_bias=(s, t, p) is given, a fraction p of the changed existing edges is
    drawn from the edges out of s and into t (Sec. 6.2 picks those with a
    higher probability).
    """
    n_inc = _round_half_up(frac[0] * B)
    n_dec = _round_half_up(frac[1] * B)
    n_ins = _round_half_up(frac[2] * B)
    n_del = B - n_inc - n_dec - n_ins
    n_old = n_inc + n_dec + n_del
    m = es.m
    if n_old > m:
        raise ValueError("batch larger than the edge set")
    if st_bias is not None:
        s, t, p = st_bias
        eu = es.keys // es.n
        ev = es.keys % es.n
        special = np.flatnonzero((eu == s) | (ev == t))
        k_sp = min(int(round(p * n_old)), special.size)
        pick_sp = rng.choice(special, size=k_sp, replace=False) if k_sp else np.zeros(0, np.int64)
        mask = np.ones(m, dtype=bool)
        mask[pick_sp] = False
        rest = np.flatnonzero(mask)
        pick_rest = rng.choice(rest, size=n_old - k_sp, replace=False)
        idx = rng.permutation(np.concatenate([pick_sp, pick_rest]))
    else:
        idx = rng.choice(m, size=n_old, replace=False)
    ku = es.keys[idx] // es.n
    kv = es.keys[idx] % es.n
    kc = es.caps[idx]
    i_inc, i_dec, i_del = idx[:n_inc], idx[n_inc:n_inc + n_dec], idx[n_inc + n_dec:]
    new_inc = kc[:n_inc] + rng.integers(1, inc_hi + 1, size=n_inc)
    old_dec = kc[n_inc:n_inc + n_dec]
    new_dec = np.floor(rng.random(n_dec) * (old_dec + 1)).astype(np.int64)
    new_dec = np.minimum(new_dec, old_dec)
    new_del = np.zeros(n_del, dtype=np.int64)
    del i_inc, i_dec, i_del
    # inserts: fresh pairs with no edge in either direction, distinct in the batch
    iu = np.zeros(0, np.int64)
    iv = np.zeros(0, np.int64)
    n = es.n
    tries = 0
    while iu.size < n_ins:
        tries += 1
        if tries > 64:
            raise RuntimeError("could not draw enough fresh pairs")
        want = (n_ins - iu.size) * 2 + 16
        cu = rng.integers(0, n, size=want)
        cv = rng.integers(0, n, size=want)
        ok = cu != cv
        cu, cv = cu[ok], cv[ok]
        ok = ~es.contains(cu, cv) & ~es.contains(cv, cu)
        cu, cv = cu[ok], cv[ok]
        allu = np.concatenate([iu, cu])
        allv = np.concatenate([iv, cv])
        pk = np.minimum(allu, allv) * n + np.maximum(allu, allv)
        _, first = np.unique(pk, return_index=True)
        first.sort()
        iu, iv = allu[first][:n_ins], allv[first][:n_ins]
    ic = rng.integers(1, ins_cap_hi + 1, size=n_ins)
    u = np.concatenate([ku, iu])
    v = np.concatenate([kv, iv])
    c = np.concatenate([new_inc, new_dec, new_del, ic])
    perm = rng.permutation(B)
    return Batch(_i32(u[perm]), _i32(v[perm]), _i32(c[perm]))


def kind_batch(es: EdgeSet, B: int, rng: np.random.Generator, kind: str, inc_hi: int = 50) -> Batch:
    """A batch of only increases ('inc'), decreases ('dec') or half/half ('mix'), Sec. 6.2.1-6.2.3."""
    idx = rng.choice(es.m, size=B, replace=False)
    u = es.keys[idx] // es.n
    v = es.keys[idx] % es.n
    c = es.caps[idx]
    inc = c + rng.integers(1, inc_hi + 1, size=B)
    dec = np.minimum(np.floor(rng.random(B) * (c + 1)).astype(np.int64), c)
    if kind == "inc":
        newc = inc
    elif kind == "dec":
        newc = dec
    elif kind == "mix":
        half = B // 2
        newc = np.concatenate([inc[:half], dec[half:]])
    else:
        raise ValueError(kind)
    return Batch(_i32(u), _i32(v), _i32(newc))


# ---------------------------------------------------------------------------
# Graph families
# ---------------------------------------------------------------------------


def random_multigraph(n: int, m: int, seed: int, cap_hi: int = 20, zero_frac: float = 0.1,
                      loops: bool = True) -> tuple:
    """Small random multigraph (parallel edges, self-loops, zero capacities) for tests."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    if not loops:
        v = np.where(u == v, (v + 1) % n, v)
    c = rng.integers(1, cap_hi + 1, size=m)
    c[rng.random(m) < zero_frac] = 0
    return _i32(u), _i32(v), _i32(c)


def erdos_renyi(n: int, m: int, seed: int, cap_lo: int = 1, cap_hi: int = 100) -> Graph:
    """Directed G(n, m): m distinct random pairs u != v, capacities U[cap_lo, cap_hi]."""
    rng = np.random.default_rng(seed)
    keys = np.zeros(0, np.int64)
    while keys.size < m:
        want = (m - keys.size) * 2 + 64
        u = rng.integers(0, n, size=want)
        v = rng.integers(0, n, size=want)
        k = (u * n + v)[u != v]
        allk = np.concatenate([keys, k])
        _, first = np.unique(allk, return_index=True)
        first.sort()
        keys = allk[first][:m]
    src, dst = keys // n, keys % n
    cap = rng.integers(cap_lo, cap_hi + 1, size=m)
    return Graph(n, _i32(src), _i32(dst), _i32(cap), 0, n - 1, name=f"er_n{n}_m{m}")


def rmat_edges(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """Raw R-MAT draws (with self-loops and duplicates), no noise."""
    rng = np.random.default_rng(seed)
    M = edge_factor << scale
    u = np.zeros(M, dtype=np.uint32)
    v = np.zeros(M, dtype=np.uint32)
    ab = a + b
    a_in_ab = a / ab
    c_in_cd = c / (1.0 - ab)
    for bit in range(scale - 1, -1, -1):
        r1 = rng.random(M, dtype=np.float32)
        r2 = rng.random(M, dtype=np.float32)
        lower = r1 >= ab                        # quadrant c or d: u bit set
        thr = np.where(lower, np.float32(c_in_cd), np.float32(a_in_ab))
        right = r2 >= thr                       # quadrant b or d: v bit set
        u[lower] |= np.uint32(1 << bit)
        v[right] |= np.uint32(1 << bit)
        del r1, r2, lower, right, thr
    return u.astype(np.int64), v.astype(np.int64)


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    keys = np.sort(keys)
    if keys.size == 0:
        return keys
    keep = np.empty(keys.size, dtype=bool)
    keep[0] = True
    np.not_equal(keys[1:], keys[:-1], out=keep[1:])
    return keys[keep]


def _csr_sym(n, src, dst):
    import scipy.sparse as sp
    data = np.ones(src.size, dtype=np.int8)
    g = sp.csr_matrix((data, (src, dst)), shape=(n, n))
    return g


def rmat(scale: int = 20, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2, cap_lo: int = 1, cap_hi: int = 1000) -> Graph:
    """R-MAT power-law digraph; self-loops dropped, duplicates merged, caps U[cap_lo, cap_hi].

    s and t: an undirected BFS from the highest-degree vertex r splits its visit
    order in two halves P and Q; s is the highest-degree vertex of P (r itself)
    and t the highest-degree vertex of Q that s reaches in the directed graph.
    """
    import scipy.sparse.csgraph as csg
    n = 1 << scale
    u, v = rmat_edges(scale, edge_factor, a, b, c, seed)
    keep = u != v
    keys = _sorted_unique(u[keep] * n + v[keep])
    del u, v, keep
    src, dst = keys // n, keys % n
    rng = np.random.default_rng(seed + 7919)
    cap = rng.integers(cap_lo, cap_hi + 1, size=keys.size)
    deg = np.bincount(src, minlength=n) + np.bincount(dst, minlength=n)
    r = int(np.argmax(deg))
    g = _csr_sym(n, src, dst)
    order = csg.breadth_first_order(g, r, directed=False, return_predecessors=False)
    half = order.size // 2
    P, Q = order[:half], order[half:]
    s = int(P[np.argmax(deg[P])])
    reach = np.zeros(n, dtype=bool)
    reach[csg.breadth_first_order(g, s, directed=True, return_predecessors=False)] = True
    cand = Q[np.lexsort((Q, -deg[Q]))]
    cand = cand[reach[cand] & (cand != s)]
    if cand.size == 0:
        raise RuntimeError("no reachable sink candidate")
    t = int(cand[0])
    return Graph(n, _i32(src), _i32(dst), _i32(cap), s, t, name=f"rmat_s{scale}_ef{edge_factor}",
                 meta={"raw_edges": edge_factor << scale, "m_merged": int(keys.size)})


# --- segmentation-shaped grid -------------------------------------------------


def _blur_periodic(img: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic Gaussian blur by FFT (transfer function exp(-2 pi^2 sigma^2 |f|^2))."""
    h, w = img.shape
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    H = np.exp(-2.0 * (math.pi ** 2) * sigma * sigma * (fy * fy + fx * fx))
    return np.fft.irfft2(np.fft.rfft2(img) * H, s=img.shape)


class GridSegmentation:
    """2D 4-connected grid shaped like a graph-cut segmentation problem.

    The image is white noise U[0,1], blurred (sigma=8 px, periodic) and min-max
    normalised.  n-links join 4-neighbours in both directions with capacity
    round(1000 exp(-d^2 / (2 * 0.1^2))), d = |I_p - I_q|.  t-links come from a
    2-component Gaussian mixture (means 0.3 / 0.7, sigma 0.15, weights 1/2):
    D_k(p) = -log(w_k N(I_p; mu_k, sigma)); cap(s, p) = q(D_bg(p)) and
    cap(p, t) = q(D_fg(p)), where q maps [min, max] of the initial D linearly
    onto [0, 1000], rounds and clamps.  s and t are two extra vertices.
    """

    MU = (0.3, 0.7)
    SIG = 0.15
    W = (0.5, 0.5)

    def __init__(self, side: int = 2048, seed: int = 3, sigma: float = 8.0, window: int = 256,
                 origin=(896, 896), step: int = 8):
        self.side = side
        self.sigma = sigma
        rng = np.random.default_rng(seed)
        img = _blur_periodic(rng.random((side, side)), sigma)
        img = (img - img.min()) / (img.max() - img.min())
        self.I = img
        self.npix = side * side
        self.s = self.npix
        self.t = self.npix + 1
        self.n = self.npix + 2
        dbg, dfg = self._D(img)
        self.qlo = float(min(dbg.min(), dfg.min()))
        self.qhi = float(max(dbg.max(), dfg.max()))
        self.window = window
        self.origin = origin
        self.step = step

    def _D(self, x):
        out = []
        for mu, w in zip(self.MU, self.W):
            pdf = np.exp(-((x - mu) ** 2) / (2 * self.SIG ** 2)) / (self.SIG * math.sqrt(2 * math.pi))
            out.append(-np.log(w * pdf))
        return out[0], out[1]

    def _q(self, D):
        x = np.rint((D - self.qlo) / (self.qhi - self.qlo) * 1000.0)
        return np.clip(x, 0, 1000).astype(np.int32)

    def graph(self) -> Graph:
        side, I = self.side, self.I
        idx = np.arange(self.npix, dtype=np.int64).reshape(side, side)
        pairs = []
        for (a, b, ia, ib) in ((I[:, :-1], I[:, 1:], idx[:, :-1], idx[:, 1:]),
                               (I[:-1, :], I[1:, :], idx[:-1, :], idx[1:, :])):
            d = np.abs(a - b).ravel()
            c = np.rint(1000.0 * np.exp(-(d * d) / (2 * 0.1 * 0.1))).astype(np.int32)
            pairs.append((ia.ravel(), ib.ravel(), c))
        pu = np.concatenate([p[0] for p in pairs])
        pv = np.concatenate([p[1] for p in pairs])
        pc = np.concatenate([p[2] for p in pairs])
        dbg, dfg = self._D(I.ravel())
        pix = np.arange(self.npix, dtype=np.int64)
        src = np.concatenate([pu, pv, np.full(self.npix, self.s, np.int64), pix])
        dst = np.concatenate([pv, pu, pix, np.full(self.npix, self.t, np.int64)])
        cap = np.concatenate([pc, pc, self._q(dbg), self._q(dfg)])
        return Graph(self.n, _i32(src), _i32(dst), _i32(cap), self.s, self.t,
                     name=f"grid{side}", meta={"n_link_pairs": int(pu.size), "t_link_pairs": 2 * self.npix})

    def window_batch(self, k: int) -> Batch:
        """Batch k: t-links re-drawn in the window at (x0 + k*step, y0)."""
        w = self.window
        x0 = self.origin[0] + self.step * k
        y0 = self.origin[1]
        rng = np.random.default_rng(100 + k)
        eta = _blur_periodic(rng.standard_normal((w, w)), self.sigma)
        sd = eta.std()
        # a window much smaller than the blur leaves no variation: no perturbation then
        eta = (eta - eta.mean()) / sd if sd > 0 else np.zeros_like(eta)
        Iw = np.clip(self.I[y0:y0 + w, x0:x0 + w] + 0.2 * eta, 0.0, 1.0)
        dbg, dfg = self._D(Iw.ravel())
        ys, xs = np.meshgrid(np.arange(y0, y0 + w), np.arange(x0, x0 + w), indexing="ij")
        pix = (ys * self.side + xs).ravel()
        u = np.concatenate([np.full(pix.size, self.s), pix])
        v = np.concatenate([pix, np.full(pix.size, self.t)])
        c = np.concatenate([self._q(dbg), self._q(dfg)])
        return Batch(_i32(u), _i32(v), _i32(c))


# --- many small instances -----------------------------------------------------


def layered_dag(n: int, seed: int, layers: int = 16, fanout: int = 8, cap_hi: int = 500) -> Graph:
    """s -> every layer-0 vertex; each vertex -> `fanout` random vertices of the next layer; last layer -> t."""
    rng = np.random.default_rng(seed)
    inner = max(n - 2, layers)
    per = np.full(layers, inner // layers)
    per[: inner % layers] += 1
    starts = np.concatenate([[0], np.cumsum(per)])
    s, t = inner, inner + 1
    src, dst = [], []
    for L in range(layers - 1):
        a0, a1, b0, b1 = starts[L], starts[L + 1], starts[L + 1], starts[L + 2]
        k = min(fanout, b1 - b0)
        for vtx in range(a0, a1):
            tgt = b0 + rng.choice(b1 - b0, size=k, replace=False)
            src.append(np.full(k, vtx))
            dst.append(tgt)
    src.append(np.full(per[0], s))
    dst.append(np.arange(starts[0], starts[1]))
    src.append(np.arange(starts[layers - 1], starts[layers]))
    dst.append(np.full(per[-1], t))
    src = np.concatenate(src)
    dst = np.concatenate(dst)
    cap = rng.integers(1, cap_hi + 1, size=src.size)
    return Graph(inner + 2, _i32(src), _i32(dst), _i32(cap), s, t, name=f"dag_n{inner + 2}")


def geometric(n: int, seed: int, avg_deg: float = 8.0, cap_hi: int = 500) -> Graph:
    """Random geometric graph in the unit square, both directions; s/t nearest to (0,0)/(1,1)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = math.sqrt(avg_deg / (math.pi * n))
    pr = cKDTree(pts).query_pairs(r, output_type="ndarray")
    pr = pr[np.lexsort((pr[:, 1], pr[:, 0]))]
    src = np.concatenate([pr[:, 0], pr[:, 1]])
    dst = np.concatenate([pr[:, 1], pr[:, 0]])
    cap = rng.integers(1, cap_hi + 1, size=src.size)
    s = int(np.argmin((pts ** 2).sum(1)))
    t = int(np.argmin(((pts - 1.0) ** 2).sum(1)))
    return Graph(n, _i32(src), _i32(dst), _i32(cap), s, t, name=f"geo_n{n}")


def batched_instances(count: int = 64, seed: int = 4, lo: float = 1e3, hi: float = 2e5,
                      cap_hi: int = 500) -> list:
    """Uneven instances: sizes log-uniform in [lo, hi]; types rotate ER (avg out-degree 8), DAG, geometric."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)
    out = []
    for i, n in enumerate(sizes):
        n = int(n)
        kind = i % 3
        if kind == 0:
            g = erdos_renyi(n, 8 * n, seed=1000 + i, cap_lo=1, cap_hi=cap_hi)
        elif kind == 1:
            g = layered_dag(n, seed=1000 + i, cap_hi=cap_hi)
        else:
            g = geometric(n, seed=1000 + i, cap_hi=cap_hi)
        out.append(g)
    return out


def serving_graphs(seed0: int = 10) -> list:
    """Sixteen R-MAT graphs of scales 18 x4, 19 x3, 20 x3, 21 x3, 22 x3, seeds 10..25."""
    scales = [18] * 4 + [19] * 3 + [20] * 3 + [21] * 3 + [22] * 3
    return [(sc, seed0 + i) for i, sc in enumerate(scales)]


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------


def er_small(seed: int = 1) -> Graph:
    """Erdos-Renyi n=4096, m=32768, caps U[1,100], s=0, t=n-1."""
    return erdos_renyi(4096, 32768, seed=seed, cap_lo=1, cap_hi=100)


def er_small_batches(g: Graph, count: int = 10, B: int = 256, seed: int = 11) -> list:
    es = EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        b = mixed_batch(es, B, rng, ins_cap_hi=100)
        es.apply(b.u, b.v, b.cap)
        out.append(b)
    return out
