"""The seeded input generators follow the recipes they state (CPU only).

The generators hold no max-flow arithmetic; these tests pin the shapes,
value ranges and mixes that the parity tests and the bench rely on.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from paper_2511_01235_gb300 import workloads as W


def _pairs(u, v, n):
    return np.asarray(u, np.int64) * n + np.asarray(v, np.int64)


@pytest.mark.parametrize("B", [256, 1000, 5, 37])
def test_mixed_batch_counts_ranges_and_fresh_inserts(B):
    g = W.erdos_renyi(400, 3000, seed=21, cap_hi=100)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    rng = np.random.default_rng(22)
    b = W.mixed_batch(es, B, rng, ins_cap_hi=77)
    assert b.size == B
    assert np.all(b.u != b.v)
    assert np.unique(_pairs(b.u, b.v, g.n)).size == B                 # no pair twice in a batch
    old = es.contains(b.u, b.v)
    fresh = ~old
    # inserts: neither direction present, caps U[1, ins_cap_hi]
    assert not np.any(es.contains(b.v[fresh], b.u[fresh]))
    assert np.all((b.cap[fresh] >= 1) & (b.cap[fresh] <= 77))
    prev = es.cap_of(b.u[old], b.v[old])
    inc = b.cap[old] > prev
    assert np.all((b.cap[old][inc] - prev[inc] >= 1) & (b.cap[old][inc] - prev[inc] <= 50))
    assert np.all(b.cap[old][~inc] <= prev[~inc])
    n_inc = math.floor(0.4 * B + 0.5)
    n_ins = math.floor(0.1 * B + 0.5)
    assert int(inc.sum()) == n_inc and int(fresh.sum()) == n_ins
    assert int((~inc).sum()) == B - n_inc - n_ins                      # decreases and deletes
    if B == 256:
        assert (n_inc, n_ins, B - 2 * n_inc - n_ins) == (102, 26, 26)


def test_mixed_batch_st_bias_draws_source_and_sink_edges():
    g = W.erdos_renyi(300, 4000, seed=23, cap_hi=100)
    es = W.EdgeSet(g.n, g.src, g.dst, g.cap)
    b = W.mixed_batch(es, 200, np.random.default_rng(24), ins_cap_hi=10, st_bias=(g.s, g.t, 0.3))
    old = es.contains(b.u, b.v)
    special = (b.u[old] == g.s) | (b.v[old] == g.t)
    n_old = int(old.sum())
    n_special = int(np.sum((es.keys // g.n == g.s) | (es.keys % g.n == g.t)))
    assert int(special.sum()) >= min(round(0.3 * n_old), n_special)


def test_erdos_renyi_distinct_pairs_and_caps():
    g = W.erdos_renyi(500, 4000, seed=25, cap_lo=1, cap_hi=100)
    assert (g.n, g.m, g.s, g.t) == (500, 4000, 0, 499)
    assert np.all(g.src != g.dst)
    assert np.unique(_pairs(g.src, g.dst, g.n)).size == g.m
    assert g.cap.min() >= 1 and g.cap.max() <= 100


def test_rmat_shape_quadrants_and_terminals():
    scale, ef = 12, 16
    u, v = W.rmat_edges(scale, ef, 0.57, 0.19, 0.19, seed=26)
    assert u.size == ef << scale and u.max() < (1 << scale) and v.max() < (1 << scale)
    top = 1 << (scale - 1)
    # the first bit decided: u's bit set with probability c + d, v's with b + d
    assert abs(np.mean(u >= top) - 0.24) < 0.01 and abs(np.mean(v >= top) - 0.24) < 0.01
    both = np.mean((u >= top) & (v >= top))
    assert abs(both - 0.05) < 0.006                                    # quadrant d
    g = W.rmat(scale, ef, 0.57, 0.19, 0.19, seed=26, cap_hi=1000)
    assert g.n == 1 << scale and np.all(g.src != g.dst)
    assert np.unique(_pairs(g.src, g.dst, g.n)).size == g.m == g.meta["m_merged"]
    assert g.cap.min() >= 1 and g.cap.max() <= 1000
    deg = np.bincount(g.src, minlength=g.n) + np.bincount(g.dst, minlength=g.n)
    assert g.s == int(np.argmax(deg)) and g.t != g.s
    A = sp.csr_matrix((np.ones(g.m, np.int8), (g.src, g.dst)), shape=(g.n, g.n))
    assert g.t in set(csg.breadth_first_order(A, g.s, directed=True, return_predecessors=False).tolist())


def test_grid_segmentation_links_and_window_batch():
    G = W.GridSegmentation(side=16, seed=3, window=4, origin=(4, 4), step=1)
    g = G.graph()
    npix = 16 * 16
    assert (g.n, g.s, g.t) == (npix + 2, npix, npix + 1)
    n_pairs = 2 * 16 * 15
    assert g.m == 2 * n_pairs + 2 * npix and g.meta["n_link_pairs"] == n_pairs
    assert g.cap.min() >= 0 and g.cap.max() <= 1000
    # n-link capacity of the first horizontal pair from its formula
    d = abs(G.I[0, 0] - G.I[0, 1])
    assert g.cap[0] == round(1000 * math.exp(-d * d / (2 * 0.1 ** 2)))
    assert (g.src[0], g.dst[0]) == (0, 1) and (g.src[n_pairs], g.dst[n_pairs]) == (1, 0)
    # t-links: s -> every pixel, every pixel -> t
    assert np.all(g.src[2 * n_pairs:2 * n_pairs + npix] == g.s) and np.all(g.dst[-npix:] == g.t)
    b = G.window_batch(2)
    assert b.size == 2 * 4 * 4
    assert b.cap.min() >= 0 and b.cap.max() <= 1000                    # also when the window is tiny
    assert np.all(b.u[:16] == g.s) and np.all(b.v[16:] == g.t)
    pix = b.v[:16]
    assert set((pix // 16).tolist()) == {4, 5, 6, 7} and set((pix % 16).tolist()) == {6, 7, 8, 9}


def test_layered_dag_structure():
    g = W.layered_dag(162, seed=27, layers=16, fanout=8, cap_hi=500)
    inner = 160
    assert (g.n, g.s, g.t) == (162, inner, inner + 1)
    per = [10] * 16
    starts = np.concatenate([[0], np.cumsum(per)])
    layer = np.searchsorted(starts, np.arange(inner), side="right") - 1
    mid = (g.src < inner) & (g.dst < inner)
    assert np.all(layer[g.dst[mid]] == layer[g.src[mid]] + 1)           # only to the next layer
    assert np.all(np.bincount(g.src[mid], minlength=inner)[: starts[15]] == 8)
    assert set(g.dst[g.src == g.s].tolist()) == set(range(0, 10))
    assert set(g.src[g.dst == g.t].tolist()) == set(range(150, 160))
    assert g.cap.min() >= 1 and g.cap.max() <= 500


def test_geometric_is_symmetric_with_about_eight_neighbours():
    g = W.geometric(400, seed=28, avg_deg=8.0)
    fwd = set(_pairs(g.src, g.dst, g.n).tolist())
    assert fwd == set(_pairs(g.dst, g.src, g.n).tolist())
    assert 4.0 < g.m / g.n < 12.0                                       # about 8 per vertex
    assert g.s != g.t


def test_batched_instances_sizes_and_rotation():
    gs = W.batched_instances(count=6, seed=4, lo=1e3, hi=5e3)
    assert len(gs) == 6
    assert all(1e3 - 1 <= g.n <= 5e3 + 2 for g in gs)
    assert [g.name.split("_")[0] for g in gs] == ["er", "dag", "geo", "er", "dag", "geo"]
    assert W.batched_instances(count=6, seed=4, lo=1e3, hi=5e3)[0].m == gs[0].m      # seeded
