"""The allocation-free heights call, checked against the ordinary one.

maxflow_global_relabel_noalloc serves callers that may not allocate device
memory while running (a serving process with a device pool fixed at
start-up, a plugin inside an application that owns the GPU allocator).  It
must give exactly the heights that maxflow_global_relabel gives on the same
residual state (integer BFS distances, so equality is the tolerance), on two
calls in a row: the second call reuses the static scratch the first one left
behind.  This file is collected last so that a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2511_01235_gb300 import native
from paper_2511_01235_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _device_csr(torch, S):
    """The solver's current residual state as caller-owned device arrays (compact rows)."""
    u, v, cap, cf = S.residual()
    n = S.n
    deg = np.bincount(u, minlength=n).astype(np.int32)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(deg)
    order = np.argsort(u, kind="stable")            # rows in order, slot order kept within a row
    u, v, cap, cf = u[order], v[order], cap[order], cf[order]
    key = u.astype(np.int64) * n + v
    rkey = v.astype(np.int64) * n + u
    srt = np.argsort(key)
    ridx = srt[np.searchsorted(key[srt], rkey)]
    pcap = (cap.astype(np.int64) + cap[ridx]).astype(np.int32)
    _, e = S.vertex_state()
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt).cuda()
    return {"off": dev(off, torch.int32), "deg": dev(deg, torch.int32), "dst": dev(v, torch.int32),
            "cf": dev(cf, torch.int32), "pcap": dev(pcap, torch.int32), "e": dev(e, torch.int64)}


def _noalloc_heights(torch, S, arrs):
    h = torch.full((S.n,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = native.maxflow_global_relabel_noalloc(
        S.n, S.s, S.t, arrs["off"].data_ptr(), arrs["deg"].data_ptr(), arrs["dst"].data_ptr(),
        arrs["cf"].data_ptr(), arrs["pcap"].data_ptr(), arrs["e"].data_ptr(), h.data_ptr(), True, stream)
    assert rc == native.OK, native.strerror(rc)
    return h.cpu().numpy()


def _state(seed, n, hubs=False):
    rng = np.random.default_rng(seed)
    src, dst, cap = W.random_multigraph(n, 6 * n, seed=seed, cap_hi=30, zero_frac=0.2)
    if hubs:   # one row above the hub threshold, to take the grid-wide frontier path
        k = 5000
        src = np.concatenate([src, np.full(k, 1), rng.integers(2, n, k)]).astype(np.int32)
        dst = np.concatenate([dst, rng.integers(2, n, k), np.full(k, 1)]).astype(np.int32)
        cap = np.concatenate([cap, rng.integers(1, 30, 2 * k)]).astype(np.int32)
    mu, mv, mc = oracle.merge(n, src, dst, cap)
    f = np.where(rng.random(mc.size) < 0.7, np.floor(rng.random(mc.size) * (mc + 1)), 0)
    f = np.minimum(f, mc).astype(np.int32)
    return src, dst, cap, mu, mv, f


def test_noalloc_heights_match_existing_entry_point_twice():
    import torch
    assert torch.cuda.is_available()
    native.load()
    for call, (seed, n, hubs) in enumerate([(4242, 5000, True), (4343, 2000, False)]):
        src, dst, cap, mu, mv, f = _state(seed, n, hubs)
        S = native.Solver(n, src, dst, cap, 0, n - 1)
        S.set_flow(mu, mv, f)
        arrs = _device_csr(torch, S)
        S.global_relabel()                         # the existing entry point
        want, _ = S.vertex_state()
        got = _noalloc_heights(torch, S, arrs)
        np.testing.assert_array_equal(got, want, err_msg=f"call {call + 1}")
        S.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    native.load()
    big = (1 << 20) + 1
    fake = C.c_void_p(16)   # never dereferenced: the size check comes first
    rc = native.maxflow_global_relabel_noalloc(big, 0, 1, fake, fake, fake, fake, fake, fake, fake, True, None)
    assert rc == native.ERR_TOO_LARGE
    rc = native.maxflow_global_relabel_noalloc(10, 3, 3, fake, fake, fake, fake, fake, fake, fake, True, None)
    assert rc == native.ERR_INVALID
