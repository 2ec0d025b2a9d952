"""The allocation-free heights call, checked against the oracle and the ordinary call.

maxflow_global_relabel_noalloc serves callers that may not allocate device
memory while running (a serving process with a device pool fixed at
start-up, a plugin inside an application that owns the GPU allocator).  On
the same residual state it must give exactly the oracle's residual distances
(integer BFS distances, so equality is the tolerance) for both root sets --
the sink and the deficient vertices, and the sink alone -- and, for the first,
exactly what maxflow_global_relabel gives.  Several calls run in a row: each
reuses the static scratch the previous one left behind.  After the prepare
call (n = 0) a call takes no device memory.  This file is collected last so
that a failure here comes after every other test has run.
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


def _call(torch, n, s, t, arrs, h, deficit_roots):
    stream = torch.cuda.current_stream().cuda_stream
    return native.maxflow_global_relabel_noalloc(
        n, s, t, arrs["off"].data_ptr(), arrs["deg"].data_ptr(), arrs["dst"].data_ptr(),
        arrs["cf"].data_ptr(), arrs["pcap"].data_ptr(), arrs["e"].data_ptr(), h.data_ptr(), deficit_roots, stream)


def _noalloc_heights(torch, S, arrs, deficit_roots):
    h = torch.full((S.n,), -1, dtype=torch.int32, device="cuda")
    rc = _call(torch, S.n, S.s, S.t, arrs, h, deficit_roots)
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


def test_noalloc_heights_match_the_oracle_and_the_existing_entry_point():
    import torch
    assert torch.cuda.is_available()
    native.load()
    calls = 0
    for seed, n, hubs in [(4242, 5000, True), (4343, 2000, False)]:
        src, dst, cap, mu, mv, f = _state(seed, n, hubs)
        R = oracle.Residual(n, src, dst, cap)
        R.set_flow(mu, mv, f)
        S = native.Solver(n, src, dst, cap, 0, n - 1)
        S.set_flow(mu, mv, f)
        arrs = _device_csr(torch, S)
        for deficit_roots in (True, False):
            want = R.heights(0, n - 1, deficit_roots=deficit_roots)
            got = _noalloc_heights(torch, S, arrs, deficit_roots)
            calls += 1
            np.testing.assert_array_equal(got, want, err_msg=f"call {calls}, deficit_roots={deficit_roots}")
        S.global_relabel()                         # the existing entry point (sink and deficits)
        existing, _ = S.vertex_state()
        np.testing.assert_array_equal(_noalloc_heights(torch, S, arrs, True), existing)
        S.close()


def test_noalloc_call_after_prepare_takes_no_device_memory():
    import torch
    native.load()
    rc = native.maxflow_global_relabel_noalloc(0, 0, 0, None, None, None, None, None, None, None, True,
                                               torch.cuda.current_stream().cuda_stream)
    assert rc == native.OK, native.strerror(rc)
    src, dst, cap, mu, mv, f = _state(4545, 3000, True)
    R = oracle.Residual(3000, src, dst, cap)
    R.set_flow(mu, mv, f)
    S = native.Solver(3000, src, dst, cap, 0, 2999)
    S.set_flow(mu, mv, f)
    arrs = _device_csr(torch, S)
    h = torch.full((S.n,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for deficit_roots in (True, False):
        assert _call(torch, S.n, S.s, S.t, arrs, h, deficit_roots) == native.OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        np.testing.assert_array_equal(h.cpu().numpy(), R.heights(0, 2999, deficit_roots=deficit_roots))
    S.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    native.load()
    big = (1 << 20) + 1
    fake = C.c_void_p(16)   # never dereferenced: the size check comes first
    rc = native.maxflow_global_relabel_noalloc(big, 0, 1, fake, fake, fake, fake, fake, fake, fake, True, None)
    assert rc == native.ERR_TOO_LARGE
    rc = native.maxflow_global_relabel_noalloc(10, 3, 3, fake, fake, fake, fake, fake, fake, fake, True, None)
    assert rc == native.ERR_INVALID
    rc = native.maxflow_global_relabel_noalloc(1, 0, 0, fake, fake, fake, fake, fake, fake, fake, True, None)
    assert rc == native.ERR_INVALID
