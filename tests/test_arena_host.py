"""The device-memory arena's placement, on the CPU.

The arena is created over a caller-provided region (here the address of a
host buffer, which the arena never dereferences), with overflow off, so no
CUDA call is made.  Checked against a plain model: live blocks never overlap
and stay inside the region, accounting matches, freeing everything coalesces
back to one block, best fit picks the smallest hole for large requests, and
small requests come from the top of the region.
"""
import numpy as np
import pytest

from paper_2511_01235_gb300 import build_ext, native

MiB = 1 << 20


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return native.load()


@pytest.fixture()
def region():
    buf = np.zeros(64 * MiB + 4096, np.uint8)
    base = (buf.ctypes.data + 255) & ~255
    return buf, base, 64 * MiB


def _arena(lib, base, nbytes):
    return native.Arena(nbytes, device=0, allow_overflow=False, base=base)


def test_bad_arguments(lib, region):
    _, base, nbytes = region
    with pytest.raises(native.MaxflowError):
        native.Arena(nbytes, allow_overflow=False, base=base + 8)        # misaligned
    with pytest.raises(native.MaxflowError):
        native.Arena(0, allow_overflow=False, base=base)


def test_best_fit_coalescing_and_small_from_the_top(lib, region):
    _, base, nbytes = region
    A = _arena(lib, base, nbytes)
    a = A.alloc(4 * MiB)
    b = A.alloc(4 * MiB)
    c = A.alloc(4 * MiB)
    assert (a, b, c) == (base, base + 4 * MiB, base + 8 * MiB)          # large: head of the block
    small = A.alloc(1000)
    assert small == base + nbytes - 1024                                 # small: tail of the highest block
    A.free(b)
    d = A.alloc(3 * MiB)
    assert d == b                                                        # best fit: the 4 MiB hole
    st = A.stats()
    assert st["in_use"] == 4 * MiB * 2 + 3 * MiB + 1024
    assert st["free_blocks"] == 2
    for p in (a, c, d, small):
        A.free(p)
    st = A.stats()
    assert st["in_use"] == 0 and st["free_blocks"] == 1 and st["largest_free"] == nbytes
    assert st["peak_in_use"] == 3 * 4 * MiB + 1024
    assert A.alloc(nbytes + 1) == 0 and A.stats()["failed"] == 1       # no overflow: the request fails
    A.close()


def test_random_sequence_matches_a_model(lib, region):
    _, base, nbytes = region
    A = _arena(lib, base, nbytes)
    rng = np.random.default_rng(5)
    live = {}
    for step in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            p = list(live)[int(rng.integers(0, len(live)))]
            A.free(p)
            del live[p]
        else:
            size = int(rng.choice([rng.integers(1, 64 * 1024), rng.integers(MiB, 6 * MiB)]))
            p = A.alloc(size)
            if p:
                live[p] = (size + 255) & ~255
            else:
                st = A.stats()                                  # failed: no free block was big enough
                assert st["largest_free"] < ((size + 255) & ~255)
        iv = sorted(live.items())
        for (p, s), (q, _) in zip(iv, iv[1:]):
            assert p + s <= q                                   # no overlap
        if iv:
            assert iv[0][0] >= base and iv[-1][0] + iv[-1][1] <= base + nbytes
        st = A.stats()
        assert st["in_use"] == sum(live.values())
        assert st["free_total"] == nbytes - st["in_use"]
    for p in list(live):
        A.free(p)
    st = A.stats()
    assert st["free_blocks"] == 1 and st["largest_free"] == nbytes
    A.close()


def test_freeing_a_foreign_pointer_is_ignored(lib, region):
    _, base, nbytes = region
    A = _arena(lib, base, nbytes)
    p = A.alloc(2 * MiB)
    A.free(p + 256)                      # inside the region but not a block start
    A.free(base - 4096)                  # outside the region
    assert A.stats()["in_use"] == 2 * MiB
    A.free(p)
    assert A.stats()["in_use"] == 0
    A.close()


def test_fits_predicts_the_allocations(lib, region):
    _, base, nbytes = region
    A = _arena(lib, base, nbytes)
    rng = np.random.default_rng(8)
    live = []
    for _ in range(400):
        # fragment the arena a little, then ask about a list and check by allocating it
        if live and rng.random() < 0.5:
            A.free(live.pop(int(rng.integers(0, len(live)))))
        p = A.alloc(int(rng.integers(MiB, 4 * MiB)))
        if p:
            live.append(p)
        sizes = [int(x) for x in rng.choice([300, 70_000, 2 * MiB, 5 * MiB, 11 * MiB], size=int(rng.integers(1, 6)))]
        want = A.fits(sizes)
        got = []
        for sz in sizes:
            q = A.alloc(sz)
            if not q:
                break
            got.append(q)
        assert want == (len(got) == len(sizes))
        for q in got:
            A.free(q)
    assert A.fits([]) is True
    A.close()
