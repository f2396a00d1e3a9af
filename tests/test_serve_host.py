"""Host logic of the serving loop, without a GPU: the value-arena ring never
hands out rows that a live bundle holds, places bundles whole, and frees
them in arrival order once their last window has closed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _ring():
    from paper_1901_01328_b300.serve import ArenaRing
    return ArenaRing


def test_ring_never_overlaps_live_rows():
    ArenaRing = _ring()
    rng = np.random.default_rng(5)
    rows = 1000
    ring = ArenaRing(rows)
    owner = np.full(rows, -1)
    w = 0
    placed = shed = 0
    for b in range(5000):
        n = int(rng.integers(1, 300))
        if rng.random() < 0.25:
            w += 1  # a window boundary passes; windows up to w - 2 close
            ring.release(w - 2)
            live = {off for off, _, _ in ring.live}
            for r in range(rows):
                if owner[r] >= 0 and owner[r] not in live:
                    owner[r] = -1
        off = ring.alloc(n, w)
        if off is None:
            shed += 1
            continue
        placed += 1
        assert 0 <= off and off + n <= rows
        assert np.all(owner[off:off + n] == -1), "rows of a live bundle handed out again"
        owner[off:off + n] = off
    assert placed > 1000 and shed > 0


def test_ring_edge_cases():
    ArenaRing = _ring()
    ring = ArenaRing(100)
    assert ring.alloc(101, 0) is None
    assert ring.alloc(100, 0) == 0
    assert ring.alloc(1, 0) is None      # full
    ring.release(0)
    assert ring.head == 0 and not ring.live
    assert ring.alloc(60, 1) == 0 and ring.alloc(30, 2) == 60
    ring.release(1)                      # frees [0, 60)
    assert ring.alloc(20, 3) == 0        # no room at the end: wraps
    assert ring.alloc(50, 3) is None     # only [20, 60) is free
    assert ring.alloc(40, 3) == 20
