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


# ------------------------------------------------------------------ window clock (no GPU)
def _clock(idle_ns):
    from paper_1901_01328_b300.serve import WindowClock
    return WindowClock(1_000_000_000, 100_000_000, idle_ns)


def _feed(clock, n_bundles, closed, period=10_000_000, t0=10_000_000_000):
    """Bundles every `period` ns of processing time; event time = t0 +
    processing time, each bundle's rows up to 100 ms late."""
    wall = 0
    for i in range(n_bundles):
        wall = i * period
        ts = t0 + wall
        for w in clock.on_bundle(ts - 100_000_000, ts, wall):
            assert w not in closed
            closed[w] = wall
        assert clock.on_idle(wall + period // 2) == []  # the source is not idle
    return wall, t0 + wall


def test_clock_stalled_source_closes_every_window_within_bound():
    L, late, idle = 1_000_000_000, 100_000_000, 200_000_000
    clock = _clock(idle)
    closed = {}
    last_wall, last_ts = _feed(clock, 350, closed)  # 3.49 s of bundles, then the source stops
    assert sorted(closed) == [9, 10, 11, 12] and clock.open_windows() == [13]
    bound = max(idle, L + late)
    t = last_wall
    while clock.open_windows():
        t += 1_000_000  # ticks every 1 ms of processing time
        for w in clock.on_idle(t):
            assert w not in closed
            closed[w] = t
            # never before the idle rule allows: its end is below the advanced watermark
            assert last_ts + (t - last_wall) - late >= (w + 1) * L
        assert t - last_wall <= bound + 1_000_000, "a window stayed open past the bound"
    assert sorted(closed) == [9, 10, 11, 12, 13]
    assert closed[13] > last_wall
    # nothing more closes while the source stays silent
    assert clock.on_idle(t + 10 * L) == [] and clock.open_windows() == []


def test_clock_without_idle_rule_keeps_windows_of_a_stalled_source_open():
    clock = _clock(None)
    closed = {}
    _feed(clock, 350, closed)
    assert clock.on_idle(10 ** 15) == [] and clock.open_windows() == [13]


def test_clock_resumes_after_a_stall():
    L = 1_000_000_000
    clock = _clock(200_000_000)
    closed = {}
    last_wall, last_ts = _feed(clock, 150, closed)  # up to event time 11.49 s
    for w in clock.on_idle(last_wall + 2 * L):
        closed[w] = -1
    assert sorted(closed) == [9, 10, 11] and clock.first_win == 12
    # the source comes back 5 s later (event time 16.5 s): the empty windows
    # in between close before its bundle lands, each once
    due = clock.on_bundle(16_400_000_000, 16_500_000_000, last_wall + 5 * L)
    assert due == [12, 13, 14, 15] and clock.open_windows() == [16]


def test_run_loop_ticks_while_waiting():
    from paper_1901_01328_b300 import serve

    class Fake:
        def __init__(self):
            self.ticks = self.admits = 0
            self.finished = False

        def tick(self, wall_ns=None):
            self.ticks += 1
            return 0

        def admit(self, *a, **k):
            self.admits += 1
            return True

        def finish(self):
            self.finished = True

    class Pool:
        def get(self, i):
            return None, None, None

    f = Fake()
    serve.run_loop(f, Pool(), np.array([0, 30_000_000, 60_000_000], np.int64), realtime=True, tick_ns=1_000_000)
    assert f.admits == 3 and f.finished and f.ticks >= 20
