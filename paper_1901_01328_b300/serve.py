"""Serving loop: record bundles arrive, tumbling windows close by watermark,
and each closed window's per-key sum, count and top-K come back to the host
(Sec. 3: bundles, watermarks and windows; Sec. 4.2 "Windowing" and "Keyed
Aggregation"; Sec. 5: the engine admits data only while memory allows).
Orchestration only: every step on the data runs in libsbh.so kernels.

Window state lives on the device.  Two window slots (the window being
filled and the one before it, which stays open until the watermark passes
its end) each hold an unsorted KPA of (key, arena row); the value column of
every admitted bundle sits in an arena ring in HBM until the last window
that uses it has closed.  Per bundle: copy its columns in (keys and
timestamps to a staging area, values to the arena), and split its rows into
the two slots by timestamp (`sbh_kpa_split_ts`, no host synchronisation).
When the watermark (max timestamp seen minus the allowed lateness) passes a
window's end, the window closes: its slot is sorted, reduced (sum and count)
and top-K'd against the arena, the results are copied to the host, and the
slot is emptied for the window after next.  `WindowClock` decides when
windows close, including, with an idle timeout, when the source stalls.

Memory is fixed at start-up from the HBM budget: a bundle that does not fit
in the arena is shed (counted); a slot that would pass its capacity sets an
overflow flag (counted).  Window-close latency is measured from the moment
the bundle that moved the watermark past the window's end was admitted to the
moment the window's results are in host memory.
"""
from __future__ import annotations

import collections
import time

import numpy as np
import torch

from . import sbh


def _u64(n, dev):
    return torch.empty(max(1, n), dtype=torch.uint64, device=dev)


def _u32(n, dev):
    return torch.empty(max(1, n), dtype=torch.uint32, device=dev)


class WindowResult:
    """One closed window, in host memory: keys (ascending), counts, sums,
    nvalid [m], top values and ptrs [m, K] (ptr = arena row)."""

    def __init__(self, w, keys, counts, sums, nvalid, tvals, tptrs, latency_s, rows):
        self.w, self.keys, self.counts, self.sums = w, keys, counts, sums
        self.nvalid, self.tvals, self.tptrs = nvalid, tvals, tptrs
        self.latency_s, self.rows = latency_s, rows


class ArenaRing:
    """Rows of the value arena as a ring: bundles are placed whole (wrapping
    to the start when the end has no room) and released in arrival order
    once the last window that uses them has closed."""

    def __init__(self, rows):
        self.rows = rows
        self.head = 0                     # next free row
        self.live = collections.deque()   # (offset, rows, last window)

    def alloc(self, n, last_w):
        if n > self.rows:
            return None
        if not self.live:
            off = 0
        else:
            tail = self.live[0][0]
            if self.head > tail:  # free: [head, end) and [0, tail)
                off = self.head if self.rows - self.head >= n else (0 if tail >= n else None)
            elif self.head < tail:  # free: [head, tail)
                off = self.head if tail - self.head >= n else None
            else:  # head == tail with bundles live: full
                off = None
        if off is None:
            return None
        self.head = off + n
        self.live.append((off, n, last_w))
        return off

    def release(self, closed_w):
        while self.live and self.live[0][2] <= closed_w:
            self.live.popleft()
        if not self.live:
            self.head = 0


class WindowClock:
    """When windows close (host logic only; no device state).

    A watermark promises that no record still to come is older than it
    (Sec. 3).  Here it is the largest timestamp seen minus the allowed
    lateness, and window [w L, (w + 1) L) closes once the watermark reaches
    its end.  A source that stops sending would leave the watermark, and so
    every open window, stuck.  The idle rule: after idle_ns of processing
    time without a bundle, event time is taken to advance at the rate of
    processing time from the last bundle's largest timestamp, and the
    watermark follows it; windows up to the newest one that holds rows then
    close.  So once the source stalls, every open window has closed within
    max(idle_ns, L + lateness) of processing time after the last bundle (plus
    the interval between ticks).  Records that arrive later than the
    watermark are dropped and counted by the split."""

    def __init__(self, win_len, lateness, idle_ns=None):
        self.L, self.lateness = int(win_len), int(lateness)
        self.idle_ns = None if idle_ns is None else int(idle_ns)
        self.wm = None         # watermark (event time, ns)
        self.first_win = None  # oldest open window
        self.last_ts = None    # largest timestamp seen
        self.last_wall = None  # processing time (ns) of the last bundle

    def _due(self, wm, limit=None):
        out = []
        while (self.first_win + 1) * self.L <= wm and (limit is None or self.first_win <= limit):
            out.append(self.first_win)
            self.first_win += 1
        return out

    def on_bundle(self, min_ts, max_ts, wall_ns):
        """A bundle with timestamps in [min_ts, max_ts] arrives: the windows
        that close before it lands, oldest first."""
        if self.first_win is None:
            self.first_win = max(0, min_ts) // self.L
        new_wm = max_ts - self.lateness if self.wm is None else max(self.wm, max_ts - self.lateness)
        due = self._due(new_wm)
        self.wm = new_wm
        self.last_ts = max_ts if self.last_ts is None else max(self.last_ts, max_ts)
        self.last_wall = wall_ns
        return due

    def on_idle(self, wall_ns):
        """Processing time wall_ns with no bundle since the last: the windows
        the idle rule closes now."""
        if self.idle_ns is None or self.last_wall is None or wall_ns - self.last_wall < self.idle_ns:
            return []
        wm = self.last_ts + (wall_ns - self.last_wall) - self.lateness
        if wm <= self.wm:
            return []
        self.wm = wm
        return self._due(wm, limit=self.last_ts // self.L)

    def open_windows(self):
        """Windows still open (the oldest up to the newest holding rows)."""
        if self.first_win is None or self.last_ts is None:
            return []
        return list(range(self.first_win, self.last_ts // self.L + 1))


class WindowServer:
    # the learned close trains on every SAMPLE_STRIDE-th key of the window
    SAMPLE_STRIDE = 400
    TRAIN = dict(steps=40, batch=4096, lr=3e-4)

    def __init__(self, win_len, lateness, slot_rows, arena_rows, max_bundle, K=3, device="cuda", keep=True,
                 out_rows=None, idle_ns=None, sort="radix"):
        """sort: "radix" sorts a closing window in place; "learned" trains the
        partition network on the window's sample and sorts into a second
        KPA (about 24 more bytes a slot row: see plan).  The learned close
        pays for keys that span most of the 64 bits; keys of a few bytes
        take few radix passes (Zipf ranks over 50M: four passes, 27.4 ms of
        device time per 250M-row window against 30.6 ms learned)."""
        if sort not in ("radix", "learned"):
            raise ValueError("sort must be 'radix' or 'learned'")
        dev = torch.device(device)
        self.sort = sort
        self.dev, self.win_len, self.lateness, self.K = dev, int(win_len), int(lateness), K
        self.clock = WindowClock(win_len, lateness, idle_ns)
        self.slots = [(_u64(slot_rows, dev), _u32(slot_rows, dev)) for _ in range(2)]
        self.fill = torch.zeros(2, dtype=torch.uint64, device=dev)
        self.dropped = torch.zeros(1, dtype=torch.uint64, device=dev)
        self.overflow = torch.zeros(1, dtype=torch.uint32, device=dev)
        self.arena = _u64(arena_rows, dev)
        self.arena_rows = arena_rows
        self.stage_keys = _u64(max_bundle, dev)
        self.stage_ts = torch.empty(max(1, max_bundle), dtype=torch.int64, device=dev)
        self.split_scr = torch.empty(sbh.split_scratch_bytes(max_bundle), dtype=torch.uint8, device=dev)
        self.slot_rows = slot_rows
        out = slot_rows if out_rows is None else min(out_rows, slot_rows)  # distinct keys a window may have
        self.out_rows = out
        if sort == "learned":
            self.lsorted = (_u64(slot_rows, dev), _u32(slot_rows, dev))
            self.sort_scr = torch.empty(max(1, sbh.sort_learned_scratch_bytes(slot_rows)), dtype=torch.uint8,
                                        device=dev)
            self.samples = _u64(slot_rows // self.SAMPLE_STRIDE + 1, dev)
            self.model = torch.zeros(sbh.LEARNED_MODEL_BYTES, dtype=torch.uint8, device=dev)
            self.train_scr = torch.empty(max(1, sbh.learned_train_scratch_bytes(self.samples.numel())),
                                         dtype=torch.uint8, device=dev)
        else:
            self.sort_scr = torch.empty(max(1, sbh.sort_scratch_bytes(slot_rows)), dtype=torch.uint8, device=dev)
        self.red = (_u64(out, dev), _u64(out, dev), _u64(out, dev), _u64(1, dev))
        self.red_scr = torch.empty(max(1, sbh.group_reduce_scratch_bytes(slot_rows, 8)), dtype=torch.uint8, device=dev)
        self.top = (_u64(out, dev), torch.empty(max(1, out), dtype=torch.uint8, device=dev),
                    _u64(out * K, dev), _u32(out * K, dev), _u64(1, dev))
        self.top_scr = torch.empty(max(1, sbh.topk_scratch_bytes(slot_rows, K, 8)), dtype=torch.uint8, device=dev)
        self.fill_h = torch.zeros(2, dtype=torch.uint64).pin_memory()
        self.nk_h = torch.zeros(1, dtype=torch.uint64).pin_memory()
        # page-locked host copies of a window's results
        self.host = (torch.empty(out, dtype=torch.uint64).pin_memory(), torch.empty(out, dtype=torch.uint64).pin_memory(),
                     torch.empty(out, dtype=torch.uint64).pin_memory(), torch.empty(out, dtype=torch.uint8).pin_memory(),
                     torch.empty(out * K, dtype=torch.uint64).pin_memory(),
                     torch.empty(out * K, dtype=torch.uint32).pin_memory())
        self.ring = ArenaRing(arena_rows)
        self.log = []          # (arena offset, rows, ts_base) of every admitted bundle
        self.results = []
        self.keep = keep
        self.shed_bundles = 0
        self.shed_rows = 0
        self.admitted_rows = 0
        self.est = {}  # host estimate of each open window's rows (a bundle counts in its newest window)
        self.truncated = 0

    # ---------------------------------------------------------------- bundles
    @property
    def first_win(self):
        return self.clock.first_win

    @property
    def wm(self):
        return self.clock.wm

    def admit(self, keys_h, vals_h, ts_rel_h, ts_base, max_ts, wall_ns=None):
        """keys_h, vals_h (uint64) and ts_rel_h (int64) are page-locked host
        tensors of one bundle; row i has timestamp ts_base + ts_rel_h[i] and
        max_ts is the largest; wall_ns is the processing time of its arrival
        (default: now).  Returns False when the bundle is shed."""
        n = keys_h.numel()
        t_admit = time.perf_counter()
        min_ts = ts_base + int(ts_rel_h.min()) if n and self.clock.first_win is None else ts_base
        # windows whose end the watermark has passed close before this bundle lands
        for w in self.clock.on_bundle(min_ts, max_ts, time.perf_counter_ns() if wall_ns is None else wall_ns):
            self._close(w, t_admit)
        w_new = max_ts // self.win_len
        # admission: the arena must have room, and the bundle's newest
        # window must stay below its slot's capacity (2% kept for late rows)
        if self.est.get(w_new, 0) + n > 0.98 * self.slot_rows:
            off = None
        else:
            off = self.ring.alloc(n, w_new)
        if off is None:
            self.shed_bundles += 1
            self.shed_rows += n
            return False
        self.est[w_new] = self.est.get(w_new, 0) + n
        if self.keep:
            self.log.append((off, n, ts_base))
        self.stage_keys[:n].copy_(keys_h, non_blocking=True)
        self.stage_ts[:n].copy_(ts_rel_h, non_blocking=True)
        self.arena[off:off + n].copy_(vals_h, non_blocking=True)
        s0, s1 = (self.slots[0], self.slots[1])
        self.split_scr = sbh.sbh_kpa_split_ts(self.stage_keys, self.stage_ts, n, ts_base, self.win_len, self.first_win,
                                              off, s0, s1, self.fill, self.dropped, self.overflow,
                                              scratch=self.split_scr)
        self.admitted_rows += n
        return True

    def tick(self, wall_ns=None):
        """Processing time passes with no bundle (the source may have
        stalled): closes the windows that the clock's idle rule releases.
        Returns how many closed."""
        due = self.clock.on_idle(time.perf_counter_ns() if wall_ns is None else wall_ns)
        t = time.perf_counter()
        for w in due:
            self._close(w, t)
        return len(due)

    def finish(self, t_now=None):
        """Close every open window (end of stream)."""
        t = time.perf_counter() if t_now is None else t_now
        for w in self.clock.open_windows():
            self._close(w, t)
        if self.clock.first_win is not None and self.clock.last_ts is not None:
            self.clock.first_win = max(self.clock.first_win, self.clock.last_ts // self.win_len + 1)

    # ---------------------------------------------------------------- window close
    def _close(self, w, t_trigger):
        """Closes window w: two host synchronisations, one to read the slot's
        size (it sizes the sort) and one when the results are in host memory
        (they are copied by kernels that read the number of keys on the
        device)."""
        s = w & 1
        keys, ptrs = self.slots[s]
        stream = torch.cuda.current_stream(self.dev)
        self.fill_h.copy_(self.fill, non_blocking=True)
        stream.synchronize()
        t1 = time.perf_counter()
        m = int(self.fill_h[s])
        K = self.K
        res = None
        dev_s = None
        if m:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            ok, op = keys[:m], ptrs[:m]
            if self.sort == "learned":
                smp = self.samples[:(m + self.SAMPLE_STRIDE - 1) // self.SAMPLE_STRIDE]
                sbh.sbh_kpa_extract(ok, 0, m, None, None, None, smp, self.SAMPLE_STRIDE)
                t = self.TRAIN
                self.train_scr = sbh.sbh_learned_train(smp, m, None, t["steps"], t["batch"], t["lr"], self.model,
                                                       scratch=self.train_scr)
                lk, lp = self.lsorted[0][:m], self.lsorted[1][:m]
                sbh.sbh_kpa_sort_learned(ok, op, lk, lp, self.model, scratch=self.sort_scr)
                ok, op = lk, lp
            else:
                sbh.sbh_kpa_sort(ok, op, ok, op, scratch=self.sort_scr)  # in place
            cap = self.out_rows
            rk, rc, rs, rn = self.red
            sbh.sbh_group_reduce(ok, op, self.arena, rk, rc, rs, cap, rn, scratch=self.red_scr)
            tk, tn, tv, tp, tnk = self.top
            sbh.sbh_topk(ok, op, self.arena, K, tk, tn, tv, tp, cap, tnk, scratch=self.top_scr)
            ev1.record(stream)
            hk, hc, hs, hn, hv, hp = self.host
            for h, d, per in ((hk, rk, 1), (hc, rc, 1), (hs, rs, 1), (hn, tn, 1), (hv, tv, K), (hp, tp, K)):
                sbh.sbh_copy_counted(d, h, rn, per, cap)
            self.nk_h.copy_(rn, non_blocking=True)
            stream.synchronize()
            dev_s = (t1 - t_trigger) + ev0.elapsed_time(ev1) / 1e3
            u = int(self.nk_h[0])
            if u > cap:
                self.truncated += 1
                u = cap
            if self.keep:
                res = [hk[:u].clone(), hc[:u].clone(), hs[:u].clone(), hn[:u].clone(), hv[:u * K].clone().view(u, K),
                       hp[:u * K].clone().view(u, K)]
        lat = time.perf_counter() - t_trigger
        self.fill[s:s + 1].zero_()
        r = (WindowResult(w, *(x.numpy() for x in res), lat, m) if res else
             WindowResult(w, None, None, None, None, None, None, lat, m))
        r.device_latency_s = dev_s if m else lat
        self.results.append(r)
        self.ring.release(w)
        self.est.pop(w, None)

    def stats(self):
        return {"shed_bundles": self.shed_bundles, "shed_rows": self.shed_rows,
                "admitted_rows": self.admitted_rows, "dropped_rows": int(self.dropped.item()),
                "overflow": int(self.overflow.item()), "truncated_windows": self.truncated}


def plan(budget_bytes, load, win_len_ns, lateness_ns, max_keys, K=3, learned=False):
    """Slot, arena and output sizes (rows) that fit the HBM budget for an
    offered load (rows/s): each slot row costs 12 B (KPA) x 2 slots + 13 B
    of sort scratch + about 5 B of top-K scratch (learned: + 12 B for the
    sorted KPA and 11 B more of sort scratch); the arena holds a window plus
    the lateness and a margin (8 B a row); outputs hold max_keys keys (24 B
    for count and sum, 9 + 12 K B for the top-K)."""
    win_rows = load * (win_len_ns + lateness_ns) * 1e-9
    arena_rows = int(1.3 * win_rows)
    out_rows = int(max_keys * 1.02) + 1024
    out_bytes = out_rows * (24 + 9 + 12 * K)
    slot_rows = int((budget_bytes - 8 * arena_rows - out_bytes) / (65 if learned else 42))
    slot_rows = max(0, min(slot_rows, int(1.15 * load * win_len_ns * 1e-9) + (1 << 20)))
    return slot_rows, arena_rows, out_rows


# -------------------------------------------------------------------- synthetic source
class BundlePool:
    """A pool of synthetic bundles in page-locked host memory (keys Zipf(s)
    over n_ids, values uniform u64, timestamps relative to the bundle's
    arrival: 0, or for a fraction `late` of the rows minus U(0, lateness))."""

    def __init__(self, gen, n_bundles, lo, hi, s, n_ids, late, lateness, seed):
        sizes = gen.uniform(seed, 1, n_bundles, lo, hi - lo + 1, np.uint64).astype(np.int64)
        self.bundles = []
        for b in range(n_bundles):
            m = int(sizes[b])
            keys = gen.zipf(seed, 100 + b, m, s, n_ids)
            vals = gen.uniform(seed, 10_000 + b, m, 0, 0, np.uint64)
            u = gen.unif01(seed, 20_000 + b, 2 * m)
            lag = np.where(u[:m] < late, np.floor(u[m:] * lateness), 0).astype(np.int64)
            self.bundles.append(tuple(torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).pin_memory()
                                      for a in (keys, vals, -lag)))
        self.sizes = sizes

    def get(self, i):
        k, v, t = self.bundles[i % len(self.bundles)]
        return k.view(torch.uint64), v.view(torch.uint64), t


def poisson_schedule(gen, seed, duration_ns, load, mean_rows):
    """Arrival times (ns) of a Poisson bundle stream offering `load` rows/s."""
    rate = load / mean_rows  # bundles per second
    n = int(duration_ns * 1e-9 * rate * 1.2) + 16
    gaps = -np.log1p(-gen.unif01(seed, 7, n)) / rate * 1e9
    t = np.cumsum(gaps)
    return t[t < duration_ns].astype(np.int64)


def run_loop(server, pool, arrivals, realtime=True, t0_ns=0, tick_ns=1_000_000):
    """Feeds the bundles at their arrival times (wall clock when realtime),
    letting the server's clock tick about every tick_ns while it waits (so
    an idle rule, when the server has one, can close windows of a stalled
    source); closes every open window at the end of the stream."""
    start = time.perf_counter()
    last_tick = time.perf_counter_ns()
    for i, a in enumerate(arrivals):
        if realtime:
            due = start + (a - arrivals[0]) * 1e-9
            while time.perf_counter() < due:
                now = time.perf_counter_ns()
                if now - last_tick >= tick_ns:
                    server.tick(now)
                    last_tick = now
        k, v, t = pool.get(i)
        base = int(t0_ns + a)
        server.admit(k, v, t, base, base)
    server.finish()
    return time.perf_counter() - start
