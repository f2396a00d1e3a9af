"""Streaming operators over record bundles and KPAs (orchestration only:
every step runs in the kernels of libsbh.so).

Sec. 4.3 states how an operator prepares its input before grouping: if the
input X is a record bundle, Extract a KPA from it; if the KPA's resident
column is not the column c the operator groups by, KeySwap it to c; then
group (Listing 2).  `as_kpa` is that rule, and every grouping operator below
calls it, so operators chain freely: a Select's KPA flows into a keyed count
on another column, a top-K, or a join, each paying only the Extract or
KeySwap it needs.  Adjacent Materialize and Extract coalesce (Sec. 4.3,
first optimisation): a derived key (a lookup table applied to a column, such
as ad -> campaign) is produced by one fused gather, never as a separate
column.

Every primitive executed is appended to `trace`, so a caller (and the tests)
can see which steps Listing 2 inserted.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import sbh


@dataclass(frozen=True, eq=False)
class Lookup:
    """A derived column: table[base column] (e.g. the campaign of each ad)."""
    name: str
    base: str
    table: torch.Tensor  # device uint64


class Bundle:
    """A record bundle (Sec. 3): named device columns of equal length, of
    which rows [begin, end) belong to the bundle.  Pointers of the KPAs made
    from it are row indices into the full columns."""

    def __init__(self, cols: dict, begin: int = 0, end: int | None = None):
        self.cols = cols
        n = next(iter(cols.values())).numel()
        self.begin, self.end = begin, n if end is None else end

    @property
    def n(self):
        return self.end - self.begin

    def rows(self, begin, end):
        return Bundle(self.cols, begin, end)

    def windows(self, ts: str, length: int, trace=None):
        """Tumbling windows of `length` on a non-decreasing timestamp column
        (Sec. 4.2 "Windowing": Partition on the timestamp column): one
        sub-bundle per window, found by the window-range kernel."""
        col = self.cols[ts]
        if self.n == 0:
            return []
        first = int(col[self.begin].item()) // length
        last = int(col[self.end - 1].item()) // length
        nwin = last - first + 1
        dev = col.device
        starts = ((torch.arange(nwin, dtype=torch.int64, device=dev) + first) * length).view(torch.uint64)
        rb = torch.empty(nwin, dtype=torch.uint64, device=dev)
        re_ = torch.empty(nwin, dtype=torch.uint64, device=dev)
        sbh.sbh_window_ranges(col[self.begin:self.end], starts, length, rb, re_)
        _log(trace, "Partition", ts)
        rb, re_ = rb.cpu().numpy(), re_.cpu().numpy()
        return [(first + w, self.rows(self.begin + int(rb[w]), self.begin + int(re_[w]))) for w in range(nwin)]

    def column(self, c):
        return self.cols[c]


@dataclass
class KPA:
    """A Key Pointer Array (Sec. 4.1): resident keys of column `column` and
    pointers into `bundle`'s rows; `sorted` when in (key, ptr) order."""
    keys: torch.Tensor
    ptrs: torch.Tensor
    column: object  # a column name or a Lookup
    bundle: Bundle
    sorted: bool = False

    @property
    def n(self):
        return self.keys.numel()


def _log(trace, *step):
    if trace is not None:
        trace.append(step)


def _name(c):
    return c.name if isinstance(c, Lookup) else c


# ------------------------------------------------------------------ Table 2 maintenance primitives
def extract(bundle: Bundle, column, trace=None) -> KPA:
    """Extract (Table 2).  A derived column's keys come from one gather
    through its table (the Materialize of the base column coalesced with the
    Extract of the new key)."""
    dev = bundle.column(column.base if isinstance(column, Lookup) else column).device
    n = bundle.n
    keys = torch.empty(n, dtype=torch.uint64, device=dev)
    ptrs = torch.empty(n, dtype=torch.uint32, device=dev)
    if isinstance(column, Lookup):
        sbh.sbh_kpa_extract(bundle.column(column.base), bundle.begin, n, keys, ptrs)
        sbh.sbh_kpa_keyswap_lookup(ptrs, bundle.column(column.base), column.table, keys)
        _log(trace, "Extract+Materialize", column.name)
    else:
        sbh.sbh_kpa_extract(bundle.column(column), bundle.begin, n, keys, ptrs)
        _log(trace, "Extract", column)
    return KPA(keys, ptrs, column, bundle)


def keyswap(kpa: KPA, column, trace=None) -> KPA:
    """KeySwap (Table 2): the KPA's keys become `column`'s values of its
    records (through the table, fused, for a derived column)."""
    keys = torch.empty_like(kpa.keys)
    if kpa.n:
        if isinstance(column, Lookup):
            sbh.sbh_kpa_keyswap_lookup(kpa.ptrs, kpa.bundle.column(column.base), column.table, keys)
        else:
            sbh.sbh_kpa_keyswap(kpa.ptrs, kpa.bundle.column(column), keys)
    _log(trace, "KeySwap", _name(column))
    return KPA(keys, kpa.ptrs, column, kpa.bundle)


def as_kpa(x, column, trace=None) -> KPA:
    """Listing 2 (Sec. 4.3): X = IsKPA(X) ? X : Extract(X); if the resident
    column of X is not `column`, KeySwap(X, column)."""
    kpa = x if isinstance(x, KPA) else extract(x, column, trace)
    if _name(kpa.column) != _name(column):
        kpa = keyswap(kpa, column, trace)
    return kpa


def sort(kpa: KPA, trace=None) -> KPA:
    """Sort (Table 2) by the resident key (a no-op on a sorted KPA)."""
    if kpa.sorted:
        return kpa
    out = KPA(torch.empty_like(kpa.keys), torch.empty_like(kpa.ptrs), kpa.column, kpa.bundle, True)
    if kpa.n:
        sbh.sbh_kpa_sort(kpa.keys, kpa.ptrs, out.keys, out.ptrs)
    _log(trace, "Sort", _name(kpa.column))
    return out


# ------------------------------------------------------------------ operators
def select(x, column: str, lo: int, hi: int, trace=None) -> KPA:
    """Select (Table 2): the records whose `column` value lies in [lo, hi).
    A bundle is first Extracted on `column`; a KPA keeps its resident key and
    reads the value through its pointers."""
    kpa = x if isinstance(x, KPA) else extract(x, column, trace)
    dev = kpa.keys.device
    ok = torch.empty(max(1, kpa.n), dtype=torch.uint64, device=dev)
    op = torch.empty(max(1, kpa.n), dtype=torch.uint32, device=dev)
    cnt = torch.zeros(1, dtype=torch.uint64, device=dev)
    if kpa.n:
        sbh.sbh_kpa_select(kpa.keys, kpa.ptrs, kpa.bundle.column(column), lo, hi, ok, op, kpa.n, cnt)
    _log(trace, "Select", column)
    m = int(cnt.item())
    return KPA(ok[:m], op[:m], kpa.column, kpa.bundle, kpa.sorted)


def count_per_key(x, key, trace=None):
    """Keyed reduction, count only: (keys, counts) as host arrays."""
    k, c, _ = sum_per_key(x, key, None, trace)
    return k, c


def sum_per_key(x, key, value: str | None, trace=None):
    """Keyed reduction (Table 2; Sec. 4.2 "Reduction primitives"): per key of
    `key`, the count and the sum of `value` (None: count only)."""
    kpa = sort(as_kpa(x, key, trace), trace)
    if kpa.n == 0:
        z = np.zeros(0, np.uint64)
        return z, z, (z if value is not None else None)
    vals = None if value is None else kpa.bundle.column(value)
    k, c, s = sbh.group_reduce(kpa.keys, kpa.ptrs, vals)
    _log(trace, "Keyed", _name(key), value)
    return k.cpu().numpy(), c.cpu().numpy(), (s.cpu().numpy() if s is not None else None)


def topk_per_key(x, key, value: str, K: int, trace=None):
    """TopK Per Key (Sec. 7): per key of `key`, the K records with the
    largest `value` as (keys, nvalid, values [m, K], ptrs [m, K])."""
    kpa = sort(as_kpa(x, key, trace), trace)
    if kpa.n == 0:
        return (np.zeros(0, np.uint64), np.zeros(0, np.uint8), np.zeros((0, K), np.uint64),
                np.zeros((0, K), np.uint32))
    out = sbh.topk(kpa.keys, kpa.ptrs, kpa.bundle.column(value), K)
    _log(trace, "TopK", _name(key), value)
    return tuple(t.cpu().numpy() for t in out)


def join(x, y, key, trace=None):
    """Join (Table 2; Sec. 4.2 "Temporal Join"): every (ptrX, ptrY) with equal
    `key`, in (key, ptrX, ptrY) order, as host arrays."""
    kx = sort(as_kpa(x, key, trace), trace)
    ky = sort(as_kpa(y, key, trace), trace)
    if kx.n == 0 or ky.n == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    pl, pr = sbh.join(kx.keys, kx.ptrs, ky.keys, ky.ptrs)
    _log(trace, "Join", _name(key))
    return pl.cpu().numpy(), pr.cpu().numpy()
