"""ORACLE -- test infrastructure only.

Plain, slow CPU statements of what the KPA grouping path of StreamBox-HBM
computes (Sec. 4.1 "KPA", Sec. 4.2 "Streaming Operations", Table 2 "KPA
primitives").  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it.

``oracle.cpp`` (std::sort, std::map, std::multimap) is compiled on first use
into ``liboracle.so``; ``mlp.py`` holds the FP64 statement of the learned
partitioner's network.

Parity status of each function (what pins it, besides itself):
  extract, sort, merge    -- brute force on tiny inputs; sortedness and
                             permutation invariants
  group_sum_count         -- brute force per distinct key; sum of counts = n;
                             sum of sums = sum of values mod 2^64; expected
                             distinct-key count (closed form)
  topk                    -- brute force per key; size = min(K, count);
                             every kept value >= every dropped one
  join                    -- nested loop; cardinality = sum_k cL(k) cR(k)
  window_ranges           -- binary search on a non-decreasing column
  partition               -- brute force on tiny inputs (a Python loop);
                             each part's keys in its range, parts in input
                             order, part sizes = rows per range
  mlp (forward/backward)  -- central finite differences; closed-form special
                             cases; one Adam step in closed form
The paper prints no worked example, so nothing is pinned to printed values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

TOPK_PAD_VAL = 0
TOPK_PAD_PTR = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the oracle library (g++ -O2; no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_extract.argtypes = [vp, u64, u64, vp, vp]
        lib.oracle_extract.restype = None
        lib.oracle_sort.argtypes = [vp, vp, u64]
        lib.oracle_sort.restype = None
        lib.oracle_merge.argtypes = [i32, vp, vp, vp, vp, vp]
        lib.oracle_merge.restype = None
        lib.oracle_group_sum_count.argtypes = [vp, vp, u64, vp, i32, vp, vp, vp]
        lib.oracle_group_sum_count.restype = u64
        lib.oracle_topk.argtypes = [vp, vp, u64, vp, i32, i32, vp, vp, vp, vp]
        lib.oracle_topk.restype = u64
        for f in (lib.oracle_join, lib.oracle_join_nested):
            f.argtypes = [vp, vp, u64, vp, vp, u64, vp, vp, u64]
            f.restype = u64
        lib.oracle_window_ranges.argtypes = [vp, i32, u64, vp, u64, u64, vp, vp]
        lib.oracle_window_ranges.restype = None
        lib.oracle_materialize.argtypes = [vp, u64, vp, i32, vp]
        lib.oracle_materialize.restype = None
        lib.oracle_select.argtypes = [vp, vp, u64, vp, i32, u64, u64, vp, vp, u64]
        lib.oracle_select.restype = u64
        lib.oracle_median_unique.argtypes = [vp, vp, u64, vp, i32, vp, vp, vp]
        lib.oracle_median_unique.restype = u64
        lib.oracle_partition.argtypes = [vp, vp, u64, vp, u64, vp, vp, vp]
        lib.oracle_partition.restype = None
        _lib = lib
    return _lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data


def extract(key_col: np.ndarray, row_begin: int, n: int):
    """KPA of rows [row_begin, row_begin + n): (keys u64, ptrs u32 = row)."""
    key_col = _c(key_col, np.uint64)
    assert row_begin + n <= key_col.size
    keys = np.empty(n, np.uint64)
    ptrs = np.empty(n, np.uint32)
    _load().oracle_extract(_p(key_col), row_begin, n, _p(keys), _p(ptrs))
    return keys, ptrs


def sort(keys: np.ndarray, ptrs: np.ndarray):
    """The KPA in (key, ptr) order (returns new arrays)."""
    k = np.array(keys, dtype=np.uint64, copy=True)
    p = np.array(ptrs, dtype=np.uint32, copy=True)
    _load().oracle_sort(_p(k), _p(p), k.size)
    return k, p


def merge(runs):
    """Merge of sorted runs [(keys, ptrs), ...] = sorted concatenation."""
    runs = [(_c(k, np.uint64), _c(p, np.uint32)) for k, p in runs]
    lens = np.array([k.size for k, _ in runs], dtype=np.uint64)
    m = int(lens.sum())
    kp = (ctypes.c_void_p * max(1, len(runs)))(*[k.ctypes.data for k, _ in runs])
    pp = (ctypes.c_void_p * max(1, len(runs)))(*[p.ctypes.data for _, p in runs])
    ok = np.empty(m, np.uint64)
    op = np.empty(m, np.uint32)
    _load().oracle_merge(len(runs), ctypes.cast(kp, ctypes.c_void_p), ctypes.cast(pp, ctypes.c_void_p),
                         _p(lens), _p(ok), _p(op))
    return ok, op


def group_sum_count(keys: np.ndarray, ptrs: np.ndarray, vals: np.ndarray | None):
    """Per distinct key (ascending): (keys, counts u64, sums u64 mod 2^64).
    With vals None, sums are zero (count only)."""
    keys = _c(keys, np.uint64)
    ptrs = _c(ptrs, np.uint32)
    vb = 0
    if vals is not None:
        vb = vals.dtype.itemsize
        assert vb in (4, 8)
        vals = np.ascontiguousarray(vals)
    n = keys.size
    ok = np.empty(n, np.uint64)
    oc = np.empty(n, np.uint64)
    osum = np.empty(n, np.uint64)
    m = _load().oracle_group_sum_count(_p(keys), _p(ptrs), n, _p(vals), vb, _p(ok), _p(oc), _p(osum))
    return ok[:m].copy(), oc[:m].copy(), osum[:m].copy()


def topk(keys: np.ndarray, ptrs: np.ndarray, vals: np.ndarray, K: int):
    """Per distinct key: (keys, nvalid u8, vals u64[m, K], ptrs u32[m, K])."""
    keys = _c(keys, np.uint64)
    ptrs = _c(ptrs, np.uint32)
    vals = np.ascontiguousarray(vals)
    vb = vals.dtype.itemsize
    n = keys.size
    ok = np.empty(n, np.uint64)
    nv = np.empty(n, np.uint8)
    ov = np.empty(n * K, np.uint64)
    op = np.empty(n * K, np.uint32)
    m = _load().oracle_topk(_p(keys), _p(ptrs), n, _p(vals), vb, K, _p(ok), _p(nv), _p(ov), _p(op))
    return ok[:m].copy(), nv[:m].copy(), ov[: m * K].reshape(m, K).copy(), op[: m * K].reshape(m, K).copy()


def _join(fn, lkeys, lptrs, rkeys, rptrs):
    lk, lp, rk, rp = _c(lkeys, np.uint64), _c(lptrs, np.uint32), _c(rkeys, np.uint64), _c(rptrs, np.uint32)
    total = fn(_p(lk), _p(lp), lk.size, _p(rk), _p(rp), rk.size, None, None, 0)
    ol = np.empty(total, np.uint32)
    orr = np.empty(total, np.uint32)
    fn(_p(lk), _p(lp), lk.size, _p(rk), _p(rp), rk.size, _p(ol), _p(orr), total)
    return ol, orr


def join(lkeys, lptrs, rkeys, rptrs):
    """All (ptrL, ptrR) with equal keys, in (key, ptrL, ptrR) order."""
    return _join(_load().oracle_join, lkeys, lptrs, rkeys, rptrs)


def join_nested(lkeys, lptrs, rkeys, rptrs):
    """The same join by a nested loop (small inputs only)."""
    return _join(_load().oracle_join_nested, lkeys, lptrs, rkeys, rptrs)


def window_ranges(ts: np.ndarray, starts: np.ndarray, length: int):
    """Row range [begin, end) of rows with ts in [start, start + length)."""
    ts = np.ascontiguousarray(ts)
    assert ts.dtype in (np.uint32, np.uint64)
    starts = _c(starts, np.uint64)
    b = np.empty(starts.size, np.uint64)
    e = np.empty(starts.size, np.uint64)
    _load().oracle_window_ranges(_p(ts), ts.dtype.itemsize, ts.size, _p(starts), length, starts.size, _p(b), _p(e))
    return b, e


def materialize(ptrs: np.ndarray, col: np.ndarray) -> np.ndarray:
    """col[ptr] for every record, in KPA order (Materialize; KeySwap when col
    is another key column)."""
    ptrs = _c(ptrs, np.uint32)
    col = np.ascontiguousarray(col)
    assert col.dtype in (np.uint32, np.uint64)
    out = np.empty(ptrs.size, col.dtype)
    _load().oracle_materialize(_p(ptrs), ptrs.size, _p(col), col.dtype.itemsize, _p(out))
    return out


def select(keys: np.ndarray, ptrs: np.ndarray, col: np.ndarray, lo: int, hi: int):
    """The records with col[ptr] in [lo, hi), in KPA order."""
    keys, ptrs = _c(keys, np.uint64), _c(ptrs, np.uint32)
    col = np.ascontiguousarray(col)
    m = _load().oracle_select(_p(keys), _p(ptrs), keys.size, _p(col), col.dtype.itemsize, lo, hi, None, None, 0)
    ok, op = np.empty(m, np.uint64), np.empty(m, np.uint32)
    _load().oracle_select(_p(keys), _p(ptrs), keys.size, _p(col), col.dtype.itemsize, lo, hi, _p(ok), _p(op), m)
    return ok, op


def median_unique(keys: np.ndarray, ptrs: np.ndarray, col: np.ndarray):
    """Per key (ascending): (keys, lower median of its values, number of
    distinct values)."""
    keys, ptrs = _c(keys, np.uint64), _c(ptrs, np.uint32)
    col = np.ascontiguousarray(col)
    n = keys.size
    ok, om, ou = np.empty(n, np.uint64), np.empty(n, np.uint64), np.empty(n, np.uint64)
    m = _load().oracle_median_unique(_p(keys), _p(ptrs), n, _p(col), col.dtype.itemsize, _p(ok), _p(om), _p(ou))
    return ok[:m], om[:m], ou[:m]


def partition(keys: np.ndarray, ptrs: np.ndarray, bounds: np.ndarray):
    """Partition (Table 2) by key ranges: (keys, ptrs, offsets[nb + 2]); part j
    = records with bounds[j - 1] <= key < bounds[j], in input order."""
    keys = _c(keys, np.uint64)
    ptrs = _c(ptrs, np.uint32)
    bounds = _c(bounds, np.uint64)
    n, nb = keys.size, bounds.size
    ok = np.empty(n, np.uint64)
    op = np.empty(n, np.uint32)
    off = np.empty(nb + 2, np.uint64)
    _load().oracle_partition(_p(keys), _p(ptrs), n, _p(bounds), nb, _p(ok), _p(op), _p(off))
    return ok, op, off
