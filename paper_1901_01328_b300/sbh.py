"""Python binding of the C ABI in include/sbh.h (ctypes).

Argument marshalling only: every step of the KPA grouping path runs in the
CUDA kernels of libsbh.so.  Tensors must be CUDA tensors (or, for the key
column of extract, a page-locked CPU tensor).  Calls run on the current
PyTorch CUDA stream unless a stream is given.  Working memory is allocated
with PyTorch.

If libsbh.so cannot be loaded, importing this module raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsbh.so")

SBH_OK, SBH_EINVAL, SBH_ENOSPACE, SBH_ETIMEOUT, SBH_ECUDA = 0, 1, 2, 3, 4
SBH_FAULT_NONE, SBH_FAULT_SKIP_PUBLISH = 0, 1
KNOB_SORT_CHUNKED_MIN, KNOB_MERGE_SEARCH_MIN_TILES, KNOB_SCATTER_GEOM = 0, 1, 2
SCATTER_GEOMS = {0: (4096, 512), 1: (2048, 256), 2: (8192, 1024)}  # tile rows, CTA threads
TOPK_PAD_VAL = 0
TOPK_PAD_PTR = 0xFFFFFFFF
TOPK_MAX_K = 8
MLP_PARAMS = 1153
LEARNED_MODEL_BYTES = 139264
LEARNED_CAPACITY = 8192
LEARNED_MAX_HEAVY = 16384
LEARNED_STATS = ("bucket_ids", "heavy_keys", "sorted_buckets", "one_key_buckets", "heavy_buckets",
                 "overflow_buckets", "overflow_rows", "largest_bucket", "radix_buckets", "radix_rows",
                 "wide_buckets", "wide_rows", "retried_buckets", "id_passes")

_ERRNAMES = {1: "SBH_EINVAL", 2: "SBH_ENOSPACE", 3: "SBH_ETIMEOUT", 4: "SBH_ECUDA"}


class SbhError(RuntimeError):
    def __init__(self, code: int, where: str, text: str):
        super().__init__(f"{where}: {_ERRNAMES.get(code, code)}: {text}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1901_01328_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32, sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)
    i64 = ctypes.c_int64
    sig = {
        "sbh_version": ([], ctypes.c_char_p),
        "sbh_last_error": ([], ctypes.c_char_p),
        "sbh_sync_status": ([vp], i32),
        "sbh_set_spin_limit": ([u32], None),
        "sbh_set_fault": ([i32], None),
        "sbh_set_knob": ([i32, u64], i32),
        "sbh_get_knob": ([i32], u64),
        "sbh_profile_enable": ([i32], None),
        "sbh_profile_collect": ([i32, vp, i32, vp], i32),
        "sbh_window_ranges": ([vp, i32, u64, vp, u64, u64, vp, vp, vp], i32),
        "sbh_kpa_extract": ([vp, u64, u64, vp, vp, vp, vp, u64, vp], i32),
        "sbh_kpa_extract_windows": ([vp, vp, u64, u64, u64, vp, vp, vp, vp], i32),
        "sbh_window_bits": ([u64], i32),
        "sbh_kpa_materialize": ([vp, u64, vp, i32, vp, vp], i32),
        "sbh_kpa_keyswap": ([vp, u64, vp, vp, vp], i32),
        "sbh_kpa_keyswap_lookup": ([vp, u64, vp, vp, u64, vp, vp, vp], i32),
        "sbh_kpa_select": ([vp, vp, u64, vp, i32, u64, u64, vp, vp, u64, vp, vp, sz, vp], i32),
        "sbh_median_unique": ([vp, vp, u64, vp, i32, vp, vp, vp, u64, vp, vp, sz, vp], i32),
        "sbh_kpa_split_ts": ([vp, vp, u64, i64, u64, u64, u32, vp, vp, u64, vp, vp, u64, vp, vp, vp, vp, sz, vp], i32),
        "sbh_kpa_sort": ([vp, vp, vp, vp, u64, vp, sz, vp], i32),
        "sbh_kpa_merge": ([i32, vp, vp, vp, vp, vp, vp, sz, vp], i32),
        "sbh_group_reduce": ([vp, vp, u64, vp, i32, vp, vp, i32, vp, u64, vp, vp, sz, vp], i32),
        "sbh_group_reduce_noalloc": ([vp, vp, u64, vp, i32, vp, vp, i32, vp, u64, vp, vp], i32),
        "sbh_topk": ([vp, vp, u64, vp, i32, i32, vp, vp, vp, vp, u64, vp, vp, sz, vp], i32),
        "sbh_join": ([vp, vp, u64, vp, vp, u64, vp, vp, u64, vp, vp, sz, vp], i32),
        "sbh_mlp_forward": ([vp, vp, u64, vp, vp], i32),
        "sbh_mlp_grad": ([vp, vp, vp, u64, vp, vp, vp, sz, vp], i32),
        "sbh_learned_train": ([vp, u64, u64, vp, i32, i32, ctypes.c_float, vp, vp, vp, vp, vp, sz, vp], i32),
        "sbh_kpa_sort_learned": ([vp, vp, vp, vp, u64, vp, vp, vp, sz, vp], i32),
        "sbh_kpa_partition": ([vp, vp, u64, vp, u64, vp, vp, vp, vp, sz, vp], i32),
        "sbh_copy_counted": ([vp, vp, i32, i32, vp, u64, u64, vp], i32),
        "sbh_kpa_merge_segments": ([i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp], i32),
        "sbh_join_segments": ([i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, u64, vp, vp, i32, vp, sz, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()
EXPORTED = ("sbh_version", "sbh_last_error", "sbh_sync_status", "sbh_set_spin_limit", "sbh_set_fault",
            "sbh_set_knob", "sbh_get_knob",
            "sbh_profile_enable", "sbh_profile_collect",
            "sbh_window_ranges", "sbh_kpa_extract", "sbh_kpa_extract_windows", "sbh_window_bits", "sbh_kpa_split_ts",
            "sbh_kpa_sort",
            "sbh_kpa_merge", "sbh_group_reduce",
            "sbh_group_reduce_noalloc", "sbh_mlp_forward", "sbh_mlp_grad", "sbh_learned_train",
            "sbh_kpa_sort_learned", "sbh_kpa_materialize", "sbh_kpa_keyswap", "sbh_kpa_keyswap_lookup",
            "sbh_kpa_select",
            "sbh_median_unique", "sbh_kpa_partition", "sbh_copy_counted", "sbh_kpa_merge_segments",
            "sbh_join_segments",
            "sbh_topk", "sbh_join")


def lib() -> ctypes.CDLL:
    return _lib


def _check(rc: int, where: str):
    if rc != SBH_OK:
        raise SbhError(rc, where, _lib.sbh_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _p(t):
    return None if t is None else t.data_ptr()


def _scratch(fn, args_before, args_after, where, device):
    """Size query, allocation and call with the (scratch, scratch_bytes) tail."""
    nbytes = ctypes.c_size_t(0)
    _check(fn(*args_before, None, ctypes.byref(nbytes), *args_after), where + " (size query)")
    buf = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=device)
    _check(fn(*args_before, buf.data_ptr(), ctypes.byref(nbytes), *args_after), where)
    return buf


def version() -> str:
    return _lib.sbh_version().decode()


def sync_status(stream=None) -> int:
    """Waits for the stream; returns SBH_OK or SBH_ETIMEOUT (device wait expired)."""
    return _lib.sbh_sync_status(_stream(stream))


def set_spin_limit(polls: int):
    _lib.sbh_set_spin_limit(polls)


def set_fault(fault: int):
    _lib.sbh_set_fault(fault)


def set_knob(knob: int, value: int):
    _check(_lib.sbh_set_knob(knob, value), "sbh_set_knob")


def get_knob(knob: int) -> int:
    return _lib.sbh_get_knob(knob)


def profile_enable(on: bool = True):
    """Start (or stop) recording an event pair around every kernel launch."""
    _lib.sbh_profile_enable(1 if on else 0)


def profile_collect():
    """[(kernel name, milliseconds)] of the recorded launches, in launch order."""
    n = _lib.sbh_profile_collect(0, None, 0, None)
    if n == 0:
        return []
    name_len = 48
    names = ctypes.create_string_buffer(n * name_len)
    ms = (ctypes.c_double * n)()
    _lib.sbh_profile_collect(n, ctypes.cast(names, ctypes.c_void_p), name_len, ctypes.cast(ms, ctypes.c_void_p))
    raw = names.raw
    return [(raw[i * name_len:(i + 1) * name_len].split(b"\0", 1)[0].decode(), ms[i]) for i in range(n)]


# ----------------------------------------------------------------- raw calls
def sbh_window_ranges(ts, starts, length, row_begin, row_end, stream=None):
    assert ts.dtype in (torch.int32, torch.uint32, torch.int64, torch.uint64)
    _check(_lib.sbh_window_ranges(_p(ts), ts.element_size(), ts.numel(), _p(starts), length, starts.numel(),
                                  _p(row_begin), _p(row_end), _stream(stream)), "sbh_window_ranges")


def sbh_kpa_extract(key_col, row_begin, n, keys_out, ptrs_out, key_or=None, samples=None, sample_stride=0,
                    stream=None):
    _check(_lib.sbh_kpa_extract(_p(key_col), row_begin, n, _p(keys_out), _p(ptrs_out), _p(key_or), _p(samples),
                                sample_stride, _stream(stream)), "sbh_kpa_extract")


def sbh_kpa_extract_windows(key_col, offsets, row_begin, n, keys_out, ptrs_out, key_or=None, stream=None):
    """offsets: device uint64 tensor of nwin + 1 row offsets."""
    _check(_lib.sbh_kpa_extract_windows(_p(key_col), _p(offsets), offsets.numel() - 1, row_begin, n, _p(keys_out),
                                        _p(ptrs_out), _p(key_or), _stream(stream)), "sbh_kpa_extract_windows")


def sbh_kpa_split_ts(keys, ts_rel, n, ts_base, win_len, first_win, ptr_base, slot0, slot1, fill, dropped, overflow,
                     scratch=None, stream=None):
    """slot0, slot1: (keys, ptrs) device tensors (their lengths are the capacities)."""
    args = (_p(keys), _p(ts_rel), n, ts_base, win_len, first_win, ptr_base, _p(slot0[0]), _p(slot0[1]),
            slot0[0].numel(), _p(slot1[0]), _p(slot1[1]), slot1[0].numel(), _p(fill), _p(dropped), _p(overflow))
    if scratch is None:
        return _scratch(_lib.sbh_kpa_split_ts, args, (_stream(stream),), "sbh_kpa_split_ts", keys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_kpa_split_ts(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_kpa_split_ts")
    return scratch


def split_scratch_bytes(n: int) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_kpa_split_ts(None, None, n, 0, 1, 0, 0, None, None, 0, None, None, 0, None, None, None, None,
                                 ctypes.byref(nbytes), None), "sbh_kpa_split_ts")
    return nbytes.value


def select_scratch_bytes(n: int) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_kpa_select(None, None, n, None, 8, 0, 0, None, None, 0, None, None, ctypes.byref(nbytes), None),
           "sbh_kpa_select")
    return nbytes.value


def window_bits(nwin: int) -> int:
    return _lib.sbh_window_bits(nwin)


def sbh_kpa_sort(keys_in, ptrs_in, keys_out, ptrs_out, scratch=None, stream=None):
    """Sorts n = keys_in.numel() pairs.  Allocates scratch if none is given;
    returns the scratch buffer used."""
    n = keys_in.numel()
    args = (_p(keys_in), _p(ptrs_in), _p(keys_out), _p(ptrs_out), n)
    if scratch is None:
        return _scratch(_lib.sbh_kpa_sort, args, (_stream(stream),), "sbh_kpa_sort", keys_in.device)
    nbytes = ctypes.c_size_t(scratch.numel() * scratch.element_size())
    _check(_lib.sbh_kpa_sort(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_kpa_sort")
    return scratch


def sort_scratch_bytes(n: int) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_kpa_sort(None, None, None, None, n, None, ctypes.byref(nbytes), None), "sbh_kpa_sort")
    return nbytes.value


def group_reduce_scratch_bytes(n: int, val_bytes: int = 8) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_group_reduce(None, None, n, None, val_bytes, None, None, 8, None, 0, None, None,
                                 ctypes.byref(nbytes), None), "sbh_group_reduce")
    return nbytes.value


def topk_scratch_bytes(n: int, K: int, val_bytes: int = 8) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_topk(None, None, n, None, val_bytes, K, None, None, None, None, 0, None, None,
                         ctypes.byref(nbytes), None), "sbh_topk")
    return nbytes.value


def join_scratch_bytes(nl: int, nr: int) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_join(None, None, nl, None, None, nr, None, None, 0, None, None, ctypes.byref(nbytes), None),
           "sbh_join")
    return nbytes.value


def sbh_kpa_merge(runs, keys_out, ptrs_out, stream=None):
    """runs: list of (keys, ptrs) CUDA tensors, each sorted."""
    r = len(runs)
    kp = (ctypes.c_void_p * max(1, r))(*[k.data_ptr() for k, _ in runs])
    pp = (ctypes.c_void_p * max(1, r))(*[p.data_ptr() for _, p in runs])
    ln = (ctypes.c_uint64 * max(1, r))(*[k.numel() for k, _ in runs])
    args = (r, ctypes.cast(kp, ctypes.c_void_p), ctypes.cast(pp, ctypes.c_void_p), ctypes.cast(ln, ctypes.c_void_p),
            _p(keys_out), _p(ptrs_out))
    _scratch(_lib.sbh_kpa_merge, args, (_stream(stream),), "sbh_kpa_merge", keys_out.device)


def _host_u64(values):
    a = (ctypes.c_uint64 * max(1, len(values)))(*[int(v) for v in values])
    return a, ctypes.cast(a, ctypes.c_void_p)


def sbh_kpa_merge_segments(a, b, a_start, a_len, b_start, b_len, keys_out, ptrs_out, stream=None):
    """a, b: (keys, ptrs) device tensors; the four segment lists are host
    sequences.  Segment g's merge lands after those of segments < g."""
    nseg = len(a_start)
    hold = [_host_u64(x) for x in (a_start, a_len, b_start, b_len)]
    args = (nseg, _p(a[0]), _p(a[1]), _p(b[0]), _p(b[1]), *[h[1] for h in hold], _p(keys_out), _p(ptrs_out))
    _scratch(_lib.sbh_kpa_merge_segments, args, (_stream(stream),), "sbh_kpa_merge_segments", keys_out.device)


def sbh_join_segments(L, l_off, R, r_start, r_len, out_l, out_r, cap, npairs, seg_pairs, scratch=None,
                      stream=None, reuse_counts=False):
    """L, R: (keys, ptrs) device tensors; l_off (nseg + 1), r_start, r_len:
    host sequences; seg_pairs: device uint64 tensor of nseg + 1 entries.
    reuse_counts: scratch holds the counts of an earlier call (cap 0) with
    the same inputs; only the pairs are written."""
    nseg = len(r_start)
    hold = [_host_u64(x) for x in (l_off, r_start, r_len)]
    args = (nseg, _p(L[0]), _p(L[1]), hold[0][1], _p(R[0]), _p(R[1]), hold[1][1], hold[2][1], _p(out_l), _p(out_r),
            cap, _p(npairs), _p(seg_pairs), 1 if reuse_counts else 0)
    if scratch is None:
        return _scratch(_lib.sbh_join_segments, args, (_stream(stream),), "sbh_join_segments", npairs.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_join_segments(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_join_segments")
    return scratch


def sbh_group_reduce(keys, ptrs, vals, out_keys, out_counts, out_sums, cap, nkeys, scratch=None, stream=None):
    """out_counts: uint64 or uint32 (each count is below 2^32)."""
    vb = 0 if vals is None else vals.element_size()
    cb = 8 if out_counts is None else out_counts.element_size()
    args = (_p(keys), _p(ptrs), keys.numel(), _p(vals), vb, _p(out_keys), _p(out_counts), cb, _p(out_sums), cap,
            _p(nkeys))
    if scratch is None:
        return _scratch(_lib.sbh_group_reduce, args, (_stream(stream),), "sbh_group_reduce", keys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_group_reduce(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_group_reduce")
    return scratch


def sbh_topk(keys, ptrs, vals, K, out_keys, out_nvalid, out_vals, out_ptrs, cap, nkeys, scratch=None, stream=None):
    args = (_p(keys), _p(ptrs), keys.numel(), _p(vals), vals.element_size(), K, _p(out_keys), _p(out_nvalid),
            _p(out_vals), _p(out_ptrs), cap, _p(nkeys))
    if scratch is None:
        return _scratch(_lib.sbh_topk, args, (_stream(stream),), "sbh_topk", keys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_topk(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_topk")
    return scratch


def sbh_join(lkeys, lptrs, rkeys, rptrs, out_l, out_r, cap, npairs, scratch=None, stream=None):
    args = (_p(lkeys), _p(lptrs), lkeys.numel(), _p(rkeys), _p(rptrs), rkeys.numel(), _p(out_l), _p(out_r), cap,
            _p(npairs))
    if scratch is None:
        return _scratch(_lib.sbh_join, args, (_stream(stream),), "sbh_join", lkeys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_join(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_join")
    return scratch


def sbh_kpa_materialize(ptrs, col, out, stream=None):
    _check(_lib.sbh_kpa_materialize(_p(ptrs), ptrs.numel(), _p(col), col.element_size(), _p(out), _stream(stream)),
           "sbh_kpa_materialize")


def sbh_copy_counted(src, dst, count, per=1, cap=None, stream=None):
    """dst[:min(count, cap) * per] = src[...]; count is a device uint64
    tensor; dst may be a page-locked CPU tensor; a 4-byte dst of an 8-byte
    src keeps each value's low 4 bytes."""
    cap = src.numel() // per if cap is None else cap
    _check(_lib.sbh_copy_counted(_p(src), _p(dst), src.element_size(), dst.element_size(), _p(count), per, cap,
                                 _stream(stream)), "sbh_copy_counted")


def sbh_kpa_keyswap(ptrs, key_col, keys_out, stream=None):
    _check(_lib.sbh_kpa_keyswap(_p(ptrs), ptrs.numel(), _p(key_col), _p(keys_out), _stream(stream)),
           "sbh_kpa_keyswap")


def sbh_kpa_keyswap_lookup(ptrs, col, table, keys_out, misses=None, stream=None):
    _check(_lib.sbh_kpa_keyswap_lookup(_p(ptrs), ptrs.numel(), _p(col), _p(table), table.numel(), _p(keys_out),
                                       _p(misses), _stream(stream)), "sbh_kpa_keyswap_lookup")


def sbh_kpa_select(keys, ptrs, col, lo, hi, out_keys, out_ptrs, cap, count, scratch=None, stream=None):
    args = (_p(keys), _p(ptrs), keys.numel(), _p(col), col.element_size(), lo, hi, _p(out_keys), _p(out_ptrs), cap,
            _p(count))
    if scratch is None:
        return _scratch(_lib.sbh_kpa_select, args, (_stream(stream),), "sbh_kpa_select", keys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_kpa_select(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_kpa_select")
    return scratch


def sbh_median_unique(keys, ptrs, vals, out_keys, out_median, out_unique, cap, nkeys, scratch=None, stream=None):
    args = (_p(keys), _p(ptrs), keys.numel(), _p(vals), vals.element_size(), _p(out_keys), _p(out_median),
            _p(out_unique), cap, _p(nkeys))
    if scratch is None:
        return _scratch(_lib.sbh_median_unique, args, (_stream(stream),), "sbh_median_unique", keys.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_median_unique(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_median_unique")
    return scratch


def sbh_kpa_partition(keys, ptrs, bounds, keys_out, ptrs_out, offsets, scratch=None, stream=None):
    """bounds: device uint64 tensor of nb non-decreasing keys; offsets: device
    uint64 tensor of nb + 2 entries."""
    nb = 0 if bounds is None else bounds.numel()
    assert offsets.numel() == nb + 2
    args = (_p(keys), _p(ptrs), keys.numel(), _p(bounds), nb, _p(keys_out), _p(ptrs_out), _p(offsets))
    if scratch is None:
        return _scratch(_lib.sbh_kpa_partition, args, (_stream(stream),), "sbh_kpa_partition", offsets.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_kpa_partition(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_kpa_partition")
    return scratch


# ----------------------------------------------------------------- conveniences
def _u64(n, dev):
    return torch.empty(n, dtype=torch.uint64, device=dev)


def _u32(n, dev):
    return torch.empty(n, dtype=torch.uint32, device=dev)


def extract(key_col, row_begin=0, n=None, device="cuda", sample_stride=0):
    """KPA of rows [row_begin, row_begin + n) -> (keys, ptrs[, key_or, samples])."""
    if n is None:
        n = key_col.numel() - row_begin
    keys, ptrs = _u64(n, device), _u32(n, device)
    key_or = _u64(1, device)
    samples = _u64((n + sample_stride - 1) // sample_stride, device) if sample_stride else None
    sbh_kpa_extract(key_col, row_begin, n, keys, ptrs, key_or, samples, sample_stride)
    if sample_stride:
        return keys, ptrs, key_or, samples
    return keys, ptrs


def sample(key_col, stride, row_begin=0, n=None):
    """Every stride-th key of rows [row_begin, row_begin + n), read straight
    from the column (no Extract)."""
    if n is None:
        n = key_col.numel() - row_begin
    samples = _u64((n + stride - 1) // stride, key_col.device)
    sbh_kpa_extract(key_col, row_begin, n, None, None, None, samples, stride)
    return samples


def sort(keys, ptrs, out=None):
    """Sorted copy (or into out=(keys_out, ptrs_out), which may alias the
    input).  ptrs=None: keys is a key column, row i's ptr is i (no Extract)."""
    if out is None:
        out = (torch.empty_like(keys), _u32(keys.numel(), keys.device) if ptrs is None else torch.empty_like(ptrs))
    sbh_kpa_sort(keys, ptrs, out[0], out[1])
    return out


def merge(runs):
    total = sum(k.numel() for k, _ in runs)
    dev = runs[0][0].device
    ok, op = _u64(total, dev), _u32(total, dev)
    sbh_kpa_merge(runs, ok, op)
    return ok, op


def group_reduce(keys, ptrs, vals=None, cap=None):
    """Per distinct key: (keys, counts, sums or None); synchronises to size the result."""
    n = keys.numel()
    cap = n if cap is None else cap
    dev = keys.device
    ok, oc = _u64(max(cap, 1), dev), _u64(max(cap, 1), dev)
    osum = _u64(max(cap, 1), dev) if vals is not None else None
    nk = _u64(1, dev)
    sbh_group_reduce(keys, ptrs, vals, ok, oc, osum, cap, nk)
    m = int(nk.item())
    m = min(m, cap)
    return ok[:m], oc[:m], (osum[:m] if osum is not None else None)


def topk(keys, ptrs, vals, K, cap=None):
    n = keys.numel()
    cap = n if cap is None else cap
    dev = keys.device
    ok = _u64(max(cap, 1), dev)
    nv = torch.empty(max(cap, 1), dtype=torch.uint8, device=dev)
    ov = _u64(max(cap, 1) * K, dev)
    op = _u32(max(cap, 1) * K, dev)
    nk = _u64(1, dev)
    sbh_topk(keys, ptrs, vals, K, ok, nv, ov, op, cap, nk)
    m = min(int(nk.item()), cap)
    return ok[:m], nv[:m], ov[: m * K].view(m, K) if m else ov[:0].view(0, K), op[: m * K].view(m, K) if m else op[:0].view(0, K)


def join(lkeys, lptrs, rkeys, rptrs, cap=None):
    """All (ptrL, ptrR) pairs; with cap None, counts first (two calls)."""
    dev = lkeys.device
    npairs = _u64(1, dev)
    if cap is None:
        sbh_join(lkeys, lptrs, rkeys, rptrs, None, None, 0, npairs)
        cap = int(npairs.item())
    ol, orr = _u32(max(cap, 1), dev), _u32(max(cap, 1), dev)
    sbh_join(lkeys, lptrs, rkeys, rptrs, ol, orr, cap, npairs)
    m = min(int(npairs.item()), cap)
    return ol[:m], orr[:m]


def partition(keys, ptrs, bounds):
    """(keys, ptrs, offsets) of the KPA split by the key ranges that bounds cut."""
    dev = keys.device
    ok, op = _u64(keys.numel(), dev), _u32(keys.numel(), dev)
    off = _u64(bounds.numel() + 2, dev)
    sbh_kpa_partition(keys, ptrs, bounds, ok, op, off)
    return ok, op, off


def window_ranges(ts, starts, length):
    rb = _u64(starts.numel(), ts.device)
    re_ = _u64(starts.numel(), ts.device)
    sbh_window_ranges(ts, starts, length, rb, re_)
    return rb, re_


# ----------------------------------------------------------------- learned partition
def sbh_mlp_forward(params, x, y, stream=None):
    _check(_lib.sbh_mlp_forward(_p(params), _p(x), x.numel(), _p(y), _stream(stream)), "sbh_mlp_forward")


def sbh_mlp_grad(params, x, t, grad, loss=None, stream=None):
    args = (_p(params), _p(x), _p(t), x.numel(), _p(grad), _p(loss))
    return _scratch(_lib.sbh_mlp_grad, args, (_stream(stream),), "sbh_mlp_grad", x.device)


def sbh_learned_train(samples, n_rows, init_params, steps, batch, lr, model, losses=None, train_x=None,
                      train_t=None, scratch=None, stream=None):
    """Allocates scratch if none is given (see learned_train_scratch_bytes);
    returns the scratch used."""
    args = (_p(samples), samples.numel(), n_rows, _p(init_params), steps, batch, ctypes.c_float(lr), _p(model),
            _p(losses), _p(train_x), _p(train_t))
    if scratch is None:
        return _scratch(_lib.sbh_learned_train, args, (_stream(stream),), "sbh_learned_train", samples.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_learned_train(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)), "sbh_learned_train")
    return scratch


def learned_train_scratch_bytes(m: int) -> int:
    """Scratch of a training call on m samples (it grows with m)."""
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_learned_train(None, m, m, None, 0, 4096, ctypes.c_float(0.0), None, None, None, None, None,
                                  ctypes.byref(nbytes), None), "sbh_learned_train")
    return nbytes.value


def sbh_kpa_sort_learned(keys_in, ptrs_in, keys_out, ptrs_out, model, stats=None, scratch=None, stream=None):
    """Queues the learned sort; stats (nullable) is a device uint64 tensor of
    len(LEARNED_STATS) entries that the call fills on the device (read it
    with stats_dict after synchronising).  Returns the scratch used."""
    args = (_p(keys_in), _p(ptrs_in), _p(keys_out), _p(ptrs_out), keys_in.numel(), _p(model), _p(stats))
    if scratch is None:
        return _scratch(_lib.sbh_kpa_sort_learned, args, (_stream(stream),), "sbh_kpa_sort_learned",
                        keys_in.device)
    nbytes = ctypes.c_size_t(scratch.numel())
    _check(_lib.sbh_kpa_sort_learned(*args, _p(scratch), ctypes.byref(nbytes), _stream(stream)),
           "sbh_kpa_sort_learned")
    return scratch


def stats_dict(stats):
    """The learned sort's statistics tensor as a dict (synchronises)."""
    return dict(zip(LEARNED_STATS, [int(x) for x in stats.cpu().tolist()]))


def sort_learned_scratch_bytes(n: int) -> int:
    nbytes = ctypes.c_size_t(0)
    _check(_lib.sbh_kpa_sort_learned(None, None, None, None, n, None, None, None, ctypes.byref(nbytes), None),
           "sbh_kpa_sort_learned")
    return nbytes.value


def learned_train(samples, n_rows, init_params, steps=150, batch=4096, lr=2e-2):
    """Model blob (uint8 CUDA tensor) and the per-step batch losses."""
    dev = samples.device
    model = torch.zeros(LEARNED_MODEL_BYTES, dtype=torch.uint8, device=dev)
    losses = torch.zeros(max(1, steps), dtype=torch.float32, device=dev)
    sbh_learned_train(samples, n_rows, init_params, steps, batch, lr, model, losses)
    return model, losses[:steps]


def model_params(model):
    """The network weights inside a model blob (a float32 view)."""
    return model[: MLP_PARAMS * 4].view(torch.float32)


def sort_learned(keys, ptrs, model):
    """Sorted copy and the statistics as a dict (synchronises to read them).
    ptrs=None: keys is a key column, row i's ptr is i (no Extract)."""
    out = (torch.empty_like(keys), _u32(keys.numel(), keys.device) if ptrs is None else torch.empty_like(ptrs))
    stats = torch.zeros(len(LEARNED_STATS), dtype=torch.uint64, device=keys.device)
    sbh_kpa_sort_learned(keys, ptrs, out[0], out[1], model, stats)
    return out[0], out[1], stats_dict(stats)


# ----------------------------------------------------------------- Table 2 record primitives and per-key statistics
def materialize(ptrs, col):
    out = torch.empty(ptrs.numel(), dtype=col.dtype, device=ptrs.device)
    sbh_kpa_materialize(ptrs, col, out)
    return out


def select(keys, ptrs, col, lo, hi):
    """(keys, ptrs) of the records with col[ptr] in [lo, hi); synchronises to size the result."""
    n = keys.numel()
    ok, op, cnt = _u64(max(n, 1), keys.device), _u32(max(n, 1), keys.device), _u64(1, keys.device)
    sbh_kpa_select(keys, ptrs, col, lo, hi, ok, op, n, cnt)
    m = int(cnt.item())
    return ok[:m], op[:m]


def median_unique(keys, ptrs, vals):
    """Per distinct key: (keys, lower median, number of distinct values)."""
    n = keys.numel()
    dev = keys.device
    ok, om, ou, nk = _u64(max(n, 1), dev), _u64(max(n, 1), dev), _u64(max(n, 1), dev), _u64(1, dev)
    sbh_median_unique(keys, ptrs, vals, ok, om, ou, n, nk)
    m = int(nk.item())
    return ok[:m], om[:m], ou[:m]
