"""Parity of the CUDA path (through the C ABI) with the oracle, element by
element, on seeded inputs: sizes that span several tiles with a ragged tail,
edge cases, and the full workload sizes (bit-exact where the oracle finishes
in seconds, by invariants beyond that)."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests import pins
from tests.gpu_util import cuda, host, same, sorted_kpa_on_device

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    return sbh


# ------------------------------------------------------------------ extract
@pytest.mark.parametrize("n,row_begin", [(0, 0), (1, 0), (5, 3), (4097, 1), (1_000_000, 0), (999_999, 7)])
def test_extract_parity(S, n, row_begin):
    col = gen.mixed_keys(row_begin + n + 5)
    d_col = cuda(col)
    keys, ptrs, key_or, samples = S.extract(d_col, row_begin, n, sample_stride=100)
    ok, op = oracle.extract(col, row_begin, n)
    assert same(keys, ok) and same(ptrs, op)
    if n:
        assert int(host(key_or)[0]) == int(np.bitwise_or.reduce(ok))
        assert same(samples, ok[::100])


@pytest.mark.parametrize("stride", [1, 3, 4, 7, 100, 4096, 2_000_000])
def test_extract_sample_strides(S, stride):
    # groups of four rows with zero, one or several sampled rows (16-byte path)
    n = 1_000_003
    col = gen.mixed_keys(n)
    keys, ptrs, key_or, samples = S.extract(cuda(col), 0, n, sample_stride=stride)
    ok, op = oracle.extract(col, 0, n)
    assert same(keys, ok) and same(ptrs, op)
    assert same(samples, ok[::stride])


def test_extract_from_pinned_host(S):
    col = gen.join_streams(300_001, key_space=1 << 24)["L"]["keys"]
    pinned = torch.from_numpy(col).pin_memory()
    keys, ptrs = S.extract(pinned, 1000, 250_000)
    ok, op = oracle.extract(col, 1000, 250_000)
    assert same(keys, ok) and same(ptrs, op)


# ------------------------------------------------------------------ sort
def _sort_case(kind, n, seed=1):
    if kind == "uniform20":
        return gen.uniform(seed, 1, n, 0, 1 << 20, np.uint64)
    if kind == "mixed":
        return gen.mixed_keys(n, seed=seed)
    if kind == "equal":
        return np.full(n, 0xDEADBEEF, dtype=np.uint64)
    if kind == "extremes":
        return np.where(gen.uniform(seed, 2, n, 0, 2, np.uint64) == 1, np.uint64(M64), np.uint64(0))
    if kind == "highbyte":  # only the top digit varies: seven passes are skipped
        return gen.uniform(seed, 3, n, 0, 256, np.uint64) << np.uint64(56)
    if kind == "full64":
        return gen.uniform(seed, 4, n, 0, 0, np.uint64)
    if kind == "gaps":  # bytes 0, 2 and 6 vary, the others are constant (not zero): passes 1, 3-5, 7 skipped
        r = gen.uniform(seed, 5, n, 0, 1 << 24, np.uint64)
        return ((r & np.uint64(0xFF)) | (((r >> np.uint64(8)) & np.uint64(0xFF)) << np.uint64(16))
                | ((r >> np.uint64(16)) << np.uint64(48)) | np.uint64(0x5A00_A5A5_5A00_5A00))
    if kind == "lowconst":  # byte 0 constant: the first pass that runs is the second
        return (gen.uniform(seed, 6, n, 0, 0, np.uint64) & ~np.uint64(0xFF)) | np.uint64(0x33)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n,offset", [("full64", 3 * 4096 + 5, 0), ("mixed", 100_003, 1), ("equal", 10_000, 0),
                                           ("highbyte", 4097, 0), ("mixed", (1 << 23) + 3, 0),
                                           ("mixed", (1 << 23) + 4099, 1), ("lowconst", (1 << 23) + 3, 0),
                                           ("gaps", (1 << 23) + 5, 0)])
def test_sort_key_column_without_extract(S, kind, n, offset):
    # ptrs_in = None: the sort reads the key column and row i's ptr is i,
    # as an Extract of the column would make it; offset 1 starts the column
    # 8 bytes past a 16-byte boundary (no bulk copies: plain loads)
    col = _sort_case(kind, n + offset)
    d = cuda(col)[offset:]
    sk, sp = S.sort(d, None)
    ok, op = oracle.sort(*oracle.extract(col[offset:], 0, n))
    assert same(sk, ok) and same(sp, op)


def test_extract_samples_only(S):
    n, stride = 1_000_003, 100
    col = gen.mixed_keys(n, seed=3)
    _, _, _, smp = S.extract(cuda(col), 7, n - 7, sample_stride=stride)
    assert same(S.sample(cuda(col), stride, 7, n - 7), smp)
    assert same(smp, col[7::stride])


@pytest.mark.parametrize("kind", ["uniform20", "mixed", "equal", "extremes", "highbyte", "full64"])
@pytest.mark.parametrize("n", [0, 1, 2, 4095, 4096, 4097, 100_003])
def test_sort_parity(S, kind, n):
    col = _sort_case(kind, n)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp = S.sort(keys, ptrs)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)
    assert same(keys, col)  # the input is not written


def test_sort_in_place_and_unordered_ptrs(S):
    n = 50_001
    col = gen.mixed_keys(n, seed=5)
    ptrs = gen.uniform(5, 9, n, 0, 1 << 31, np.uint32)  # arbitrary pointers: ties keep input order
    k, p = cuda(col), cuda(ptrs)
    S.sort(k, p, out=(k, p))
    order = np.argsort(col, kind="stable")
    assert same(k, col[order]) and same(p, ptrs[order])
    # odd number of passes (20-bit keys: three digits), in place
    col = _sort_case("uniform20", n)
    k, p = cuda(col), cuda(np.arange(n, dtype=np.uint32))
    S.sort(k, p, out=(k, p))
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(k, ok) and same(p, op)


def test_sort_tumbling_window_full_size(S):
    w = gen.tumbling_window(1_000_000)
    keys, ptrs = S.extract(cuda(w["keys"]), 0, 1_000_000)
    sk, sp = S.sort(keys, ptrs)
    ok, op = oracle.sort(*oracle.extract(w["keys"], 0, 1_000_000))
    assert same(sk, ok) and same(sp, op)


def test_sort_mixed_keys_16m_bit_exact(S):
    n = 16_000_000
    col = gen.mixed_keys(n)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp = S.sort(keys, ptrs)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


def test_sort_mixed_keys_256m_invariants(S):
    n = 256_000_000
    col = torch.empty(n, dtype=torch.uint64)
    gen.mixed_keys(n, out=col.numpy())
    d_col = col.cuda()
    keys, ptrs = S.extract(d_col, 0, n)
    del col
    S.sort(keys, ptrs, out=(keys, ptrs))
    sorted_kpa_on_device(d_col, 0, keys, ptrs)
    # sampled rows against the oracle's sort of the same rows: the rank of a
    # sampled (key, ptr) pair equals the number of pairs below it
    idx = torch.linspace(0, n - 1, 257, dtype=torch.int64).cuda()
    sk = (d_col.view(torch.int64) ^ torch.iinfo(torch.int64).min)
    for i in host(idx)[:: 32]:
        kk, pp = keys[i].view(torch.int64) ^ torch.iinfo(torch.int64).min, int(ptrs[i])
        below = int((sk < kk).sum()) + int(((sk == kk) & (torch.arange(n, device="cuda") < pp)).sum())
        assert below == int(i)


def test_sort_timeout_hook_reports_and_recovers(S):
    n = 3 * 4096 + 17
    col = _sort_case("full64", n)
    keys, ptrs = S.extract(cuda(col), 0, n)
    S.sync_status()
    S.set_spin_limit(2000)
    S.set_fault(S.SBH_FAULT_SKIP_PUBLISH)
    try:
        S.sort(keys, ptrs)
        assert S.sync_status() == S.SBH_ETIMEOUT
    finally:
        S.set_spin_limit(0)
        S.set_fault(S.SBH_FAULT_NONE)
    sk, sp = S.sort(keys, ptrs)
    assert S.sync_status() == S.SBH_OK
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


def test_sort_chunked_path_tiny_wait_budget_reports_and_recovers(S):
    # the chunked passes wait only on their own bulk copies; with a poll
    # budget of one, a copy that has not landed at the first poll ends its
    # chunk: the CTA lets its copies in flight land and leaves, the timeout
    # is recorded, and the next sort with the normal budget is correct
    n = (1 << 23) + 4097
    col = _sort_case("mixed", n, seed=4)
    keys, ptrs = S.extract(cuda(col), 0, n)
    S.sync_status()
    S.set_spin_limit(1)
    try:
        S.sort(keys, ptrs)
        st = S.sync_status()
    finally:
        S.set_spin_limit(0)
    assert st in (S.SBH_OK, S.SBH_ETIMEOUT)
    sk, sp = S.sort(keys, ptrs)
    assert S.sync_status() == S.SBH_OK
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


def test_sort_scratch_too_small(S):
    keys, ptrs = S.extract(cuda(_sort_case("full64", 1000)), 0, 1000)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.SbhError) as e:
        S.sbh_kpa_sort(keys, ptrs, torch.empty_like(keys), torch.empty_like(ptrs), scratch=small)
    assert e.value.code == S.SBH_ENOSPACE


# ------------------------------------------------------------------ group reduce
def _sorted_kpa(S, col):
    n = col.size
    keys, ptrs = S.extract(cuda(col), 0, n)
    return S.sort(keys, ptrs)


def _oracle_sorted(col):
    """The oracle's own sorted KPA of a whole column: the input the oracle's
    grouping functions get, so that no CUDA output feeds the expected values."""
    return oracle.sort(*oracle.extract(col, 0, col.size))


@pytest.mark.parametrize("vbytes", [4, 8])
@pytest.mark.parametrize("n,space", [(1, 4), (4096, 7), (4097, 1), (100_003, 1000), (100_003, 1 << 40)])
def test_group_reduce_parity(S, vbytes, n, space):
    col, _ = gen.tiny_kpa(n, space, seed=n)
    vals = gen.uniform(7, 7, n, 0, 0, np.uint64 if vbytes == 8 else np.uint32)  # full range: sums wrap
    sk, sp = _sorted_kpa(S, col)
    gk, gc, gs = S.group_reduce(sk, sp, cuda(vals))
    ok, oc, osum = oracle.group_sum_count(*_oracle_sorted(col), vals)
    assert same(gk, ok) and same(gc, oc) and same(gs, osum)


def test_group_reduce_tumbling_window_and_count_only(S):
    w = gen.tumbling_window(1_000_000)
    sk, sp = _sorted_kpa(S, w["keys"])
    gk, gc, gs = S.group_reduce(sk, sp, cuda(w["vals"]))
    ok, oc, osum = oracle.group_sum_count(*oracle.sort(*oracle.extract(w["keys"], 0, 1_000_000)), w["vals"])
    assert same(gk, ok) and same(gc, oc) and same(gs, osum)
    ck, cc, cs = S.group_reduce(sk, sp, None)
    assert cs is None and same(ck, ok) and same(cc, oc)


def test_group_reduce_heavy_key_spans_tiles_and_cap(S):
    n = 300_000
    col = gen.mixed_keys(n, seed=11)
    col[1000:200_000] = 1  # one key over ~49 tiles
    vals = gen.uniform(3, 3, n, 0, 0, np.uint64)
    sk, sp = _sorted_kpa(S, col)
    gk, gc, gs = S.group_reduce(sk, sp, cuda(vals))
    ok, oc, osum = oracle.group_sum_count(*_oracle_sorted(col), vals)
    assert same(gk, ok) and same(gc, oc) and same(gs, osum)
    # capacity below the number of keys: the first cap rows, the full count
    cap = ok.size // 3
    out_k = torch.zeros(cap, dtype=torch.uint64, device="cuda")
    out_c = torch.zeros(cap, dtype=torch.uint64, device="cuda")
    out_s = torch.zeros(cap, dtype=torch.uint64, device="cuda")
    nk = torch.zeros(1, dtype=torch.uint64, device="cuda")
    S.sbh_group_reduce(sk, sp, cuda(vals), out_k, out_c, out_s, cap, nk)
    assert int(host(nk)[0]) == ok.size
    assert same(out_k, ok[:cap]) and same(out_c, oc[:cap]) and same(out_s, osum[:cap])


@pytest.mark.parametrize("offset", [0, 1, 511])
def test_group_count_runs_at_warp_range_boundaries(S, offset):
    # a warp reads 512 consecutive rows; counts-only skips the rows of a
    # range whose first and last keys are equal.  Runs that start, end or
    # fill a range exactly (and one that ends at the last row) must still
    # give every key its head and count
    lengths = [offset or 1, 512, 511, 513, 1, 1024, 4096, 4097, 3, 512 * 9, 1, 1, 700, 512 + 511]
    lengths = lengths * 6 + [2 * 4096 + 5]
    col = np.repeat(np.arange(len(lengths), dtype=np.uint64) * 7 + 3, lengths)
    n = col.size
    sk, sp = _sorted_kpa(S, col)
    gk, gc, _ = S.group_reduce(sk, sp, None)
    ok, oc, _ = oracle.group_sum_count(*_oracle_sorted(col), None)
    assert same(gk, ok) and same(gc, oc) and int(oc.sum()) == n


def test_group_reduce_four_byte_counts(S):
    # counts written as uint32 equal the uint64 ones (every count is below 2^32)
    n = 300_001
    col = gen.mixed_keys(n, seed=13)
    vals = gen.uniform(6, 6, n, 0, 0, np.uint64)
    sk, sp = _sorted_kpa(S, col)
    ok, oc, osum = oracle.group_sum_count(*_oracle_sorted(col), vals)
    for with_vals in (False, True):
        out_k = torch.zeros(n, dtype=torch.uint64, device="cuda")
        out_c = torch.zeros(n, dtype=torch.uint32, device="cuda")
        out_s = torch.zeros(n, dtype=torch.uint64, device="cuda") if with_vals else None
        nk = torch.zeros(1, dtype=torch.uint64, device="cuda")
        S.sbh_group_reduce(sk, sp, cuda(vals) if with_vals else None, out_k, out_c, out_s, n, nk)
        m = int(host(nk)[0])
        assert m == ok.size and same(out_k[:m], ok) and same(out_c[:m], oc.astype(np.uint32))
        assert int(host(out_c)[m]) == 0  # nothing written past the last key
        if with_vals:
            assert same(out_s[:m], osum)


def test_copy_counted_narrows_counts(S):
    # the counted copy of 8-byte counts into 4 bytes (page-locked host memory
    # and device memory), only the first count rows
    n = 100_000
    src = cuda(gen.uniform(8, 8, n, 0, 1 << 31, np.uint64))
    cnt = torch.tensor([77_777], dtype=torch.uint64, device="cuda")
    for dst in (torch.zeros(n, dtype=torch.uint32).pin_memory(), torch.zeros(n, dtype=torch.uint32, device="cuda")):
        S.sbh_copy_counted(src, dst, cnt)
        torch.cuda.synchronize()
        got = host(dst)
        assert same(got[:77_777], host(src)[:77_777].astype(np.uint32)) and not got[77_777:].any()


def test_group_count_mixed_keys_16m(S):
    n = 16_000_000
    col = gen.mixed_keys(n)
    sk, sp = _sorted_kpa(S, col)
    gk, gc, _ = S.group_reduce(sk, sp, None)
    ok, oc, _ = oracle.group_sum_count(col, np.arange(n, dtype=np.uint32), None)
    assert same(gk, ok) and same(gc, oc)


# ------------------------------------------------------------------ top-K
@pytest.mark.parametrize("K", [1, 3, 5, 8])
@pytest.mark.parametrize("vbytes", [4, 8])
@pytest.mark.parametrize("n,space,vspan", [(1, 4, 8), (4097, 3, 5), (100_003, 5000, 0), (60_000, 1, 100)])
def test_topk_parity(S, K, vbytes, n, space, vspan):
    col, _ = gen.tiny_kpa(n, space, seed=n + K)
    vals = gen.uniform(4, 4, n, 0, vspan, np.uint64 if vbytes == 8 else np.uint32)
    sk, sp = _sorted_kpa(S, col)
    tk, tn, tv, tp = S.topk(sk, sp, cuda(vals), K)
    ok, onv, ov, op = oracle.topk(*_oracle_sorted(col), vals, K)
    assert same(tk, ok) and same(tn, onv) and same(tv, ov) and same(tp, op)


@pytest.mark.parametrize("K", [3, 8])
def test_topk_segment_size_boundaries_and_cap(S, K):
    # runs at the per-thread limit (64 / 65 rows), the per-warp limit (4096 /
    # 4097) and the chunk size (16384 / 16385 rows), runs of several chunks,
    # short runs between them
    counts = [1, 64, 65, 2, 4096, 4097, 16384, 16385, 40_000, 3, 100_000, 7]
    col = np.repeat(np.arange(len(counts), dtype=np.uint64) * 11, counts)
    n = col.size
    vals = gen.uniform(6, 6, n, 0, 50, np.uint64)
    sk, sp = _sorted_kpa(S, col)
    tk, tn, tv, tp = S.topk(sk, sp, cuda(vals), K)
    ok, onv, ov, op = oracle.topk(*_oracle_sorted(col), vals, K)
    assert same(tk, ok) and same(tn, onv) and same(tv, ov) and same(tp, op)
    # a capacity below the number of keys: the first cap keys are written
    cap = 4
    okk = torch.zeros(cap, dtype=torch.uint64, device="cuda")
    onn = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    ovv = torch.zeros(cap * K, dtype=torch.uint64, device="cuda")
    opp = torch.zeros(cap * K, dtype=torch.uint32, device="cuda")
    nk = torch.zeros(1, dtype=torch.uint64, device="cuda")
    S.sbh_topk(sk, sp, cuda(vals), K, okk, onn, ovv, opp, cap, nk)
    assert int(host(nk)[0]) == len(counts)
    assert same(okk, ok[:cap]) and same(onn, onv[:cap]) and same(ovv, ov[:cap].reshape(-1))
    assert same(opp, op[:cap].reshape(-1))


def test_topk_batched_window_shape(S):
    b = gen.batched_windows(8, 4)
    col, vals = b["keys"], b["vals"]
    sk, sp = _sorted_kpa(S, col)
    tk, tn, tv, tp = S.topk(sk, sp, cuda(vals), 3)
    ok, onv, ov, op = oracle.topk(*_oracle_sorted(col), vals, 3)
    assert same(tk, ok) and same(tn, onv) and same(tv, ov) and same(tp, op)


# ------------------------------------------------------------------ merge
@pytest.mark.parametrize("lens", [[5, 0], [4096, 4097], [250_000] * 4, [1, 30_000, 0, 7777, 100_001], [10] * 9])
def test_merge_parity(S, lens):
    total = sum(lens)
    col, _ = gen.tiny_kpa(total, 1 << 12, seed=len(lens))
    runs_d, runs_h, off = [], [], 0
    for L in lens:
        k, p = oracle.sort(*oracle.extract(col, off, L))
        runs_h.append((k, p))
        runs_d.append((cuda(k), cuda(p)))
        off += L
    mk, mp = S.merge(runs_d)
    ok, op = oracle.merge(runs_h)
    assert same(mk, ok) and same(mp, op)


# ------------------------------------------------------------------ join
@pytest.mark.parametrize("nl,nr,space", [(0, 10, 4), (10, 0, 4), (300, 200, 5), (4097, 5000, 1 << 12),
                                         (100_000, 90_000, 1 << 24)])
def test_join_parity(S, nl, nr, space):
    lk, _ = gen.tiny_kpa(nl, space, seed=nl + 1)
    rk, _ = gen.tiny_kpa(nr, space, seed=nr + 2, stream=3)
    L = _sorted_kpa(S, lk)
    R = _sorted_kpa(S, rk)
    gl, gr = S.join(*L, *R)
    ol, orr = oracle.join(lk, np.arange(nl, dtype=np.uint32), rk, np.arange(nr, dtype=np.uint32))
    assert same(gl, ol) and same(gr, orr)


def test_join_sliding_window_full_size_and_cap(S):
    # one 1M-row window of each stream, keys uniform over 2^24
    s = gen.join_streams(1_250_000)
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    L = S.sort(*S.extract(cuda(lcol), 250_000, 1_000_000))
    R = S.sort(*S.extract(cuda(rcol), 250_000, 1_000_000))
    gl, gr = S.join(*L, *R)
    lk, lp = oracle.sort(*oracle.extract(lcol, 250_000, 1_000_000))
    rk, rp = oracle.sort(*oracle.extract(rcol, 250_000, 1_000_000))
    ol, orr = oracle.join(lk, lp, rk, rp)
    assert same(gl, ol) and same(gr, orr)
    pins.check_join(lcol, rcol, host(gl), host(gr), pins.join_cardinality(lk, rk))
    cap = ol.size // 2
    out_l = torch.zeros(cap, dtype=torch.uint32, device="cuda")
    out_r = torch.zeros(cap, dtype=torch.uint32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.uint64, device="cuda")
    S.sbh_join(*L, *R, out_l, out_r, cap, npairs)
    assert int(host(npairs)[0]) == ol.size and same(out_l, ol[:cap]) and same(out_r, orr[:cap])


# ------------------------------------------------------------------ windows
def test_window_ranges_parity(S):
    ts = np.sort(gen.uniform(2, 2, 200_000, 0, 1 << 30, np.uint64))
    starts = np.sort(gen.uniform(2, 3, 509, 0, 1 << 30, np.uint64))
    rb, re_ = S.window_ranges(cuda(ts), cuda(starts), 1 << 22)
    ob, oe = oracle.window_ranges(ts, starts, 1 << 22)
    assert same(rb, ob) and same(re_, oe)
    ts32 = np.arange(1_000_000, dtype=np.uint32)
    starts = np.arange(0, 1_000_000, 250_000, dtype=np.uint64)
    rb, re_ = S.window_ranges(cuda(ts32), cuda(starts), 1_000_000)
    ob, oe = oracle.window_ranges(ts32, starts, 1_000_000)
    assert same(rb, ob) and same(re_, oe)


@pytest.fixture
def chunked_from_2m(S):
    """Sorts from 2^21 pairs take the per-chunk count/scan/scatter passes."""
    old = S.get_knob(S.KNOB_SORT_CHUNKED_MIN)
    S.set_knob(S.KNOB_SORT_CHUNKED_MIN, 1 << 21)
    yield
    S.set_knob(S.KNOB_SORT_CHUNKED_MIN, old)


@pytest.mark.parametrize("kind", ["uniform20", "mixed", "highbyte", "extremes", "gaps", "lowconst"])
def test_sort_chunked_path_ragged(S, kind, chunked_from_2m):
    # above the size where passes switch to per-chunk count/scan/scatter,
    # with a ragged last tile.  Each scatter pass leaves every row's digit
    # of the next pass that runs for that pass's chunk counts: "gaps" skips
    # passes between the ones that run, "lowconst" skips the first
    n = (1 << 21) + 4097
    col = _sort_case(kind, n, seed=3)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp = S.sort(keys, ptrs)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


def test_sort_chunked_path_default_threshold(S):
    # just above the default threshold (2^23 pairs), mixed keys
    n = (1 << 23) + 3
    col = gen.mixed_keys(n, seed=8)
    sk, sp = S.sort(*S.extract(cuda(col), 0, n))
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


@pytest.mark.parametrize("kind", ["mixed", "uniform20", "gaps"])
def test_sort_chunked_in_place(S, kind, chunked_from_2m):
    # in place through the chunked passes (the passes alternate between the
    # scratch and the output, and each leaves the next pass's digit bytes);
    # arbitrary pointers: ties keep input order
    n = (1 << 21) + 777
    col = _sort_case(kind, n, seed=11)
    ptrs = gen.uniform(11, 9, n, 0, 1 << 31, np.uint32)
    k, p = cuda(col), cuda(ptrs)
    S.sort(k, p, out=(k, p))
    order = np.argsort(col, kind="stable")
    assert same(k, col[order]) and same(p, ptrs[order])


def test_sort_unaligned_views(S, chunked_from_2m):
    # views that start 8 bytes into a buffer cannot use bulk copies (both paths)
    for n in (50_001, (1 << 21) + 11):
        col = gen.mixed_keys(n + 1, seed=6)
        keys, ptrs = S.extract(cuda(col), 0, n + 1)
        kv, pv = keys[1:], ptrs[1:]
        ok_, op_ = torch.empty_like(keys)[1:], torch.empty_like(ptrs)[1:]
        S.sbh_kpa_sort(kv, pv, ok_, op_)
        ek, ep = oracle.sort(col[1:], np.arange(1, n + 1, dtype=np.uint32))
        assert same(ok_, ek) and same(op_, ep)


# ------------------------------------------------------------------ Table 2 record primitives, median, unique
@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_materialize_and_keyswap_parity(S, dtype):
    n = 300_001
    col = gen.uniform(12, 1, n, 0, 0 if dtype == np.uint64 else 1 << 32, np.uint64).astype(dtype)
    keys, _ = gen.tiny_kpa(n, 1000, seed=12)
    sk, sp = _sorted_kpa(S, keys)
    _, osp = _oracle_sorted(keys)
    got = S.materialize(sp, cuda(col))
    assert same(got, oracle.materialize(osp, col))
    if dtype == np.uint64:
        k2 = torch.empty(n, dtype=torch.uint64, device="cuda")
        S.sbh_kpa_keyswap(sp, cuda(col), k2)
        assert same(k2, oracle.materialize(osp, col))


@pytest.mark.parametrize("n,lo,hi", [(1, 0, 10), (4097, 3, 9), (1_000_003, 100, 60_000), (200_000, 7, 7)])
def test_select_parity(S, n, lo, hi):
    keys, _ = gen.tiny_kpa(n, 5000, seed=n)
    vals = gen.uniform(13, 2, n, 0, 65_536, np.uint32)
    sk, sp = _sorted_kpa(S, keys)
    ok, op = S.select(sk, sp, cuda(vals), lo, hi)
    ek, ep = oracle.select(*_oracle_sorted(keys), vals, lo, hi)
    assert same(ok, ek) and same(op, ep)


@pytest.mark.parametrize("n,space,vspan,vb", [(1, 3, 5, 8), (4097, 9, 4, 4), (500_000, 3000, 1000, 8),
                                              (300_000, 2, 0, 8), (2_500_000, 1 << 20, 1 << 30, 8)])
def test_median_unique_parity(S, n, space, vspan, vb):
    keys, _ = gen.tiny_kpa(n, space, seed=n + 1)
    vals = gen.uniform(14, 3, n, 0, vspan, np.uint64 if vb == 8 else np.uint32)
    sk, sp = _sorted_kpa(S, keys)
    gk, gm, gu = S.median_unique(sk, sp, cuda(vals))
    ek, em, eu = oracle.median_unique(*_oracle_sorted(keys), vals)
    assert same(gk, ek) and same(gm, em) and same(gu, eu)


def test_partition_sorted_kpa_by_key_ranges(S):
    # Partition (Table 2) of a sorted KPA into key ranges is the window-range
    # search over its (non-decreasing) key column
    n = 1_000_003
    keys, _ = gen.tiny_kpa(n, 1 << 20, seed=21)
    sk, sp = _sorted_kpa(S, keys)
    starts = np.arange(0, 1 << 20, 1 << 14, dtype=np.uint64)
    rb, re_ = S.window_ranges(sk, cuda(starts), 1 << 14)
    hk, _ = _oracle_sorted(keys)
    ob, oe = oracle.window_ranges(hk, starts, 1 << 14)
    assert same(rb, ob) and same(re_, oe)
    for w in (0, 17, 63):
        part = hk[int(ob[w]):int(oe[w])]
        assert part.size == np.sum((keys >= starts[w]) & (keys < starts[w] + (1 << 14)))


def test_worked_example_on_the_gpu(S):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    keys = cuda(np.array(g["keys"], np.uint64))
    vals = cuda(np.array(g["values"], np.uint64))
    k, p = S.sort(*S.extract(keys, 0, 8))
    assert host(k).tolist() == g["sorted"]["keys"] and host(p).tolist() == g["sorted"]["ptrs"]
    uk, uc, us = S.group_reduce(k, p, vals)
    assert [host(x).tolist() for x in (uk, uc, us)] == [g["sum_count"][x] for x in ("keys", "counts", "sums")]
    tk, tn, tv, tp = S.topk(k, p, vals, 2)
    t = g["top2"]
    assert host(tv).tolist() == t["vals"] and host(tp).tolist() == t["ptrs"] and host(tn).tolist() == t["nvalid"]
    mk, mm, mu = S.median_unique(k, p, vals)
    assert host(mm).tolist() == g["median_unique"]["median"] and host(mu).tolist() == g["median_unique"]["unique"]
    L = S.sort(*S.extract(keys, 0, 4))
    R = S.sort(*S.extract(keys, 4, 4))
    jl, jr = S.join(*L, *R)
    assert host(jl).tolist() == g["join"]["ptr_l"] and host(jr).tolist() == g["join"]["ptr_r"]
    sk, sp = S.select(k, p, vals, 20, 45)
    assert host(sk).tolist() == g["select_20_45"]["keys"] and host(sp).tolist() == g["select_20_45"]["ptrs"]
