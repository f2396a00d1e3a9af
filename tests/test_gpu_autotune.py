"""The autotuner on the GPU: it times both sort paths and both merge-cut
searches, sets the knobs to values drawn from what it measured, and the
results stay bit-identical to the oracle whichever path a knob selects."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests.gpu_util import cuda, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import autotune, sbh
    yield autotune
    sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, 1 << 23)
    sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, 2047)
    sbh.set_knob(sbh.KNOB_SCATTER_GEOM, 0)


def test_tuning_sets_knobs_from_measurements(A, tmp_path):
    from paper_1901_01328_b300 import sbh
    r = A.tune_sort_threshold(sizes=(1 << 18, 1 << 20, 1 << 21))
    assert r["value"] in (1 << 18, 1 << 20, 1 << 21, 1 << 22)
    assert sbh.get_knob(sbh.KNOB_SORT_CHUNKED_MIN) == r["value"]
    assert all(set(v) == {"onesweep", "chunked"} and min(v.values()) > 0 for v in r["timings_ms"].values())
    m = A.tune_merge_search(totals=(1 << 20, 1 << 22))
    assert sbh.get_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES) == m["value"]
    # a cache file round trip
    cache = str(tmp_path / "knobs.json")
    saved = A.autotune(cache, quick=True)
    sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, 7)
    assert A.autotune(cache) == saved and sbh.get_knob(sbh.KNOB_SORT_CHUNKED_MIN) == saved["SBH_KNOB_SORT_CHUNKED_MIN"]


@pytest.mark.parametrize("thr", [0, 1 << 40])
def test_both_sort_paths_and_both_merge_searches_are_exact(A, thr):
    from paper_1901_01328_b300 import sbh
    sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, thr)
    sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, thr)
    try:
        n = 1_000_003
        col = gen.mixed_keys(n, seed=31)
        sk, sp = sbh.sort(*sbh.extract(cuda(col), 0, n))
        ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
        assert same(sk, ok) and same(sp, op)
        half = n // 2
        a = sbh.sort(*sbh.extract(cuda(col), 0, half))
        b = sbh.sort(*sbh.extract(cuda(col), half, n - half))
        mk, mp = sbh.merge([a, b])
        assert same(mk, ok) and same(mp, op)
    finally:
        sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, 1 << 23)
        sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, 2047)


def test_batched_schedule_choice(A):
    b = gen.batched_windows(32, 8, size_hi=50_000)
    choice, t = A.batched_schedule(cuda(b["keys"]), cuda(b["vals"]), b["offsets"], sample_windows=16)
    assert choice in ("batched", "loop") and t[choice] == min(t.values())


def test_scatter_geometry_tuning_and_every_geometry_is_exact(A):
    from paper_1901_01328_b300 import sbh
    r = A.tune_scatter_geometry(sizes=(1 << 22,))
    assert r["value"] in sbh.SCATTER_GEOMS and sbh.get_knob(sbh.KNOB_SCATTER_GEOM) == r["value"]
    assert r["timings_ms"][1 << 22][r["value"]] == min(r["timings_ms"][1 << 22].values())
    with pytest.raises(sbh.SbhError):
        sbh.set_knob(sbh.KNOB_SCATTER_GEOM, 3)
    old = sbh.get_knob(sbh.KNOB_SORT_CHUNKED_MIN)
    sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, 1 << 20)  # the chunked passes from 2^20 pairs
    try:
        n = (1 << 21) + 4097  # ragged last tile in every geometry
        for kind, col in (("mixed", gen.mixed_keys(n, seed=33)), ("uniform20", gen.uniform(33, 1, n, 0, 1 << 20,
                                                                                              np.uint64))):
            ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
            for geom in sbh.SCATTER_GEOMS:
                sbh.set_knob(sbh.KNOB_SCATTER_GEOM, geom)
                sk, sp = sbh.sort(*sbh.extract(cuda(col), 0, n))
                assert same(sk, ok) and same(sp, op), (kind, geom)
            # in place
            sbh.set_knob(sbh.KNOB_SCATTER_GEOM, 2)
            k, p = sbh.extract(cuda(col), 0, n)
            sbh.sort(k, p, out=(k, p))
            assert same(k, ok) and same(p, op)
    finally:
        sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, old)
        sbh.set_knob(sbh.KNOB_SCATTER_GEOM, 0)
