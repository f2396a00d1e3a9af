"""The C ABI library loads on a machine without a GPU, exports every entry
point include/sbh.h declares, and rejects bad arguments on the host before
any launch (no call below reaches the GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1901_01328_b300 import build
    build.build()
    from paper_1901_01328_b300 import sbh
    return sbh


def _declared():
    text = open(os.path.join(ROOT, "include", "sbh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sbh_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert "sbh_kpa_sort" in names and "sbh_join" in names
    lib = ctypes.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.EXPORTED)


def test_version_and_error_text(L):
    assert "sm_103a" in L.version()


def test_scratch_size_queries_need_no_gpu(L):
    lib = L.lib()
    nb = ctypes.c_size_t(0)
    assert lib.sbh_kpa_sort(None, None, None, None, 256_000_000, None, ctypes.byref(nb), None) == 0
    # ping-pong copy (12 B per pair), the next pass's digit byte and the chunk tables
    assert 256_000_000 * 13 <= nb.value < 256_000_000 * 13 + 200_000_000
    for fn, args in ((lib.sbh_group_reduce, (None, None, 10_000, None, 8, None, None, 8, None, 0, None)),
                     (lib.sbh_topk, (None, None, 10_000, None, 8, 3, None, None, None, None, 0, None)),
                     (lib.sbh_join, (None, None, 10_000, None, None, 10, None, None, 0, None))):
        nb = ctypes.c_size_t(0)
        assert fn(*args, None, ctypes.byref(nb), None) == 0 and nb.value > 0


def test_host_side_argument_errors(L):
    lib = L.lib()
    nb = ctypes.c_size_t(0)
    assert lib.sbh_kpa_sort(None, None, None, None, 1 << 33, None, ctypes.byref(nb), None) == L.SBH_EINVAL
    assert b"2^32" in lib.sbh_last_error()
    assert lib.sbh_topk(None, None, 10, None, 8, 0, None, None, None, None, 0, None, None, ctypes.byref(nb),
                        None) == L.SBH_EINVAL
    assert lib.sbh_topk(None, None, 10, None, 8, 9, None, None, None, None, 0, None, None, ctypes.byref(nb),
                        None) == L.SBH_EINVAL
    # scratch present but too small
    fake = ctypes.c_void_p(1 << 20)
    small = ctypes.c_size_t(16)
    assert lib.sbh_kpa_sort(fake, fake, fake, fake, 100_000, fake, ctypes.byref(small), None) == L.SBH_ENOSPACE
    # scratch_bytes missing
    assert lib.sbh_group_reduce(None, None, 10, None, 8, None, None, 8, None, 0, None, None, None, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract(fake, (1 << 32) - 5, 10, fake, fake, None, None, 0, None) == L.SBH_EINVAL
    # a key column sorted without an Extract (ptrs_in NULL) cannot be sorted in place
    need = ctypes.c_size_t(0)
    assert lib.sbh_kpa_sort(None, None, None, None, 100_000, None, ctypes.byref(need), None) == L.SBH_OK
    assert lib.sbh_kpa_sort(fake, None, fake, fake, 100_000, fake, ctypes.byref(need), None) == L.SBH_EINVAL
    # Extract: keys and ptrs both or neither; samples only, without the OR
    assert lib.sbh_kpa_extract(fake, 0, 10, None, fake, None, None, 0, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract(fake, 0, 10, None, None, None, None, 0, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract(fake, 0, 10, None, None, fake, fake, 2, None) == L.SBH_EINVAL
    assert lib.sbh_window_ranges(fake, 3, 10, fake, 5, 2, fake, fake, None) == L.SBH_EINVAL


def test_window_bits_and_batched_extract_arguments(L):
    assert [L.window_bits(x) for x in (1, 2, 3, 4096, 4097)] == [1, 2, 2, 13, 13]
    lib = L.lib()
    fake = ctypes.c_void_p(1 << 20)
    assert lib.sbh_kpa_extract_windows(fake, fake, 0, 0, 10, fake, fake, None, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract_windows(fake, fake, 4, (1 << 32) - 5, 10, fake, fake, None, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract_windows(None, fake, 4, 0, 10, fake, fake, None, None) == L.SBH_EINVAL
    assert lib.sbh_kpa_extract_windows(None, None, 4, 0, 0, None, None, None, None) == L.SBH_OK


def test_knobs_set_and_get_without_a_gpu(L):
    assert L.get_knob(L.KNOB_SORT_CHUNKED_MIN) == 1 << 23
    assert L.get_knob(L.KNOB_MERGE_SEARCH_MIN_TILES) == 2047
    L.set_knob(L.KNOB_SORT_CHUNKED_MIN, 12345)
    assert L.get_knob(L.KNOB_SORT_CHUNKED_MIN) == 12345
    L.set_knob(L.KNOB_SORT_CHUNKED_MIN, 1 << 23)
    lib = L.lib()
    assert lib.sbh_set_knob(7, 1) == L.SBH_EINVAL and lib.sbh_get_knob(7) == 0
    # the sort's scratch depends on the path the knob picks
    nb_small, nb_large = ctypes.c_size_t(0), ctypes.c_size_t(0)
    L.set_knob(L.KNOB_SORT_CHUNKED_MIN, 1 << 40)   # onesweep: look-back records
    assert lib.sbh_kpa_sort(None, None, None, None, 1 << 22, None, ctypes.byref(nb_small), None) == 0
    L.set_knob(L.KNOB_SORT_CHUNKED_MIN, 0)         # chunked: chunk tables
    assert lib.sbh_kpa_sort(None, None, None, None, 1 << 22, None, ctypes.byref(nb_large), None) == 0
    L.set_knob(L.KNOB_SORT_CHUNKED_MIN, 1 << 23)
    assert nb_small.value != nb_large.value


def test_binding_constants_match_the_header(L):
    S = L
    text = open(os.path.join(ROOT, "include", "sbh.h")).read()
    defs = {m.group(1): int(m.group(2), 0) for m in re.finditer(r"#define (SBH_\w+) (0x[0-9A-Fa-f]+|\d+)", text)}
    assert defs["SBH_MLP_PARAMS"] == S.MLP_PARAMS
    assert defs["SBH_LEARNED_MODEL_BYTES"] == S.LEARNED_MODEL_BYTES
    assert defs["SBH_LEARNED_CAPACITY"] == S.LEARNED_CAPACITY
    assert defs["SBH_LEARNED_MAX_HEAVY"] == S.LEARNED_MAX_HEAVY
    assert defs["SBH_LEARNED_STATS"] == len(S.LEARNED_STATS)
    assert defs["SBH_TOPK_MAX_K"] == S.TOPK_MAX_K
    assert (defs["SBH_OK"], defs["SBH_EINVAL"], defs["SBH_ENOSPACE"], defs["SBH_ETIMEOUT"], defs["SBH_ECUDA"]) == (
        S.SBH_OK, S.SBH_EINVAL, S.SBH_ENOSPACE, S.SBH_ETIMEOUT, S.SBH_ECUDA)
    assert (defs["SBH_KNOB_SORT_CHUNKED_MIN"], defs["SBH_KNOB_MERGE_SEARCH_MIN_TILES"]) == (
        S.KNOB_SORT_CHUNKED_MIN, S.KNOB_MERGE_SEARCH_MIN_TILES)
