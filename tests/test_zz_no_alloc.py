"""sbh_group_reduce_noalloc: the keyed reduction for callers that cannot
allocate device memory when they call (it keeps its working memory in a fixed
device array).  Checked through the C ABI against sbh_group_reduce, which
takes caller scratch, on two calls in a row, and against the oracle's
grouping of the oracle's own sort, up to a window of more than 4096 tiles
(where the fixed array also holds the block totals of the tile scan).  This
file is collected last so that a run stopping at its first failure has run
every other test first."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    return sbh


def _run(S, sk, sp, vals, scratch_for_reference=False):
    lib = S.lib()
    n = sk.numel()
    dev = sk.device
    ok = torch.full((n,), 7, dtype=torch.uint64, device=dev)
    oc = torch.full((n,), 7, dtype=torch.uint64, device=dev)
    osum = torch.full((n,), 7, dtype=torch.uint64, device=dev)
    nk = torch.full((1,), 7, dtype=torch.uint64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    vb = 8 if vals is None else vals.element_size()
    vp = None if vals is None else vals.data_ptr()
    sump = None if vals is None else osum.data_ptr()
    args = [sk.data_ptr(), sp.data_ptr(), n, vp, vb, ok.data_ptr(), oc.data_ptr(), 8, sump, n, nk.data_ptr()]
    if scratch_for_reference:
        nb = ctypes.c_size_t(0)
        assert lib.sbh_group_reduce(*args, None, ctypes.byref(nb), stream) == 0
        buf = torch.empty(nb.value, dtype=torch.uint8, device=dev)
        rc = lib.sbh_group_reduce(*args, buf.data_ptr(), ctypes.byref(nb), stream)
    else:
        rc = lib.sbh_group_reduce_noalloc(*args, stream)
    assert rc == 0, lib.sbh_last_error()
    torch.cuda.synchronize()
    m = int(nk.item())
    return ok[:m].cpu().numpy(), oc[:m].cpu().numpy(), osum[:m].cpu().numpy()


@pytest.mark.parametrize("vbytes", [4, 8])
def test_noalloc_matches_scratch_version_twice(S, vbytes):
    # two different windows, one after the other: the second call must not
    # see anything the first one left in the shared array
    for seed, n in ((1, 1_000_003), (2, 300_000)):
        col = gen.mixed_keys(n, seed=seed)
        vals = gen.uniform(seed, 8, n, 0, 0, np.uint64 if vbytes == 8 else np.uint32)
        keys, ptrs = S.extract(torch.from_numpy(col).cuda(), 0, n)
        sk, sp = S.sort(keys, ptrs)
        d_vals = torch.from_numpy(vals).cuda()
        ref = _run(S, sk, sp, d_vals, scratch_for_reference=True)
        got = _run(S, sk, sp, d_vals)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)
        ok, oc, osum = oracle.group_sum_count(*oracle.sort(*oracle.extract(col, 0, n)), vals)
        assert np.array_equal(got[0], ok) and np.array_equal(got[1], oc) and np.array_equal(got[2], osum)


def test_noalloc_count_only_above_4096_tiles(S):
    # 20M rows = 4883 tiles of 4096: the tile scan goes through block totals,
    # which also live in the fixed array; then a small window right after
    for seed, n in ((3, 20_000_000), (4, 5_000)):
        col = gen.mixed_keys(n, seed=seed)
        keys, ptrs = S.extract(torch.from_numpy(col).cuda(), 0, n)
        sk, sp = S.sort(keys, ptrs)
        got = _run(S, sk, sp, None)
        ok, oc, _ = oracle.group_sum_count(col, np.arange(n, dtype=np.uint32), None)
        assert np.array_equal(got[0], ok) and np.array_equal(got[1], oc)
        assert int(got[1].sum()) == n


def test_noalloc_rejects_rows_beyond_its_array(S):
    lib = S.lib()
    dummy = torch.empty(1, dtype=torch.uint64, device="cuda")
    p = dummy.data_ptr()
    rc = lib.sbh_group_reduce_noalloc(p, p, (1 << 28) + 1, None, 8, p, p, 8, None, 0, p,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == S.SBH_EINVAL
    assert b"at most" in lib.sbh_last_error()
