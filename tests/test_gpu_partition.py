"""Partition (Table 2) on the GPU through the C ABI against the oracle:
unsorted KPAs with arbitrary pointers split by key ranges, bit-exact (keys,
pointers and part offsets), over one and two digit passes, both sort paths,
empty and single parts, repeated bounds and keys equal to a bound."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests import pins
from tests.gpu_util import cuda, host, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    return sbh


def _bounds(kind, col):
    if kind == "none":
        return np.zeros(0, np.uint64)
    if kind == "one":
        return np.array([1 << 20], np.uint64)
    if kind == "repeated":  # empty parts between equal bounds, keys equal to a bound
        return np.array([5, 5, 5, 1000, 1000, 1 << 40], np.uint64)
    if kind == "quantiles255":  # 256 parts: one pass
        return np.unique(np.sort(col)[np.linspace(0, col.size - 1, 255).astype(np.int64)]) if col.size else \
            np.arange(1, 256, dtype=np.uint64)
    if kind == "random5000":  # 5001 parts: two passes
        return np.sort(gen.mixed_keys(5000, seed=31))
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["none", "one", "repeated", "quantiles255", "random5000"])
@pytest.mark.parametrize("n", [0, 1, 4097, 1_000_003])
def test_partition_parity(S, kind, n):
    col = gen.mixed_keys(n, seed=30)
    ptrs = gen.uniform(30, 5, n, 0, 1 << 32, np.uint32)  # any pointers, repeats allowed
    bounds = _bounds(kind, col)
    ok, op, off = oracle.partition(col, ptrs, bounds)
    gk, gp, goff = S.partition(cuda(col), cuda(ptrs), cuda(bounds))
    assert same(gk, ok) and same(gp, op) and same(goff, off)
    assert same(cuda(col), col)  # the input is not written


def test_partition_chunked_path_in_place(S):
    # above the sort's chunked threshold, in place, 257 parts (two passes
    # whose upper digit takes two values)
    n = (1 << 23) + 11
    col = gen.mixed_keys(n, seed=32)
    ptrs = np.arange(n, dtype=np.uint32)
    bounds = np.sort(gen.mixed_keys(256, seed=33))
    k, p = cuda(col), cuda(ptrs)
    off = torch.empty(bounds.size + 2, dtype=torch.uint64, device="cuda")
    S.sbh_kpa_partition(k, p, cuda(bounds), k, p, off)
    ok, op, oo = oracle.partition(col, ptrs, bounds)
    assert same(k, ok) and same(p, op) and same(off, oo)


def test_partition_timestamps_into_windows(S):
    # Sec. 4.2 "Windowing": Partition on the timestamp column with the window
    # length as the range; out-of-order timestamps (5% up to 100 ms late)
    n = 2_000_000
    ts = np.arange(n, dtype=np.uint64) * np.uint64(1000)
    late = gen.uniform(34, 1, n, 0, 20, np.uint64) == 0
    ts[late] -= np.minimum(ts[late], gen.uniform(34, 2, int(late.sum()), 0, 100_000_000, np.uint64))
    bounds = np.arange(1, 8, dtype=np.uint64) * np.uint64(250_000_000)
    ptrs = np.arange(n, dtype=np.uint32)
    gk, gp, goff = S.partition(cuda(ts), cuda(ptrs), cuda(bounds))
    pins.check_partition(ts, ptrs, bounds, host(gk), host(gp), host(goff))
