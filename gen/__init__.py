"""Seeded synthetic inputs for the KPA grouping path.

This package is shared by the oracle tests, the GPU parity tests and the
benchmark.  It draws keys, values, timestamps and window sizes only; it holds
none of the grouping arithmetic (no sorting, grouping, joining or MLP code).

The C helper ``sbhgen.c`` is compiled on first use into ``libsbhgen.so`` next
to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbhgen.c")
_LIB = os.path.join(_HERE, "libsbhgen.so")
_lib = None

# One seed per workload: 0x5B4B0000 + workload number.
SEED_BASE = 0x5B4B0000


def build(force: bool = False) -> str:
    """Compile the generator library (gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, dbl, i32, vp = ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.sbhgen_uniform.argtypes = [u64, u64, u64, u64, u64, vp, i32, i32]
        lib.sbhgen_zipf_lognormal_mix.argtypes = [u64, u64, dbl, dbl, u64, dbl, dbl, vp, i32, i32]
        lib.sbhgen_zipf.argtypes = [u64, u64, u64, dbl, u64, vp, i32]
        lib.sbhgen_lognormal_sizes.argtypes = [u64, u64, u64, dbl, dbl, u64, u64, vp]
        lib.sbhgen_unif01.argtypes = [u64, u64, u64, vp]
        for f in (lib.sbhgen_uniform, lib.sbhgen_zipf_lognormal_mix, lib.sbhgen_zipf,
                  lib.sbhgen_lognormal_sizes, lib.sbhgen_unif01):
            f.restype = None
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- primitives
def uniform(seed: int, stream: int, n: int, lo: int, span: int, dtype=np.uint64, out=None) -> np.ndarray:
    """out[i] = lo + floor(r_i * span / 2^64); span = 0 draws the whole 64-bit range."""
    dtype = np.dtype(dtype)
    a = np.empty(n, dtype=dtype) if out is None else out
    assert a.dtype == dtype and a.size == n and a.flags.c_contiguous
    _load().sbhgen_uniform(seed, stream, n, lo, span, _ptr(a), dtype.itemsize, _threads())
    return a


def zipf(seed: int, stream: int, n: int, s: float, n_ids: int, out=None) -> np.ndarray:
    """Zipf(s) ranks in [1, n_ids] (rank r drawn with probability ~ r^-s)."""
    a = np.empty(n, dtype=np.uint64) if out is None else out
    _load().sbhgen_zipf(seed, stream, n, float(s), n_ids, _ptr(a), _threads())
    return a


def zipf_lognormal_mix(seed: int, n: int, zipf_frac: float, s: float, n_ids: int, mu: float, sigma: float,
                       out=None, hashed: bool = False) -> np.ndarray:
    """Per element: a Zipf(s) rank over [1, n_ids] with probability zipf_frac, else
    floor(exp(N(mu, sigma^2))) redrawn until it is below 2^64.  hashed: each
    Zipf rank r is replaced by mix64(r), the SplitMix64 output function (a
    bijection of 64-bit words), which keeps the multiplicities but spreads the
    ranks over the whole key range."""
    a = np.empty(n, dtype=np.uint64) if out is None else out
    _load().sbhgen_zipf_lognormal_mix(seed, n, float(zipf_frac), float(s), n_ids, float(mu), float(sigma),
                                      _ptr(a), _threads(), int(bool(hashed)))
    return a


def lognormal_sizes(seed: int, stream: int, n: int, mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    a = np.empty(n, dtype=np.uint64)
    _load().sbhgen_lognormal_sizes(seed, stream, n, float(mu), float(sigma), lo, hi, _ptr(a))
    return a


def unif01(seed: int, stream: int, n: int) -> np.ndarray:
    a = np.empty(n, dtype=np.float64)
    _load().sbhgen_unif01(seed, stream, n, _ptr(a))
    return a


from .workloads import *  # noqa: E402,F401,F403
