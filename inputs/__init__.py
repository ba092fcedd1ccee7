"""Seeded synthetic inputs for the sort workloads (arXiv 1511.03404, Sec. 3-4).

The comparison study sorts six input distributions (uniform, Gaussian, zero,
bucket, sorted, sorted descending) of 32- and 64-bit keys and key-value pairs
drawn from a Mersenne Twister (Sec. 3).  The generators live in ``gen.cpp``
(raw ``std::mt19937`` / ``std::mt19937_64`` outputs, whose values the C++
standard fixes) and are reached here through ctypes; the arrays come back as
numpy arrays in host memory.

This module is the one piece shared by the tests, the oracle's checks and the
benchmark.  It contains no part of the sort itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librsgen.so")

DISTS = {
    "uniform": 0,
    "gaussian": 1,
    "zero": 2,
    "sorted": 3,
    "sorted_desc": 4,
    "bucket": 5,
    "entropy16": 6,
}
# The six distributions named in Sec. 4; "entropy16" is an extra workload whose
# keys carry only 16 random low bits (it exercises digit passes that can be
# skipped).
PAPER_DISTS = ("uniform", "gaussian", "zero", "bucket", "sorted", "sorted_desc")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gen.cpp`` into ``_build/librsgen.so`` (g++, host code only)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            vp = ctypes.c_void_p
            lib.rsgen_mt19937.argtypes = [u32, u64, vp]
            lib.rsgen_mt19937_64.argtypes = [u64, u64, vp]
            lib.rsgen_keys_u32.argtypes = [i32, u64, u32, vp]
            lib.rsgen_keys_u64.argtypes = [i32, u64, u64, vp]
            lib.rsgen_segment_lengths.argtypes = [u64, u32, u32, vp]
            for f in (lib.rsgen_mt19937, lib.rsgen_mt19937_64, lib.rsgen_keys_u32,
                      lib.rsgen_keys_u64, lib.rsgen_segment_lengths):
                f.restype = i32
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


def mt19937(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of ``std::mt19937(seed)``."""
    out = np.empty(count, dtype=np.uint32)
    _check(_load().rsgen_mt19937(seed, count, out.ctypes.data), "mt19937")
    return out


def mt19937_64(seed: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of ``std::mt19937_64(seed)``."""
    out = np.empty(count, dtype=np.uint64)
    _check(_load().rsgen_mt19937_64(seed, count, out.ctypes.data), "mt19937_64")
    return out


def keys(dtype, dist: str, n: int, seed: int = 1) -> np.ndarray:
    """``n`` keys of ``dtype`` (np.uint32 or np.uint64) from distribution ``dist``."""
    dtype = np.dtype(dtype)
    code = DISTS[dist]
    out = np.empty(n, dtype=dtype)
    lib = _load()
    if dtype == np.uint32:
        rc = lib.rsgen_keys_u32(code, n, seed, out.ctypes.data)
    elif dtype == np.uint64:
        rc = lib.rsgen_keys_u64(code, n, seed, out.ctypes.data)
    else:
        raise TypeError(f"unsupported key dtype {dtype}")
    _check(rc, f"keys({dtype}, {dist}, {n})")
    return out


def float_keys(dtype, n: int, seed: int = 1) -> np.ndarray:
    """``n`` IEEE-754 keys as bit patterns (np.uint32 for binary32, np.uint64
    for binary64): mostly finite values of both signs spread over a wide
    range of exponents, about 1/8 special patterns (+-0, +-inf, quiet and
    signalling NaNs of both signs, subnormals, the largest finite values),
    and many repeated values (every fourth key repeats an earlier one)."""
    dtype = np.dtype(dtype)
    if dtype == np.uint32:
        raw = mt19937(seed, 4 * n).astype(np.uint64)
        ebits, fbits, bias = 8, 23, 127
    elif dtype == np.uint64:
        raw = mt19937_64(seed, 4 * n)
        ebits, fbits, bias = 11, 52, 1023
    else:
        raise TypeError(f"unsupported key dtype {dtype}")
    w = ebits + fbits + 1
    a, b, c, d = raw[0::4], raw[1::4], raw[2::4], raw[3::4]
    sign = (a & 1) << (w - 1)
    exp = (bias - 40 + (a >> 1) % 81) << fbits          # 2^-40 .. 2^40
    frac = b & ((1 << fbits) - 1)
    out = sign | exp | frac
    emax = ((1 << ebits) - 1) << fbits
    specials = np.array([0, 1 << (w - 1), emax, emax | (1 << (w - 1)), emax | 1,
                         emax | (1 << (fbits - 1)), emax | (1 << (fbits - 1)) | (1 << (w - 1)),
                         emax | ((1 << fbits) - 1) | (1 << (w - 1)), 1, (1 << (w - 1)) | 3,
                         emax - 1, (emax - 1) | (1 << (w - 1))], dtype=np.uint64)
    pick = (c % 8) == 0
    out[pick] = specials[(c[pick] >> 3) % len(specials)]
    rep = (d % 4) == 0
    src = (d >> 2) % np.maximum(np.arange(n, dtype=np.uint64), 1)
    out[rep] = out[src[rep].astype(np.int64)]
    return out.astype(dtype)


def values(dtype, n: int) -> np.ndarray:
    """Values of a key-value workload: value[i] = i, the original index."""
    return np.arange(n, dtype=np.dtype(dtype))


def segment_lengths(nseg: int, seed: int = 1, max_log2: int = 20) -> np.ndarray:
    """Log-uniform segment lengths in [1, 2^max_log2] (batched workload)."""
    out = np.empty(nseg, dtype=np.uint64)
    _check(_load().rsgen_segment_lengths(nseg, seed, max_log2, out.ctypes.data),
           "segment_lengths")
    return out


def scale_lengths(lengths: np.ndarray, total: int) -> np.ndarray:
    """Scale lengths so that they add up to about ``total`` (floor, minimum 1)."""
    s = int(lengths.sum())
    scaled = np.floor(lengths.astype(np.float64) * (total / s)).astype(np.uint64)
    return np.maximum(scaled, 1).astype(np.uint64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    """Segment offsets (n_seg + 1 entries, first 0) for the given lengths."""
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths.astype(np.uint64), out=off[1:])
    return off
