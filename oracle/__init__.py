"""Oracle for the LSD radix sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
(and ``--impl reference``) leg may import this package.  The library under
``paper_1511_03404_gb300/`` never imports it, and the two share no code.

``rs_oracle.c`` is a plain single-threaded CPU LSD counting sort written from
arXiv 1511.03404 Sec. 2.6 (digits of r bits, least significant first, one
stable counting sort per digit).  These wrappers take numpy arrays, sort
copies and return them; nothing here touches a GPU.

Pins (what checks the oracle against something other than itself) are in
``tests/test_oracle.py`` and ``tests/test_oracle_mutants.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "rs_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librs_oracle.so")

_lock = threading.Lock()
_lib = None


def compile_library(src: str, out: str, extra_flags=()) -> str:
    """Compile a C oracle source into a shared library with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)):
        return _LIB_PATH
    return compile_library(SOURCE, _LIB_PATH)


def bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.oracle_num_passes.argtypes = [i32, i32, i32, i32]
    lib.oracle_lsd_sort_u32.argtypes = [vp, vp, u64, i32, i32, i32]
    lib.oracle_lsd_sort_u64.argtypes = [vp, vp, u64, i32, i32, i32]
    lib.oracle_digit_counts_u64.argtypes = [vp, u64, i32, i32, i32, i32, vp]
    lib.oracle_digit_offsets.argtypes = [vp, i32, i32, vp]
    lib.oracle_segmented_sort_u32.argtypes = [vp, vp, vp, u64, i32, i32, i32]
    lib.oracle_segmented_sort_u64.argtypes = [vp, vp, vp, u64, i32, i32, i32]
    lib.oracle_order_keys_u32.argtypes = [vp, vp, u64, i32, i32]
    lib.oracle_order_keys_u64.argtypes = [vp, vp, u64, i32, i32]
    for name in ("oracle_num_passes", "oracle_lsd_sort_u32", "oracle_lsd_sort_u64",
                 "oracle_digit_counts_u64", "oracle_digit_offsets",
                 "oracle_segmented_sort_u32", "oracle_segmented_sort_u64",
                 "oracle_order_keys_u32", "oracle_order_keys_u64"):
        getattr(lib, name).restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _key_bits(dtype) -> int:
    dtype = np.dtype(dtype)
    if dtype == np.uint32:
        return 32
    if dtype == np.uint64:
        return 64
    raise TypeError(f"oracle sorts uint32 or uint64 keys, got {dtype}")


def num_passes(key_bits: int, begin_bit: int, end_bit: int, r: int) -> int:
    return _load().oracle_num_passes(key_bits, begin_bit, end_bit, r)


def lsd_sort(keys: np.ndarray, vals: np.ndarray | None = None, begin_bit: int = 0,
             end_bit: int | None = None, r: int = 8, lib=None):
    """Stable LSD radix sort of copies of ``keys`` (and ``vals``).

    Returns ``(sorted_keys, sorted_vals_or_None)``.
    """
    lib = lib or _load()
    bits = _key_bits(keys.dtype)
    end_bit = bits if end_bit is None else end_bit
    k = np.ascontiguousarray(keys).copy()
    v = None
    if vals is not None:
        if vals.dtype != keys.dtype or vals.shape != keys.shape:
            raise TypeError("values must have the keys' dtype and length")
        v = np.ascontiguousarray(vals).copy()
    fn = lib.oracle_lsd_sort_u32 if bits == 32 else lib.oracle_lsd_sort_u64
    rc = fn(_ptr(k), _ptr(v), k.size, begin_bit, end_bit, r)
    if rc != 0:
        raise ValueError(f"oracle_lsd_sort failed with code {rc}")
    return k, v


KEY_UNSIGNED, KEY_SIGNED, KEY_FLOAT = 0, 1, 2


def order_keys(keys: np.ndarray, kind: int = KEY_UNSIGNED, descending: bool = False, lib=None):
    """The unsigned order key of every bit pattern in ``keys`` (uint32 or
    uint64 views of the caller's keys): its ascending order is the order
    asked for (unsigned, two's-complement signed or IEEE-754 total order;
    reversed when descending)."""
    bits = _key_bits(keys.dtype)
    k = np.ascontiguousarray(keys)
    out = np.empty_like(k)
    lib = lib or _load()
    fn = lib.oracle_order_keys_u32 if bits == 32 else lib.oracle_order_keys_u64
    rc = fn(_ptr(k), _ptr(out), k.size, int(kind), int(bool(descending)))
    if rc != 0:
        raise ValueError(f"oracle_order_keys failed with code {rc}")
    return out


def ordered_sort(keys: np.ndarray, vals: np.ndarray | None = None, kind: int = KEY_UNSIGNED,
                 descending: bool = False, begin_bit: int = 0, end_bit: int | None = None,
                 r: int = 8, lib=None):
    """Stable sort of the bit patterns ``keys`` (uint32 / uint64 views) in the
    order of ``kind`` / ``descending``: the LSD sort orders the order keys
    (over their bits [begin_bit, end_bit)) and carries each element's input
    position, which then permutes the original keys and values."""
    n = keys.size
    m = order_keys(keys, kind, descending, lib)
    idx = np.arange(n, dtype=keys.dtype)
    _, perm = lsd_sort(m, idx, begin_bit, end_bit, r, lib)
    perm = perm.astype(np.int64)
    return keys[perm], (None if vals is None else vals[perm])


def digit_counts(keys: np.ndarray, begin_bit: int = 0, end_bit: int | None = None,
                 r: int = 8) -> np.ndarray:
    """Per-pass digit histograms, shape (passes, 2^r), dtype uint64."""
    bits = _key_bits(keys.dtype)
    end_bit = bits if end_bit is None else end_bit
    lib = _load()
    p = lib.oracle_num_passes(bits, begin_bit, end_bit, r)
    if p < 0:
        raise ValueError("bad digit layout")
    k = np.ascontiguousarray(keys).astype(np.uint64)
    out = np.zeros((max(p, 0), 1 << r), dtype=np.uint64)
    rc = lib.oracle_digit_counts_u64(_ptr(k), k.size, bits, begin_bit, end_bit, r, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_digit_counts failed with code {rc}")
    return out


def digit_offsets(counts: np.ndarray, r: int = 8) -> np.ndarray:
    """Exclusive prefix of each row of ``counts`` (the per-pass digit offsets)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.zeros_like(c)
    rc = _load().oracle_digit_offsets(_ptr(c), c.shape[0], r, _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_digit_offsets failed with code {rc}")
    return out


def segmented_sort(keys: np.ndarray, vals: np.ndarray | None, offsets: np.ndarray,
                   begin_bit: int = 0, end_bit: int | None = None, r: int = 8):
    """The sort applied to each segment [offsets[s], offsets[s+1]) independently."""
    lib = _load()
    bits = _key_bits(keys.dtype)
    end_bit = bits if end_bit is None else end_bit
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    fn = lib.oracle_segmented_sort_u32 if bits == 32 else lib.oracle_segmented_sort_u64
    rc = fn(_ptr(k), _ptr(v), _ptr(off), len(off) - 1, begin_bit, end_bit, r)
    if rc != 0:
        raise ValueError(f"oracle_segmented_sort failed with code {rc}")
    return k, v
