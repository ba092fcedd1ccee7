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


def sample_partition(keys: np.ndarray, vals: np.ndarray, block: int, samples: int, buckets: int,
                     lib=None):
    """Deterministic regular-sampling partition of sample sort (Sec. 2.7, the
    variant of Dehne et al.), step by step:

    1. split the input into blocks of ``block`` elements and sort each block
       stably (the LSD sort above);
    2. from each sorted block of length L take ``samples`` equidistant
       elements, at positions floor(j L / samples), j = 0 .. samples - 1
       (the block's minimum and then every (L / samples)-th element);
    3. sort all samples; the splitters are the sorted samples at positions
       floor((k + 1) M / buckets), k = 0 .. buckets - 2 (M samples in all);
    4. an element x belongs to bucket b = the number of splitters < x, so
       equal keys always share a bucket;
    5. bucket b collects, block after block, each sorted block's run of
       bucket-b elements.

    Returns ``(keys, vals, bucket_offsets[buckets + 1], splitters)``; keys and
    values are the partitioned copies (uint32)."""
    n = keys.size
    k = np.ascontiguousarray(keys).copy()
    v = np.ascontiguousarray(vals).copy()
    nblk = (n + block - 1) // block
    for i in range(nblk):
        a, b = i * block, min(n, (i + 1) * block)
        k[a:b], v[a:b] = lsd_sort(k[a:b], v[a:b], lib=lib)
    picked = []
    for i in range(nblk):
        a, b = i * block, min(n, (i + 1) * block)
        L = b - a
        for j in range(samples):
            picked.append(k[a + (j * L) // samples])
    sample = np.array(picked, dtype=keys.dtype)
    sample, _ = lsd_sort(sample, None, lib=lib)
    M = sample.size
    splitters = np.array([sample[((q + 1) * M) // buckets] for q in range(buckets - 1)],
                         dtype=keys.dtype) if M else np.zeros(0, dtype=keys.dtype)
    counts = np.zeros((buckets, nblk), dtype=np.int64)
    runs = []
    for i in range(nblk):
        a, b = i * block, min(n, (i + 1) * block)
        bucket = np.searchsorted(splitters, k[a:b], side="left")  # splitters < x
        counts[:, i] = np.bincount(bucket, minlength=buckets)
        runs.append(bucket)
    offsets = np.zeros(buckets + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(counts.sum(axis=1))
    ok = np.empty_like(k)
    ov = np.empty_like(v)
    for q in range(buckets):
        pos = int(offsets[q])
        for i in range(nblk):
            a = i * block
            sel = np.nonzero(runs[i] == q)[0]
            ok[pos:pos + sel.size] = k[a + sel]
            ov[pos:pos + sel.size] = v[a + sel]
            pos += sel.size
    return ok, ov, offsets, splitters


def sample_sort(keys: np.ndarray, vals: np.ndarray, block: int, samples: int, buckets: int,
                lib=None):
    """Sample sort: the partition above, then every bucket sorted by the LSD
    sort (the "alternative sort" of Sec. 2.7)."""
    k, v, off, _ = sample_partition(keys, vals, block, samples, buckets, lib)
    return segmented_sort(k, v, off) if lib is None else _segmented_with(lib, k, v, off)


def _segmented_with(lib, k, v, off):
    fn = lib.oracle_segmented_sort_u32 if _key_bits(k.dtype) == 32 else lib.oracle_segmented_sort_u64
    k = k.copy(); v = v.copy()
    rc = fn(_ptr(k), _ptr(v), _ptr(np.ascontiguousarray(off, dtype=np.uint64)), len(off) - 1, 0,
            _key_bits(k.dtype), 8)
    if rc != 0:
        raise ValueError(f"oracle_segmented_sort failed with code {rc}")
    return k, v


def sort_wide(keys128: np.ndarray, vals: np.ndarray | None = None, lib=None):
    """Stable ascending sort of 128-bit unsigned keys given as an (n, 2)
    uint64 array of (low word, high word): the key's value is
    low + 2^64 * high.  Written out as the LSD sort's definition over two
    64-bit digits: a stable sort by the low word, then a stable sort by the
    high word, each carrying the input positions (the LSD sort above)."""
    k = np.ascontiguousarray(keys128, dtype=np.uint64).reshape(-1, 2)
    n = k.shape[0]
    idx = np.arange(n, dtype=np.uint64)
    _, p1 = lsd_sort(k[:, 0].copy(), idx, lib=lib)          # by the low word
    p1 = p1.astype(np.int64)
    _, p2 = lsd_sort(k[p1, 1].copy(), idx.copy(), lib=lib)  # then by the high word, stably
    perm = p1[p2.astype(np.int64)]
    return k[perm].copy(), (None if vals is None else vals[perm].copy())
