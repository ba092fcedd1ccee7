"""Pins of the oracle's 128-bit key sort against numpy's stable lexsort,
Python's stable sorted() on the integer values, and the invariants of a
stable sort."""
import itertools

import numpy as np

import inputs
import oracle


def wide_keys(n, seed, few=False):
    lo = inputs.keys(np.uint64, "uniform", n, seed)
    hi = inputs.keys(np.uint64, "entropy16" if few else "uniform", n, seed + 1)
    if few:
        hi = hi % np.uint64(3)
        lo = lo % np.uint64(5)
    return np.stack([lo, hi], axis=1)


def test_matches_lexsort():
    for n, few in ((0, False), (1, False), (1000, False), (50000, True), (70001, False)):
        k = wide_keys(n, 7, few)
        v = np.arange(n, dtype=np.uint64)
        sk, sv = oracle.sort_wide(k, v)
        perm = np.lexsort((k[:, 0], k[:, 1]))  # last key primary; stable
        assert np.array_equal(sv, perm.astype(np.uint64))
        assert np.array_equal(sk, k[perm])


def test_brute_force_small():
    alphabet = [(0, 0), (2**64 - 1, 0), (0, 1), (1, 1), (0, 2**63)]
    for L in range(6):
        for seq in itertools.product(range(len(alphabet)), repeat=L):
            k = np.array([alphabet[i] for i in seq], dtype=np.uint64).reshape(-1, 2)
            v = np.arange(L, dtype=np.uint64)
            _, sv = oracle.sort_wide(k, v)
            ref = sorted(range(L), key=lambda i: int(k[i, 0]) + (int(k[i, 1]) << 64))
            assert sv.tolist() == ref
