"""Pins of the oracle's key orders beyond unsigned keys (signed integers,
IEEE-754 floats, descending order), each checked against something other
than the oracle: numpy's stable sort of the typed values, Python's stable
``sorted`` under IEEE-754 totalOrder written out from the encoding (sign,
exponent, fraction), and the special cases the standard fixes.

The pin functions take the oracle library so that the mutant tests can run
them against planted mistakes.
"""
import itertools

import numpy as np
import pytest

import inputs
import oracle

U = {4: np.uint32, 8: np.uint64}
S = {4: np.int32, 8: np.int64}
F = {4: np.float32, 8: np.float64}
FIELDS = {4: (8, 23), 8: (11, 52)}  # exponent, fraction bits


def total_order_key(bits: int, nbytes: int):
    """IEEE-754 totalOrder as a sort key: every negative pattern below every
    positive one; positives by (exponent, fraction) ascending, negatives by
    (exponent, fraction) descending.  NaNs land at the ends by sign."""
    ebits, fbits = FIELDS[nbytes]
    sign = bits >> (ebits + fbits)
    exp = (bits >> fbits) & ((1 << ebits) - 1)
    frac = bits & ((1 << fbits) - 1)
    return (1, exp, frac) if sign == 0 else (0, -exp, -frac)


def pin_signed(lib=None):
    for nb in (4, 8):
        info = np.iinfo(S[nb])
        k = inputs.keys(U[nb], "uniform", 5000).view(S[nb]).copy()
        k[::7] = k[3]  # ties
        k[:6] = [info.min, -1, 0, 1, info.max, info.min + 1]
        small = (inputs.keys(U[nb], "entropy16", 3000).astype(np.int64) % 201 - 100).astype(S[nb])
        for arr in (k, small, k[:1], k[:0]):
            v = np.arange(arr.size, dtype=U[nb])
            sk, sv = oracle.ordered_sort(arr.view(U[nb]), v, kind=oracle.KEY_SIGNED, lib=lib)
            perm = np.argsort(arr, kind="stable")
            assert np.array_equal(sk.view(S[nb]), arr[perm])
            assert np.array_equal(sv, perm.astype(U[nb]))


def pin_float_numpy(lib=None):
    # numpy orders floats like totalOrder apart from NaNs and the sign of
    # zero: keep neither here
    for nb in (4, 8):
        bits = inputs.float_keys(U[nb], 6000, seed=5)
        f = bits.view(F[nb]).copy()
        f[np.isnan(f) | ((f == 0) & np.signbit(f))] = 1.0
        v = np.arange(f.size, dtype=U[nb])
        sk, sv = oracle.ordered_sort(f.view(U[nb]), v, kind=oracle.KEY_FLOAT, lib=lib)
        perm = np.argsort(f, kind="stable")
        assert np.array_equal(sk, f[perm].view(U[nb]))
        assert np.array_equal(sv, perm.astype(U[nb]))


def special_patterns(nb):
    ebits, fbits = FIELDS[nb]
    w = 8 * nb
    top = 1 << (w - 1)
    emax = ((1 << ebits) - 1) << fbits
    one = ((1 << (ebits - 1)) - 1) << fbits
    return [0, top, emax, emax | top, emax | 1, emax | (1 << (fbits - 1)) | top, 1, top | 1,
            one, one | top, emax - 1, (emax - 1) | top]


def pin_float_total_order(lib=None):
    for nb in (4, 8):
        pats = special_patterns(nb)
        rng = np.random.default_rng(7)
        cases = [list(c) for c in itertools.permutations(pats[:6], 4)][::7]
        cases += [list(rng.choice(pats, size=int(rng.integers(1, 40)))) for _ in range(60)]
        for case in cases:
            k = np.array(case, dtype=U[nb])
            v = np.arange(k.size, dtype=U[nb])
            sk, sv = oracle.ordered_sort(k, v, kind=oracle.KEY_FLOAT, lib=lib)
            perm = sorted(range(k.size), key=lambda i: total_order_key(int(k[i]), nb))
            assert sv.tolist() == perm and sk.tolist() == k[perm].tolist()
        # the facts the order fixes, on one array
        f = np.array([np.nan, 1.0, -0.0, np.inf, 0.0, -np.inf, -np.nan, -1.0], dtype=F[nb])
        sk, _ = oracle.ordered_sort(f.view(U[nb]), kind=oracle.KEY_FLOAT, lib=lib)
        s = sk.view(F[nb])
        assert np.isnan(s[0]) and np.signbit(s[0]) and np.isnan(s[-1]) and not np.signbit(s[-1])
        assert s[1] == -np.inf and s[-2] == np.inf
        z = np.nonzero(s == 0)[0]
        assert np.signbit(s[z[0]]) and not np.signbit(s[z[1]])


def pin_descending(lib=None):
    for nb in (4, 8):
        u = inputs.keys(U[nb], "entropy16", 4000) % np.array(50, dtype=U[nb])  # many ties
        cases = {oracle.KEY_UNSIGNED: (u, lambda x: -int(x)),
                 oracle.KEY_SIGNED: (u.view(S[nb]) - 25, lambda x: -int(x)),
                 oracle.KEY_FLOAT: (inputs.float_keys(U[nb], 4000, seed=9), None)}
        for kind, (arr, neg) in cases.items():
            bits = arr.view(U[nb])
            v = np.arange(bits.size, dtype=U[nb])
            sk, sv = oracle.ordered_sort(bits, v, kind=kind, descending=True, lib=lib)
            if kind == oracle.KEY_FLOAT:
                key = lambda i: tuple(-x for x in total_order_key(int(bits[i]), nb))
            else:
                typed = arr
                key = lambda i: neg(typed[i])
            perm = sorted(range(bits.size), key=key)  # stable: ties keep input order
            assert sv.tolist() == perm and np.array_equal(sk, bits[perm])


def pin_bit_range(lib=None):
    # a bit range applies to the order key: descending on bits [8, 24) of
    # unsigned keys is the stable descending sort of that field
    k = inputs.keys(np.uint32, "uniform", 3000)
    v = np.arange(k.size, dtype=np.uint32)
    sk, sv = oracle.ordered_sort(k, v, descending=True, begin_bit=8, end_bit=24, lib=lib)
    field = ((k >> 8) & 0xFFFF).astype(np.int64)
    perm = sorted(range(k.size), key=lambda i: -field[i])
    assert sv.tolist() == perm


PINS = {"signed": pin_signed, "float_numpy": pin_float_numpy,
        "float_total_order": pin_float_total_order, "descending": pin_descending,
        "bit_range": pin_bit_range}


@pytest.mark.parametrize("name", sorted(PINS))
def test_key_order_pin(name):
    PINS[name]()


def test_unsigned_order_key_is_identity():
    k = inputs.keys(np.uint64, "uniform", 1000)
    assert np.array_equal(oracle.order_keys(k), k)
    assert np.array_equal(oracle.order_keys(k, descending=True), ~k)
