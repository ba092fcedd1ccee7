"""Pins for the oracle (plain CPU LSD radix sort of arXiv 1511.03404 Sec. 2.6).

Each check compares the oracle with something other than itself:
  * a library routine that computes the same result (numpy's stable argsort,
    Python's ``sorted``, ``np.bincount`` / ``np.cumsum`` for the per-digit
    counts and offsets);
  * a brute-force stable insertion sort over every short sequence of a small
    key alphabet;
  * invariants (non-decreasing, multiset hash, stability, bijective values);
  * closed forms of the degenerate distributions (zero, sorted, reverse
    sorted, 16-bit entropy, bucket);
  * independence of the result from the digit width r.
``tests/test_oracle_mutants.py`` plants mistakes in copies of the oracle and
checks that these pins catch each of them.
"""
import hashlib
import itertools
import json
import os

import numpy as np
import pytest

import inputs
import oracle

M64 = (1 << 64) - 1


def stable_reference(keys, begin_bit=0, end_bit=None):
    """Library stable sort by the key bits [begin_bit, end_bit)."""
    bits = keys.dtype.itemsize * 8
    end_bit = bits if end_bit is None else end_bit
    width = end_bit - begin_bit
    k = keys.astype(np.uint64)
    if width < 64:
        field = (k >> np.uint64(begin_bit)) & np.uint64((1 << width) - 1)
    else:
        field = k
    perm = np.argsort(field, kind="stable")
    return keys[perm], perm


def splitmix64(x):
    x = x.astype(np.uint64)
    with np.errstate(over="ignore"):
        x = x + np.uint64(0x9E3779B97F4A7C15)
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return x ^ (x >> np.uint64(31))


def multiset_hash(keys, vals):
    h1 = splitmix64(keys)
    rot = ((vals.astype(np.uint64) << np.uint64(17)) | (vals.astype(np.uint64) >> np.uint64(47)))
    h2 = splitmix64(keys.astype(np.uint64) ^ rot)
    with np.errstate(over="ignore"):
        return (int(h1.sum(dtype=np.uint64)), int(np.bitwise_xor.reduce(h1)),
                int(h2.sum(dtype=np.uint64)), int(np.bitwise_xor.reduce(h2)))


def check_invariants(k_in, v_in, k_out, v_out):
    """Sorted, same multiset of pairs, stable (values are indices), bijection."""
    assert np.all(k_out[1:] >= k_out[:-1])
    assert multiset_hash(k_in, v_in) == multiset_hash(k_out, v_out)
    eq = k_out[1:] == k_out[:-1]
    assert np.all(v_out[1:][eq] > v_out[:-1][eq])
    assert np.array_equal(np.sort(v_out), np.arange(len(v_out), dtype=v_out.dtype))
    assert np.array_equal(k_in[v_out.astype(np.int64)], k_out)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("dist", list(inputs.DISTS))
@pytest.mark.parametrize("n", [0, 1, 2, 31, 33, 4095, 3 * 2**14])
def test_matches_library_stable_sort(dtype, dist, n):
    k = inputs.keys(dtype, dist, n)
    v = inputs.values(dtype, n)
    sk, sv = oracle.lsd_sort(k, v)
    rk, perm = stable_reference(k)
    assert np.array_equal(sk, rk)
    assert np.array_equal(sv, perm.astype(dtype))
    if n:
        check_invariants(k, v, sk, sv)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_keys_only_matches_sort(dtype):
    k = inputs.keys(dtype, "uniform", 50000)
    sk, sv = oracle.lsd_sort(k)
    assert sv is None
    assert np.array_equal(sk, np.sort(k))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_heavy_ties_python_sorted(dtype):
    rng = inputs.mt19937(7, 4096)
    for n in range(0, 65):
        k = (rng[:n] & 0xF).astype(dtype)  # 4-bit keys: many ties
        v = np.arange(n, dtype=dtype)
        sk, sv = oracle.lsd_sort(k, v)
        order = sorted(range(n), key=lambda i: int(k[i]))  # Python's sort is stable
        assert sk.tolist() == [int(k[i]) for i in order]
        assert sv.tolist() == order


def insertion_sort_pairs(keys):
    """Textbook stable insertion sort; returns (keys, original indices)."""
    items = [(int(x), i) for i, x in enumerate(keys)]
    for j in range(1, len(items)):
        cur = items[j]
        i = j - 1
        while i >= 0 and items[i][0] > cur[0]:  # strict: equal keys stay put
            items[i + 1] = items[i]
            i -= 1
        items[i + 1] = cur
    return [a for a, _ in items], [b for _, b in items]


@pytest.mark.parametrize("dtype,alphabet", [
    (np.uint32, [0, 1, 2**31, 2**32 - 1]),
    (np.uint64, [0, 1, 2**63, 2**64 - 1]),
])
def test_brute_force_all_short_sequences(dtype, alphabet):
    for length in range(0, 7):
        for seq in itertools.product(alphabet, repeat=length):
            k = np.array(seq, dtype=dtype)
            v = np.arange(length, dtype=dtype)
            sk, sv = oracle.lsd_sort(k, v)
            bk, bv = insertion_sort_pairs(seq)
            assert sk.tolist() == bk and sv.tolist() == bv, seq


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_digit_width_independence(dtype):
    k = inputs.keys(dtype, "gaussian", 20000)
    k[::7] = k[3]  # add ties
    v = inputs.values(dtype, len(k))
    base = oracle.lsd_sort(k, v, r=8)
    for r in (1, 3, 4, 5, 7, 11, 13, 16):
        got = oracle.lsd_sort(k, v, r=r)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1]), r


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_bit_range(dtype):
    bits = np.dtype(dtype).itemsize * 8
    k = inputs.keys(dtype, "uniform", 30000)
    v = inputs.values(dtype, len(k))
    for begin, end in [(0, bits), (0, 1), (3, 17), (bits - 8, bits), (5, 5), (4, bits - 3)]:
        for r in (4, 8, 11):
            sk, sv = oracle.lsd_sort(k, v, begin_bit=begin, end_bit=end, r=r)
            rk, perm = stable_reference(k, begin, end)
            assert np.array_equal(sk, rk), (begin, end, r)
            assert np.array_equal(sv, perm.astype(dtype)), (begin, end, r)


def test_num_passes():
    assert oracle.num_passes(32, 0, 32, 8) == 4
    assert oracle.num_passes(64, 0, 64, 8) == 8
    assert oracle.num_passes(32, 0, 32, 11) == 3
    assert oracle.num_passes(32, 3, 17, 8) == 2
    assert oracle.num_passes(32, 5, 5, 8) == 0
    assert oracle.num_passes(32, 0, 33, 8) == -1
    assert oracle.num_passes(32, 0, 32, 0) == -1


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_closed_forms(dtype):
    n = 3 * 2**13
    v = inputs.values(dtype, n)
    # zero: output = input, values = identity
    z = inputs.keys(dtype, "zero", n)
    sk, sv = oracle.lsd_sort(z, v)
    assert not sk.any() and np.array_equal(sv, v)
    # sorted: values = identity
    s = inputs.keys(dtype, "sorted", n)
    sk, sv = oracle.lsd_sort(s, v)
    assert np.array_equal(sk, s) and np.array_equal(sv, v)
    # reverse sorted: reversed, except that runs of equal keys stay ascending
    d = inputs.keys(dtype, "sorted_desc", n)
    d[100:140] = d[100]  # plant a run of ties
    d[n - 5:] = d[n - 5]
    sk, sv = oracle.lsd_sort(d, v)
    assert np.array_equal(sk, d[::-1])
    run_end = np.empty(n, dtype=np.int64)  # exclusive end of each element's run
    end = n
    for j in range(n - 1, -1, -1):
        if j < n - 1 and sk[j] != sk[j + 1]:
            end = j + 1
        run_end[j] = end
    run_start = np.empty(n, dtype=np.int64)
    start = 0
    for j in range(n):
        if j > 0 and sk[j] != sk[j - 1]:
            start = j
        run_start[j] = start
    j = np.arange(n, dtype=np.int64)
    want = n - run_end + (j - run_start)
    assert np.array_equal(sv.astype(np.int64), want)
    # 16-bit entropy: output = counting sort over 2^16 bins
    e = inputs.keys(dtype, "entropy16", n)
    sk, _ = oracle.lsd_sort(e, v)
    hist = np.bincount(e.astype(np.int64), minlength=2**16)
    assert np.array_equal(sk, np.repeat(np.arange(2**16), hist).astype(dtype))
    # bucket: output chunk j holds exactly the keys of bucket j
    b = inputs.keys(dtype, "bucket", 8192 * 6)
    sk, _ = oracle.lsd_sort(b, inputs.values(dtype, len(b)))
    bits = np.dtype(dtype).itemsize * 8
    top = (sk >> np.array(bits - 13, dtype=dtype)).astype(np.int64)
    assert np.array_equal(top, np.repeat(np.arange(8192), 6))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
@pytest.mark.parametrize("r", [4, 8, 11])
def test_digit_counts_and_offsets(dtype, r):
    bits = np.dtype(dtype).itemsize * 8
    k = inputs.keys(dtype, "bucket", 40000)
    cnt = oracle.digit_counts(k, r=r)
    off = oracle.digit_offsets(cnt, r=r)
    passes = -(-bits // r)
    assert cnt.shape == (passes, 1 << r)
    for p in range(passes):
        lo = p * r
        width = min(r, bits - lo)
        field = ((k.astype(np.uint64) >> np.uint64(lo)) & np.uint64((1 << width) - 1)).astype(np.int64)
        want = np.bincount(field, minlength=1 << r)
        assert np.array_equal(cnt[p], want)
        assert np.array_equal(off[p], np.concatenate([[0], np.cumsum(want)[:-1]]))


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_segmented(dtype):
    L = inputs.segment_lengths(300, seed=3, max_log2=10)
    off = inputs.offsets_from_lengths(L)
    n = int(off[-1])
    k = inputs.keys(dtype, "gaussian", n)
    v = inputs.values(dtype, n)
    sk, sv = oracle.segmented_sort(k, v, off)
    for s in range(len(L)):
        a, b = int(off[s]), int(off[s + 1])
        rk, perm = stable_reference(k[a:b])
        assert np.array_equal(sk[a:b], rk)
        assert np.array_equal(sv[a:b], (perm + a).astype(dtype))
    # empty segments are allowed
    off2 = np.array([0, 0, 3, 3, 7], dtype=np.uint64)
    k2 = np.array([5, 4, 3, 2, 9, 1, 1], dtype=dtype)
    sk2, sv2 = oracle.segmented_sort(k2, np.arange(7, dtype=dtype), off2)
    assert sk2.tolist() == [3, 4, 5, 1, 1, 2, 9]
    assert sv2.tolist() == [2, 1, 0, 5, 6, 3, 4]


def test_stored_oracle_hashes():
    """Hashes written by tests/golden/make_golden.py catch platform drift
    (the oracle must give the same bytes on x86_64 and aarch64 hosts)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_sha256.json")
    with open(path) as f:
        golden = json.load(f)
    for key, want in list(golden.items())[::3]:
        dtype, dist, n = key.split(":")
        k = inputs.keys(np.dtype(dtype), dist, int(n))
        sk, sv = oracle.lsd_sort(k, inputs.values(np.dtype(dtype), int(n)))
        assert hashlib.sha256(sk.tobytes()).hexdigest() == want["keys"], key
        assert hashlib.sha256(sv.tobytes()).hexdigest() == want["vals"], key
