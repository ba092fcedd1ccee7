"""Pins of the oracle's sample-sort partition (Sec. 2.7, regular sampling
after Dehne et al.) against what the definition fixes, independent of how
the oracle computes it:

- every bucket q holds exactly the keys x with s[q-1] < x <= s[q];
- the partition is a permutation, and inside a bucket the elements come
  block by block, each block's run in stable sorted order;
- the splitters are the order statistics of the regular sample, computed
  here with numpy's sort and partition (library routines);
- regular sampling bounds every bucket of distinct keys by 2n/B + one block;
- sample sort (partition, then each bucket sorted) equals the stable sort.
"""
import numpy as np
import pytest

import inputs
import oracle

BLOCK = 4096


def check_partition(k, v, samples, buckets):
    pk, pv, off, spl = oracle.sample_partition(k, v, BLOCK, samples, buckets)
    n = k.size
    off = off.astype(np.int64)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert np.array_equal(np.sort(pk), np.sort(k)) and np.array_equal(np.sort(pv), v)
    assert np.array_equal(pk, k[pv.astype(np.int64)])  # keys travel with their values
    lo = np.concatenate([[None], spl])
    for q in range(buckets):
        x = pk[off[q]:off[q + 1]].astype(np.int64)
        idx = pv[off[q]:off[q + 1]].astype(np.int64)
        if q > 0:
            assert np.all(x > int(lo[q]))
        if q < buckets - 1:
            assert np.all(x <= int(spl[q]))
        blk = idx // BLOCK
        assert np.all(np.diff(blk) >= 0)  # block after block
        for b in np.unique(blk):
            r = blk == b
            xs, ids = x[r], idx[r]
            assert np.all(np.diff(xs) >= 0)
            assert np.all((np.diff(xs) > 0) | (np.diff(ids) > 0))  # stable
    # splitters: order statistics of the regular sample
    nblk = (n + BLOCK - 1) // BLOCK
    picked = []
    for i in range(nblk):
        blk_sorted = np.sort(k[i * BLOCK:(i + 1) * BLOCK], kind="stable")
        L = blk_sorted.size
        picked.extend(blk_sorted[[j * L // samples for j in range(samples)]])
    sample = np.array(picked, dtype=k.dtype)
    M = sample.size
    for q in range(buckets - 1):
        r = (q + 1) * M // buckets
        assert spl[q] == np.partition(sample, r)[r]
    return pk, pv, off, spl


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "bucket", "sorted", "sorted_desc",
                                  "zero", "entropy16"])
def test_partition_definition(dist):
    for n, s, b in ((1, 4, 2), (4095, 8, 8), (40000, 64, 64), (100003, 32, 256)):
        k = inputs.keys(np.uint32, dist, n)
        check_partition(k, inputs.values(np.uint32, n), s, b)


def test_regular_sampling_bound():
    # distinct keys: no bucket exceeds 2n/B + one block
    n, s, b = 200000, 64, 64
    k = np.random.default_rng(3).permutation(n).astype(np.uint32) * np.uint32(7919)
    _, _, off, _ = check_partition(k, inputs.values(np.uint32, n), s, b)
    assert np.diff(off).max() <= 2 * n / b + BLOCK


def test_sample_sort_is_the_stable_sort():
    for dist in ("uniform", "gaussian", "zero", "bucket"):
        k = inputs.keys(np.uint32, dist, 70001)
        v = inputs.values(np.uint32, 70001)
        sk, sv = oracle.sample_sort(k, v, BLOCK, 32, 128)
        ek, ev = oracle.lsd_sort(k, v)
        assert np.array_equal(sk, ek) and np.array_equal(sv, ev)


def test_empty_input():
    k = np.zeros(0, dtype=np.uint32)
    pk, pv, off, spl = oracle.sample_partition(k, k.copy(), BLOCK, 16, 8)
    assert pk.size == 0 and off.tolist() == [0] * 9 and spl.size == 0
