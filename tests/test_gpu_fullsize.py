"""Parity at the benchmark's full sizes, in the configuration bench.py times
(the C ABI, the tuned variant choice): u32 pairs at n = 2^26 for the six
distributions and in the signed and IEEE-754 orders (ascending and
descending), u64 keys and u64 pairs at n = 2^27 for the six and 16-bit
entropy keys, and the batched segmented workload (20,000 segments, about
1.5e9 pairs).  The oracle takes minutes
at these sizes, so the result is checked on the device by properties that
together define the stable sort uniquely (values are the input positions):

- the keys are non-decreasing as unsigned integers;
- the values are a permutation of 0 .. n-1;
- every output key equals the input key at its value's position;
- equal keys keep their input order (their values increase).

Keys-only sorts are checked against torch's sort of the same keys mapped to
the signed order (x ^ sign bit), an independent library routine."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import from_dev, to_dev

torch = pytest.importorskip("torch")

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu


def ordered(t):
    """Signed tensor whose order is the unsigned order of t's bits."""
    top = -(1 << 31) if t.dtype == torch.int32 else -(1 << 63)
    return t ^ top


def run(kb, vb, k_host):
    n = k_host.size
    dk = to_dev(k_host, torch)
    src = dk.clone()
    ka = torch.empty_like(dk)
    dv = va = None
    if vb:
        dv = torch.arange(n, dtype=torch.int32 if vb == 4 else torch.int64, device="cuda")
        va = torch.empty_like(dv)
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort(kb, vb, dk.data_ptr(), dv.data_ptr() if vb else None, ka.data_ptr(),
                            va.data_ptr() if vb else None, n, 0, 8 * kb, ws.data_ptr(),
                            ws.numel(), h)
    rs.check(st, "rs_sort")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    out_k = ka if in_alt else dk
    out_v = (va if in_alt else dv) if vb else None
    return src, out_k, out_v


def check_pairs(src, out_k, out_v):
    n = src.numel()
    o = ordered(out_k)
    assert bool((o[1:] >= o[:-1]).all()), "keys not sorted"
    idx = out_v.long()
    assert int(idx.min()) == 0 and int(idx.max()) == n - 1
    seen = torch.zeros(n, dtype=torch.int32, device="cuda")
    seen.scatter_add_(0, idx, torch.ones(n, dtype=torch.int32, device="cuda"))
    assert bool((seen == 1).all()), "values are not a permutation"
    assert bool((src[idx] == out_k).all()), "a key left its value"
    eq = o[1:] == o[:-1]
    assert bool((idx[1:][eq] > idx[:-1][eq]).all()), "equal keys out of input order"


@pytest.mark.parametrize("dist", list(inputs.PAPER_DISTS))
def test_u32_pairs_2p26(dist):
    k = inputs.keys(np.uint32, dist, 1 << 26)
    src, out_k, out_v = run(4, 4, k)
    check_pairs(src, out_k, out_v)


@pytest.mark.parametrize("dist", list(inputs.PAPER_DISTS) + ["entropy16"])
def test_u64_keys_2p27(dist):
    k = inputs.keys(np.uint64, dist, 1 << 27)
    src, out_k, _ = run(8, 0, k)
    want = ordered(torch.sort(ordered(src)).values)
    assert bool((out_k == want).all())


@pytest.mark.parametrize("dist", list(inputs.PAPER_DISTS) + ["entropy16"])
def test_u64_pairs_2p27(dist):
    k = inputs.keys(np.uint64, dist, 1 << 27)
    src, out_k, out_v = run(8, 8, k)
    check_pairs(src, out_k, out_v)


@pytest.mark.parametrize("vb", [0, 4], ids=["keys", "pairs"])
def test_largest_array(vb):
    """n = RS_MAX_N = 2^30 - 1: the look-back counts use their full 30 bits."""
    n = rs.RS_MAX_N
    k = inputs.keys(np.uint32, "uniform", n, seed=5)
    src, out_k, out_v = run(4, vb, k)
    del k
    if vb:
        check_pairs(src, out_k, out_v)
    else:
        want = ordered(torch.sort(ordered(src)).values)
        assert bool((out_k == want).all())


def check_segmented(src, out_k, out_v, off):
    """Every segment of the batched sort sorted stably, on the device.  The
    values are the input positions 0 .. n-1, so the four properties of
    check_pairs taken per segment fix the result uniquely: keys
    non-decreasing inside each segment, the values a permutation of 0 .. n-1
    in which every value stays inside its own position's segment, every
    output key equal to the input key at its value, and equal keys of a
    segment in increasing value order."""
    n = src.numel()
    dev = src.device
    lengths = torch.from_numpy(np.diff(off).astype(np.int64)).to(dev)
    seg = torch.repeat_interleave(torch.arange(lengths.numel(), dtype=torch.int32, device=dev),
                                  lengths, output_size=n)
    same = seg[1:] == seg[:-1]
    o = ordered(out_k)
    assert bool(((o[1:] >= o[:-1]) | ~same).all()), "a segment is not sorted"
    idx = out_v.long()
    assert int(idx.min()) == 0 and int(idx.max()) == n - 1
    seen = torch.zeros(n, dtype=torch.uint8, device=dev)
    seen[idx] = 1
    assert bool(seen.bool().all()), "values are not a permutation"
    del seen
    assert bool((seg[idx] == seg).all()), "a value left its segment"
    assert bool((src[idx] == out_k).all()), "a key left its value"
    eq = (o[1:] == o[:-1]) & same
    assert bool(((idx[1:] > idx[:-1]) | ~eq).all()), "equal keys out of input order"


def test_segmented_twenty_thousand_segments_full_size():
    """The batched workload itself: 20,000 segments, lengths log-uniform in
    [1, 2^20] (seed 1), about 1.5e9 u32 pairs in all -- more elements than
    RS_MAX_N and byte offsets beyond 2^32.  Checked on the device as a whole
    (check_segmented), and against the oracle on sampled segments: the last
    ones (the largest offsets), the longest ones and random ones."""
    L = inputs.segment_lengths(20000, seed=1, max_log2=20)
    off = inputs.offsets_from_lengths(L)
    n = int(off[-1])
    assert n > rs.RS_MAX_N and 4 * n > 2**32
    k = inputs.keys(np.uint32, "uniform", n, seed=1)
    dk = to_dev(k, torch)
    src = dk.clone()
    dv = torch.arange(n, dtype=torch.int32, device="cuda")
    ka, va = torch.empty_like(dk), torch.empty_like(dv)
    doff = to_dev(off.astype(np.uint64), torch)
    st, need = rs.rs_segmented_workspace_bytes(n, len(L), 0, 32)
    rs.check(st, "rs_segmented_workspace_bytes")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_segmented_sort_pairs(dk.data_ptr(), dv.data_ptr(), ka.data_ptr(),
                                            va.data_ptr(), n, doff.data_ptr(), len(L), 0, 32,
                                            ws.data_ptr(), ws.numel(), h)
    rs.check(st, "rs_segmented_sort_pairs")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    out_k, out_v = (ka, va) if in_alt else (dk, dv)
    del ws
    check_segmented(src, out_k, out_v, off)
    rng = np.random.default_rng(3)
    picks = set(range(len(L) - 40, len(L)))
    picks |= set(np.argsort(L, kind="stable")[-20:].tolist())
    picks |= set(rng.choice(len(L), 200, replace=False).tolist())
    for s in sorted(picks):
        a, b = int(off[s]), int(off[s + 1])
        ek, ev = oracle.lsd_sort(k[a:b], np.arange(a, b, dtype=np.uint32))
        assert np.array_equal(from_dev(out_k[a:b], np.uint32), ek), s
        assert np.array_equal(from_dev(out_v[a:b], np.uint32), ev), s


def total_order(t):
    """Signed tensor whose order is IEEE-754 totalOrder of binary32 bit patterns
    held in an int32 tensor: negative patterns have every bit but the sign
    flipped, non-negative ones are kept."""
    return t ^ ((t >> 31) & 0x7FFFFFFF)


def check_pairs_order(src, out_k, out_v, o):
    """As check_pairs, for a sort by the order whose signed key is o."""
    n = src.numel()
    assert bool((o[1:] >= o[:-1]).all()), "keys not in order"
    idx = out_v.long()
    seen = torch.zeros(n, dtype=torch.uint8, device="cuda")
    seen[idx] = 1
    assert bool(seen.bool().all()), "values are not a permutation"
    assert bool((src[idx] == out_k).all()), "a key left its value"
    eq = o[1:] == o[:-1]
    assert bool(((idx[1:] > idx[:-1]) | ~eq).all()), "equal keys out of input order"


@pytest.mark.parametrize("kind,descending", [(1, False), (1, True), (2, False), (2, True)],
                         ids=["signed", "signed_desc", "float", "float_desc"])
def test_u64_keys_2p26_key_orders(kind, descending):
    """64-bit keys only in the signed and IEEE-754 orders, ascending and
    descending, at 2^26 (the tuned pass stages these keys in place): the
    output is the sorted multiset of the input under that order."""
    n = 1 << 26
    k = inputs.keys(np.uint64, "uniform", n) if kind == 1 else inputs.float_keys(np.uint64, n)
    dk = to_dev(k, torch)
    src = dk.clone()
    ka = torch.empty_like(dk)
    st, need = rs.rs_workspace_bytes(8, 0, n, 0, 64)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort(8, 0, dk.data_ptr(), None, ka.data_ptr(), None, n, 0, 64,
                            ws.data_ptr(), ws.numel(), h, key_kind=kind, descending=descending)
    rs.check(st, "rs_sort")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    out_k = ka if in_alt else dk

    def order(t):  # signed int64 whose order is the requested one
        o = t if kind == 1 else t ^ ((t >> 63) & 0x7FFFFFFFFFFFFFFF)
        return ~o if descending else o

    o = order(out_k)
    assert bool((o[1:] >= o[:-1]).all()), "keys not in order"
    assert torch.equal(o, torch.sort(order(src)).values), "not the input's multiset"


@pytest.mark.parametrize("kind,descending", [(1, False), (1, True), (2, False), (2, True)],
                         ids=["signed", "signed_desc", "float", "float_desc"])
def test_u32_pairs_2p26_key_orders(kind, descending):
    """Signed and IEEE-754 orders, ascending and descending, at the benchmark
    size: stable in every mode (equal keys keep their input order)."""
    n = 1 << 26
    k = inputs.keys(np.uint32, "uniform", n) if kind == 1 else inputs.float_keys(np.uint32, n)
    dk = to_dev(k, torch)
    src = dk.clone()
    dv = torch.arange(n, dtype=torch.int32, device="cuda")
    ka, va = torch.empty_like(dk), torch.empty_like(dv)
    st, need = rs.rs_workspace_bytes(4, 4, n, 0, 32)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort(4, 4, dk.data_ptr(), dv.data_ptr(), ka.data_ptr(), va.data_ptr(), n,
                            0, 32, ws.data_ptr(), ws.numel(), h, key_kind=kind,
                            descending=descending)
    rs.check(st, "rs_sort")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    out_k, out_v = (ka, va) if in_alt else (dk, dv)
    o = out_k if kind == 1 else total_order(out_k)
    if descending:
        o = ~o  # reverses the signed order
    check_pairs_order(src, out_k, out_v, o)
