"""Parity at the benchmark's full sizes, in the configuration bench.py times
(the C ABI, the tuned variant choice): u32 pairs at n = 2^26 for the six
distributions, u64 keys and u64 pairs at n = 2^27.  The oracle takes minutes
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
from gpu_util import to_dev

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


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "entropy16"])
def test_u64_keys_2p27(dist):
    k = inputs.keys(np.uint64, dist, 1 << 27)
    src, out_k, _ = run(8, 0, k)
    want = ordered(torch.sort(ordered(src)).values)
    assert bool((out_k == want).all())


@pytest.mark.parametrize("dist", ["uniform", "entropy16"])
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
