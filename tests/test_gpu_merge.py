"""GPU parity of the merge sort (Sec. 2.4) with the oracle, bit for bit:
32- and 64-bit keys against the LSD sort, 128-bit keys against the wide-key
oracle, with and without values, at tile boundaries, ragged lengths and a
million elements (ten merge passes), on inputs with many ties (stability)."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import from_dev, to_dev

torch = pytest.importorskip("torch")

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu
TILE = 4096
SIZES = (0, 1, 2, 7, 2047, 2049, TILE - 1, TILE, TILE + 1, 3 * TILE + 5, 2**17 + 3, 2**20 + 7)


def make(kb, dist, n):
    if kb == 16:
        lo = inputs.keys(np.uint64, dist, n)
        hi = inputs.keys(np.uint64, "entropy16", n, seed=2) % np.uint64(3)
        return np.ascontiguousarray(np.stack([lo, hi], axis=1))
    return inputs.keys(np.uint32 if kb == 4 else np.uint64, dist, n)


def gpu_merge(k, v, kb, vb):
    n = k.shape[0]
    dk = to_dev(k, torch)
    ka = torch.empty_like(dk)
    dv = to_dev(v, torch) if vb else None
    va = torch.empty_like(dv) if vb else None
    st, need = rs.rs_merge_workspace_bytes(kb, vb, n)
    rs.check(st, "rs_merge_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    st, in_alt = rs.rs_merge_sort(kb, vb, dk.data_ptr(), ptr(dv), ka.data_ptr(), ptr(va), n,
                                  ws.data_ptr(), ws.numel(), torch.cuda.current_stream().cuda_stream)
    rs.check(st, "rs_merge_sort")
    rk = from_dev(ka if in_alt else dk, k.dtype).reshape(k.shape)
    rv = from_dev(va if in_alt else dv, v.dtype) if vb else None
    return rk, rv


@pytest.mark.parametrize("kb,vb", [(4, 0), (4, 4), (8, 0), (8, 8), (16, 0), (16, 8)],
                         ids=["k32", "kv32", "k64", "kv64", "k128", "k128v64"])
def test_merge_sort_matches_oracle(kb, vb):
    for dist in ("uniform", "entropy16", "zero", "sorted_desc"):
        for n in SIZES:
            k = make(kb, dist, n)
            vdt = np.uint32 if vb == 4 else np.uint64
            v = np.arange(n, dtype=vdt) if vb else None
            gk, gv = gpu_merge(k, v, kb, vb)
            if kb == 16:
                ek, ev = oracle.sort_wide(k, v)
            else:
                ek, ev = oracle.lsd_sort(k, v)
            assert np.array_equal(gk, ek), (kb, vb, dist, n)
            if vb:
                assert np.array_equal(gv, ev), (kb, vb, dist, n)


def test_merge_sort_arguments():
    h = torch.cuda.current_stream().cuda_stream
    d = torch.zeros(1024, dtype=torch.int64, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    for kb, vb in ((2, 0), (4, 8), (16, 4), (16, 16)):
        assert rs.rs_merge_workspace_bytes(kb, vb, 100)[0] == rs.RS_ERR_INVALID
    assert rs.rs_merge_sort(4, 0, p, None, p, None, 100, ws.data_ptr(), ws.numel(),
                            h)[0] == rs.RS_ERR_INVALID  # aliasing
    assert rs.rs_merge_sort(16, 0, p + 8, None, p + 4096, None, 100, ws.data_ptr(), ws.numel(),
                            h)[0] == rs.RS_ERR_INVALID  # 16-byte keys misaligned
    assert rs.rs_merge_sort(4, 0, p, None, p + 4096, None, 100, ws.data_ptr(), 0,
                            h)[0] == rs.RS_ERR_WORKSPACE
