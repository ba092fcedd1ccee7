"""GPU parity of the sample-sort partition and sample sort (Sec. 2.7)
against the oracle, bit for bit: the partitioned keys and values, the
bucket offsets and the splitters, and the sorted result (equal to the LSD
sort's).  Covers ragged block counts, a single partial block, heavy ties
(all keys equal: every key lands in the last bucket), more samples than a
block holds, and the argument checks."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import from_dev, to_dev

torch = pytest.importorskip("torch")

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu
BLOCK = 4096


def run_partition(k, v, samples, buckets, sort=False):
    n = k.size
    dk, dv = to_dev(k, torch), to_dev(v, torch)
    ko = torch.empty_like(dk)
    vo = torch.empty_like(dv)
    off = torch.zeros(buckets + 1, dtype=torch.int64, device="cuda")
    spl = torch.zeros(max(buckets - 1, 1), dtype=torch.int32, device="cuda")
    st, need = rs.rs_sample_workspace_bytes(n, samples, buckets)
    rs.check(st, "rs_sample_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    if sort:
        st, in_alt = rs.rs_sample_sort_pairs_u32(dk.data_ptr(), dv.data_ptr(), ko.data_ptr(),
                                                 vo.data_ptr(), n, samples, buckets,
                                                 off.data_ptr(), ws.data_ptr(), ws.numel(), h)
        rs.check(st, "rs_sample_sort_pairs_u32")
        rk, rv = (ko, vo) if in_alt else (dk, dv)
        return from_dev(rk, np.uint32), from_dev(rv, np.uint32)
    st = rs.rs_sample_partition_pairs_u32(dk.data_ptr(), dv.data_ptr(), ko.data_ptr(),
                                          vo.data_ptr(), n, samples, buckets, off.data_ptr(),
                                          spl.data_ptr(), ws.data_ptr(), ws.numel(), h)
    rs.check(st, "rs_sample_partition_pairs_u32")
    torch.cuda.synchronize()
    return (from_dev(ko, np.uint32), from_dev(vo, np.uint32),
            off.cpu().numpy().astype(np.uint64), from_dev(spl, np.uint32)[:buckets - 1])


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "zero", "bucket", "sorted",
                                  "sorted_desc", "entropy16"])
def test_partition_matches_oracle(dist):
    for n, s, b in ((1, 4, 2), (5000, 16, 8), (3 * BLOCK + 17, 64, 64), (2**17 + 5, 32, 256),
                    (2**20 + 3, 256, 1024), (4095, 4096, 16)):
        k = inputs.keys(np.uint32, dist, n)
        v = inputs.values(np.uint32, n)
        gk, gv, goff, gspl = run_partition(k, v, s, b)
        ek, ev, eoff, espl = oracle.sample_partition(k, v, BLOCK, s, b)
        assert np.array_equal(goff, eoff), (dist, n, s, b)
        assert np.array_equal(gspl, espl), (dist, n, s, b)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev), (dist, n, s, b)


@pytest.mark.parametrize("dist", ["uniform", "gaussian", "zero", "bucket"])
def test_sample_sort_matches_stable_sort(dist):
    for n, s, b in ((70001, 32, 128), (2**21 + 11, 128, 512)):
        k = inputs.keys(np.uint32, dist, n)
        v = inputs.values(np.uint32, n)
        gk, gv = run_partition(k, v, s, b, sort=True)
        ek, ev = oracle.lsd_sort(k, v)
        assert np.array_equal(gk, ek) and np.array_equal(gv, ev), (dist, n)


def test_sample_sort_arguments():
    h = torch.cuda.current_stream().cuda_stream
    d = torch.zeros(64, dtype=torch.int32, device="cuda")
    off = torch.zeros(9, dtype=torch.int64, device="cuda")
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    p = d.data_ptr()
    for samples, buckets in ((0, 8), (4097, 8), (16, 1), (16, 4097)):
        assert rs.rs_sample_workspace_bytes(64, samples, buckets)[0] == rs.RS_ERR_INVALID
    # output aliasing the input
    assert rs.rs_sample_partition_pairs_u32(p, p + 256, p, p + 512, 16, 4, 8, off.data_ptr(),
                                            None, ws.data_ptr(), ws.numel(),
                                            h) == rs.RS_ERR_INVALID
    # workspace too small
    a = torch.zeros(4 * 64, dtype=torch.int32, device="cuda")
    q = a.data_ptr()
    assert rs.rs_sample_partition_pairs_u32(q, q + 256, q + 512, q + 768, 64, 4, 8,
                                            off.data_ptr(), None, ws.data_ptr(), 256,
                                            h) == rs.RS_ERR_WORKSPACE
