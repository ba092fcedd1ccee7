"""GPU parity of the batched segmented sort (row a5: the sort of arXiv
1511.03404 Sec. 2.6 applied independently to every segment) against the
oracle's segmented sort, bit for bit."""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
from gpu_util import from_dev, to_dev  # noqa: E402

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu


def run_segmented(k, v, off, begin_bit=0, end_bit=32, check_status=True, ws=None):
    n = k.size
    dk, dv = to_dev(k, torch), to_dev(v, torch)
    ka, va = torch.empty_like(dk), torch.empty_like(dv)
    doff = to_dev(off.astype(np.uint64), torch)
    st, need = rs.rs_segmented_workspace_bytes(n, len(off) - 1, begin_bit, end_bit)
    rs.check(st, "rs_segmented_workspace_bytes")
    if ws is None:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_segmented_sort_pairs(dk.data_ptr(), dv.data_ptr(), ka.data_ptr(),
                                            va.data_ptr(), n, doff.data_ptr(), len(off) - 1,
                                            begin_bit, end_bit, ws.data_ptr(), ws.numel(), h)
    rs.check(st, "rs_segmented_sort_pairs")
    dst, info = rs.rs_workspace_status(ws.data_ptr(), h)
    if check_status:
        rs.check(dst, f"device status {info}")
    ok = from_dev(ka if in_alt else dk, np.uint32)
    ov = from_dev(va if in_alt else dv, np.uint32)
    return ok, ov, in_alt, dst


def check(dist, lengths, begin_bit=0, end_bit=32):
    off = inputs.offsets_from_lengths(np.asarray(lengths, dtype=np.uint64))
    n = int(off[-1])
    k = inputs.keys(np.uint32, dist, n)
    v = inputs.values(np.uint32, n)
    gk, gv, in_alt, _ = run_segmented(k, v, off, begin_bit, end_bit)
    ek, ev = oracle.segmented_sort(k, v, off, begin_bit=begin_bit, end_bit=end_bit)
    assert np.array_equal(gk, ek), (dist, begin_bit, end_bit)
    assert np.array_equal(gv, ev), (dist, begin_bit, end_bit)
    passes = -(-(end_bit - begin_bit) // 8)
    assert in_alt == (passes & 1)


EDGE = [0, 1, 2, 0, 31, 4095, 4096, 4097, 8191, 8192, 8193, 32767, 32768, 32769, 0, 70001, 3,
        1, 131072 + 4095]


@pytest.mark.parametrize("dist", list(inputs.DISTS))
def test_edge_lengths(dist):
    check(dist, EDGE)


@pytest.mark.parametrize("begin,end", [(0, 32), (0, 24), (8, 16), (5, 29), (0, 1)])
def test_bit_ranges(begin, end):
    check("uniform", EDGE, begin, end)
    check("entropy16", EDGE, begin, end)


def test_log_uniform_mix():
    L = inputs.segment_lengths(3000, seed=5, max_log2=17)
    check("uniform", L)
    check("gaussian", L)


def test_twenty_thousand_segments_scaled():
    """The batched workload's segment count and length law, lengths scaled
    so that the total is about 2^25 elements."""
    L = inputs.scale_lengths(inputs.segment_lengths(20000, seed=1, max_log2=20), 2**25)
    check("uniform", L)


def test_single_segment_matches_plain_sort():
    n = 3 * 2**18 + 77
    check("bucket", [n])


def test_bad_offsets_reported_not_written():
    k = inputs.keys(np.uint32, "uniform", 10000)
    v = inputs.values(np.uint32, 10000)
    off = np.array([0, 6000, 5000, 10000], dtype=np.uint64)  # not monotonic
    gk, gv, _, st = run_segmented(k, v, off, check_status=False)
    assert st == rs.RS_ERR_INVALID
    assert np.array_equal(gk, k) and np.array_equal(gv, v)
    off = np.array([0, 6000, 9000], dtype=np.uint64)  # does not end at n
    _, _, _, st = run_segmented(k, v, off, check_status=False)
    assert st == rs.RS_ERR_INVALID


def test_graph_capture_and_replay():
    """The whole batched sort captured once in a CUDA graph and replayed on
    new data in the same buffers."""
    L = inputs.segment_lengths(500, seed=9, max_log2=16)
    off = inputs.offsets_from_lengths(L)
    n = int(off[-1])
    dk = torch.empty(n, dtype=torch.int32, device="cuda")
    dv, ka, va = torch.empty_like(dk), torch.empty_like(dk), torch.empty_like(dk)
    doff = to_dev(off, torch)
    st, need = rs.rs_segmented_workspace_bytes(n, len(L))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    # one ordinary call first: kernel attributes are set outside the capture
    rs.check(rs.rs_segmented_sort_pairs(dk.data_ptr(), dv.data_ptr(), ka.data_ptr(),
                                        va.data_ptr(), n, doff.data_ptr(), len(L), 0, 32,
                                        ws.data_ptr(), ws.numel(), s.cuda_stream)[0])
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    result = {}
    with torch.cuda.graph(g, stream=s):
        st, in_alt = rs.rs_segmented_sort_pairs(dk.data_ptr(), dv.data_ptr(), ka.data_ptr(),
                                                va.data_ptr(), n, doff.data_ptr(), len(L), 0, 32,
                                                ws.data_ptr(), ws.numel(), s.cuda_stream)
        result["st"], result["in_alt"] = st, in_alt
    rs.check(result["st"])
    for dist in ("uniform", "sorted_desc", "gaussian"):
        k = inputs.keys(np.uint32, dist, n)
        v = inputs.values(np.uint32, n)
        dk.copy_(to_dev(k, torch))
        dv.copy_(to_dev(v, torch))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        rs.check(rs.rs_workspace_status(ws.data_ptr(), 0)[0])
        ek, ev = oracle.segmented_sort(k, v, off)
        src_k, src_v = (ka, va) if result["in_alt"] else (dk, dv)
        assert np.array_equal(from_dev(src_k, np.uint32), ek), dist
        assert np.array_equal(from_dev(src_v, np.uint32), ev), dist


# ---- the same sort for the other data types (rs_segmented_sort)

TYPED = [(4, 0), (4, 4), (8, 0), (8, 8)]
TYPED_IDS = ["k32", "kv32", "k64", "kv64"]
EDGE64 = EDGE + [2047, 2048, 2049, 6143, 6144, 6145]


def run_typed(kb, vb, k, v, off, begin_bit=0, end_bit=None):
    end_bit = 8 * kb if end_bit is None else end_bit
    n = k.size
    dk = to_dev(k, torch)
    ka = torch.empty_like(dk)
    dv = to_dev(v, torch) if vb else None
    va = torch.empty_like(dv) if vb else None
    doff = to_dev(off.astype(np.uint64), torch)
    st, need = rs.rs_segmented_workspace_bytes_typed(kb, vb, n, len(off) - 1, begin_bit, end_bit)
    rs.check(st, "rs_segmented_workspace_bytes_typed")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    st, in_alt = rs.rs_segmented_sort(kb, vb, p(dk), p(dv), p(ka), p(va), n, doff.data_ptr(),
                                      len(off) - 1, begin_bit, end_bit, p(ws), ws.numel(), h)
    rs.check(st, "rs_segmented_sort")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    assert in_alt == (-(-(end_bit - begin_bit) // 8) & 1)
    ok = from_dev(ka if in_alt else dk, k.dtype)
    ov = from_dev(va if in_alt else dv, v.dtype) if vb else None
    return ok, ov


def check_typed(kb, vb, dist, lengths, begin_bit=0, end_bit=None):
    dt = np.uint32 if kb == 4 else np.uint64
    off = inputs.offsets_from_lengths(np.asarray(lengths, dtype=np.uint64))
    n = int(off[-1])
    k = inputs.keys(dt, dist, n)
    v = inputs.values(dt, n) if vb else None
    gk, gv = run_typed(kb, vb, k, v, off, begin_bit, end_bit)
    ek, ev = oracle.segmented_sort(k, v, off, begin_bit=begin_bit, end_bit=end_bit)
    assert np.array_equal(gk, ek), (kb, vb, dist, begin_bit, end_bit)
    if vb:
        assert np.array_equal(gv, ev), (kb, vb, dist, begin_bit, end_bit)


@pytest.mark.parametrize("kb,vb", TYPED, ids=TYPED_IDS)
@pytest.mark.parametrize("dist", ["uniform", "entropy16", "zero", "sorted_desc", "gaussian"])
def test_typed_edge_lengths(kb, vb, dist):
    check_typed(kb, vb, dist, EDGE64)


@pytest.mark.parametrize("kb,vb", TYPED, ids=TYPED_IDS)
def test_typed_bit_ranges_and_mix(kb, vb):
    for b, e in ((0, 8 * kb), (0, 24), (5, 29), (8 * kb - 12, 8 * kb)):
        check_typed(kb, vb, "uniform", EDGE64, b, e)
    check_typed(kb, vb, "bucket", inputs.segment_lengths(1500, seed=7, max_log2=17))


def test_typed_entry_matches_pairs_entry():
    """rs_segmented_sort(4, 4, ...) and rs_segmented_sort_pairs are one sort."""
    L = inputs.segment_lengths(400, seed=3, max_log2=16)
    off = inputs.offsets_from_lengths(L)
    n = int(off[-1])
    k = inputs.keys(np.uint32, "gaussian", n)
    v = inputs.values(np.uint32, n)
    gk, gv = run_typed(4, 4, k, v, off)
    pk, pv, _, _ = run_segmented(k, v, off)
    assert np.array_equal(gk, pk) and np.array_equal(gv, pv)


def test_torch_segmented_sort_helper():
    """rs.segmented_sort over torch tensors: in place, every type, unsigned order."""
    L = inputs.segment_lengths(300, seed=13, max_log2=15)
    off = inputs.offsets_from_lengths(L)
    n = int(off[-1])
    doff = to_dev(off.astype(np.uint64), torch)
    for dt in (np.uint32, np.uint64):
        k = inputs.keys(dt, "sorted_desc", n)
        v = inputs.values(dt, n)
        dk, dv = to_dev(k, torch), to_dev(v, torch)
        rs.segmented_sort(dk, doff, dv)
        ek, ev = oracle.segmented_sort(k, v, off)
        assert np.array_equal(from_dev(dk, dt), ek) and np.array_equal(from_dev(dv, dt), ev)
        dk = to_dev(k, torch)
        rs.segmented_sort(dk, doff)
        assert np.array_equal(from_dev(dk, dt), oracle.segmented_sort(k, None, off)[0])
