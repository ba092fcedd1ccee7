"""GPU parity: the CUDA LSD radix sort against the oracle, bit for bit.

Every case runs the library through its C ABI on seeded inputs and compares
keys and values element by element with the oracle's result (arXiv
1511.03404 Sec. 2.6 semantics: ascending, unsigned, stable).  Sizes span
several tiles and ragged tails, the 2^n + 2^(n-1) lengths of Sec. 3, and the
degenerate cases (n = 0, 1, one digit value, every pass skipped).
"""
import time

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
from gpu_util import from_dev, sort_via_abi, to_dev  # noqa: E402

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu

TYPES = [(np.uint32, False), (np.uint32, True), (np.uint64, False), (np.uint64, True)]
TYPE_IDS = ["k32", "kv32", "k64", "kv64"]


def variants(kb, vb):
    return [rs.rs_variant_info(kb, vb, i) | {"index": i} for i in range(rs.rs_num_variants(kb, vb))]


def expected(k, v, begin_bit=0, end_bit=None):
    return oracle.lsd_sort(k, v, begin_bit=begin_bit, end_bit=end_bit)


def check_case(dtype, pairs, dist, n, **kw):
    k = inputs.keys(dtype, dist, n)
    v = inputs.values(dtype, n) if pairs else None
    gk, gv, _ = sort_via_abi(torch, k, v, **kw)
    ek, ev = expected(k, v, kw.get("begin_bit", 0), kw.get("end_bit"))
    assert np.array_equal(gk, ek), (dtype, pairs, dist, n, kw)
    if pairs:
        assert np.array_equal(gv, ev), (dtype, pairs, dist, n, kw)


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
@pytest.mark.parametrize("dist", list(inputs.DISTS))
def test_default_choice_all_distributions(dtype, pairs, dist):
    for n in (0, 1, 2, 31, 32, 33, 1000, 3 * 2**12, 3 * 2**15, 2**17 + 5):
        check_case(dtype, pairs, dist, n)


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_every_variant_tile_boundaries(dtype, pairs):
    kb = np.dtype(dtype).itemsize
    vb = kb if pairs else 0
    for var in variants(kb, vb):
        tile = var["threads"] * var["items"]
        sizes = {2, 3, 31, 32, 33, tile - 1, tile, tile + 1, 2 * tile + 7, 5 * tile}
        if var["max_n"] <= 1 << 17:  # one-CTA and one-cluster kinds: their largest arrays
            sizes |= {var["max_n"] - 1, var["max_n"]}
        for n in sorted(s for s in sizes if s <= var["max_n"]):
            for dist in ("uniform", "entropy16", "zero", "sorted_desc"):
                check_case(dtype, pairs, dist, n, variant=var["index"])


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_resident_cta_variants_many_tiles_per_cta(dtype, pairs):
    """Variants whose CTAs stay resident and take tile after tile: sizes that
    give every CTA several tiles (the boundary test above gives each one)."""
    kb = np.dtype(dtype).itemsize
    vb = kb if pairs else 0
    for var in variants(kb, vb):
        if var["kind"] not in (2, 3):  # resident CTAs; one cooperative launch
            continue
        tile = var["threads"] * var["items"]
        for n in (152 * 4 * tile * 3 + 12345, 152 * 4 * tile * 5):
            check_case(dtype, pairs, "uniform", n, variant=var["index"])
        check_case(dtype, pairs, "sorted_desc", 152 * 4 * tile * 2 + 7, variant=var["index"])


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_typed_entry_points(dtype, pairs):
    for n in (5000, 70001):
        check_case(dtype, pairs, "bucket", n, api="typed")


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_paper_lengths(dtype, pairs):
    # 2^n and 2^n + 2^(n-1) for n = 15..20 (Sec. 3 tests both forms)
    for e in range(15, 21):
        for n in (2**e, 2**e + 2**(e - 1)):
            check_case(dtype, pairs, "gaussian", n)


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_bit_ranges(dtype, pairs):
    bits = np.dtype(dtype).itemsize * 8
    for begin, end in [(0, 1), (3, 17), (bits - 8, bits), (4, bits - 3), (0, 12), (7, 7)]:
        for n in (3000, 50001):
            check_case(dtype, pairs, "uniform", n, begin_bit=begin, end_bit=end)


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_unaligned_buffers(dtype, pairs):
    for off in (1, 2, 3):
        for n in (4097, 100003):
            check_case(dtype, pairs, "uniform", n, offset_elems=off)


@pytest.mark.parametrize("dtype,pairs", TYPES, ids=TYPE_IDS)
def test_unaligned_buffers_every_multi_cta_variant(dtype, pairs):
    """Every one-CTA-per-tile and resident-CTA variant (warp and half-warp
    ranking units) on buffers 1-3 elements past a 16-byte boundary, over
    several tiles and a ragged tail: the bulk copies start at the aligned
    part and the head and tail elements are loaded by threads."""
    kb = np.dtype(dtype).itemsize
    vb = kb if pairs else 0
    for var in variants(kb, vb):
        if var["kind"] not in (0, 2):
            continue
        tile = var["threads"] * var["items"]
        for off in (1, 3):
            check_case(dtype, pairs, "uniform", 3 * tile + 5, offset_elems=off,
                       variant=var["index"])


def test_non_default_stream():
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        check_case(np.uint32, True, "uniform", 300001, stream=s)


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_digit_counts_and_scan(dtype):
    """Rows a1/a2: per-pass digit histograms and their exclusive scans."""
    kb = np.dtype(dtype).itemsize
    for dist in ("uniform", "zero", "entropy16", "bucket"):
        n = 3 * 2**16 + 11
        k = inputs.keys(dtype, dist, n)
        passes = 8 * kb // 8
        want_c = oracle.digit_counts(k, r=8)
        want_o = oracle.digit_offsets(want_c, r=8)
        dk = to_dev(k, torch)
        dc = torch.zeros(passes * 256, dtype=torch.int32, device="cuda")
        do = torch.zeros_like(dc)
        dm = torch.zeros(1, dtype=torch.int32, device="cuda")
        st, nbytes = rs.rs_workspace_bytes(kb, 0, n, 0, 8 * kb)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        h = torch.cuda.current_stream().cuda_stream
        rs.check(rs.rs_digit_counts(kb, dk.data_ptr(), n, 0, 8 * kb, 8, dc.data_ptr(),
                                    do.data_ptr(), dm.data_ptr(), ws.data_ptr(), ws.numel(), h))
        got_c = from_dev(dc, np.uint32).reshape(passes, 256).astype(np.uint64)
        got_o = from_dev(do, np.uint32).reshape(passes, 256).astype(np.uint64)
        assert np.array_equal(got_c, want_c), dist
        assert np.array_equal(got_o, want_o), dist
        moving = [int(want_c[p].max()) != n for p in range(passes)]
        mask = int(from_dev(dm, np.uint32)[0])
        want_mask = sum(1 << p for p in range(passes) if moving[p])
        if bin(want_mask).count("1") % 2 != passes % 2:
            low = next(p for p in range(passes) if not moving[p])
            want_mask |= 1 << low
        assert mask == want_mask, (dist, hex(mask), hex(want_mask))


def test_result_location_rule():
    """result_in_alt follows the pass count (ceil(bits / r)) for the onesweep
    path even when passes are skipped; the small path sorts in place."""
    k = inputs.keys(np.uint32, "entropy16", 200000)
    for begin, end, want in ((0, 32, 0), (0, 24, 1), (0, 8, 1), (8, 24, 0)):
        _, _, in_alt = sort_via_abi(torch, k, None, begin_bit=begin, end_bit=end)
        assert in_alt == want, (begin, end)
    _, _, in_alt = sort_via_abi(torch, k[:1000], None, begin_bit=0, end_bit=24)
    assert in_alt == 0


def test_repeated_calls_reuse_workspace():
    n = 2**18 + 3
    kb = 4
    st, nbytes = rs.rs_workspace_bytes(kb, kb, n, 0, 32)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    for dist in ("uniform", "zero", "sorted", "gaussian"):
        k = inputs.keys(np.uint32, dist, n)
        v = inputs.values(np.uint32, n)
        dk, dv = to_dev(k, torch), to_dev(v, torch)
        ka, va = torch.empty_like(dk), torch.empty_like(dv)
        st, in_alt = rs.rs_sort_pairs_u32(dk.data_ptr(), dv.data_ptr(), ka.data_ptr(),
                                          va.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), h)
        rs.check(st)
        rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0])
        ek, ev = oracle.lsd_sort(k, v)
        assert np.array_equal(from_dev(ka if in_alt else dk, np.uint32), ek)
        assert np.array_equal(from_dev(va if in_alt else dv, np.uint32), ev)


def test_argument_errors_on_device_buffers():
    n = 100000
    d = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    a = torch.zeros(n + 8, dtype=torch.int32, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, need = rs.rs_workspace_bytes(4, 0, n, 0, 32)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    # workspace too small / misaligned / missing
    assert rs.rs_sort_keys_u32(d.data_ptr(), a.data_ptr(), n, 0, 32, ws.data_ptr(), need - 1,
                               h)[0] == rs.RS_ERR_WORKSPACE
    assert rs.rs_sort_keys_u32(d.data_ptr(), a.data_ptr(), n, 0, 32, ws.data_ptr() + 4, need - 4,
                               h)[0] == rs.RS_ERR_WORKSPACE
    assert rs.rs_sort_keys_u32(d.data_ptr(), a.data_ptr(), n, 0, 32, None, 0, h)[0] == \
        rs.RS_ERR_WORKSPACE
    # same buffer twice, bad bits, misaligned keys
    assert rs.rs_sort_keys_u32(d.data_ptr(), d.data_ptr(), n, 0, 32, ws.data_ptr(), need,
                               h)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_keys_u32(d.data_ptr(), a.data_ptr(), n, 0, 33, ws.data_ptr(), need,
                               h)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_keys_u32(d.data_ptr() + 2, a.data_ptr(), n, 0, 32, ws.data_ptr(), need,
                               h)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_keys_u32(d.data_ptr(), a.data_ptr(), rs.RS_MAX_N + 1, 0, 32, ws.data_ptr(),
                               need, h)[0] == rs.RS_ERR_INVALID


@pytest.mark.parametrize("vb", [0, 4], ids=["k32", "kv32"])
def test_every_multi_cta_form_gives_up_in_bounded_time(vb):
    """The same dropped tile under every form that waits on other CTAs (one
    CTA per tile, resident CTAs taking tile after tile, one cooperative
    launch with grid barriers): each reports RS_ERR_TIMEOUT in bounded time,
    and the context sorts correctly afterwards."""
    n = 2**20
    k = inputs.keys(np.uint32, "uniform", n)
    v = inputs.values(np.uint32, n)
    h = torch.cuda.current_stream().cuda_stream
    tested = set()
    for var in variants(4, vb):
        if var["kind"] not in (0, 2, 3) or var["max_n"] < n:
            continue
        tested.add(var["kind"])
        try:
            rs.check(rs.rs_debug_set(rs.RS_DEBUG_TIMEOUT_NS, 20_000_000))
            rs.check(rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_PASS, 1))
            rs.check(rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_TILE, 3))
            dk, dv = to_dev(k, torch), to_dev(v, torch)
            ka, va = torch.empty_like(dk), torch.empty_like(dv)
            st, need = rs.rs_workspace_bytes(4, vb, n, 0, 32, 0, var["index"])
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            t0 = time.time()
            rs.check(rs.rs_sort(4, vb, dk.data_ptr(), dv.data_ptr() if vb else None,
                                ka.data_ptr(), va.data_ptr() if vb else None, n, 0, 32,
                                ws.data_ptr(), need, h, 0, var["index"])[0])
            st, info = rs.rs_workspace_status(ws.data_ptr(), h)
            assert st == rs.RS_ERR_TIMEOUT, (var, st)
            assert info > 3, (var, info)
            assert time.time() - t0 < 30, var
        finally:
            rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_TILE, -1)
            rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_PASS, -1)
            rs.rs_debug_set(rs.RS_DEBUG_TIMEOUT_NS, 1_000_000_000)
        check_case(np.uint32, vb > 0, "uniform", n, variant=var["index"])
    assert tested == {0, 2, 3}


def test_lookback_wait_is_bounded():
    """A tile that never publishes makes its successors' bounded waits run
    out: the call reports RS_ERR_TIMEOUT and the context stays usable."""
    k = inputs.keys(np.uint32, "uniform", 2**20)
    try:
        rs.check(rs.rs_debug_set(rs.RS_DEBUG_TIMEOUT_NS, 20_000_000))
        rs.check(rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_PASS, 1))
        rs.check(rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_TILE, 3))
        dk = to_dev(k, torch)
        ka = torch.empty_like(dk)
        st, need = rs.rs_workspace_bytes(4, 0, k.size, 0, 32)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        h = torch.cuda.current_stream().cuda_stream
        rs.check(rs.rs_sort_keys_u32(dk.data_ptr(), ka.data_ptr(), k.size, 0, 32, ws.data_ptr(),
                                     need, h)[0])
        st, info = rs.rs_workspace_status(ws.data_ptr(), h)
        assert st == rs.RS_ERR_TIMEOUT
        assert info > 3
    finally:
        rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_TILE, -1)
        rs.rs_debug_set(rs.RS_DEBUG_DROP_PUBLISH_PASS, -1)
        rs.rs_debug_set(rs.RS_DEBUG_TIMEOUT_NS, 1_000_000_000)
    # the same context sorts correctly afterwards
    check_case(np.uint32, False, "uniform", 2**20)


def test_without_dependent_launch_same_result():
    """With RS_NO_PDL set (read once per process) the passes are launched the
    ordinary way; the sorted output is the same."""
    import subprocess
    import sys
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "import numpy as np, inputs, oracle, torch\n"
        "from gpu_util import sort_via_abi\n"
        "for n in (5 * 4352 + 3, 1 << 21, (1 << 23) + 5):\n"
        "    k = inputs.keys(np.uint32, 'uniform', n); v = inputs.values(np.uint32, n)\n"
        "    gk, gv, _ = sort_via_abi(torch, k, v)\n"
        "    ek, ev = oracle.lsd_sort(k, v)\n"
        "    assert np.array_equal(gk, ek) and np.array_equal(gv, ev)\n"
        "print('ok')\n" % (root, os.path.join(root, "tests")))
    env = dict(os.environ, RS_NO_PDL="1")
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stderr[-2000:]
