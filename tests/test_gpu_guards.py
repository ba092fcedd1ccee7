"""Guard canaries around every buffer the kernels write, and the bounds-
checked debug build.  Both stand in for compute-sanitizer's out-of-bounds
check, which is closed on this machine.

Every output, alternate and workspace buffer of a call sits between two
4 KiB guards of a seeded byte pattern, and every guard must be intact after
the call.  This holds for the tile-boundary suite (every compiled variant of
every key type at sizes around its tile), the segmented edge suite, the
sample-sort partition and the merge sort, each also compared with the
oracle.  The same tests run again in a child process that loads the debug
build (RS_LIBRARY=debug), whose kernels check the index of every global store
against its array's length; there rs_debug_status must report no failed
check after every call, and a planted bad index (a debug-only knob whose
stores the checks drop) must be reported."""
import os
import subprocess
import sys

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
from gpu_util import from_dev  # noqa: E402

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu
GUARD = 4096
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NP_SIGNED = {1: np.int8, 4: np.int32, 8: np.int64}


class Guarded:
    """Device buffers, each between two guards of a seeded pattern."""

    def __init__(self):
        self.regions = []

    def alloc(self, nbytes: int):
        nb = int(nbytes)
        raw = torch.empty(2 * GUARD + nb, dtype=torch.uint8, device="cuda")
        rng = np.random.default_rng(1000 + len(self.regions))
        pat = torch.from_numpy(rng.integers(0, 256, 2 * GUARD, dtype=np.uint8)).cuda()
        raw[:GUARD] = pat[:GUARD]
        raw[GUARD + nb:] = pat[GUARD:]
        self.regions.append((raw, nb, pat))
        return raw[GUARD:GUARD + nb]

    def put(self, a: np.ndarray):
        """A guarded device copy of a host array."""
        body = self.alloc(a.nbytes)
        if a.size:
            body.copy_(torch.from_numpy(np.ascontiguousarray(a).view(np.uint8).reshape(-1)))
        return body

    def check(self, what):
        torch.cuda.synchronize()
        for i, (raw, nb, pat) in enumerate(self.regions):
            assert torch.equal(raw[:GUARD], pat[:GUARD]), f"{what}: guard before buffer {i}"
            assert torch.equal(raw[GUARD + nb:], pat[GUARD:]), f"{what}: guard after buffer {i}"
        if rs.debug_library():
            st, is_debug, site, index = rs.rs_debug_status()
            assert is_debug, "RS_LIBRARY=debug but the library is not the debug build"
            assert st == rs.RS_OK, f"{what}: bounds check failed at site {site}, index {index}"


def ptr(t):
    return None if t is None else t.data_ptr()


def host(t, dtype):
    return t.cpu().numpy().view(dtype)


def guarded_sort(kb, vb, dist, n, variant):
    dt = np.uint32 if kb == 4 else np.uint64
    k = inputs.keys(dt, dist, n)
    v = inputs.values(dt, n) if vb else None
    g = Guarded()
    dk, ka = g.put(k), g.alloc(n * kb)
    dv = g.put(v) if vb else None
    va = g.alloc(n * vb) if vb else None
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb, variant=variant)
    rs.check(st)
    ws = g.alloc(max(need, 256))
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort(kb, vb, ptr(dk), ptr(dv), ptr(ka), ptr(va), n, 0, 8 * kb, ptr(ws),
                            ws.numel(), h, variant=variant)
    rs.check(st, "rs_sort")
    rs.check(rs.rs_workspace_status(ptr(ws), h)[0], "device status")
    what = f"sort k{kb} v{vb} {dist} n={n} variant {variant}"
    g.check(what)
    ek, ev = oracle.lsd_sort(k, v)
    assert np.array_equal(host(ka if in_alt else dk, dt), ek), what
    if vb:
        assert np.array_equal(host(va if in_alt else dv, dt), ev), what


@pytest.mark.parametrize("kb,vb", [(4, 0), (4, 4), (8, 0), (8, 8)],
                         ids=["k32", "kv32", "k64", "kv64"])
def test_tile_boundary_suite_guards_intact(kb, vb):
    for i in range(rs.rs_num_variants(kb, vb)):
        var = rs.rs_variant_info(kb, vb, i)
        tile = var["threads"] * var["items"]
        sizes = {2, 33, tile - 1, tile, tile + 1, 2 * tile + 7}
        if var["max_n"] <= 1 << 17:
            sizes |= {var["max_n"]}
        for n in sorted(s for s in sizes if s <= var["max_n"]):
            for dist in ("uniform", "sorted_desc"):
                guarded_sort(kb, vb, dist, n, i)


EDGE = [0, 1, 2, 0, 31, 4095, 4096, 4097, 8191, 8192, 8193, 32767, 32768, 32769, 0, 70001, 3,
        1, 131072 + 4095]


@pytest.mark.parametrize("begin,end", [(0, 32), (5, 29)])
@pytest.mark.parametrize("dist", ["uniform", "entropy16", "zero"])
def test_segmented_edge_suite_guards_intact(dist, begin, end):
    off = inputs.offsets_from_lengths(np.asarray(EDGE, dtype=np.uint64))
    n = int(off[-1])
    k = inputs.keys(np.uint32, dist, n)
    v = inputs.values(np.uint32, n)
    g = Guarded()
    dk, dv, ka, va = g.put(k), g.put(v), g.alloc(4 * n), g.alloc(4 * n)
    doff = g.put(off.astype(np.uint64))
    st, need = rs.rs_segmented_workspace_bytes(n, len(EDGE), begin, end)
    rs.check(st)
    ws = g.alloc(need)
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_segmented_sort_pairs(ptr(dk), ptr(dv), ptr(ka), ptr(va), n, ptr(doff),
                                            len(EDGE), begin, end, ptr(ws), ws.numel(), h)
    rs.check(st, "rs_segmented_sort_pairs")
    rs.check(rs.rs_workspace_status(ptr(ws), h)[0], "device status")
    g.check(f"segmented {dist} [{begin},{end})")
    ek, ev = oracle.segmented_sort(k, v, off, begin_bit=begin, end_bit=end)
    assert np.array_equal(host(ka if in_alt else dk, np.uint32), ek)
    assert np.array_equal(host(va if in_alt else dv, np.uint32), ev)


@pytest.mark.parametrize("kb,vb", [(4, 0), (8, 0), (8, 8)], ids=["k32", "k64", "kv64"])
def test_typed_segmented_guards_intact(kb, vb):
    lengths = EDGE + [2047, 2048, 2049]
    off = inputs.offsets_from_lengths(np.asarray(lengths, dtype=np.uint64))
    n = int(off[-1])
    dt = np.uint32 if kb == 4 else np.uint64
    k = inputs.keys(dt, "entropy16", n)
    v = inputs.values(dt, n) if vb else None
    g = Guarded()
    dk, ka = g.put(k), g.alloc(kb * n)
    dv = g.put(v) if vb else None
    va = g.alloc(vb * n) if vb else None
    doff = g.put(off.astype(np.uint64))
    st, need = rs.rs_segmented_workspace_bytes_typed(kb, vb, n, len(lengths))
    rs.check(st)
    ws = g.alloc(need)
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_segmented_sort(kb, vb, ptr(dk), ptr(dv), ptr(ka), ptr(va), n, ptr(doff),
                                      len(lengths), 0, 8 * kb, ptr(ws), ws.numel(), h)
    rs.check(st, "rs_segmented_sort")
    rs.check(rs.rs_workspace_status(ptr(ws), h)[0], "device status")
    g.check(f"typed segmented k{kb} v{vb}")
    ek, ev = oracle.segmented_sort(k, v, off)
    assert np.array_equal(host(ka if in_alt else dk, dt), ek)
    if vb:
        assert np.array_equal(host(va if in_alt else dv, dt), ev)


@pytest.mark.parametrize("n,s,b", [(5000, 16, 8), (3 * 4096 + 17, 64, 64), (2**17 + 5, 32, 256)])
def test_sample_partition_guards_intact(n, s, b):
    k = inputs.keys(np.uint32, "gaussian", n)
    v = inputs.values(np.uint32, n)
    g = Guarded()
    dk, dv, ko, vo = g.put(k), g.put(v), g.alloc(4 * n), g.alloc(4 * n)
    off, spl = g.alloc(8 * (b + 1)), g.alloc(4 * (b - 1))
    st, need = rs.rs_sample_workspace_bytes(n, s, b)
    rs.check(st)
    ws = g.alloc(need)
    h = torch.cuda.current_stream().cuda_stream
    rs.check(rs.rs_sample_partition_pairs_u32(ptr(dk), ptr(dv), ptr(ko), ptr(vo), n, s, b,
                                              ptr(off), ptr(spl), ptr(ws), ws.numel(), h))
    g.check(f"sample partition n={n}")
    ek, ev, eoff, espl = oracle.sample_partition(k, v, 4096, s, b)
    assert np.array_equal(host(ko, np.uint32), ek) and np.array_equal(host(vo, np.uint32), ev)
    assert np.array_equal(host(off, np.uint64), eoff) and np.array_equal(host(spl, np.uint32), espl)


@pytest.mark.parametrize("kb,vb", [(4, 4), (8, 0), (16, 8)], ids=["kv32", "k64", "k128v64"])
def test_merge_sort_guards_intact(kb, vb):
    for n in (2, 4095, 4097, 3 * 4096 + 5, 2**17 + 3):
        if kb == 16:
            lo = inputs.keys(np.uint64, "uniform", n)
            k = np.ascontiguousarray(np.stack([lo, lo % np.uint64(5)], axis=1))
        else:
            k = inputs.keys(np.uint32 if kb == 4 else np.uint64, "entropy16", n)
        vdt = np.uint32 if vb == 4 else np.uint64
        v = np.arange(n, dtype=vdt) if vb else None
        g = Guarded()
        dk, ka = g.put(k), g.alloc(n * kb)
        dv = g.put(v) if vb else None
        va = g.alloc(n * vb) if vb else None
        st, need = rs.rs_merge_workspace_bytes(kb, vb, n)
        rs.check(st)
        ws = g.alloc(max(need, 256))
        st, in_alt = rs.rs_merge_sort(kb, vb, ptr(dk), ptr(dv), ptr(ka), ptr(va), n, ptr(ws),
                                      ws.numel(), torch.cuda.current_stream().cuda_stream)
        rs.check(st, "rs_merge_sort")
        g.check(f"merge k{kb} v{vb} n={n}")
        ek, ev = oracle.sort_wide(k, v) if kb == 16 else oracle.lsd_sort(k, v)
        got = host(ka if in_alt else dk, np.uint64 if kb == 16 else k.dtype).reshape(k.shape)
        assert np.array_equal(got, ek)
        if vb:
            assert np.array_equal(host(va if in_alt else dv, vdt), ev)


def test_debug_build_catches_a_planted_bad_index():
    """Only in the debug build: one tile of pass 0 computes every scatter
    index past the array; the bounds checks drop those stores and
    rs_debug_status reports the key-scatter site.  The release build refuses
    the knob."""
    if not rs.debug_library():
        assert rs.rs_debug_set(rs.RS_DEBUG_BAD_INDEX_TILE, 3) == rs.RS_ERR_INVALID
        pytest.skip("the planted index runs only in the debug build")
    n = 1 << 20
    k = inputs.keys(np.uint32, "uniform", n)
    multi = [i for i in range(rs.rs_num_variants(4, 4)) if rs.rs_variant_info(4, 4, i)["kind"] in (0, 2)]
    g = Guarded()
    dk, dv = g.put(k), g.put(inputs.values(np.uint32, n))
    ka, va = g.alloc(4 * n), g.alloc(4 * n)
    st, need = rs.rs_workspace_bytes(4, 4, n, 0, 32, variant=multi[0])
    ws = g.alloc(need)
    h = torch.cuda.current_stream().cuda_stream
    assert rs.rs_debug_status()[0] == rs.RS_OK
    rs.check(rs.rs_debug_set(rs.RS_DEBUG_BAD_INDEX_TILE, 3))
    try:
        rs.check(rs.rs_sort(4, 4, ptr(dk), ptr(dv), ptr(ka), ptr(va), n, 0, 32, ptr(ws),
                            ws.numel(), h, variant=multi[0])[0])
        torch.cuda.synchronize()
        st, _, site, index = rs.rs_debug_status()
    finally:
        rs.rs_debug_set(rs.RS_DEBUG_BAD_INDEX_TILE, -1)
    assert st == rs.RS_ERR_DEVICE and site == 7 and index >= n, (st, site, index)
    for raw, nb, pat in g.regions:  # the dropped stores wrote nowhere
        assert torch.equal(raw[:GUARD], pat[:GUARD]) and torch.equal(raw[GUARD + nb:], pat[GUARD:])
    assert rs.rs_debug_status()[0] == rs.RS_OK  # read and cleared


def test_same_suites_under_the_debug_build():
    """This file's tests again, in a process that loads librs_debug.so."""
    if rs.debug_library():
        pytest.skip("already the debug build")
    env = dict(os.environ, RS_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.abspath(__file__), "-m", "gpu",
                        "-x", "-q", "-p", "no:cacheprovider", "-k", "not under_the_debug_build"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
