"""rs_sort_keys_u32_noalloc: the 32-bit key sort for callers that cannot
allocate device memory where they sort -- a framework that owns every device
byte through its own pool, a real-time or callback context where an
allocation could block or synchronize, memory reserved once at start-up.
Its scratch is a fixed device array inside the library instead of a caller
workspace.

It is compared, through the C ABI, with the existing entry point
rs_sort_keys_u32 (which takes a caller-allocated workspace) and with the
oracle, on two calls in a row, so the second call runs on the array as the
first one left it; after every call its device status is read back through
rs_sort_keys_u32_noalloc_status.  Keys are integers, so the tolerance is
zero: the outputs must be identical.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
from gpu_util import from_dev, to_dev  # noqa: E402

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu


def sort_existing(k, begin_bit, end_bit):
    dk = to_dev(k, torch)
    ka = torch.empty_like(dk)
    st, need = rs.rs_workspace_bytes(4, 0, k.size, begin_bit, end_bit)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort_keys_u32(dk.data_ptr(), ka.data_ptr(), k.size, begin_bit, end_bit,
                                     ws.data_ptr(), ws.numel(), h)
    rs.check(st, "rs_sort_keys_u32")
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    return from_dev(ka if in_alt else dk, np.uint32)


def sort_noalloc(k, begin_bit, end_bit):
    dk = to_dev(k, torch)
    ka = torch.empty_like(dk)
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort_keys_u32_noalloc(dk.data_ptr(), ka.data_ptr(), k.size, begin_bit,
                                             end_bit, h)
    rs.check(st, "rs_sort_keys_u32_noalloc")
    st, info = rs.rs_sort_keys_u32_noalloc_status(h)
    rs.check(st, f"rs_sort_keys_u32_noalloc device status (info {info})")
    return from_dev(ka if in_alt else dk, np.uint32)


CASES = [("uniform", 3 * 2**20 + 5, 0, 32), ("gaussian", rs.RS_NOALLOC_MAX_N, 0, 32),
         ("entropy16", 100003, 0, 24), ("bucket", 5000, 0, 32)]


def test_noalloc_matches_existing_entry_on_two_calls_in_a_row():
    for dist, n, b, e in CASES:
        k = inputs.keys(np.uint32, dist, n)
        want = sort_existing(k, b, e)
        first = sort_noalloc(k, b, e)
        second = sort_noalloc(k, b, e)
        assert np.array_equal(first, want), (dist, n)
        assert np.array_equal(second, want), (dist, n)
        ek, _ = oracle.lsd_sort(k, None, begin_bit=b, end_bit=e)
        assert np.array_equal(first, ek), (dist, n)


def test_noalloc_keeps_to_its_array_whatever_the_tuned_table_says():
    """A tuned table that picks, for the largest accepted size, a tile shape
    whose workspace is larger than the array: the entry point takes a shape
    that fits instead and still sorts correctly."""
    n = rs.RS_NOALLOC_MAX_N
    big = [i for i in range(rs.rs_num_variants(4, 0))
           if rs.rs_variant_info(4, 0, i)["max_n"] >= n
           and rs.rs_workspace_bytes(4, 0, n, 0, 32, variant=i)[1] > rs.RS_NOALLOC_SCRATCH_BYTES]
    if not big:
        pytest.skip("every compiled shape fits the array")
    try:
        rs.check(rs.rs_tune_set(4, 0, n, big[0]))
        assert rs.rs_workspace_bytes(4, 0, n, 0, 32)[1] > rs.RS_NOALLOC_SCRATCH_BYTES
        k = inputs.keys(np.uint32, "uniform", n, seed=7)
        first = sort_noalloc(k, 0, 32)
        second = sort_noalloc(k, 0, 32)
    finally:
        rs.rs_tune_clear()
        rs._apply_tuned_table(rs.load())
    want = sort_existing(k, 0, 32)
    assert np.array_equal(first, want) and np.array_equal(second, want)


def test_noalloc_rejects_sizes_beyond_its_array():
    n = rs.RS_NOALLOC_MAX_N + 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    a = torch.empty_like(d)
    st, _ = rs.rs_sort_keys_u32_noalloc(d.data_ptr(), a.data_ptr(), n, 0, 32,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == rs.RS_ERR_INVALID
