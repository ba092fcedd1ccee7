"""rs_sort_keys_u32_noalloc: the 32-bit key sort for callers that cannot
allocate device memory (a framework that owns every device byte, a real-time
or callback context, memory reserved once at start-up).  Its scratch is a
fixed device array inside the library instead of a caller workspace.

It is compared, through the C ABI, with the existing entry point
rs_sort_keys_u32 (which takes a caller-allocated workspace) on two calls in
a row, so the second call runs on the array as the first one left it.  Keys
are integers, so the tolerance is zero: the outputs must be identical.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import inputs

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
    torch.cuda.synchronize()
    return from_dev(ka if in_alt else dk, np.uint32)


def test_noalloc_matches_existing_entry_on_two_calls_in_a_row():
    cases = [("uniform", 3 * 2**20 + 5, 0, 32), ("gaussian", rs.RS_NOALLOC_MAX_N, 0, 32),
             ("entropy16", 100003, 0, 24), ("bucket", 5000, 0, 32)]
    for dist, n, b, e in cases:
        k = inputs.keys(np.uint32, dist, n)
        want = sort_existing(k, b, e)
        first = sort_noalloc(k, b, e)
        second = sort_noalloc(k, b, e)
        assert np.array_equal(first, want), (dist, n)
        assert np.array_equal(second, want), (dist, n)


def test_noalloc_rejects_sizes_beyond_its_array():
    n = rs.RS_NOALLOC_MAX_N + 1
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    a = torch.empty_like(d)
    st, _ = rs.rs_sort_keys_u32_noalloc(d.data_ptr(), a.data_ptr(), n, 0, 32,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == rs.RS_ERR_INVALID
