"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/*.h declares, and rejects bad arguments on the host before it
touches CUDA.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

from paper_1511_03404_gb300 import _build, rs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rs_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = rs.load()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same names
    assert not [n for n in names if not hasattr(rs, n) and n not in ("rs_status_string",)]


def test_built_for_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(_build.LIB_PATH)


def test_status_strings_and_version():
    assert rs.status_string(rs.RS_OK) == "RS_OK"
    assert "TIMEOUT" in rs.status_string(rs.RS_ERR_TIMEOUT)
    assert re.match(r"\d+\.\d+\.\d+", rs.rs_version())


def test_variants_described():
    for kb, vb in ((4, 0), (4, 4), (8, 0), (8, 8)):
        n = rs.rs_num_variants(kb, vb)
        assert n >= 2
        kinds = set()
        for i in range(n):
            info = rs.rs_variant_info(kb, vb, i)
            assert 4 <= info["radix_bits"] <= 8 and info["threads"] % 32 == 0
            kinds.add(info["kind"])
        assert {0, 1} <= kinds <= {0, 1, 2, 3, 4}
    assert rs.rs_num_variants(4, 8) == 0
    with pytest.raises(rs.RsError):
        rs.rs_variant_info(4, 4, 99)


def test_workspace_sizes():
    st, b = rs.rs_workspace_bytes(4, 4, 0, 0, 32)
    assert st == rs.RS_OK and b == 0
    st, b = rs.rs_workspace_bytes(4, 4, 1000, 0, 32)  # one-CTA path: no workspace
    assert st == rs.RS_OK and b == 0
    # variant 0 named explicitly: the tuned table may pick another tile shape
    st, b1 = rs.rs_workspace_bytes(4, 4, 2**26, 0, 32, variant=0)
    assert st == rs.RS_OK
    # onesweep: 256 B control + counts + offsets + look-back words of every
    # pass (per tile, plus two per group of 32 tiles)
    info = rs.rs_variant_info(4, 4, 0)
    tiles = -(-2**26 // (info["threads"] * info["items"]))
    groups = -(-tiles // 32)
    words = 4 * (tiles + 2 * groups) * 256
    assert b1 >= 4 * words + 2 * 4 * 256 * 4
    assert b1 < 4 * words + 16384
    st, b2 = rs.rs_workspace_bytes(8, 0, 2**26, 0, 64)
    assert st == rs.RS_OK and b2 > b1
    assert rs.rs_workspace_bytes(4, 4, rs.RS_MAX_N + 1, 0, 32)[0] == rs.RS_ERR_INVALID
    assert rs.rs_workspace_bytes(4, 4, 100, 0, 33)[0] == rs.RS_ERR_INVALID
    assert rs.rs_workspace_bytes(4, 8, 100, 0, 32)[0] == rs.RS_ERR_INVALID


def test_host_argument_checks_without_gpu():
    fake = 1 << 40  # never dereferenced: every call below fails its host checks
    # wrong type combination
    assert rs.rs_sort(4, 8, fake, fake + 4096, fake + 8192, fake + 12288, 100, 0, 32, None, 0,
                      None)[0] == rs.RS_ERR_INVALID
    # values given for a keys-only sort
    assert rs.rs_sort(4, 0, fake, fake + 4096, fake + 8192, None, 100, 0, 32, None, 0,
                      None)[0] == rs.RS_ERR_INVALID
    # bit range
    assert rs.rs_sort_keys_u32(fake, fake + 4096, 100, 5, 4, None, 0, None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_keys_u64(fake, fake + 4096, 100, 0, 65, None, 0, None)[0] == rs.RS_ERR_INVALID
    # too many elements
    assert rs.rs_sort_keys_u32(fake, fake + 4096, rs.RS_MAX_N + 1, 0, 32, None, 0,
                               None)[0] == rs.RS_ERR_INVALID
    # missing workspace for a multi-CTA sort
    assert rs.rs_sort_keys_u32(fake, fake + 2**30, 2**20, 0, 32, None, 0,
                               None)[0] == rs.RS_ERR_WORKSPACE
    # trivially sorted inputs return at once, in place
    assert rs.rs_sort_keys_u32(fake, fake + 4096, 1, 0, 32, None, 0, None) == (rs.RS_OK, 0)
    assert rs.rs_sort_pairs_u64(fake, fake + 8, fake + 16, fake + 24, 500, 9, 9, None, 0,
                                None) == (rs.RS_OK, 0)
    assert rs.rs_debug_set(99, 1) == rs.RS_ERR_INVALID
    assert rs.rs_profile_end()[0] == rs.RS_ERR_INVALID


def test_server_entry_points_reject_null_without_gpu():
    """The server's query and policy entry points check their arguments on
    the host: a NULL server or output is RS_ERR_INVALID, nothing is touched."""
    lib = rs.load()
    import ctypes
    out = ctypes.c_size_t()
    cfg = rs.rs_server_config(1 << 14, 1 << 22, 1 << 21, 2, 1)
    assert lib.rs_server_get_config(None, ctypes.byref(cfg)) == rs.RS_ERR_INVALID
    assert lib.rs_server_set_config(None, ctypes.byref(cfg)) == rs.RS_ERR_INVALID
    assert lib.rs_server_trace(None, None, 0, ctypes.byref(out)) == rs.RS_ERR_INVALID
    assert lib.rs_server_completed(None, None, 0, ctypes.byref(out)) == rs.RS_ERR_INVALID
    assert lib.rs_server_stats(None, None) == rs.RS_ERR_INVALID
    assert lib.rs_poll(None, 1, None) == rs.RS_ERR_INVALID


def test_noalloc_array_fits_a_compiled_shape_at_every_size():
    """rs_sort_keys_u32_noalloc takes the tuned shape when its workspace fits
    the library's fixed array, else the shape with the smallest workspace:
    some shape must fit at every accepted size, whatever the tuned table says."""
    count = rs.rs_num_variants(4, 0)
    for n in (2, 4097, 65537, 1 << 20, (1 << 22) + 3, rs.RS_NOALLOC_MAX_N):
        sizes = [rs.rs_workspace_bytes(4, 0, n, 0, 32, variant=i)[1] for i in range(count)
                 if rs.rs_variant_info(4, 0, i)["max_n"] >= n]
        assert sizes and min(sizes) <= rs.RS_NOALLOC_SCRATCH_BYTES, n


def test_host_buffer_sort_checks_arguments_before_enqueuing():
    fake = 1 << 40  # never dereferenced: every call below fails its host checks
    h = 1 << 41
    # wrong type combination
    assert rs.rs_sort_host(4, 8, h, h, h, h, 100, 0, 32, fake, fake + 4096, fake + 8192,
                           fake + 12288, None, 0, None)[0] == rs.RS_ERR_INVALID
    # host values without a value type, and a missing host output
    assert rs.rs_sort_host(4, 0, h, h, h, None, 100, 0, 32, fake, None, fake + 4096, None, None,
                           0, None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_host(4, 0, h, None, None, None, 100, 0, 32, fake, None, fake + 4096, None,
                           None, 0, None)[0] == rs.RS_ERR_INVALID
    # same key buffer twice, bad bit range, too many elements
    assert rs.rs_sort_host(4, 0, h, None, h, None, 100, 0, 32, fake, None, fake, None, None, 0,
                           None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_host(4, 0, h, None, h, None, 100, 0, 40, fake, None, fake + 4096, None,
                           None, 0, None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_host(4, 0, h, None, h, None, rs.RS_MAX_N + 1, 0, 32, fake, None,
                           fake + 2**33, None, None, 0, None)[0] == rs.RS_ERR_INVALID
    # misaligned keys, a bad key order
    assert rs.rs_sort_host(8, 0, h, None, h, None, 100, 0, 64, fake + 4, None, fake + 4096, None,
                           None, 0, None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_sort_host(4, 0, h, None, h, None, 100, 0, 32, fake, None, fake + 4096, None,
                           None, 0, None, key_kind=7)[0] == rs.RS_ERR_INVALID
    # missing workspace for a multi-CTA sort
    assert rs.rs_sort_host(4, 0, h, None, h, None, 2**20, 0, 32, fake, None, fake + 2**30, None,
                           None, 0, None)[0] == rs.RS_ERR_WORKSPACE


def test_stats_entry_rejects_null_output():
    lib = rs.load()
    assert lib.rs_workspace_stats(None, None, None) == rs.RS_ERR_INVALID


def test_typed_segmented_sort_checks_arguments_without_gpu():
    fake = 1 << 40
    ok = rs.rs_segmented_workspace_bytes_typed
    assert ok(4, 8, 100, 2)[0] == rs.RS_ERR_INVALID
    assert ok(8, 0, 100, 2, 0, 65)[0] == rs.RS_ERR_INVALID
    assert ok(8, 8, 100, 2)[0] == rs.RS_OK
    # values given for keys only, missing values for pairs, same buffer twice
    assert rs.rs_segmented_sort(8, 0, fake, fake + 8192, fake + 4096, None, 100, fake, 2, 0, 64,
                                None, 0, None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_segmented_sort(4, 4, fake, None, fake + 4096, None, 100, fake, 2, 0, 32, None, 0,
                                None)[0] == rs.RS_ERR_INVALID
    assert rs.rs_segmented_sort(4, 0, fake, None, fake, None, 100, fake, 2, 0, 32, None, 0,
                                None)[0] == rs.RS_ERR_INVALID


_DEFAULT_TABLE_PROBE = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
from paper_1511_03404_gb300 import _build, rs
lib = ctypes.CDLL(_build.LIB_PATH)  # the library alone: the binding installs nothing
lib.rs_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
def ws(kb, vb, n, variant=-1):
    out = ctypes.c_size_t()
    cfg = None if variant < 0 else ctypes.byref(rs.rs_config(0, variant, 0, 0))
    assert lib.rs_workspace_bytes(kb, vb, n, 0, 8 * kb, cfg, ctypes.byref(out)) == 0
    return out.value
table = json.load(open(rs.TUNED_TABLE))
rows = []
for e in table["entries"]:
    if e.get("ms") is None:
        continue
    n = int(e["n_max"])
    rows.append([ws(e["key_bytes"], e["val_bytes"], n), ws(e["key_bytes"], e["val_bytes"], n, e["variant"])])
print(json.dumps(rows))
"""


def _default_table_rows(env_extra):
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k != "RS_NO_TUNED_TABLE"}
    env.update(env_extra)
    res = subprocess.run([sys.executable, "-c", _DEFAULT_TABLE_PROBE, ROOT], capture_output=True,
                         text=True, env=env, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_library_starts_with_the_tuned_table():
    """A C caller that never installs a table gets the tuned choices: with no
    configuration, every tuned size sorts with the table's variant (seen
    through its workspace size), which the build compiled in from
    tuned.json; RS_NO_TUNED_TABLE turns the built-in table off."""
    rows = _default_table_rows({})
    assert rows and all(default == tuned for default, tuned in rows)
    off = _default_table_rows({"RS_NO_TUNED_TABLE": "1"})
    # without the table the built-in choice differs from the tuned one somewhere
    assert any(default != tuned for default, tuned in off)
