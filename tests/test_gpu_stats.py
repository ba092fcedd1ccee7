"""Per-call statistics (rs_workspace_stats), the host-buffer entry point
(rs_sort_host) and the NVTX switch, on the GPU through the C ABI.

The stats record which digit passes of Sec. 2.6 moved the data and which
were skipped because one digit value held every key; with 64-bit keys that
carry 16 random bits, six of the eight 8-bit passes are skipped.  The
host-buffer sort is compared with the oracle bit for bit."""
import os
import subprocess
import sys

import numpy as np
import pytest

import inputs
import oracle

torch = pytest.importorskip("torch")
from gpu_util import from_dev, to_dev  # noqa: E402

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sort_and_stats(kb, vb, k, variant=-1):
    n = k.size
    dk = to_dev(k, torch)
    ka = torch.empty_like(dk)
    dv = va = None
    if vb:
        dv = torch.arange(n, dtype=dk.dtype, device="cuda")
        va = torch.empty_like(dv)
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb, variant=variant)
    rs.check(st)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    ws.fill_(0xA5)  # the record must not depend on what the workspace held
    h = torch.cuda.current_stream().cuda_stream
    st, in_alt = rs.rs_sort(kb, vb, dk.data_ptr(), dv.data_ptr() if vb else None, ka.data_ptr(),
                            va.data_ptr() if vb else None, n, 0, 8 * kb, ws.data_ptr(),
                            ws.numel(), h, variant=variant)
    rs.check(st, "rs_sort")
    st, s = rs.rs_workspace_stats(ws.data_ptr(), h)
    rs.check(st, "rs_workspace_stats")
    out = from_dev(ka if in_alt else dk, k.dtype)
    return s, out


def test_skipped_passes_of_16_bit_entropy_u64_keys():
    n = 1 << 24
    k = inputs.keys(np.uint64, "entropy16", n)
    s, out = sort_and_stats(8, 0, k)
    assert s["status"] == rs.RS_OK and s["form"] in (1, 2)
    assert s["passes"] == 8 and s["n"] == n and s["key_bytes"] == 8 and s["val_bytes"] == 0
    assert s["moved_mask"] == 0b11 and s["skipped_mask"] == 0b11111100
    assert all(t > 0 for t in s["pass_ms"][:2]) and all(t == 0 for t in s["pass_ms"][2:])
    assert s["bytes"] == n * 8 + 2 * (2 * n * 8)
    assert 0 < s["upsweep_ms"] < s["total_ms"] < 1000
    assert np.array_equal(out, np.sort(k))


def test_every_pass_moves_uniform_u32_pairs():
    n = 1 << 22
    k = inputs.keys(np.uint32, "uniform", n)
    s, _ = sort_and_stats(4, 4, k)
    assert s["form"] in (1, 2) and s["moved_mask"] == 0xF and s["skipped_mask"] == 0
    assert all(t > 0 for t in s["pass_ms"]) and s["bytes"] == n * 4 + 4 * 2 * n * 8
    assert s["total_ms"] >= max(s["pass_ms"])


def test_zero_keys_skip_every_pass():
    """All keys equal: no pass moves data (4 skipped, an even count, so the
    result stays in place), and the record says so."""
    n = 1 << 21
    s, out = sort_and_stats(4, 4, np.zeros(n, dtype=np.uint32))
    assert s["form"] in (1, 2) and s["moved_mask"] == 0 and s["skipped_mask"] == 0xF


@pytest.mark.parametrize("kind,form", [(3, 2), (4, 3), (2, 1)],
                         ids=["one_launch", "cluster", "resident_ctas"])
def test_record_of_every_sort_form(kind, form):
    """The record of the one-launch (cooperative), cluster and resident-CTA
    forms: shape, moved passes and times, and the same sorted result."""
    for kb, vb in ((4, 0), (4, 4), (8, 0), (8, 8)):
        cands = [i for i in range(rs.rs_num_variants(kb, vb))
                 if rs.rs_variant_info(kb, vb, i)["kind"] == kind]
        if not cands:
            continue
        info = rs.rs_variant_info(kb, vb, cands[0])
        n = min(info["max_n"], 3 * info["threads"] * info["items"] + 77)
        dt = np.uint32 if kb == 4 else np.uint64
        k = inputs.keys(dt, "uniform", n, seed=17)
        s, out = sort_and_stats(kb, vb, k, variant=cands[0])
        passes = 8 * kb // info["radix_bits"]
        assert s["form"] == form and s["n"] == n and s["passes"] == passes, (kb, vb, s)
        assert s["key_bytes"] == kb and s["val_bytes"] == vb
        assert s["moved_mask"] == (1 << passes) - 1 and s["total_ms"] > 0
        if form != 3:
            assert all(t > 0 for t in s["pass_ms"]) and s["upsweep_ms"] > 0
            assert s["bytes"] == n * kb + passes * 2 * n * (kb + vb)
        else:
            assert s["bytes"] == 2 * n * (kb + vb)
        assert np.array_equal(out, oracle.lsd_sort(k)[0])


def test_one_cta_and_no_op_records():
    k = inputs.keys(np.uint32, "uniform", 3000)
    small = [i for i in range(rs.rs_num_variants(4, 0)) if rs.rs_variant_info(4, 0, i)["kind"] == 1]
    s, out = sort_and_stats(4, 0, k, variant=small[0])
    assert s["form"] == 3 and s["moved_mask"] == 0xF and s["n"] == 3000
    assert np.array_equal(out, np.sort(k))
    s, _ = sort_and_stats(4, 0, k[:1])
    assert s["form"] == 0 and s["status"] == rs.RS_OK


@pytest.mark.parametrize("kb,vb", [(4, 0), (4, 4), (8, 0), (8, 8)])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_buffer_sort_matches_oracle(kb, vb, pinned):
    dt = np.uint32 if kb == 4 else np.uint64
    n = 3 * 2**19 + 123
    k = inputs.keys(dt, "gaussian", n)
    v = inputs.values(dt, n) if vb else None
    sdt = torch.int32 if kb == 4 else torch.int64
    hk = torch.from_numpy(k.view(np.int32 if kb == 4 else np.int64).copy())
    hv = torch.from_numpy(v.view(np.int32 if kb == 4 else np.int64).copy()) if vb else None
    ok, ov = torch.empty_like(hk), (torch.empty_like(hv) if vb else None)
    if pinned:
        hk, ok = hk.pin_memory(), ok.pin_memory()
        if vb:
            hv, ov = hv.pin_memory(), ov.pin_memory()
    dk = torch.empty(n, dtype=sdt, device="cuda")
    ka = torch.empty_like(dk)
    dv = torch.empty_like(dk) if vb else None
    va = torch.empty_like(dk) if vb else None
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    st, in_alt = rs.rs_sort_host(kb, vb, p(hk), p(hv), p(ok), p(ov), n, 0, 8 * kb, p(dk), p(dv),
                                 p(ka), p(va), p(ws), ws.numel(), s.cuda_stream)
    rs.check(st, "rs_sort_host")
    rs.check(rs.rs_workspace_status(p(ws), s.cuda_stream)[0], "device status")
    ek, ev = oracle.lsd_sort(k, v)
    assert np.array_equal(ok.numpy().view(dt), ek)
    if vb:
        assert np.array_equal(ov.numpy().view(dt), ev)
    # the device buffers it names hold the same result
    assert np.array_equal(from_dev(ka if in_alt else dk, dt), ek)


def test_host_buffer_pipeline_on_three_streams():
    """Calls on three streams with their own buffers overlap copy-in, sort
    and copy-out; every step's output is the stable sort of its input."""
    n = 1 << 21
    sets = []
    for j in range(3):
        k = inputs.keys(np.uint32, ("uniform", "bucket", "sorted_desc")[j], n)
        hk = torch.from_numpy(k.view(np.int32).copy()).pin_memory()
        hv = torch.arange(n, dtype=torch.int32).pin_memory()
        d = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(4)]
        st, need = rs.rs_workspace_bytes(4, 4, n, 0, 32)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        sets.append((k, hk, hv, torch.empty_like(hk).pin_memory(), torch.empty_like(hv).pin_memory(),
                     d, ws, torch.cuda.Stream()))
    for _ in range(2):
        for k, hk, hv, ok, ov, d, ws, s in sets:
            st, _ = rs.rs_sort_host(4, 4, hk.data_ptr(), hv.data_ptr(), ok.data_ptr(),
                                    ov.data_ptr(), n, 0, 32, d[0].data_ptr(), d[1].data_ptr(),
                                    d[2].data_ptr(), d[3].data_ptr(), ws.data_ptr(), ws.numel(),
                                    s.cuda_stream)
            rs.check(st, "rs_sort_host")
    torch.cuda.synchronize()
    for k, hk, hv, ok, ov, d, ws, s in sets:
        ek, ev = oracle.lsd_sort(k, np.arange(n, dtype=np.uint32))
        assert np.array_equal(ok.numpy().view(np.uint32), ek)
        assert np.array_equal(ov.numpy().view(np.uint32), ev)


def test_nvtx_ranges_switch():
    """With RS_NVTX set the library opens NVTX ranges around its calls and
    launches (no tool attached: they cost a check); the sort is unchanged."""
    code = ("import sys, numpy as np, torch; sys.path.insert(0, %r); sys.path.insert(0, %r); "
            "import inputs, oracle; from paper_1511_03404_gb300 import rs; "
            "k = inputs.keys(np.uint32, 'uniform', 1 << 20); "
            "out = rs.sort(torch.from_numpy(k.view(np.int32)).cuda(), key_kind=rs.RS_KEY_UNSIGNED)[0]; "
            "assert np.array_equal(out.cpu().numpy().view(np.uint32), np.sort(k)); print('ok')"
            % (ROOT, os.path.join(ROOT, "tests")))
    env = dict(os.environ, RS_NVTX="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]
