"""GPU parity of the key orders beyond unsigned keys (signed integers,
IEEE-754 floats, descending order) against the oracle's ordered sort, bit
for bit, through the C ABI.  The transform is applied by the first digit
pass that moves data and undone by the last one, so the cases include
inputs whose low or high digit passes are skipped, arrays small enough for
the one-CTA path, ragged multi-tile arrays and every compiled variant."""
import numpy as np
import pytest

import inputs
import oracle
from gpu_util import sort_via_abi

torch = pytest.importorskip("torch")

from paper_1511_03404_gb300 import rs  # noqa: E402

pytestmark = pytest.mark.gpu

U = {4: np.uint32, 8: np.uint64}
S = {4: np.int32, 8: np.int64}
KINDS = [(oracle.KEY_UNSIGNED, True), (oracle.KEY_SIGNED, False), (oracle.KEY_SIGNED, True),
         (oracle.KEY_FLOAT, False), (oracle.KEY_FLOAT, True)]
KIND_IDS = ["unsigned_desc", "signed", "signed_desc", "float", "float_desc"]


def make_keys(nb, kind, n, flavour, seed=1):
    """Bit patterns for the case: 'wide' spreads over all digit passes;
    'narrow' keeps the high passes constant (they are skipped); 'lowconst'
    keeps the low byte constant (the first pass is skipped)."""
    u = U[nb]
    if kind == oracle.KEY_FLOAT:
        k = inputs.float_keys(u, n, seed=seed)
        if flavour == "narrow":  # small integers as floats: few distinct high bytes
            k = (inputs.keys(u, "entropy16", n, seed) % u(200)).astype(np.float64) - 100.0
            k = k.astype(np.float32 if nb == 4 else np.float64).view(u)
    else:
        k = inputs.keys(u, "uniform", n, seed)
        if flavour == "narrow":
            k = ((inputs.keys(u, "entropy16", n, seed).astype(np.int64) % 2001) - 1000)
            k = k.astype(S[nb]).view(u)
    if flavour == "lowconst":
        k = (k & ~u(0xFF)) | u(0x5A)
    return np.ascontiguousarray(k)


def check(nb, pairs, kind, desc, n, flavour="wide", **kw):
    k = make_keys(nb, kind, n, flavour)
    v = inputs.values(U[nb], n) if pairs else None
    gk, gv, _ = sort_via_abi(torch, k, v, key_kind=kind, descending=desc, **kw)
    ek, ev = oracle.ordered_sort(k, v, kind=kind, descending=desc,
                                 begin_bit=kw.get("begin_bit", 0), end_bit=kw.get("end_bit"))
    assert np.array_equal(gk, ek), (nb, pairs, kind, desc, n, flavour, kw)
    if pairs:
        assert np.array_equal(gv, ev), (nb, pairs, kind, desc, n, flavour, kw)


@pytest.mark.parametrize("nb,pairs", [(4, False), (4, True), (8, False), (8, True)],
                         ids=["k32", "kv32", "k64", "kv64"])
@pytest.mark.parametrize("kind,desc", KINDS, ids=KIND_IDS)
def test_key_orders_default_choice(nb, pairs, kind, desc):
    for n in (0, 1, 2, 33, 4095, 4097, 3 * 2**12 + 5, 2**17 + 3, 2**20 + 7):
        for flavour in ("wide", "narrow", "lowconst"):
            check(nb, pairs, kind, desc, n, flavour)


@pytest.mark.parametrize("nb,pairs", [(4, False), (4, True), (8, False), (8, True)],
                         ids=["k32", "kv32", "k64", "kv64"])
def test_key_orders_every_variant(nb, pairs):
    vb = nb if pairs else 0
    for i in range(rs.rs_num_variants(nb, vb)):
        info = rs.rs_variant_info(nb, vb, i)
        tile = info["threads"] * info["items"]
        n = min(info["max_n"], 7 * tile + 13)
        for kind, desc in ((oracle.KEY_FLOAT, False), (oracle.KEY_SIGNED, True)):
            check(nb, pairs, kind, desc, n, variant=i)
            check(nb, pairs, kind, desc, n, "narrow", variant=i)


def test_key_order_bit_range():
    # the bits of the transformed key: descending on [8, 24), signed on [0, 12)
    check(4, True, oracle.KEY_UNSIGNED, True, 50001, begin_bit=8, end_bit=24)
    check(8, False, oracle.KEY_SIGNED, False, 30001, begin_bit=0, end_bit=12)


def test_key_order_arguments():
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    a = torch.empty_like(d)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    h = torch.cuda.current_stream().cuda_stream
    for kind, desc in ((3, 0), (-1, 0), (0, 2)):
        st, _ = rs.rs_sort(4, 0, d.data_ptr(), None, a.data_ptr(), None, 16, 0, 32,
                           ws.data_ptr(), ws.numel(), h, 0, -1, kind, desc)
        assert st == rs.RS_ERR_INVALID


def test_torch_convenience_orders():
    g = torch.Generator().manual_seed(3)
    x = torch.randn(100003, generator=g).to("cuda")
    x[::97] = -0.0
    y = x.clone()
    rs.sort(y)
    ref = np.sort(x.cpu().numpy(), kind="stable")
    assert np.array_equal(y.cpu().numpy(), ref)  # equal as numbers (-0.0 == 0.0)
    i = torch.randint(-2**31, 2**31 - 1, (70001,), generator=g, dtype=torch.int64).to(torch.int32)
    di = i.to("cuda")
    idx = torch.arange(i.numel(), dtype=torch.int32, device="cuda")
    rs.sort(di, idx, descending=True)
    perm = np.argsort(-i.numpy().astype(np.int64), kind="stable")
    assert np.array_equal(idx.cpu().numpy(), perm)
