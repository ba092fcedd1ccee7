"""Helpers for the GPU tests: move numpy arrays to torch device tensors with
the same bits, and run one sort through the C ABI (include/rs.h)."""
from __future__ import annotations

import numpy as np

from paper_1511_03404_gb300 import rs

SIGNED = {4: np.int32, 8: np.int64}


def to_dev(a: np.ndarray, torch, device="cuda"):
    """Device tensor with the bits of ``a`` (uint32/uint64 viewed as int32/int64)."""
    return torch.from_numpy(np.ascontiguousarray(a).view(SIGNED[a.dtype.itemsize])).to(device)


def from_dev(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def sort_via_abi(torch, keys: np.ndarray, vals: np.ndarray | None = None, begin_bit=0,
                 end_bit=None, radix_bits=0, variant=-1, api="generic", stream=None,
                 offset_elems=0, check_status=True, key_kind=0, descending=False):
    """Sort host arrays on the GPU through the C ABI; returns host arrays.

    ``offset_elems`` places the arrays that many elements into larger device
    buffers (unaligned starts).  ``api`` picks rs_sort or the typed entry
    point (rs_sort_keys_u32 ...).
    """
    kb = keys.dtype.itemsize
    vb = 0 if vals is None else vals.dtype.itemsize
    n = keys.size
    end_bit = 8 * kb if end_bit is None else end_bit
    off = offset_elems
    pad = np.zeros(off, dtype=keys.dtype)
    dk_full = to_dev(np.concatenate([pad, keys]), torch)
    dk = dk_full[off:]
    ka_full = torch.empty(n + off, dtype=dk.dtype, device=dk.device)
    ka = ka_full[off:]
    dv = va = None
    if vb:
        dv = to_dev(np.concatenate([pad.astype(vals.dtype), vals]), torch)[off:]
        va = torch.empty(n + off, dtype=dv.dtype, device=dv.device)[off:]
    st, nbytes = rs.rs_workspace_bytes(kb, vb, n, begin_bit, end_bit, radix_bits, variant)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dk.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    h = s.cuda_stream
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    if api == "generic" or radix_bits or variant >= 0 or key_kind or descending:
        st, in_alt = rs.rs_sort(kb, vb, ptr(dk), ptr(dv), ptr(ka), ptr(va), n, begin_bit,
                                end_bit, ws.data_ptr(), ws.numel(), h, radix_bits, variant,
                                key_kind, descending)
    else:
        fn = {(4, 0): rs.rs_sort_keys_u32, (8, 0): rs.rs_sort_keys_u64,
              (4, 4): rs.rs_sort_pairs_u32, (8, 8): rs.rs_sort_pairs_u64}[(kb, vb)]
        if vb:
            st, in_alt = fn(ptr(dk), ptr(dv), ptr(ka), ptr(va), n, begin_bit, end_bit,
                            ws.data_ptr(), ws.numel(), h)
        else:
            st, in_alt = fn(ptr(dk), ptr(ka), n, begin_bit, end_bit, ws.data_ptr(),
                            ws.numel(), h)
    rs.check(st, "sort")
    dev_st, info = rs.rs_workspace_status(ws.data_ptr(), h)
    if check_status:
        rs.check(dev_st, f"device status (info {info})")
    out_k = from_dev(ka if in_alt else dk, keys.dtype)
    out_v = from_dev(va if in_alt else dv, vals.dtype) if vb else None
    return out_k, out_v, in_alt
