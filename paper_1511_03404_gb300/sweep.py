"""Sort-rate sweep in the format of the paper's experiments (Sec. 3-4).

For every key type (32-bit keys, 32-bit pairs, 64-bit keys, 64-bit pairs),
every input distribution of Sec. 4 and every length n = 2^e and
2^e + 2^(e-1) (e = 15 .. 25 for 32-bit keys, 15 .. 24 for 64-bit keys, as
in Sec. 3), the sort is timed as the paper times it: only the sort (the
input is already on the device; a device-to-device copy of the pristine
input runs before each repetition, outside the CUDA events), repeated
``reps`` times (50 in the paper), reporting the median and the mean.  Each
case's output is checked on the device: keys non-decreasing and, for pairs,
equal keys keep their input order (the values are the input indices).

    python -m paper_1511_03404_gb300.sweep [--reps 50] [--types k32,kv32,k64,kv64]
        [--dists uniform,...] [--max-log2 25] [--out sweep.json] [--markdown sweep.md]

The rate is n / median time, in Mkeys/s (the paper's unit).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

from . import rs

TYPES = {"k32": (4, 0), "kv32": (4, 4), "k64": (8, 0), "kv64": (8, 8)}
DISTS = ("uniform", "gaussian", "zero", "bucket", "sorted", "sorted_desc")
MAX_LOG2 = {4: 25, 8: 24}


def lengths(key_bytes: int, max_log2: int | None = None) -> list[int]:
    top = MAX_LOG2[key_bytes] if max_log2 is None else min(max_log2, MAX_LOG2[key_bytes])
    out = []
    for e in range(15, top + 1):
        out.append(1 << e)
        if e < top:
            out.append((1 << e) + (1 << (e - 1)))
    return out


def _as_ordered(torch, t):
    """Signed view whose order is the unsigned order of t's bits."""
    top = -(1 << 31) if t.dtype == torch.int32 else -(1 << 63)
    return t ^ top


def check_output(torch, keys, vals) -> bool:
    o = _as_ordered(torch, keys)
    if keys.numel() < 2:
        return True
    if not bool((o[1:] >= o[:-1]).all()):
        return False
    if vals is not None:
        eq = o[1:] == o[:-1]
        if not bool((vals[1:][eq] > vals[:-1][eq]).all()):
            return False
    return True


def time_case(torch, key_bytes, val_bytes, keys_h, reps, stream):
    """Median and mean (ms) of ``reps`` CUDA-event timed sorts, and the check."""
    dev = torch.device("cuda")
    sdt = torch.int32 if key_bytes == 4 else torch.int64
    n = keys_h.size
    base = torch.from_numpy(keys_h.view(np.int32 if key_bytes == 4 else np.int64)).to(dev)
    vals0 = torch.arange(n, dtype=sdt, device=dev) if val_bytes else None
    k = torch.empty_like(base)
    ka = torch.empty_like(base)
    v = torch.empty_like(vals0) if val_bytes else None
    va = torch.empty_like(vals0) if val_bytes else None
    st, need = rs.rs_workspace_bytes(key_bytes, val_bytes, n, 0, 8 * key_bytes)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    h = stream.cuda_stream
    times = []
    in_alt = 0
    with torch.cuda.stream(stream):
        for r in range(reps + 1):
            k.copy_(base)
            if val_bytes:
                v.copy_(vals0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, in_alt = rs.rs_sort(key_bytes, val_bytes, k.data_ptr(),
                                    v.data_ptr() if val_bytes else None, ka.data_ptr(),
                                    va.data_ptr() if val_bytes else None, n, 0, 8 * key_bytes,
                                    ws.data_ptr(), ws.numel(), h)
            e1.record(stream)
            rs.check(st, "rs_sort")
            e1.synchronize()
            if r:  # the first run warms up
                times.append(e0.elapsed_time(e1))
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    ok = check_output(torch, ka if in_alt else k, (va if in_alt else v) if val_bytes else None)
    return statistics.median(times), statistics.fmean(times), ok


def sweep(types=tuple(TYPES), dists=DISTS, reps=50, max_log2=None, log=None):
    import torch

    import inputs

    rs.load()
    stream = torch.cuda.Stream()
    rows = []
    for tname in types:
        kb, vb = TYPES[tname]
        udt = np.uint32 if kb == 4 else np.uint64
        for dist in dists:
            for n in lengths(kb, max_log2):
                keys_h = inputs.keys(udt, dist, n)
                med, mean, ok = time_case(torch, kb, vb, keys_h, reps, stream)
                row = {"type": tname, "dist": dist, "n": n, "median_ms": med, "mean_ms": mean,
                       "mkeys_per_s": n / med / 1e3, "ok": ok}
                rows.append(row)
                if log:
                    log(f"{tname:5s} {dist:12s} n={n:>9d} {med:9.4f} ms "
                        f"{row['mkeys_per_s']:10.1f} Mkeys/s {'ok' if ok else 'WRONG'}")
    return {"device": torch.cuda.get_device_name(0), "reps": reps,
            "timing": "median / mean of CUDA-event timed sorts, input restored outside the "
                      "events before each, first run discarded", "rows": rows}


def markdown(result) -> str:
    """One table per key type: rows n, columns the distributions, Mkeys/s."""
    out = []
    rows = result["rows"]
    for tname in dict.fromkeys(r["type"] for r in rows):
        sub = [r for r in rows if r["type"] == tname]
        dists = list(dict.fromkeys(r["dist"] for r in sub))
        ns = sorted(set(r["n"] for r in sub))
        out.append(f"**{tname}** (Mkeys/s, median of {result['reps']})\n")
        out.append("| n | " + " | ".join(dists) + " |")
        out.append("|---|" + "---|" * len(dists))
        for n in ns:
            cells = []
            for d in dists:
                r = next(x for x in sub if x["n"] == n and x["dist"] == d)
                cells.append(f"{r['mkeys_per_s']:.0f}" + ("" if r["ok"] else " (WRONG)"))
            e = n.bit_length() - 1
            label = f"2^{e}" if n == 1 << e else f"2^{e}+2^{e - 1}"
            out.append(f"| {label} | " + " | ".join(cells) + " |")
        out.append("")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--types", default=",".join(TYPES))
    ap.add_argument("--dists", default=",".join(DISTS))
    ap.add_argument("--max-log2", type=int, default=None)
    ap.add_argument("--out", default=None, help="write the rows as JSON")
    ap.add_argument("--markdown", default=None, help="write the tables as markdown")
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    res = sweep(args.types.split(","), args.dists.split(","), args.reps, args.max_log2,
                log=lambda s: print(s, flush=True))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    md = markdown(res)
    if args.markdown:
        with open(args.markdown, "w") as f:
            f.write(md + "\n")
    print(md)
    bad = [r for r in res["rows"] if not r["ok"]]
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
