"""Autotuner: pick the compiled variant (digit width, tile shape, items per
thread) of each data type for each size band, on the GPU at hand.

For every (key bytes, value bytes) and every size n of the sweep, each
compiled variant that can sort n is timed on uniform keys (median of a few
CUDA-event timed sorts, inputs restored before each, outside the events).
The fastest variant of size n becomes the table entry "n_max = n"; a sort of
m elements then uses the entry with the smallest n_max >= m.  The variant of
the largest size swept also gets an entry up to the largest sortable array,
so that larger sorts keep the tile shape that won at the top of the sweep
(without it the library's built-in choice would apply there).  The table is written to
``tuned.json`` next to this file, which the binding loads at start-up.

    python -m paper_1511_03404_gb300.autotune [--quick] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

from . import rs

TYPES = ((4, 0), (4, 4), (8, 0), (8, 8))
# the lengths of the paper's grid (Sec. 3): 2^e and 2^e + 2^(e-1); a band per
# half octave, so that no length of the grid falls between two measured sizes
SIZES = tuple(sorted({2**e for e in range(12, 27)} | {2**e + 2**(e - 1) for e in range(12, 26)}))


def _time_variant(torch, kb, vb, n, variant, keys, vals, reps):
    dk = torch.empty_like(keys)
    ka = torch.empty_like(keys)
    dv = torch.empty_like(vals) if vb else None
    va = torch.empty_like(vals) if vb else None
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb, 0, variant)
    if st != rs.RS_OK:
        return None
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=keys.device)
    stream = torch.cuda.current_stream()
    h = stream.cuda_stream
    times = []
    for r in range(reps + 1):
        dk.copy_(keys)
        if vb:
            dv.copy_(vals)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = rs.rs_sort(kb, vb, dk.data_ptr(), dv.data_ptr() if vb else None, ka.data_ptr(),
                           va.data_ptr() if vb else None, n, 0, 8 * kb, ws.data_ptr(),
                           ws.numel(), h, 0, variant)
        e1.record(stream)
        rs.check(st, "rs_sort (autotune)")
        torch.cuda.synchronize()
        if r:  # the first run warms up
            times.append(e0.elapsed_time(e1))
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "autotune device status")
    return statistics.median(times)


def tune(sizes=SIZES, types=TYPES, reps=5, log=print, verbose=False) -> dict:
    import torch

    rs.load()
    rs.rs_tune_clear()  # time the variants themselves, not a previous table
    dev = torch.device("cuda")
    entries = []
    for kb, vb in types:
        dt = np.uint32 if kb == 4 else np.uint64
        sdt = np.int32 if kb == 4 else np.int64
        nvar = rs.rs_num_variants(kb, vb)
        infos = [rs.rs_variant_info(kb, vb, i) for i in range(nvar)]
        for n in sizes:
            raw = np.random.default_rng(1).integers(0, np.iinfo(dt).max, n, dtype=dt,
                                                    endpoint=True)
            keys = torch.from_numpy(raw.view(sdt)).to(dev)
            vals = torch.from_numpy(np.arange(n, dtype=dt).view(sdt)).to(dev) if vb else None
            results = {}
            for i, info in enumerate(infos):
                if n > info["max_n"]:
                    continue
                if verbose:
                    print(f"  k{kb} v{vb} n={n} variant {i}", file=sys.stderr, flush=True)
                try:
                    ms = _time_variant(torch, kb, vb, n, i, keys, vals, reps)
                except rs.RsError as err:  # a form this GPU cannot launch: leave it out
                    log(f"k{kb} v{vb} n={n} variant {i}: skipped ({err})")
                    continue
                if ms is not None:
                    results[i] = ms
            best = min(results, key=results.get)
            entries.append({"key_bytes": kb, "val_bytes": vb, "n_max": n, "variant": best,
                            "ms": results[best],
                            "gkeys_per_s": n / (results[best] / 1e3) / 1e9,
                            "candidates": {str(i): round(ms, 5) for i, ms in results.items()},
                            "variant_info": infos[best]})
            log(f"k{kb} v{vb} n={n}: best variant {best} "
                f"({infos[best]}) {results[best]:.4f} ms")
            del keys, vals
        torch.cuda.empty_cache()
        extend_to_max(entries, kb, vb, infos)
    return {"device": torch.cuda.get_device_name(dev), "sizes": list(sizes),
            "entries": entries,
            "method": "median of %d CUDA-event timed sorts of uniform keys per variant" % reps}


def extend_to_max(entries: list, kb: int, vb: int, infos: list) -> None:
    """Append an entry n_max = RS_MAX_N for (kb, vb) that repeats the variant of
    the largest size swept, when that variant sorts arrays of any size."""
    mine = [e for e in entries if e["key_bytes"] == kb and e["val_bytes"] == vb]
    if not mine:
        return
    top = max(mine, key=lambda e: e["n_max"])
    if top["n_max"] >= rs.RS_MAX_N or infos[top["variant"]]["max_n"] < rs.RS_MAX_N:
        return
    entries.append({"key_bytes": kb, "val_bytes": vb, "n_max": rs.RS_MAX_N,
                    "variant": top["variant"], "ms": None, "gkeys_per_s": None,
                    "extrapolated_from": top["n_max"], "variant_info": top["variant_info"]})


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=rs.TUNED_TABLE)
    ap.add_argument("--quick", action="store_true", help="fewer sizes and repetitions")
    ap.add_argument("--verbose", action="store_true", help="name each variant before timing it")
    args = ap.parse_args(argv)
    sizes = (2**12, 2**16, 2**20, 2**24) if args.quick else SIZES
    table = tune(sizes=sizes, reps=3 if args.quick else 5, verbose=args.verbose)
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1)
        f.write("\n")
    print(f"wrote {args.out} ({len(table['entries'])} entries)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
