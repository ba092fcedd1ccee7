"""Named, timed workloads of the library's entry points: the LSD sort of any
key type (Sec. 2.6), merge sort (Sec. 2.4), the sample-sort partition
(Sec. 2.7) and the batched segmented sort, on seeded keys.

Each function runs its entry point on the device, times it with CUDA events
on the launching stream (the input restored outside the events, L2 flushed
before each timed call), and reads the per-kernel durations the library
records (``rs_profile_begin/end``).  ``python -m paper_1511_03404_gb300.workloads
merge --n 16777216`` runs one of them alone, e.g. under a profiler.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import numpy as np

from . import rs

_L2_FLUSH_BYTES = 256 << 20


def _uniform_u32(n: int, seed: int = 1):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:  # the seeded generators live beside the package
        sys.path.insert(0, root)
    import inputs  # seeded generators shared with the tests; no sort arithmetic
    return inputs.keys(np.uint32, "uniform", n, seed=seed)


def _timed(torch, stream, restore, call, reps: int):
    """Median CUDA-event time (ms) of ``call`` over ``reps`` runs after two
    warm-ups, plus the library's per-kernel records of the timed runs."""
    flush = torch.empty(_L2_FLUSH_BYTES, dtype=torch.uint8, device=stream.device)
    times = []
    for r in range(reps + 2):
        restore()
        flush.fill_(r & 0xFF)
        if r == 2:
            rs.check(rs.rs_profile_begin(64 * reps + 64), "rs_profile_begin")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        stream.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    st, prof = rs.rs_profile_end()
    rs.check(st, "rs_profile_end")
    return statistics.median(times), prof


def _kernel_rate(p: dict, peak_gbs):
    if not p["launches"] or p["ms"] <= 0:
        return None
    gbs = p["bytes"] / 1e9 / (p["ms"] / 1e3)
    return {"launches": p["launches"], "ms": p["ms"], "GB/s": gbs,
            "frac_of_hbm": (gbs / peak_gbs) if peak_gbs else None}


def merge(n: int = 1 << 26, key_bytes: int = 4, val_bytes: int = 0, reps: int = 5,
          peak_gbs=None, device: int = 0) -> dict:
    """Stable merge sort of n uniform u32 keys (values = index when val_bytes
    is 4) through ``rs_merge_sort``."""
    import torch
    if key_bytes != 4 or val_bytes not in (0, 4):
        raise ValueError("this workload takes u32 keys, optionally u32 values")
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    keys0 = torch.from_numpy(_uniform_u32(n).view(np.int32)).to(dev)
    k, ka = torch.empty_like(keys0), torch.empty_like(keys0)
    v = torch.arange(n, dtype=torch.int32, device=dev) if val_bytes else None
    v0 = v.clone() if val_bytes else None
    va = torch.empty_like(keys0) if val_bytes else None
    st, need = rs.rs_merge_workspace_bytes(key_bytes, val_bytes, n)
    rs.check(st, "rs_merge_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    out = {}

    def restore():
        with torch.cuda.stream(stream):
            k.copy_(keys0)
            if val_bytes:
                v.copy_(v0)

    def call():
        st_, alt = rs.rs_merge_sort(key_bytes, val_bytes, k.data_ptr(),
                                    v.data_ptr() if val_bytes else None, ka.data_ptr(),
                                    va.data_ptr() if val_bytes else None, n, ws.data_ptr(),
                                    ws.numel(), stream.cuda_stream)
        rs.check(st_, "rs_merge_sort")
        out["alt"] = alt

    ms, prof = _timed(torch, stream, restore, call, reps)
    res = (k if out["alt"] == 0 else ka).to(torch.int64) & 0xFFFFFFFF
    if n > 1 and not bool(torch.all(res[1:] >= res[:-1]).item()):
        raise SystemExit("workloads.merge: output is not sorted")
    return {"workload": f"merge sort, u32 keys{' + u32 values' if val_bytes else ''}, n={n}, "
                        "uniform (mt19937 seed 1)",
            "ms": ms, "gkeys_per_s": n / (ms / 1e3) / 1e9,
            "kernels": _kernel_rate(prof["merge"], peak_gbs),
            "bytes_per_launch": "2 n (key bytes + value bytes): one read and one write"}


def sample_partition(n: int = 1 << 26, samples: int = 64, buckets: int = 64, reps: int = 5,
                     peak_gbs=None, device: int = 0) -> dict:
    """Regular-sampling partition of n uniform u32 pairs (values = index)
    into ``buckets`` buckets through ``rs_sample_partition_pairs_u32``."""
    import torch
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    keys0 = torch.from_numpy(_uniform_u32(n).view(np.int32)).to(dev)
    vals0 = torch.arange(n, dtype=torch.int32, device=dev)
    k, v = torch.empty_like(keys0), torch.empty_like(keys0)
    ko, vo = torch.empty_like(keys0), torch.empty_like(keys0)
    off = torch.zeros(buckets + 1, dtype=torch.int64, device=dev)
    st, need = rs.rs_sample_workspace_bytes(n, samples, buckets)
    rs.check(st, "rs_sample_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)

    def restore():
        with torch.cuda.stream(stream):
            k.copy_(keys0)
            v.copy_(vals0)

    def call():
        rs.check(rs.rs_sample_partition_pairs_u32(k.data_ptr(), v.data_ptr(), ko.data_ptr(),
                                                  vo.data_ptr(), n, samples, buckets,
                                                  off.data_ptr(), None, ws.data_ptr(),
                                                  ws.numel(), stream.cuda_stream),
                 "rs_sample_partition_pairs_u32")

    ms, prof = _timed(torch, stream, restore, call, reps)
    sizes = np.diff(off.cpu().numpy())
    if sizes.sum() != n:
        raise SystemExit("workloads.sample_partition: bucket sizes do not add up to n")
    return {"workload": f"sample-sort partition, u32 pairs, n={n}, s={samples}, B={buckets}, "
                        "uniform (mt19937 seed 1)",
            "ms": ms, "gkeys_per_s": n / (ms / 1e3) / 1e9,
            "largest_bucket_over_mean": float(sizes.max()) * buckets / n,
            # the blocks are sorted in shared memory: one read and one write of the pairs
            "block_sort": _kernel_rate(dict(prof["segmented"], bytes=2.0 * n * 8 * reps), peak_gbs),
            "count_and_copy": _kernel_rate(prof["sample"], peak_gbs),
            "bytes": "block sort: 2 n (4 + 4); bucket counts: 4 n; run copy: 2 n (4 + 4)"}


def segmented(n: int = 1 << 24, nseg: int = 1000, reps: int = 5, peak_gbs=None,
              device: int = 0, stated: bool = False) -> dict:
    """Batched segmented sort of u32 pairs (values = index): nseg segments of
    log-uniform lengths in [1, 2^20] (seed 1) scaled to n elements in all
    (stated: the lengths as drawn, not scaled; n is then ignored), through
    ``rs_segmented_sort_pairs``."""
    import torch
    _uniform_u32(1)  # puts the input generators on the path
    import inputs
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    lengths = inputs.segment_lengths(nseg, seed=1, max_log2=20)
    if not stated:
        lengths = inputs.scale_lengths(lengths, n)
    off = inputs.offsets_from_lengths(lengths)
    total = int(off[-1])
    keys0 = torch.from_numpy(_uniform_u32(total).view(np.int32)).to(dev)
    vals0 = torch.arange(total, dtype=torch.int32, device=dev)
    k, v = torch.empty_like(keys0), torch.empty_like(keys0)
    ka, va = torch.empty_like(keys0), torch.empty_like(keys0)
    doff = torch.from_numpy(off.view(np.int64)).to(dev)
    st, need = rs.rs_segmented_workspace_bytes(total, len(lengths), 0, 32)
    rs.check(st, "rs_segmented_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)

    def restore():
        with torch.cuda.stream(stream):
            k.copy_(keys0)
            v.copy_(vals0)

    def call():
        st_, _ = rs.rs_segmented_sort_pairs(k.data_ptr(), v.data_ptr(), ka.data_ptr(),
                                            va.data_ptr(), total, doff.data_ptr(), len(lengths),
                                            0, 32, ws.data_ptr(), ws.numel(), stream.cuda_stream)
        rs.check(st_, "rs_segmented_sort_pairs")

    ms, prof = _timed(torch, stream, restore, call, reps)
    law = "as drawn" if stated else "scaled"
    return {"workload": f"segmented sort, u32 pairs, {len(lengths)} log-uniform segments ({law}), "
                        f"n={total}, uniform keys (mt19937 seed 1)",
            "ms": ms, "gkeys_per_s": total / (ms / 1e3) / 1e9,
            "kernels": _kernel_rate(prof["segmented"], peak_gbs),
            "bytes": "histograms 4 n, then 2 n (4 + 4) per pass"}


def sort(n: int = 1 << 26, key_bytes: int = 4, val_bytes: int = 4, dist: str = "uniform",
         variant: int = -1, reps: int = 5, peak_gbs=None, device: int = 0) -> dict:
    """One LSD sort (rs_sort) of n seeded keys of `dist` (values = index when
    val_bytes > 0), with the library's tile shape unless `variant` names one:
    the sort time, each kernel kind's rate, and the per-pass device times and
    moved / skipped passes of the last call (rs_workspace_stats)."""
    import torch
    _uniform_u32(1)  # puts the input generators on the path
    import inputs
    dev = torch.device("cuda", device)
    stream = torch.cuda.Stream(dev)
    dt, sdt = (np.uint32, torch.int32) if key_bytes == 4 else (np.uint64, torch.int64)
    keys0 = torch.from_numpy(inputs.keys(dt, dist, n).view(np.int32 if key_bytes == 4
                                                            else np.int64)).to(dev)
    k, ka = torch.empty_like(keys0), torch.empty_like(keys0)
    vals0 = torch.arange(n, dtype=sdt, device=dev) if val_bytes else None
    v = torch.empty_like(keys0) if val_bytes else None
    va = torch.empty_like(keys0) if val_bytes else None
    st, need = rs.rs_workspace_bytes(key_bytes, val_bytes, n, 0, 8 * key_bytes, variant=variant)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731

    def restore():
        with torch.cuda.stream(stream):
            k.copy_(keys0)
            if val_bytes:
                v.copy_(vals0)

    def call():
        st_, _ = rs.rs_sort(key_bytes, val_bytes, ptr(k), ptr(v), ptr(ka), ptr(va), n, 0,
                            8 * key_bytes, ws.data_ptr(), ws.numel(), stream.cuda_stream,
                            variant=variant)
        rs.check(st_, "rs_sort")

    ms, prof = _timed(torch, stream, restore, call, reps)
    st, stats = rs.rs_workspace_stats(ws.data_ptr(), stream.cuda_stream)
    rs.check(st, "rs_workspace_stats")
    rs.check(stats["status"], "device status")
    return {"workload": f"LSD sort, {8 * key_bytes}-bit keys" +
                        (f" + {8 * val_bytes}-bit values" if val_bytes else "") +
                        f", n={n}, {dist} (mt19937 seed 1), variant {variant}",
            "ms": ms, "gkeys_per_s": n / (ms / 1e3) / 1e9,
            "upsweep": _kernel_rate(prof["upsweep"], peak_gbs),
            "passes": _kernel_rate(prof["onesweep"], peak_gbs),
            "pass_ms": [round(t, 4) for t in stats["pass_ms"]],
            "upsweep_ms": round(stats["upsweep_ms"], 4),
            "moved_mask": stats["moved_mask"], "skipped_mask": stats["skipped_mask"],
            "bytes": "upsweep n K; each moving pass 2 n (K + V)"}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description="run one named workload and print its timing")
    ap.add_argument("workload", choices=("sort", "merge", "merge_pairs", "sample_partition",
                                         "segmented"))
    ap.add_argument("--n", type=int, default=1 << 26)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--buckets", type=int, default=64)
    ap.add_argument("--key-bytes", type=int, default=4, choices=(4, 8))
    ap.add_argument("--val-bytes", type=int, default=4, choices=(0, 4, 8))
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--segments", type=int, default=1000)
    ap.add_argument("--stated", action="store_true",
                    help="segmented: the log-uniform lengths as drawn (20,000 segments: about "
                         "1.5e9 pairs), not scaled to --n")
    args = ap.parse_args(argv)
    rs.load()
    if args.workload == "sort":
        r = sort(args.n, args.key_bytes, args.val_bytes, args.dist, args.variant, args.reps)
    elif args.workload == "merge":
        r = merge(args.n, 4, 0, args.reps)
    elif args.workload == "merge_pairs":
        r = merge(args.n, 4, 4, args.reps)
    elif args.workload == "segmented":
        r = segmented(args.n, args.segments, args.reps, stated=args.stated)
    else:
        r = sample_partition(args.n, args.buckets, args.buckets, args.reps)
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
