"""Benchmark: LSD radix sort rate on GB300 (arXiv 1511.03404, Sec. 3-4 protocol).

One step = one complete sort (upsweep + every digit pass) of one array of
2^26 32-bit key + 32-bit value pairs; the steps cycle through the six input
distributions of Sec. 4 (uniform, gaussian, zero, bucket, sorted,
sorted descending).  As in Sec. 3, only the sort is timed: the data is
already on the device (a device-to-device copy of the pristine input and an
L2 flush run before each step, outside the events).  ``value`` is the whole
job's sort rate in Gkeys/s.  ``e2e`` times the same sorts through the C ABI
from pinned host buffers (host->device copy, sort, device->host copy).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank sorts its own replica (the sort does not
shard); the slowest rank's time counts.  ``--impl reference`` times the CPU
oracle (the slow, plain LSD counting sort) on bounded samples instead.
"""
from __future__ import annotations

import argparse
import faulthandler
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402

METRIC = "Gkeys/s & % HBM peak, radix sort 32/64-bit KV; batched vs plain; p99 latency"
N_KEYS = 1 << 26
DISTS = ("uniform", "gaussian", "zero", "bucket", "sorted", "sorted_desc")
WORKLOAD = ("u32 key + u32 value (value = index) pairs, n=2^26, mt19937 seed 1, six "
            "distributions (uniform, gaussian, zero, bucket, sorted, sorted_desc) one per step "
            "in turn; LSD radix sort, 8-bit digits, 4 passes")
L2_FLUSH_BYTES = 256 << 20

# DRAM traffic of one onesweep launch from an ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of pass 0 of a 2^26-pair sort), keyed by the hash of the
# kernel sources it was taken on; when they change the figure no longer applies
# and traffic is null.
NCU_TRAFFIC = {
    "0f7b97d11c47d4db": {"bytes_per_launch": 1027530240, "n": 1 << 26,
                         "kernel": "k_onesweep_persist<u32,4,8,256,45,2,16>"},
}

ONESWEEP_SOURCES = ("rs_kernels.cuh", "rs_common.h", "rs_launch.cuh", "rs_inst_kv32.cu")


def kernel_source_hash() -> str:
    """Hash of the code (comments and blank lines left out) of the files that
    make the onesweep pass and its launch."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1511_03404_gb300", "csrc")
    for f in ONESWEEP_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(n: int, dists=DISTS):
    keys = {d: inputs.keys(np.uint32, d, n) for d in dists}
    vals = inputs.values(np.uint32, n)
    return keys, vals


def cpu_oracle_rate(sample_n: int, dists=DISTS, budget_s: float = 30.0,
                    lib_budget_s: float = 10.0) -> dict:
    """The oracle (single thread) on bounded samples of the same workload: whole
    arrays of the distributions in turn until about budget_s of CPU work."""
    import oracle

    vals = inputs.values(np.uint32, sample_n)
    done, t_total, used = 0, 0.0, []
    for d in dists:
        k = inputs.keys(np.uint32, d, sample_n)
        t0 = time.perf_counter()
        oracle.lsd_sort(k, vals)
        t_total += time.perf_counter() - t0
        done += sample_n
        used.append(d)
        if t_total > budget_s:
            break
    # a library stable sort beside it on the same arrays (numpy: one thread)
    t_lib, done_lib = 0.0, 0
    for d in used:
        k = inputs.keys(np.uint32, d, sample_n)
        t0 = time.perf_counter()
        order = np.argsort(k, kind="stable")
        k[order], vals[order]  # the sorted pairs
        t_lib += time.perf_counter() - t0
        done_lib += sample_n
        if t_lib > lib_budget_s:
            break
    return {"value": done / t_total / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(used)} arrays of 2^{int(np.log2(sample_n))} u32 pairs "
                      f"({', '.join(used)}), single-threaded C LSD counting sort, "
                      f"{t_total:.1f} s",
            "library_stable_sort": {"value": done_lib / t_lib / 1e9, "unit": "Gkeys/s", "cores": 1,
                                    "what": "numpy.argsort(kind='stable') and the gather of keys "
                                            f"and values, the first {done_lib // sample_n} of the "
                                            "same arrays"}}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the slowest rank's time), via one all-reduce."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, n: int, max_ms: float) -> float:
    """Keys sorted by all ranks / slowest rank's time, in Gkeys/s."""
    return world * steps * n / (max_ms / 1e3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    sample_n = 1 << 22
    vals = inputs.values(np.uint32, sample_n)
    samples = [inputs.keys(np.uint32, DISTS[i % len(DISTS)], sample_n)
               for i in range(args.warmup + args.steps)]
    import oracle

    for i in range(args.warmup):
        oracle.lsd_sort(samples[i], vals)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.lsd_sort(samples[args.warmup + i], vals)
    dt = time.perf_counter() - t0
    value = args.steps * sample_n / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": "each step sorts one 2^22-pair "
                   "sample of the workload, in turn over the six distributions, so that the "
                   "run stays within minutes"},
        "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed arrays of 2^22 u32 pairs"},
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_1511_03404_gb300 import rs

    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    n = args.n
    dists = (args.dist,) if args.dist else DISTS
    keys_h, vals_h = make_inputs(n, dists)
    # pristine inputs on the device, plus the sort's double buffer and workspace
    pristine = {d: torch.from_numpy(keys_h[d].view(np.int32)).to(dev) for d in dists}
    vals0 = torch.from_numpy(vals_h.view(np.int32)).to(dev)
    k, v = torch.empty_like(vals0), torch.empty_like(vals0)
    ka, va = torch.empty_like(vals0), torch.empty_like(vals0)
    st, nbytes = rs.rs_workspace_bytes(4, 4, n, 0, 32)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    h = stream.cuda_stream

    def one_sort(i, ev0=None, ev1=None):
        d = dists[i % len(dists)]
        k.copy_(pristine[d])
        v.copy_(vals0)
        flush.fill_(i & 0xFF)
        if ev0 is not None:
            ev0.record(stream)
        st, in_alt = rs.rs_sort_pairs_u32(k.data_ptr(), v.data_ptr(), ka.data_ptr(),
                                          va.data_ptr(), n, 0, 32, ws.data_ptr(), ws.numel(), h)
        if ev1 is not None:
            ev1.record(stream)
        rs.check(st, "rs_sort_pairs_u32")
        return d, in_alt

    # correctness of the timed configuration: every distribution once, checked
    # against the properties that fix a stable sort (sorted keys, values are a
    # permutation, keys_in[vals_out] == keys_out, equal keys keep index order)
    for i in range(0 if args.quick else len(dists)):
        d, in_alt = one_sort(i)
        st, info = rs.rs_workspace_status(ws.data_ptr(), h)
        rs.check(st, "device status")
        if i == 0 and rank == 0:
            ok = check_sorted(torch, (ka if in_alt else k), (va if in_alt else v), pristine[d])
            if not ok:
                raise SystemExit("bench: sorted output failed its property check")

    for i in range(args.warmup):
        one_sort(i)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(dev.index or 0) as clocks:
        torch.cuda.synchronize()
        for i in range(args.steps):
            one_sort(i, starts[i], ends[i])
        torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # per-kernel times: the same steps again with events around every launch
    # (kept out of the timed steps above: an event between two kernels also
    # stops the next one from being scheduled before the last one ends)
    rs.check(rs.rs_profile_begin(16 * args.steps + 16), "rs_profile_begin")
    for i in range(args.steps):
        one_sort(i)
    torch.cuda.synchronize()
    st, prof = rs.rs_profile_end()
    rs.check(st, "rs_profile_end")
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, pg, dev)
    value = whole_job_rate(world, args.steps, n, total_ms)

    # end to end through the C ABI: pinned host -> device, sort, device -> host
    e2e = {"value": None, "ms_per_step": None, "h2d": 0, "d2h": 0}
    stage(f"timed sorts done: {total_ms / args.steps:.3f} ms per sort")
    serving = None
    if not (args.no_extras or args.quick) and world == 1:
        # first, before this process pins host memory for the end-to-end leg:
        # host copies (and with them the served latencies) slow down as a
        # process, or the host, holds more pinned memory
        stage("serving: Poisson trace")
        serving = bench_serving_process(args.serve_seconds)
    if not args.quick:
        stage("end to end (host buffers)")
        e2e = e2e_rate(torch, rs, keys_h, vals_h, n, dev, ws, args, dists)
    if pg and not args.quick:
        e2e["value"] = whole_job_rate(world, 1, n, max_over_ranks(e2e["ms_per_step"], pg, dev))

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    os_p = prof["onesweep"]
    achieved = (os_p["bytes"] / 1e9) / (os_p["ms"] / 1e3) if os_p["ms"] > 0 else None
    launches = sum(p["launches"] for p in prof.values())
    traffic = None
    src = kernel_source_hash()
    t = NCU_TRAFFIC.get(src)
    if t is not None and t.get("n") == n:
        traffic = t["bytes_per_launch"]
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world,
        "value_by_distribution": {d: n / (statistics.mean(step_ms[i::len(dists)]) / 1e3) / 1e9
                                  for i, d in enumerate(dists) if step_ms[i::len(dists)]},
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "digit_bits": 8,
                   "l2": "256 MiB written before every timed sort; inputs (512 MiB) exceed L2",
                   "timing": "CUDA events around each sort call on its stream; per-kernel times "
                             "(roofline) from a second pass over the same steps with events around "
                             "every launch",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if (achieved and hbm) else None,
                     "traffic": traffic, "kernel": "k_onesweep (one digit pass)",
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else None,
                     "algorithmic_bytes_per_launch": "2 n (4 + 4) for a pass that moves data"},
        "per_kernel": {k_: {"launches": p["launches"], "ms": p["ms"],
                            "GB/s": (p["bytes"] / 1e9) / (p["ms"] / 1e3) if p["ms"] else None}
                       for k_, p in prof.items() if p["launches"]},
        "per_dist_ms": {d: statistics.mean(step_ms[i::len(dists)])
                        for i, d in enumerate(dists) if step_ms[i::len(dists)]},
        "cpu_baseline": None,
        "e2e": {"value": e2e["value"], "unit": "Gkeys/s",
                "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
                "runs": e2e.get("runs_gkeys_per_s"),
                "serial": e2e.get("serial"), "link_bound": e2e.get("link_bound"),
                "entry": e2e.get("entry"), "pipelining": e2e.get("pipelining")},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
        "kernel_source": src,
    }
    if not (args.no_extras or args.quick) and world == 1:
        line["serving"] = serving
        stage("u32 keys, 2^20 (launch-bound)")
        line["u32_keys_2p20"] = bench_u32_keys_small(torch, rs, dev)
        stage("u64 keys and pairs, 2^27")
        line["u64_2p27"] = bench_u64(torch, rs, dev)
        stage("segmented: batched vs plain")
        line["segmented"] = bench_segmented(torch, rs, dev, args.seg_scaled)
        stage("merge sort and sample-sort partition, 2^26")
        from paper_1511_03404_gb300 import workloads
        line["merge_2p26"] = {"keys": workloads.merge(n, 4, 0, peak_gbs=hbm, device=dev.index or 0),
                              "pairs": workloads.merge(n, 4, 4, peak_gbs=hbm,
                                                       device=dev.index or 0)}
        line["sample_partition_2p26"] = workloads.sample_partition(n, 64, 64, peak_gbs=hbm,
                                                                   device=dev.index or 0)
    if not (args.no_cpu_baseline or args.quick):
        stage("cpu baseline (oracle)")
        line["cpu_baseline"] = cpu_oracle_rate(n)
        line["cpu_baseline"]["host"] = host_description()
    line["summary"] = summary(line)
    stage("summary " + json.dumps(line["summary"]))
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def summary(line: dict) -> dict:
    """The headline figures of every leg in a few hundred bytes, the last key
    of the bench line (and the last stderr line), so that a reader who keeps
    only the end of the output still has them."""
    r = lambda x, d=2: None if x is None else round(float(x), d)  # noqa: E731
    out = {"gkeys_per_s": r(line["value"]),
           "uniform_gkeys_per_s": r(line["value_by_distribution"].get("uniform")),
           "onesweep_frac_of_hbm": r(line["roofline"]["frac"], 3),
           "e2e_gkeys_per_s": r(line["e2e"]["value"])}
    u64 = line.get("u64_2p27")
    if u64:
        out["u64_2p27_gkeys_per_s"] = {d: [r(u64[d]["keys_gkeys_per_s"]),
                                           r(u64[d]["pairs_gkeys_per_s"])]
                                       for d in ("uniform", "gaussian", "entropy16") if d in u64}
    seg = line.get("segmented")
    if seg:
        out["segmented"] = {"elements": seg["elements"], "batched_gkeys_per_s":
                            r(seg["batched_gkeys_s"]), "plain_gkeys_per_s": r(seg["plain_gkeys_s"]),
                            "batched_over_plain": r(seg["batched_over_plain"])}
    srv = line.get("serving")
    if srv:
        svp = srv.get("served_vs_plain", {})
        out["serving"] = {"p50_ms": r(srv["p50_ms"]), "p99_ms": r(srv["p99_ms"]),
                          "gkeys_per_s": r(srv["gkeys_per_s"]),
                          "offered_gkeys_per_s": r(srv["offered_gkeys_per_s"]),
                          "saturated_gkeys_per_s": r(svp.get("served_gkeys_per_s")),
                          "plain_gkeys_per_s": r(svp.get("plain_gkeys_per_s")),
                          "served_over_plain": r(svp.get("served_over_plain"))}
    small = line.get("u32_keys_2p20")
    if small:
        out["u32_keys_2p20_ms"] = r(small.get("ms_per_call", small.get("ms")), 4)
    cpu = line.get("cpu_baseline")
    if cpu:
        out["cpu_oracle_gkeys_per_s"] = r(cpu["value"], 4)
    return out


def host_description() -> str:
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for l_ in f:
                if l_.lower().startswith(("model name", "cpu part")):
                    model = l_.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{os.cpu_count()} cores {model}".strip()


def check_sorted(torch, k_out, v_out, k_in) -> bool:
    ko = k_out.to(torch.int64) & 0xFFFFFFFF
    if not bool((ko[1:] >= ko[:-1]).all()):
        return False
    idx = v_out.to(torch.int64)
    if not bool((torch.sort(idx).values == torch.arange(idx.numel(), device=idx.device)).all()):
        return False
    if not bool((k_in[idx] == k_out).all()):
        return False
    eq = ko[1:] == ko[:-1]
    return bool((idx[1:][eq] > idx[:-1][eq]).all())


def check_segmented(torch, src, out_k, out_v, off) -> bool:
    """Every segment sorted stably, checked on the device.  The values are
    the input positions, so these properties fix the result: keys
    non-decreasing inside each segment; the values a permutation of 0 .. n-1
    with every value inside its own position's segment; src[value] equal to
    the output key; equal keys of a segment in increasing value order."""
    n = src.numel()
    dev = src.device
    lengths = torch.from_numpy(np.diff(off).astype(np.int64)).to(dev)
    seg = torch.repeat_interleave(torch.arange(lengths.numel(), dtype=torch.int32, device=dev),
                                  lengths, output_size=n)
    same = seg[1:] == seg[:-1]
    o = out_k ^ -(1 << 31)  # unsigned order as signed order
    if not bool(((o[1:] >= o[:-1]) | ~same).all()):
        return False
    idx = out_v.long()
    if int(idx.min()) != 0 or int(idx.max()) != n - 1:
        return False
    seen = torch.zeros(n, dtype=torch.uint8, device=dev)
    seen[idx] = 1
    ok = bool(seen.bool().all())
    del seen
    ok = ok and bool((seg[idx] == seg).all()) and bool((src[idx] == out_k).all())
    eq = (o[1:] == o[:-1]) & same
    return ok and bool(((idx[1:] > idx[:-1]) | ~eq).all())


def e2e_rate(torch, rs, keys_h, vals_h, n, dev, ws, args, dists) -> dict:
    """Host -> device copy, sort, device -> host copy, per step, through the
    C ABI's host-buffer entry point rs_sort_host (one call per step does all
    three on its stream).

    Steps go round robin over three streams, each with its own device buffers
    and pinned host outputs, so the copy-in of step i + 1, the sort of step i
    and the copy-out of step i - 1 overlap (stream order keeps each buffer
    set's reuse in order).  ``serial`` is one stream (no overlap), and
    ``link_bound`` the step time the host link alone allows (both directions
    at once, measured here)."""
    hk = {d: torch.from_numpy(keys_h[d].view(np.int32)).pin_memory() for d in dists}
    hv = torch.from_numpy(vals_h.view(np.int32)).pin_memory()
    nsets = 3
    sets = []
    for j in range(nsets):
        k = torch.empty(n, dtype=torch.int32, device=dev)
        sets.append({
            "k": k, "v": torch.empty_like(k), "ka": torch.empty_like(k), "va": torch.empty_like(k),
            "ok": torch.empty(n, dtype=torch.int32).pin_memory(),
            "ov": torch.empty(n, dtype=torch.int32).pin_memory(),
            "ws": ws if j == 0 else torch.empty_like(ws),
        })
    streams = [torch.cuda.Stream(dev) for _ in range(nsets)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)  # the link-bound probe

    def timed(nb, steps):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(streams[0])
        for s in streams[1:nb]:
            s.wait_event(t0)
        for i in range(steps):
            d = dists[i % len(dists)]
            sl, s = sets[i % nb], streams[i % nb]
            st, _ = rs.rs_sort_host(4, 4, hk[d].data_ptr(), hv.data_ptr(), sl["ok"].data_ptr(),
                                    sl["ov"].data_ptr(), n, 0, 32, sl["k"].data_ptr(),
                                    sl["v"].data_ptr(), sl["ka"].data_ptr(), sl["va"].data_ptr(),
                                    sl["ws"].data_ptr(), sl["ws"].numel(), s.cuda_stream)
            rs.check(st, "rs_sort_host")
        for s in streams[1:nb]:
            streams[0].wait_stream(s)
        t1.record(streams[0])
        torch.cuda.synchronize()
        # the last outputs are complete and sorted
        last = sets[(steps - 1) % nb]
        assert np.all(np.diff(last["ok"].numpy().view(np.uint32)) >= 0)
        return t0.elapsed_time(t1) / steps

    def link_ms():
        # one step's bytes in both directions at once, on two copy streams
        a, b = sets[0], sets[1]
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s_in)
        s_out.wait_event(t0)
        with torch.cuda.stream(s_in):
            a["k"].copy_(hk[dists[0]], non_blocking=True)
            a["v"].copy_(hv, non_blocking=True)
        with torch.cuda.stream(s_out):
            b["ok"].copy_(b["k"], non_blocking=True)
            b["ov"].copy_(b["v"], non_blocking=True)
        s_in.wait_stream(s_out)
        t1.record(s_in)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    steps = max(6, min(args.steps, 15))
    timed(1, 2)
    ms_serial = timed(1, max(4, steps // 2))
    timed(nsets, steps)  # a whole pipelined run as warm-up: the first one was often slower
    # the pipelined run five times, the median reported: on these hosts a
    # single run now and then loses its copy overlap (the sort is unchanged)
    ms_runs = [timed(nsets, steps) for _ in range(5)]
    ms = statistics.median(ms_runs)
    link = min(link_ms() for _ in range(3))
    return {"value": n / (ms / 1e3) / 1e9, "ms_per_step": ms, "h2d": 2 * 4 * n, "d2h": 2 * 4 * n,
            "runs_gkeys_per_s": [n / (m / 1e3) / 1e9 for m in ms_runs],
            "serial": {"value": n / (ms_serial / 1e3) / 1e9, "ms_per_step": ms_serial},
            "link_bound": {"value": n / (link / 1e3) / 1e9, "ms_per_step": link,
                           "what": "the step's host->device and device->host bytes copied at once, "
                                   "no sort"},
            "entry": "rs_sort_host (C ABI: host->device copies, sort, device->host copies "
                     "on one stream)",
            "pipelining": "one rs_sort_host call per step, round robin over three streams and "
                          "buffer sets: step i + 1 loads while step i sorts and step i - 1 "
                          "returns; serial: one stream"}


def _time_sorts(torch, rs, kb, vb, keys, vals, reps, stream):
    """Median CUDA-event time (ms) of `reps` sorts of fresh copies of keys/vals."""
    n = keys.numel()
    k, ka = torch.empty_like(keys), torch.empty_like(keys)
    v = torch.empty_like(vals) if vb else None
    va = torch.empty_like(vals) if vb else None
    st, need = rs.rs_workspace_bytes(kb, vb, n, 0, 8 * kb)
    rs.check(st, "rs_workspace_bytes")
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=keys.device)
    h = stream.cuda_stream
    times = []
    for r in range(reps + 2):
        k.copy_(keys)
        if vb:
            v.copy_(vals)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = rs.rs_sort(kb, vb, k.data_ptr(), v.data_ptr() if vb else None, ka.data_ptr(),
                           va.data_ptr() if vb else None, n, 0, 8 * kb, ws.data_ptr(),
                           ws.numel(), h)
        e1.record(stream)
        rs.check(st, "rs_sort")
        stream.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "device status")
    return statistics.median(times)


def bench_u32_keys_small(torch, rs, dev, reps: int = 20) -> dict:
    """32-bit keys only, n = 2^20, uniform: a launch-bound, L2-resident sort,
    timed per call and as a replayed CUDA graph of the same call."""
    n = 1 << 20
    keys = torch.from_numpy(inputs.keys(np.uint32, "uniform", n).view(np.int32)).to(dev)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ms = _time_sorts(torch, rs, 4, 0, keys, None, reps, stream)
    k, ka = torch.empty_like(keys), torch.empty_like(keys)
    st, need = rs.rs_workspace_bytes(4, 0, n, 0, 32)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    h = stream.cuda_stream
    with torch.cuda.stream(stream):
        k.copy_(keys)
        rs.check(rs.rs_sort_keys_u32(k.data_ptr(), ka.data_ptr(), n, 0, 32, ws.data_ptr(),
                                     ws.numel(), h)[0])
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        st, in_alt = rs.rs_sort_keys_u32(k.data_ptr(), ka.data_ptr(), n, 0, 32, ws.data_ptr(),
                                         ws.numel(), h)
    rs.check(st, "captured sort")
    times = []
    for r in range(reps + 2):
        with torch.cuda.stream(stream):
            k.copy_(keys)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
        stream.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    gms = statistics.median(times)
    out_k = (ka if in_alt else k).cpu().numpy().view(np.uint32)
    if not np.array_equal(out_k, np.sort(keys.cpu().numpy().view(np.uint32))):
        raise SystemExit("bench: 2^20-key sort (graph replay) is not sorted")
    sort_bytes = n * (4 + 4 * 2 * 4)  # one histogram read + four passes of read + write
    return {"workload": "u32 keys only, n=2^20, uniform, 8-bit digits (4 passes); inputs fit L2",
            "ms": ms, "gkeys_per_s": n / (ms / 1e3) / 1e9,
            "graph_ms": gms, "graph_gkeys_per_s": n / (gms / 1e3) / 1e9,
            "l2_resident_gb_per_s": sort_bytes / (gms / 1e3) / 1e9,
            "l2_note": "36 B/key algorithmic over the graph-replay time; the 4 MiB array lives "
                       "in L2, so this is not an HBM figure (launch- and latency-bound)"}


def bench_u64(torch, rs, dev, reps: int = 3) -> dict:
    """64-bit keys and 64-bit pairs, n = 2^27: uniform, gaussian and 16-bit
    entropy keys (the last skips six of eight digit passes)."""
    n = 1 << 27
    stream = torch.cuda.Stream(dev)
    out = {}
    vals = torch.from_numpy(np.arange(n, dtype=np.int64)).to(dev)
    for dist in ("uniform", "gaussian", "entropy16"):
        keys = torch.from_numpy(inputs.keys(np.uint64, dist, n).view(np.int64)).to(dev)
        with torch.cuda.stream(stream):
            mk = _time_sorts(torch, rs, 8, 0, keys, None, reps, stream)
            mkv = _time_sorts(torch, rs, 8, 8, keys, vals, reps, stream)
        out[dist] = {"keys_ms": mk, "keys_gkeys_per_s": n / (mk / 1e3) / 1e9,
                     "pairs_ms": mkv, "pairs_gkeys_per_s": n / (mkv / 1e3) / 1e9}
        del keys
    del vals
    torch.cuda.empty_cache()
    out["workload"] = "n=2^27, 64-bit keys / 64-bit key + 64-bit value pairs, 8-bit digits"
    return out


def bench_segmented(torch, rs, dev, scaled: bool, reps: int = 3) -> dict:
    """20,000 segments of u32 pairs with log-uniform lengths in [1, 2^20]:
    one batched launch sequence (captured once in a CUDA graph, replayed) vs
    one plain rs_sort_pairs_u32 call per segment, same data, same stream."""
    lengths = inputs.segment_lengths(20000, seed=1, max_log2=20)
    law = "log-uniform in [1, 2^20], 20,000 segments, as stated"
    if scaled:
        lengths = inputs.scale_lengths(lengths, 1 << 28)
        law = "log-uniform in [1, 2^20], 20,000 segments, scaled to total 2^28"
    off = inputs.offsets_from_lengths(lengths)
    n = int(off[-1])
    keys = inputs.keys(np.uint32, "uniform", n, seed=1)
    vals = np.arange(n, dtype=np.uint32)
    pk = torch.from_numpy(keys.view(np.int32)).to(dev)
    pv = torch.from_numpy(vals.view(np.int32)).to(dev)
    del keys, vals
    k, v = torch.empty_like(pk), torch.empty_like(pv)
    ka, va = torch.empty_like(pk), torch.empty_like(pv)
    doff = torch.from_numpy(off.view(np.int64)).to(dev)
    st, need = rs.rs_segmented_workspace_bytes(n, len(lengths))
    rs.check(st, "rs_segmented_workspace_bytes")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    h = stream.cuda_stream

    def seg_call():
        return rs.rs_segmented_sort_pairs(k.data_ptr(), v.data_ptr(), ka.data_ptr(),
                                          va.data_ptr(), n, doff.data_ptr(), len(lengths), 0, 32,
                                          ws.data_ptr(), ws.numel(), h)

    with torch.cuda.stream(stream):
        k.copy_(pk)
        v.copy_(pv)
        rs.check(seg_call()[0], "rs_segmented_sort_pairs")  # warm-up outside the capture
    stream.synchronize()
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "segmented device status")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        st, in_alt = seg_call()
    rs.check(st, "captured rs_segmented_sort_pairs")
    batched = []
    for _ in range(reps):
        with torch.cuda.stream(stream):
            k.copy_(pk)
            v.copy_(pv)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()  # on the current stream, which is `stream` here
            e1.record(stream)
        stream.synchronize()
        batched.append(e0.elapsed_time(e1))
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "segmented device status")
    # the timed output, checked whole on the device (keys and values)
    if not check_segmented(torch, pk, ka if in_alt else k, va if in_alt else v, off):
        raise SystemExit("bench: the batched segmented sort failed its property check")
    # plain: one sort per segment through the typed entry point
    maxlen = int(lengths.max())
    st, need_p = rs.rs_workspace_bytes(4, 4, maxlen, 0, 32)
    wsp = torch.empty(max(need_p, 256), dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        k.copy_(pk)
        v.copy_(pv)
    stream.synchronize()
    bk, bv, bka, bva = k.data_ptr(), v.data_ptr(), ka.data_ptr(), va.data_ptr()
    offs = off.tolist()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(len(lengths)):
        a = offs[s] * 4
        st, _ = rs.rs_sort_pairs_u32(bk + a, bv + a, bka + a, bva + a, offs[s + 1] - offs[s], 0,
                                     32, wsp.data_ptr(), wsp.numel(), h)
        if st:
            rs.check(st, "rs_sort_pairs_u32 (plain per segment)")
    e1.record(stream)
    stream.synchronize()
    plain_ms = e0.elapsed_time(e1)
    b_ms = min(batched)
    out = {"law": law, "segments": len(lengths), "elements": n,
           "batched_ms": b_ms, "batched_gkeys_s": n / (b_ms / 1e3) / 1e9,
           "plain_ms": plain_ms, "plain_gkeys_s": n / (plain_ms / 1e3) / 1e9,
           "batched_over_plain": plain_ms / b_ms,
           "checked": "the timed output, whole, on the device: keys sorted in every segment, "
                      "values a permutation kept in their segments, keys follow their values, "
                      "ties in input order",
           "batched": "one CUDA graph replay: memset + planning kernel + short-segment kernel + histogram kernel + one persistent kernel",
           "plain": "one rs_sort_pairs_u32 call per segment on the same stream"}
    del pk, pv, k, v, ka, va, ws, wsp
    torch.cuda.empty_cache()
    return out


def bench_serving(torch, rs, seconds: float = 10.0, rate: float = 5000.0,
                  budget: int = 24 << 30, streams: int = 8, compare_requests: int = 10000,
                  policy: dict | None = None) -> dict:
    """Poisson arrivals at `rate` requests/s of log-uniform size [2^10, 2^24],
    half u32 pairs, half u64 keys (uniform keys), through the sort server
    with a 24 GiB admission budget; p50/p99 latency and aggregate Gkeys/s.

    Then the first `compare_requests` requests of the same trace twice more,
    with no arrival schedule: ``saturated`` submits them all as fast as the
    server admits them (its capacity: continuous batching, copies and sorts
    of different requests overlapping on its streams), ``plain`` runs them one
    after another as one rs_sort_host call each (copy in, sort, copy out) on
    one stream, from and to the same pinned host buffers."""
    count = int(seconds * rate)
    raw = inputs.mt19937(1, 3 * count)
    u = raw.astype(np.float64) / 2.0**32
    gaps = -np.log1p(-u[0::3][:count]) / rate
    sizes = np.floor(2.0 ** (10 + 14 * u[1::3][:count])).astype(np.int64)
    is_pairs = (raw[2::3][:count] % 2) == 0
    pool_n = 1 << 25
    k32 = torch.from_numpy(inputs.keys(np.uint32, "uniform", pool_n, seed=2).view(np.int32)).pin_memory()
    k64 = torch.from_numpy(inputs.keys(np.uint64, "uniform", pool_n, seed=3).view(np.int64)).pin_memory()
    iota = torch.arange(1 << 24, dtype=torch.int32).pin_memory()
    ring_bytes = 3 << 30  # outputs of the requests in flight; submission waits when it is full
    ring = torch.empty(ring_bytes, dtype=torch.uint8).pin_memory()
    ring_base = ring.data_ptr()
    link_before = host_link_gbs(torch, ring)
    offsets = (raw[0::3][:count].astype(np.int64) % (pool_n - (1 << 24)))
    arrival = np.cumsum(gaps)

    def request(i, out):
        n = int(sizes[i])
        o = int(offsets[i])
        if is_pairs[i]:
            return rs.rs_request(4, 4, n, 0, 32, k32.data_ptr() + 4 * o, iota.data_ptr(),
                                 ring_base + out, ring_base + out + 4 * n)
        return rs.rs_request(8, 0, n, 0, 64, k64.data_ptr() + 8 * o, None, ring_base + out, None)

    def serve(idx, paced: bool):
        """Submit requests idx through a new server (paced: at their arrival
        times); returns the server's stats and the client's wall time."""
        st, srv = rs.rs_server_create(budget, streams)
        rs.check(st, "rs_server_create")
        if policy:
            st, cfg = rs.rs_server_get_config(srv)
            rs.check(st, "rs_server_get_config")
            cfg.update(policy)
            rs.check(rs.rs_server_set_config(srv, cfg), "rs_server_set_config")
        pending = {}        # handle -> (ring start, ring end)
        live = []           # ring regions in use, in allocation order
        head = 0
        reqs = []           # keep the ctypes structs alive

        def poll_some(block=False):
            # one call takes every finished handle off the server's completion
            # queue; polling each pending handle instead kept the server's lock
            # busy and starved its scheduler thread
            st_, finished = rs.rs_server_completed(srv, 4096)
            rs.check(st_, "rs_server_completed")
            for hnd in finished:
                st_, done = rs.rs_poll(srv, hnd)
                if st_ != rs.RS_OK or not done:
                    raise SystemExit(f"bench: server request failed: {rs.status_string(st_)}")
                live.remove(pending.pop(hnd))
            if block and pending:
                time.sleep(0.0002)

        def reserve(nbytes):
            nonlocal head
            while True:
                start = head if head + nbytes <= ring_bytes else 0
                end = start + nbytes
                if not any(a_ < end and start < b_ for a_, b_ in live):
                    head = end
                    live.append((start, end))
                    return start
                poll_some(block=True)

        # no cyclic garbage collection while the client keeps the arrival
        # schedule: a full collection over a large heap stalls it for tens of ms
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        for i in idx:
            while paced:
                rem = arrival[i] - (time.perf_counter() - t0)
                if rem <= 0:
                    break
                poll_some()
                if rem > 3e-4:
                    time.sleep(1e-4)  # far from the next arrival: leave the lock alone
            r = request(i, reserve(8 * int(sizes[i])))
            while True:
                st, hnd = rs.rs_submit(srv, r)
                if st != rs.RS_ERR_BUSY:
                    break
                poll_some(block=True)  # queue full: wait for completions
            rs.check(st, "rs_submit")
            reqs.append(r)
            pending[hnd] = live[-1]
            if len(reqs) > 4096:
                reqs = reqs[-4096:]
        while pending:
            poll_some(block=True)
        wall = time.perf_counter() - t0
        gc.enable()
        st, stats = rs.rs_server_stats(srv)
        rs.check(st, "rs_server_stats")
        rs.rs_server_destroy(srv)
        return stats, wall

    stats, _ = serve(range(count), paced=True)
    offered = float(sizes.sum()) / float(arrival[-1]) / 1e9
    link_after = host_link_gbs(torch, ring)

    # capacity: the first compare_requests requests, no arrival schedule
    sub = list(range(min(compare_requests, count)))
    sub_keys = float(sizes[sub].sum())
    sat, sat_wall = serve(sub, paced=False)
    # plain: one rs_sort_host per request, one stream, same pinned buffers
    maxn = int(sizes[sub].max())
    dev_k = torch.empty(maxn * 8, dtype=torch.uint8, device="cuda")
    dev_v = torch.empty(maxn * 8, dtype=torch.uint8, device="cuda")
    dev_ka = torch.empty_like(dev_k)
    dev_va = torch.empty_like(dev_v)
    need = max(rs.rs_workspace_bytes(4, 4, maxn, 0, 32)[1], rs.rs_workspace_bytes(8, 0, maxn, 0, 64)[1])
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    h = stream.cuda_stream
    out = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in sub:
        n = int(sizes[i])
        if out + 8 * n > ring_bytes:
            out = 0
        r = request(i, out)
        out += 8 * n
        st, _ = rs.rs_sort_host(r.key_bytes, r.val_bytes, r.h_keys, r.h_vals, r.h_out_keys,
                                r.h_out_vals, n, r.begin_bit, r.end_bit, dev_k.data_ptr(),
                                dev_v.data_ptr() if r.val_bytes else None, dev_ka.data_ptr(),
                                dev_va.data_ptr() if r.val_bytes else None, ws.data_ptr(),
                                ws.numel(), h)
        rs.check(st, "rs_sort_host (plain)")
    e1.record(stream)
    stream.synchronize()
    plain_wall = time.perf_counter() - t0
    plain_gpu_s = e0.elapsed_time(e1) / 1e3
    rs.check(rs.rs_workspace_status(ws.data_ptr(), h)[0], "plain device status")
    del dev_k, dev_v, dev_ka, dev_va, ws
    return {"requests": count, "rate_per_s": rate, "budget_gib": budget / 2**30,
            "streams": streams, "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
            "max_ms": stats["max_ms"], "wait_p99_ms": stats["wait_p99_ms"],
            "service_p50_ms": stats["service_p50_ms"],
            "service_p99_ms": stats["service_p99_ms"], "gkeys_per_s": stats["gkeys_per_s"],
            "offered_gkeys_per_s": offered, "batches": stats["batches"],
            "batched_requests": stats["batched_requests"], "max_queued": stats["max_queued"],
            "pool_peak_gib": stats["pool_peak_bytes"] / 2**30,
            "served_vs_plain": {
                "requests": len(sub), "keys": sub_keys,
                "served_gkeys_per_s": sub_keys / sat_wall / 1e9,
                "served_p50_ms": sat["p50_ms"], "served_p99_ms": sat["p99_ms"],
                "served_batches": sat["batches"], "served_batched_requests": sat["batched_requests"],
                "plain_gkeys_per_s": sub_keys / plain_wall / 1e9,
                "plain_gpu_gkeys_per_s": sub_keys / plain_gpu_s / 1e9,
                "served_over_plain": plain_wall / sat_wall,
                "what": "the first requests of the same trace submitted at once: served = "
                        "through the server (its capacity); plain = one rs_sort_host call per "
                        "request on one stream; both from and to pinned host memory, "
                        "wall-clock first submit -> last completion"},
            "host_link_gb_per_s": {"before": link_before, "after": link_after,
                                   "what": "256 MiB pinned copies, each direction alone"},
            "latency": "submit -> completion callback, host pinned buffers in and out; wait = "
                       "submit -> admission, service = admission -> completion"}


def host_link_gbs(torch, host_u8) -> dict:
    """Host<->device copy bandwidth (GB/s) right now, 256 MiB each way: the
    serving latencies depend on it, and on a shared host it varies."""
    nb = 256 << 20
    dev_buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    h = host_u8[:nb]
    out = {}
    for name in ("h2d", "d2h"):
        best = None
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if name == "h2d":
                dev_buf.copy_(h, non_blocking=True)
            else:
                h.copy_(dev_buf, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        out[name] = nb / (best / 1e3) / 1e9
    return out


def bench_serving_process(seconds: float) -> dict:
    """The serving trace in a child process of its own, the way a sort server
    runs: the benchmark's own process holds tens of GB of device and pinned
    host buffers by then, which a serving process does not."""
    code = ("import json, sys; sys.path.insert(0, %r); import torch, bench; "
            "from paper_1511_03404_gb300 import rs; rs.load(); "
            "print('SERVING ' + json.dumps(bench.bench_serving(torch, rs, seconds=%r)))"
            % (ROOT, float(seconds)))
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=600)
    for line in res.stdout.splitlines():
        if line.startswith("SERVING "):
            out = json.loads(line[len("SERVING "):])
            out["process"] = "own process (a dedicated serving process)"
            return out
    raise SystemExit(f"bench: serving child failed ({res.returncode}): {res.stderr[-2000:]}")


def stage(msg: str) -> None:
    """Progress marker on stderr (stdout carries only the JSON line)."""
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def main(argv=None):
    faulthandler.enable()
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=6)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=N_KEYS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="timed sorts only (no CPU baseline, no end-to-end leg, no check); "
                         "for profiler captures")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the segmented (batched vs plain) and serving measurements")
    ap.add_argument("--seg-scaled", action="store_true",
                    help="segment lengths scaled to a 2^28 total instead of the stated law")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--dist", choices=DISTS, default=None,
                    help="sort only this distribution (default: all six in turn)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
