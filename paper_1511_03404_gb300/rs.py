"""Python binding of the rs C ABI (include/rs.h): ctypes, argument marshalling only.

Every function named ``rs_*`` here calls the C entry point of the same name
in ``_build/librs.so`` with plain integers (device pointers, sizes, a
``cudaStream_t`` handle) and returns what it returns; every step of the sort
runs in the library's CUDA kernels.  There is no CPU fallback: if the library
cannot be built or loaded, loading raises.

``sort()`` and ``segmented_sort()`` at the bottom are conveniences over torch
tensors: torch only provides the device memory and the stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

RS_OK = 0
RS_ERR_INVALID = 1
RS_ERR_NOMEM = 2
RS_ERR_CUDA = 3
RS_ERR_TIMEOUT = 4
RS_ERR_BUSY = 5
RS_ERR_WORKSPACE = 6
RS_ERR_DEVICE = 7
RS_ERR_CANCELLED = 8
RS_ERR_NOT_FOUND = 9
RS_MAX_N = (1 << 30) - 1

(RS_KERNEL_UPSWEEP, RS_KERNEL_ONESWEEP, RS_KERNEL_SMALL, RS_KERNEL_SEGMENTED, RS_KERNEL_MERGE,
 RS_KERNEL_SAMPLE) = range(6)
RS_KERNEL_KINDS = 6
KERNEL_NAMES = ("upsweep", "onesweep", "small", "segmented", "merge", "sample")

(RS_DEBUG_TIMEOUT_NS, RS_DEBUG_DROP_PUBLISH_TILE, RS_DEBUG_DROP_PUBLISH_PASS, RS_DEBUG_TRACE_PTR,
 RS_DEBUG_TRACE_TILES, RS_DEBUG_TRACE_PASS, RS_DEBUG_LB_SMALL, RS_DEBUG_BAD_INDEX_TILE) = range(8)


class RsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}")


class rs_config(ctypes.Structure):
    _fields_ = [("radix_bits", ctypes.c_int), ("variant", ctypes.c_int),
                ("key_kind", ctypes.c_int), ("descending", ctypes.c_int)]


class rs_request(ctypes.Structure):
    _fields_ = [("key_bytes", ctypes.c_int), ("val_bytes", ctypes.c_int),
                ("n", ctypes.c_size_t), ("begin_bit", ctypes.c_int), ("end_bit", ctypes.c_int),
                ("h_keys", ctypes.c_void_p), ("h_vals", ctypes.c_void_p),
                ("h_out_keys", ctypes.c_void_p), ("h_out_vals", ctypes.c_void_p)]


class rs_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("keys", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batched_requests", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("max_queued", ctypes.c_uint64), ("pool_peak_bytes", ctypes.c_size_t),
                ("pool_used_bytes", ctypes.c_size_t), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("gkeys_per_s", ctypes.c_double),
                ("wait_p50_ms", ctypes.c_double), ("wait_p99_ms", ctypes.c_double),
                ("service_p50_ms", ctypes.c_double), ("service_p99_ms", ctypes.c_double)]


class rs_server_config(ctypes.Structure):
    _fields_ = [("batch_max_n", ctypes.c_size_t), ("max_batch_keys", ctypes.c_size_t),
                ("large_n", ctypes.c_size_t), ("max_large", ctypes.c_int),
                ("large_low_priority", ctypes.c_int), ("shared_copy_queues", ctypes.c_int)]


class rs_sort_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("info", ctypes.c_uint32), ("form", ctypes.c_int),
                ("key_bytes", ctypes.c_int), ("val_bytes", ctypes.c_int),
                ("passes", ctypes.c_int), ("n", ctypes.c_uint64),
                ("moved_mask", ctypes.c_uint32), ("skipped_mask", ctypes.c_uint32),
                ("upsweep_ms", ctypes.c_double), ("pass_ms", ctypes.c_double * 16),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class rs_trace_record(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("n", ctypes.c_uint64),
                ("key_bytes", ctypes.c_int), ("val_bytes", ctypes.c_int),
                ("stream", ctypes.c_int), ("batched", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_vp, _sz, _i, _u32p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
_SIGS = {
    "rs_status_string": ([_i], ctypes.c_char_p),
    "rs_version": ([], ctypes.c_char_p),
    "rs_num_variants": ([_i, _i], _i),
    "rs_variant_info": ([_i, _i, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "rs_workspace_bytes": ([_i, _i, _sz, _i, _i, _vp, _vp], _i),
    "rs_sort_keys_u32": ([_vp, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp], _i),
    "rs_sort_keys_u64": ([_vp, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp], _i),
    "rs_sort_pairs_u32": ([_vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp], _i),
    "rs_sort_pairs_u64": ([_vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp], _i),
    "rs_sort_keys_u32_noalloc": ([_vp, _vp, _sz, _i, _i, _vp, _vp], _i),
    "rs_sort_keys_u32_noalloc_status": ([_vp, _vp], _i),
    "rs_sort_host": ([_i, _i, _vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                      _vp, _vp], _i),
    "rs_workspace_stats": ([_vp, _vp, _vp], _i),
    "rs_sort": ([_i, _i, _vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _vp, _sz, _vp, _vp], _i),
    "rs_digit_counts": ([_i, _vp, _sz, _i, _i, _i, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "rs_workspace_status": ([_vp, _vp, _vp], _i),
    "rs_segmented_sort_pairs": ([_vp, _vp, _vp, _vp, _sz, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp],
                                _i),
    "rs_segmented_workspace_bytes": ([_sz, _sz, _i, _i, _vp], _i),
    "rs_segmented_sort": ([_i, _i, _vp, _vp, _vp, _vp, _sz, _vp, _sz, _i, _i, _vp, _sz, _vp, _vp],
                          _i),
    "rs_segmented_workspace_bytes_typed": ([_i, _i, _sz, _sz, _i, _i, _vp], _i),
    "rs_sample_workspace_bytes": ([_sz, _i, _i, _vp], _i),
    "rs_merge_workspace_bytes": ([_i, _i, _sz, _vp], _i),
    "rs_merge_sort": ([_i, _i, _vp, _vp, _vp, _vp, _sz, _vp, _sz, _vp, _vp], _i),
    "rs_sample_partition_pairs_u32": ([_vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _vp, _vp, _sz, _vp],
                                      _i),
    "rs_sample_sort_pairs_u32": ([_vp, _vp, _vp, _vp, _sz, _i, _i, _vp, _vp, _sz, _vp, _vp], _i),
    "rs_server_create": ([_sz, _i, _vp], _i),
    "rs_server_destroy": ([_vp], _i),
    "rs_submit": ([_vp, _vp, _vp], _i),
    "rs_poll": ([_vp, ctypes.c_uint64, _vp], _i),
    "rs_cancel": ([_vp, ctypes.c_uint64], _i),
    "rs_server_stats": ([_vp, _vp], _i),
    "rs_server_reset_stats": ([_vp], _i),
    "rs_server_trace": ([_vp, _vp, _sz, _vp], _i),
    "rs_server_get_config": ([_vp, _vp], _i),
    "rs_server_completed": ([_vp, _vp, _sz, _vp], _i),
    "rs_server_set_config": ([_vp, _vp], _i),
    "rs_tune_set": ([_i, _i, _sz, _i], _i),
    "rs_tune_clear": ([], _i),
    "rs_profile_begin": ([_i], _i),
    "rs_profile_end": ([_vp, _vp, _vp], _i),
    "rs_debug_set": ([_i, ctypes.c_longlong], _i),
    "rs_debug_status": ([_vp, _vp, _vp], _i),
}


def debug_library() -> bool:
    """Whether this process uses the debug build (RS_LIBRARY=debug)."""
    return os.environ.get("RS_LIBRARY", "") == "debug"


def library_path() -> str:
    return _build.DEBUG_LIB_PATH if debug_library() else _build.LIB_PATH


def load():
    """Build (if needed) and load librs.so (librs_debug.so when the
    environment sets RS_LIBRARY=debug); raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=debug_library())
            lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            for name, (args, res) in _SIGS.items():
                if not hasattr(lib, name):
                    continue  # a library built from an older header
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
            _apply_tuned_table(lib)
    return _lib


TUNED_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def _apply_tuned_table(lib, path: str | None = None) -> int:
    """Load the autotuner's table (tuned.json next to this file) into the library.

    Returns the number of entries applied (0 when there is no table, or when
    RS_NO_TUNED_TABLE is set)."""
    import json
    path = path or TUNED_TABLE
    if os.environ.get("RS_NO_TUNED_TABLE") or not os.path.exists(path):
        return 0
    with open(path) as f:
        table = json.load(f)
    applied = 0
    for e in table.get("entries", []):
        if lib.rs_tune_set(e["key_bytes"], e["val_bytes"], e["n_max"], e["variant"]) == RS_OK:
            applied += 1
    return applied


def declared_symbols() -> list[str]:
    return list(_SIGS)


def status_string(status: int) -> str:
    return load().rs_status_string(status).decode()


def check(status: int, what: str = "rs") -> None:
    if status != RS_OK:
        raise RsError(status, what)


def _out_int():
    return ctypes.c_int(0)


# ------------------------------------------------------------------ C ABI
# Same names and arguments as include/rs.h; pointers are Python ints.

def rs_version() -> str:
    return load().rs_version().decode()


def rs_num_variants(key_bytes: int, val_bytes: int) -> int:
    return load().rs_num_variants(key_bytes, val_bytes)


def rs_variant_info(key_bytes: int, val_bytes: int, index: int):
    r, t, it, k = (ctypes.c_int() for _ in range(4))
    mx = ctypes.c_size_t()
    st = load().rs_variant_info(key_bytes, val_bytes, index, ctypes.byref(r), ctypes.byref(t),
                                ctypes.byref(it), ctypes.byref(k), ctypes.byref(mx))
    check(st, "rs_variant_info")
    return {"radix_bits": r.value, "threads": t.value, "items": it.value, "kind": k.value,
            "max_n": mx.value}


RS_KEY_UNSIGNED, RS_KEY_SIGNED, RS_KEY_FLOAT = range(3)


def _cfg(radix_bits=0, variant=-1, key_kind=RS_KEY_UNSIGNED, descending=False):
    if radix_bits == 0 and variant < 0 and key_kind == RS_KEY_UNSIGNED and not descending:
        return None
    return ctypes.byref(rs_config(radix_bits, variant, key_kind, int(descending)))


def rs_workspace_bytes(key_bytes, val_bytes, n, begin_bit, end_bit, radix_bits=0, variant=-1):
    out = ctypes.c_size_t()
    st = load().rs_workspace_bytes(key_bytes, val_bytes, n, begin_bit, end_bit,
                                   _cfg(radix_bits, variant), ctypes.byref(out))
    return st, out.value


def rs_sort_keys_u32(keys, keys_alt, n, begin_bit, end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_sort_keys_u32(keys, keys_alt, n, begin_bit, end_bit, ws, ws_bytes, stream,
                                 ctypes.byref(r))
    return st, r.value


def rs_sort_keys_u64(keys, keys_alt, n, begin_bit, end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_sort_keys_u64(keys, keys_alt, n, begin_bit, end_bit, ws, ws_bytes, stream,
                                 ctypes.byref(r))
    return st, r.value


def rs_sort_pairs_u32(keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_sort_pairs_u32(keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, ws,
                                  ws_bytes, stream, ctypes.byref(r))
    return st, r.value


def rs_sort_pairs_u64(keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_sort_pairs_u64(keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, ws,
                                  ws_bytes, stream, ctypes.byref(r))
    return st, r.value


RS_NOALLOC_MAX_N = 1 << 23
RS_NOALLOC_SCRATCH_BYTES = 9 << 20


def rs_sort_keys_u32_noalloc(keys, keys_alt, n, begin_bit, end_bit, stream):
    r = _out_int()
    st = load().rs_sort_keys_u32_noalloc(keys, keys_alt, n, begin_bit, end_bit, stream,
                                         ctypes.byref(r))
    return st, r.value


def rs_sort_keys_u32_noalloc_status(stream):
    info = ctypes.c_uint32()
    st = load().rs_sort_keys_u32_noalloc_status(stream, ctypes.byref(info))
    return st, info.value


def rs_sort_host(key_bytes, val_bytes, h_keys, h_vals, h_out_keys, h_out_vals, n, begin_bit,
                 end_bit, keys, vals, keys_alt, vals_alt, ws, ws_bytes, stream, radix_bits=0,
                 variant=-1, key_kind=RS_KEY_UNSIGNED, descending=False):
    r = _out_int()
    st = load().rs_sort_host(key_bytes, val_bytes, h_keys, h_vals, h_out_keys, h_out_vals, n,
                             begin_bit, end_bit, _cfg(radix_bits, variant, key_kind, descending),
                             keys, vals, keys_alt, vals_alt, ws, ws_bytes, stream,
                             ctypes.byref(r))
    return st, r.value


def rs_workspace_stats(ws, stream):
    """(status, dict) with the fields of rs_sort_stats; pass_ms as a list of `passes` floats."""
    out = rs_sort_stats()
    st = load().rs_workspace_stats(ws, stream, ctypes.byref(out))
    d = {name: getattr(out, name) for name, _ in rs_sort_stats._fields_}
    d["pass_ms"] = list(out.pass_ms)[:max(0, out.passes)]
    return st, d


def rs_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, begin_bit, end_bit, ws,
            ws_bytes, stream, radix_bits=0, variant=-1, key_kind=RS_KEY_UNSIGNED,
            descending=False):
    r = _out_int()
    st = load().rs_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, begin_bit,
                        end_bit, _cfg(radix_bits, variant, key_kind, descending), ws, ws_bytes,
                        stream, ctypes.byref(r))
    return st, r.value


def rs_digit_counts(key_bytes, keys, n, begin_bit, end_bit, radix_bits, d_counts, d_offsets,
                    d_exec_mask, ws, ws_bytes, stream):
    return load().rs_digit_counts(key_bytes, keys, n, begin_bit, end_bit, radix_bits, d_counts,
                                  d_offsets, d_exec_mask, ws, ws_bytes, stream)


def rs_segmented_sort_pairs(keys, vals, keys_alt, vals_alt, n, d_offsets, n_seg, begin_bit,
                            end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_segmented_sort_pairs(keys, vals, keys_alt, vals_alt, n, d_offsets, n_seg,
                                        begin_bit, end_bit, ws, ws_bytes, stream,
                                        ctypes.byref(r))
    return st, r.value


def rs_segmented_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, d_offsets, n_seg,
                      begin_bit, end_bit, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_segmented_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n,
                                  d_offsets, n_seg, begin_bit, end_bit, ws, ws_bytes, stream,
                                  ctypes.byref(r))
    return st, r.value


def rs_segmented_workspace_bytes_typed(key_bytes, val_bytes, n, n_seg, begin_bit=0, end_bit=None):
    out = ctypes.c_size_t()
    end_bit = 8 * key_bytes if end_bit is None else end_bit
    st = load().rs_segmented_workspace_bytes_typed(key_bytes, val_bytes, n, n_seg, begin_bit,
                                                   end_bit, ctypes.byref(out))
    return st, out.value


def rs_segmented_workspace_bytes(n, n_seg, begin_bit=0, end_bit=32):
    out = ctypes.c_size_t()
    st = load().rs_segmented_workspace_bytes(n, n_seg, begin_bit, end_bit, ctypes.byref(out))
    return st, out.value


def rs_sample_workspace_bytes(n, samples, buckets):
    out = ctypes.c_size_t()
    st = load().rs_sample_workspace_bytes(n, samples, buckets, ctypes.byref(out))
    return st, out.value


def rs_sample_partition_pairs_u32(keys, vals, keys_out, vals_out, n, samples, buckets,
                                  d_bucket_offsets, d_splitters, ws, ws_bytes, stream):
    return load().rs_sample_partition_pairs_u32(keys, vals, keys_out, vals_out, n, samples,
                                                buckets, d_bucket_offsets, d_splitters, ws,
                                                ws_bytes, stream)


def rs_sample_sort_pairs_u32(keys, vals, keys_out, vals_out, n, samples, buckets,
                             d_bucket_offsets, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_sample_sort_pairs_u32(keys, vals, keys_out, vals_out, n, samples, buckets,
                                         d_bucket_offsets, ws, ws_bytes, stream, ctypes.byref(r))
    return st, r.value


def rs_merge_workspace_bytes(key_bytes, val_bytes, n):
    out = ctypes.c_size_t()
    st = load().rs_merge_workspace_bytes(key_bytes, val_bytes, n, ctypes.byref(out))
    return st, out.value


def rs_merge_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, ws, ws_bytes, stream):
    r = _out_int()
    st = load().rs_merge_sort(key_bytes, val_bytes, keys, vals, keys_alt, vals_alt, n, ws,
                              ws_bytes, stream, ctypes.byref(r))
    return st, r.value


def rs_workspace_status(ws, stream):
    info = ctypes.c_uint32()
    st = load().rs_workspace_status(ws, stream, ctypes.byref(info))
    return st, info.value


def rs_server_create(budget_bytes: int, streams: int):
    out = ctypes.c_void_p()
    st = load().rs_server_create(budget_bytes, streams, ctypes.byref(out))
    return st, out.value


def rs_server_destroy(server) -> int:
    return load().rs_server_destroy(server)


def rs_submit(server, req: rs_request):
    h = ctypes.c_uint64()
    st = load().rs_submit(server, ctypes.byref(req), ctypes.byref(h))
    return st, h.value


def rs_poll(server, handle: int):
    done = ctypes.c_int()
    st = load().rs_poll(server, handle, ctypes.byref(done))
    return st, bool(done.value)


def rs_cancel(server, handle: int) -> int:
    return load().rs_cancel(server, handle)


def rs_server_stats(server):
    out = rs_server_stats_t()
    st = load().rs_server_stats(server, ctypes.byref(out))
    return st, {name: getattr(out, name) for name, _ in rs_server_stats_t._fields_}


def rs_server_reset_stats(server) -> int:
    return load().rs_server_reset_stats(server)


def rs_server_completed(server, cap: int = 1024):
    """(status, handles of requests finished since the last call, oldest first)."""
    buf = (ctypes.c_uint64 * max(cap, 1))()
    count = ctypes.c_size_t()
    st = load().rs_server_completed(server, buf, cap, ctypes.byref(count))
    return st, [buf[i] for i in range(count.value)]


def rs_server_get_config(server):
    out = rs_server_config()
    st = load().rs_server_get_config(server, ctypes.byref(out))
    return st, {name: getattr(out, name) for name, _ in rs_server_config._fields_}


def rs_server_set_config(server, cfg: dict) -> int:
    return load().rs_server_set_config(server, ctypes.byref(rs_server_config(**cfg)))


def rs_server_trace(server):
    """(status, list of per-request dicts) for every completed request."""
    total = ctypes.c_size_t()
    st = load().rs_server_trace(server, None, 0, ctypes.byref(total))
    if st != RS_OK:
        return st, []
    buf = (rs_trace_record * max(total.value, 1))()
    st = load().rs_server_trace(server, buf, total.value, ctypes.byref(total))
    names = [name for name, _ in rs_trace_record._fields_]
    return st, [{k: getattr(buf[i], k) for k in names} for i in range(min(total.value, len(buf)))]


def rs_tune_set(key_bytes: int, val_bytes: int, n_max: int, variant: int) -> int:
    return load().rs_tune_set(key_bytes, val_bytes, n_max, variant)


def rs_tune_clear() -> int:
    return load().rs_tune_clear()


def rs_profile_begin(capacity: int) -> int:
    return load().rs_profile_begin(capacity)


def rs_profile_end():
    launches = (ctypes.c_int * RS_KERNEL_KINDS)()
    ms = (ctypes.c_double * RS_KERNEL_KINDS)()
    by = (ctypes.c_double * RS_KERNEL_KINDS)()
    st = load().rs_profile_end(launches, ms, by)
    return st, {KERNEL_NAMES[k]: {"launches": launches[k], "ms": ms[k], "bytes": by[k]}
                for k in range(RS_KERNEL_KINDS)}


def rs_debug_status():
    """(status, debug_build, site, index) of the bounds checks of a debug build."""
    dbg, site, index = ctypes.c_int(), ctypes.c_uint32(), ctypes.c_uint64()
    st = load().rs_debug_status(ctypes.byref(dbg), ctypes.byref(site), ctypes.byref(index))
    return st, bool(dbg.value), site.value, index.value


def rs_debug_set(knob: int, value: int) -> int:
    return load().rs_debug_set(knob, value)


# ------------------------------------------------------- torch conveniences

def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# dtype name -> (bytes, key kind)
_KEY_TYPES = {"uint32": (4, RS_KEY_UNSIGNED), "int32": (4, RS_KEY_SIGNED),
              "uint64": (8, RS_KEY_UNSIGNED), "int64": (8, RS_KEY_SIGNED),
              "float32": (4, RS_KEY_FLOAT), "float64": (8, RS_KEY_FLOAT)}


def _key_type(t):
    name = str(t.dtype).replace("torch.", "")
    if name not in _KEY_TYPES:
        raise TypeError(f"expected a 32- or 64-bit integer or float tensor, got {t.dtype}")
    return _KEY_TYPES[name]


def _key_bytes(t) -> int:
    return _key_type(t)[0]


def workspace(key_bytes, val_bytes, n, begin_bit=0, end_bit=None, radix_bits=0, variant=-1,
              device=None):
    """A torch uint8 device tensor large enough for one sort."""
    torch = _torch()
    end_bit = 8 * key_bytes if end_bit is None else end_bit
    st, nbytes = rs_workspace_bytes(key_bytes, val_bytes, n, begin_bit, end_bit, radix_bits,
                                    variant)
    check(st, "rs_workspace_bytes")
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device or "cuda")


def sort(keys, vals=None, begin_bit=0, end_bit=None, radix_bits=0, variant=-1, stream=None,
         ws=None, alt=None, descending=False, key_kind=None):
    """Sort contiguous device tensors in place (stable).

    ``keys`` (and ``vals``, any dtype of the keys' width) are overwritten with
    the sorted sequence.  The key order follows the dtype: unsigned, signed
    (int32 / int64) or IEEE float (float32 / float64, -0.0 before +0.0, NaNs
    by sign at the ends); ``key_kind`` overrides it (for instance
    ``RS_KEY_UNSIGNED`` to sort int32 storage as unsigned bit patterns).
    Returns ``(keys, vals)``.
    """
    torch = _torch()
    if not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    kb, kind = _key_type(keys)
    if key_kind is not None:
        kind = key_kind
    vb = 0
    if vals is not None:
        vb = _key_bytes(vals)
        if vb != kb or vals.numel() != keys.numel() or not vals.is_contiguous():
            raise ValueError("vals must match the keys' width and length")
    n = keys.numel()
    end_bit = 8 * kb if end_bit is None else end_bit
    if ws is None:
        ws = workspace(kb, vb, n, begin_bit, end_bit, radix_bits, variant, keys.device)
    if alt is None:
        ka = torch.empty_like(keys)
        va = torch.empty_like(vals) if vals is not None else None
    else:
        ka, va = alt
    st, in_alt = rs_sort(kb, vb, keys.data_ptr(), vals.data_ptr() if vals is not None else None,
                         ka.data_ptr(), va.data_ptr() if va is not None else None, n, begin_bit,
                         end_bit, ws.data_ptr(), ws.numel(), _stream_handle(stream), radix_bits,
                         variant, kind, descending)
    check(st, "rs_sort")
    if in_alt:
        keys.copy_(ka)
        if vals is not None:
            vals.copy_(va)
    return keys, vals


def segmented_sort(keys, offsets, vals=None, begin_bit=0, end_bit=None, stream=None, ws=None):
    """Sort every segment [offsets[s], offsets[s+1]) of contiguous device
    tensors in place (stable), in one launch sequence (rs_segmented_sort).

    ``keys`` and ``vals`` are 32- or 64-bit tensors of one width (``vals``
    optional); the keys are ordered as unsigned bit patterns over
    [begin_bit, end_bit).  ``offsets`` is a uint64/int64 device tensor of
    n_seg + 1 entries.  Returns ``(keys, vals)``.
    """
    torch = _torch()
    if not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    kb = _key_bytes(keys)
    vb = 0
    if vals is not None:
        vb = _key_bytes(vals)
        if vb != kb or vals.numel() != keys.numel() or not vals.is_contiguous():
            raise ValueError("vals must match the keys' width and length")
    if offsets.dtype not in (torch.int64, torch.uint64) or not offsets.is_contiguous():
        raise ValueError("offsets must be a contiguous 64-bit integer tensor")
    n, nseg = keys.numel(), offsets.numel() - 1
    end_bit = 8 * kb if end_bit is None else end_bit
    if ws is None:
        st, need = rs_segmented_workspace_bytes_typed(kb, vb, n, nseg, begin_bit, end_bit)
        check(st, "rs_segmented_workspace_bytes_typed")
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=keys.device)
    ka = torch.empty_like(keys)
    va = torch.empty_like(vals) if vals is not None else None
    ptr = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    st, in_alt = rs_segmented_sort(kb, vb, ptr(keys), ptr(vals), ptr(ka), ptr(va), n,
                                   offsets.data_ptr(), nseg, begin_bit, end_bit, ws.data_ptr(),
                                   ws.numel(), _stream_handle(stream))
    check(st, "rs_segmented_sort")
    if in_alt:
        keys.copy_(ka)
        if vals is not None:
            vals.copy_(va)
    return keys, vals
