"""Build the rs CUDA library in-tree: csrc/*.cu -> _build/librs.so (sm_103a).

Each translation unit is compiled by its own nvcc process (in parallel),
then linked into one shared library that exports the C ABI of
include/rs.h.  A stamp of the sources and flags skips rebuilds.

The debug flavour (_build/librs_debug.so, compiled with RS_DEBUG) checks the
index of every global store of its kernels (rs_debug_status); the binding
loads it instead of librs.so when the environment sets RS_LIBRARY=debug.

The package's tuned variant table (tuned.json) is compiled into the library
as its default table (_build/rs_tuned_table.inc), so that callers of the C
ABI get the tuned choices without the binding.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "librs.so")
DEBUG_LIB_PATH = os.path.join(OUT_DIR, "librs_debug.so")
DEBUG_FLAGS = ("-DRS_DEBUG",)
INCLUDE = os.path.join(ROOT, "include")
TUNED_JSON = os.path.join(HERE, "tuned.json")
TUNED_INC = os.path.join(OUT_DIR, "rs_tuned_table.inc")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the rs CUDA library cannot be built")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _stamp(extra=()) -> str:
    h = hashlib.sha256()
    files = sources() + sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                               if f.endswith((".h", ".cuh")))
    files.append(os.path.join(INCLUDE, "rs.h"))
    if os.path.exists(TUNED_JSON):
        files.append(TUNED_JSON)
    for f in files:
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()


def _compile(src: str, extra, suffix: str = ".o") -> str:
    obj = os.path.join(OUT_DIR, os.path.basename(src) + suffix)
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", OUT_DIR, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if "spill" in (res.stderr or "") and "0 bytes spill" not in res.stderr:
        print(res.stderr)
    return obj


def write_tuned_table(json_path: str = TUNED_JSON, out_path: str = TUNED_INC) -> int:
    """Write the entries of the tuned table as C initialisers
    ``{key_bytes, val_bytes, n_max, variant},`` (none when there is no table).
    Returns the number of entries written."""
    import json
    entries = []
    if os.path.exists(json_path):
        with open(json_path) as f:
            entries = json.load(f).get("entries", [])
    lines = ["// written by the build step from tuned.json; not edited by hand"]
    for e in entries:
        lines.append("{%d, %d, %dull, %d}," % (int(e["key_bytes"]), int(e["val_bytes"]),
                                              int(e["n_max"]), int(e["variant"])))
    tmp = out_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(tmp, out_path)
    return len(entries)


def _flavours(debug: bool | None):
    rel = (LIB_PATH, "librs.stamp", ".o", ())
    dbg = (DEBUG_LIB_PATH, "librs_debug.stamp", ".dbg.o", DEBUG_FLAGS)
    return {None: [rel, dbg], False: [rel], True: [dbg]}[debug]


def build(force: bool = False, extra_flags=(), jobs: int | None = None,
          debug: bool | None = False) -> str:
    """Compile every translation unit for sm_103a and link librs.so
    (debug=True: librs_debug.so; debug=None: both, compiled together).
    Returns the path of the (first) library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    todo = []
    for lib, stamp_name, suffix, flags in _flavours(debug):
        stamp_path = os.path.join(OUT_DIR, stamp_name)
        stamp = _stamp(tuple(extra_flags) + flags)
        if not force and os.path.exists(lib) and os.path.exists(stamp_path):
            with open(stamp_path) as f:
                if f.read() == stamp:
                    continue
        todo.append((lib, stamp_path, stamp, suffix, tuple(extra_flags) + flags))
    if todo:
        write_tuned_table()
        srcs = sources()
        units = [(src, t) for t in todo for src in srcs]
        jobs = jobs or min(len(units), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(jobs) as ex:
            objs = list(ex.map(lambda u: _compile(u[0], u[1][4], u[1][3]), units))
        for i, (lib, stamp_path, stamp, _, _) in enumerate(todo):
            tmp = lib + f".tmp{os.getpid()}"
            mine = objs[i * len(srcs):(i + 1) * len(srcs)]
            cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *mine]
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
            os.replace(tmp, lib)
            with open(stamp_path, "w") as f:
                f.write(stamp)
    return _flavours(debug)[0][0]


if __name__ == "__main__":
    print(build(force=True, debug=None))
