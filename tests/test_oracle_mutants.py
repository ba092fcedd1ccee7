"""Plant mistakes in copies of the oracle and check that the pins catch them.

Each mutant is a plausible slip in the LSD counting sort of arXiv 1511.03404
Sec. 2.6 (unstable scatter, wrong digit order, wrong digit field, wrong
prefix, values not moved with their keys, a pass dropped), or in the order
keys of signed, float and descending sorts.  The mutated
source is compiled into a temporary library (on the CPU only) and the pin
checks of ``tests/test_oracle.py`` run against it in a child process; every
mutant must fail at least one of them.  The unmodified source must pass.
"""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))

MUTANTS = {
    "reverse_scatter_order": (
        "for (uint64_t i = 0; i < n; ++i) { /* input order: stable */",
        "for (uint64_t i = n; i-- > 0;) { /* input order: stable */"),
    "msd_first": (
        "for (int p = 0; p < passes; ++p) { /* least significant digit first */",
        "for (int p = passes - 1; p >= 0; --p) {"),
    "digit_too_narrow": ("int hi = lo + r;", "int hi = lo + r - 1;"),
    "digit_ignores_end_bit": ("if (hi > end_bit) hi = end_bit;", ""),
    "descending_prefix": (
        "for (uint64_t v = 0; v < radix; ++v) {\n    start[v] = run;",
        "for (uint64_t v = radix; v-- > 0;) {\n    start[v] = run;"),
    "values_left_behind": ("if (val) val_out[dst] = val[i];", "if (val) val_out[dst] = val[dst];"),
    "one_pass_short": ("return (end_bit - begin_bit + r - 1) / r;", "return (end_bit - begin_bit) / r;"),
    # key orders beyond unsigned keys
    "signed_read_as_unsigned": ("u = bits >= half ? bits - half : bits + half;", "u = bits;"),
    "float_sign_flip_only": ("u = (bits & half) ? half - 1 - m : half + m;", "u = bits ^ half;"),
    "float_zero_signs_merged": ("u = (bits & half) ? half - 1 - m : half + m;",
                                "u = (bits & half) ? half - m : half + m;"),
    "descending_ignored": ("return descending ? all - u : u;", "return u;"),
}

CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import inputs, oracle
import test_oracle as T
lib = oracle.bind(ctypes.CDLL({lib!r}))
fails = []
def check(name, fn):
    try:
        fn()
    except Exception as e:  # a pin failed
        fails.append(name)
def library_sort():
    for dtype in (np.uint32, np.uint64):
        for dist in ("uniform", "gaussian", "bucket", "entropy16"):
            k = inputs.keys(dtype, dist, 3000); v = inputs.values(dtype, 3000)
            sk, sv = oracle.lsd_sort(k, v, lib=lib)
            rk, perm = T.stable_reference(k)
            assert np.array_equal(sk, rk) and np.array_equal(sv, perm.astype(dtype))
def brute():
    import itertools
    for L in range(7):
        for seq in itertools.product([0, 1, 2**31, 2**32 - 1], repeat=L):
            k = np.array(seq, dtype=np.uint32)
            sk, sv = oracle.lsd_sort(k, np.arange(L, dtype=np.uint32), lib=lib)
            bk, bv = T.insertion_sort_pairs(seq)
            assert sk.tolist() == bk and sv.tolist() == bv
def bit_ranges():
    k = inputs.keys(np.uint32, "uniform", 2000); v = inputs.values(np.uint32, 2000)
    for b, e in [(0, 32), (3, 17), (4, 29)]:
        for r in (4, 8, 11):
            sk, sv = oracle.lsd_sort(k, v, begin_bit=b, end_bit=e, r=r, lib=lib)
            rk, perm = T.stable_reference(k, b, e)
            assert np.array_equal(sk, rk) and np.array_equal(sv, perm.astype(np.uint32))
def invariants():
    k = inputs.keys(np.uint64, "gaussian", 5000); k[::5] = k[1]
    v = inputs.values(np.uint64, 5000)
    sk, sv = oracle.lsd_sort(k, v, lib=lib)
    T.check_invariants(k, v, sk, sv)
check("library_sort", library_sort)
check("brute", brute)
check("bit_ranges", bit_ranges)
check("invariants", invariants)
import test_oracle_keyorder as KO
for name, pin in KO.PINS.items():
    check("keyorder_" + name, lambda: pin(lib))
print(",".join(fails))
"""


def run_pins(lib_path):
    code = CHILD.format(tests=HERE, root=os.path.dirname(HERE), lib=lib_path)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         timeout=300)
    assert res.returncode == 0, res.stderr
    out = res.stdout.strip().splitlines()
    return [f for f in (out[-1] if out else "").split(",") if f]


def test_unmodified_oracle_passes_pins(tmp_path):
    lib = oracle.compile_library(oracle.SOURCE, str(tmp_path / "liborig.so"))
    assert run_pins(lib) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    with open(oracle.SOURCE) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutated = tmp_path / f"{name}.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.compile_library(str(mutated), str(tmp_path / f"lib{name}.so"))
    caught = run_pins(lib)
    assert caught, f"mutant {name} survived every pin"
