"""Host logic of the sort-rate sweep (no GPU): the paper's length grid and
the table layout."""
from paper_1511_03404_gb300 import sweep


def test_paper_length_grid():
    n32 = sweep.lengths(4)
    assert n32[0] == 2**15 and n32[1] == 2**15 + 2**14 and n32[-1] == 2**25
    assert len(n32) == 2 * (25 - 15) + 1
    n64 = sweep.lengths(8)
    assert n64[-1] == 2**24 and len(n64) == 2 * (24 - 15) + 1
    assert sweep.lengths(4, max_log2=17) == [2**15, 3 * 2**14, 2**16, 3 * 2**15, 2**17]


def test_markdown_table():
    rows = [{"type": "kv32", "dist": d, "n": n, "median_ms": 1.0, "mean_ms": 1.0,
             "mkeys_per_s": n / 1e3, "ok": d != "zero"}
            for n in (2**15, 3 * 2**14) for d in ("uniform", "zero")]
    md = sweep.markdown({"reps": 50, "rows": rows})
    lines = md.splitlines()
    assert lines[0].startswith("**kv32**") and "| n | uniform | zero |" in lines
    assert "| 2^15 | 33 | 33 (WRONG) |" in lines
    assert "| 2^15+2^14 | 49 | 49 (WRONG) |" in lines
