"""Host logic of the autotuner's table (no GPU): the largest swept size's
variant is extended to the largest sortable array, and only when that
variant can sort arrays of any size."""
from paper_1511_03404_gb300 import autotune, rs


def _entry(kb, vb, n, variant):
    return {"key_bytes": kb, "val_bytes": vb, "n_max": n, "variant": variant, "ms": 1.0,
            "variant_info": {"max_n": 0}}


def test_extend_to_max_repeats_the_top_variant():
    infos = [{"max_n": rs.RS_MAX_N}, {"max_n": 8192}, {"max_n": rs.RS_MAX_N}]
    entries = [_entry(4, 4, 1 << 24, 0), _entry(4, 4, 1 << 26, 2), _entry(8, 0, 1 << 26, 0)]
    autotune.extend_to_max(entries, 4, 4, infos)
    extra = [e for e in entries if e["n_max"] == rs.RS_MAX_N]
    assert len(extra) == 1
    assert (extra[0]["key_bytes"], extra[0]["val_bytes"], extra[0]["variant"]) == (4, 4, 2)
    assert extra[0]["extrapolated_from"] == 1 << 26
    autotune.extend_to_max(entries, 4, 4, infos)  # already extended: nothing more
    assert sum(e["n_max"] == rs.RS_MAX_N for e in entries) == 1


def test_extend_to_max_skips_bounded_variants_and_missing_types():
    infos = [{"max_n": rs.RS_MAX_N}, {"max_n": 8192}]
    entries = [_entry(4, 0, 8192, 1)]
    autotune.extend_to_max(entries, 4, 0, infos)  # a one-CTA form cannot take larger arrays
    assert len(entries) == 1
    autotune.extend_to_max(entries, 8, 8, infos)  # no entries of that type
    assert len(entries) == 1


def test_tuned_sizes_cover_the_paper_grid():
    """Every length of the paper's grid (Sec. 3: 2^e and 2^e + 2^(e-1)) is a
    measured size of the autotuner, so that no length the sweep reports falls
    between two tuned bands; and the committed table has an entry at each."""
    import json
    from paper_1511_03404_gb300 import sweep
    grid = set(sweep.lengths(4)) | set(sweep.lengths(8))
    assert grid <= set(autotune.SIZES)
    with open(rs.TUNED_TABLE) as f:
        table = json.load(f)
    for kb, vb in autotune.TYPES:
        have = {e["n_max"] for e in table["entries"] if (e["key_bytes"], e["val_bytes"]) == (kb, vb)}
        assert set(sweep.lengths(kb)) <= have, (kb, vb)
