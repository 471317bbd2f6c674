"""The cutoff table (sq_set_cutoff_table / sq_cutoff_for) and the autotuner's
host logic, without a GPU: lookup by floor(log2 n), validation, clearing, and
loading a tuning file."""
import json

import pytest


@pytest.fixture()
def sq():
    from paper_2407_14801_gb300 import build

    build.build()
    import paper_2407_14801_gb300 as sq

    sq.lib()
    saved = {d: [sq.cutoff_for(d, 1 << lg) for lg in range(64)] for d in sq.DTYPES}
    yield sq
    for d in sq.DTYPES:
        sq.set_cutoff_table(d, [])
        default = sq.get_cutoff(d)
        sq.set_cutoff_table(d, [c if c != default else 0 for c in saved[d]])


def test_lookup_by_floor_log2(sq):
    sq.set_cutoff_table("u32", {20: 4096, 21: 8192})
    default = sq.get_cutoff("u32")
    assert sq.cutoff_for("u32", (1 << 20) - 1) == default
    assert sq.cutoff_for("u32", 1 << 20) == 4096
    assert sq.cutoff_for("u32", (1 << 21) - 1) == 4096
    assert sq.cutoff_for("u32", 1 << 21) == 8192
    assert sq.cutoff_for("u32", 1 << 22) == default
    assert sq.cutoff_for("u32", 0) == default
    sq.set_cutoff_table("u64", [])
    assert sq.cutoff_for("u64", 1 << 20) == sq.get_cutoff("u64")  # per key type


def test_table_replaces_and_clears(sq):
    sq.set_cutoff_table("f32", {10: 2048})
    sq.set_cutoff_table("f32", {11: 16384})
    assert sq.cutoff_for("f32", 1 << 10) == sq.get_cutoff("f32")
    assert sq.cutoff_for("f32", 1 << 11) == 16384
    sq.set_cutoff_table("f32", [])
    assert sq.cutoff_for("f32", 1 << 11) == sq.get_cutoff("f32")


def test_an_explicit_cutoff_overrides_the_table(sq):
    sq.set_cutoff_table("u32", {5: 64})
    assert sq.cutoff_for("u32", 40) == 64
    sq.set_cutoff("u32", 300)
    try:
        assert sq.cutoff_for("u32", 40) == 300 and sq.cutoff_for("u32", 1000) == 300
    finally:
        sq.set_cutoff("u32", 0)
    assert sq.cutoff_for("u32", 40) == 64 and sq.cutoff_for("u32", 1000) == sq.get_cutoff("u32")


def test_rejects_bad_tables(sq):
    import ctypes

    L = sq.lib()
    sq.set_cutoff_table("u32", {7: 512})
    with pytest.raises(sq.SquareSortError):
        sq.set_cutoff_table("u32", {3: 1})
    with pytest.raises(sq.SquareSortError):
        sq.set_cutoff_table("u32", {3: sq.max_leaf("u32") + 1})
    assert sq.cutoff_for("u32", 1 << 7) == 512  # a rejected table changes nothing
    buf = (ctypes.c_uint32 * 65)()
    assert L.sq_set_cutoff_table(0, buf, 65) == 1
    assert L.sq_set_cutoff_table(0, None, 3) == 1
    assert L.sq_set_cutoff_table(9, buf, 1) == 1
    assert L.sq_cutoff_for(9, 100) == 0


def test_load_tuning_file(sq, tmp_path):
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps({"cutoff_by_log2n": {"u64": {"18": 8192, "19": 16384}}}))
    assert sq.load_tuning(str(path))
    assert sq.cutoff_for("u64", 1 << 18) == 8192 and sq.cutoff_for("u64", 3 << 18) == 16384
    assert not sq.load_tuning(str(tmp_path / "absent.json"))


def test_fill_takes_the_nearest_measured_size():
    from paper_2407_14801_gb300.autotune import fill

    t = fill({"16": 8192, "20": 32768, "24": 65536})
    assert len(t) == 64
    assert t["0"] == t["15"] == t["16"] == t["17"] == t["18"] == 8192  # 18: tie, smaller size wins
    assert t["19"] == t["20"] == t["21"] == t["22"] == 32768
    assert t["23"] == t["24"] == t["63"] == 65536
    assert fill({}) == {}


def test_choose_prefers_larger_cutoffs_within_the_tie():
    from paper_2407_14801_gb300.autotune import choose, retable

    assert choose({"2048": 1.0, "65536": 1.5}) == 2048
    assert choose({"2048": 1.0, "65536": 1.015}) == 65536
    assert choose({"8192": 2.0, "32768": 1.9, "65536": 2.1}) == 32768
    t = retable({"u32": {"20": {"8192": 1.0, "65536": 1.3}, "24": {"8192": 1.0, "65536": 1.0}}})
    assert t["u32"]["20"] == 8192 and t["u32"]["24"] == 65536 and t["u32"]["0"] == 8192


def test_sweep_report_and_level_steps():
    """The cutoff-experiment report (no GPU): normalised time is
    ms * 1e6 / (n log2 n); a table row per size; an extra recursion level is
    read where the round count rises with n."""
    from paper_2407_14801_gb300 import autotune as at

    assert abs(at.normalised_ns(1.0, 1 << 20) - 1e6 / ((1 << 20) * 20)) < 1e-12
    doc = {"cutoffs": [64, 65536], "points": {"u32": {
        "10": {"64": {"ns_per_n_log2n": 1.0, "rounds": 3}, "65536": {"ns_per_n_log2n": 0.5, "rounds": 1}},
        "12": {"64": {"ns_per_n_log2n": 1.1, "rounds": 3}, "65536": {"ns_per_n_log2n": 0.4, "rounds": 1}},
        "14": {"64": {"ns_per_n_log2n": 1.3, "rounds": 5}, "65536": {"ns_per_n_log2n": 0.3, "rounds": 1}},
        "18": {"64": {"ns_per_n_log2n": 1.4, "rounds": 5}, "65536": {"ns_per_n_log2n": 0.6, "rounds": 4}}}}}
    text = at.report(doc)
    assert "| 2^14 | 1.3000 (5) | 0.3000 (1) |" in text
    assert at.level_steps(doc, "u32", 64) == [14]
    assert at.level_steps(doc, "u32", 65536) == [18]


def test_radix_classes_setting(sq):
    """sq_set_radix_classes / sq_get_radix_classes (no GPU): per key type, only
    classes 2..10 kept, uint64 refused, and a tuning file applies its masks."""
    import os
    import tempfile

    before = {d: sq.get_radix_classes(d) for d in ("u32", "f32")}
    try:
        assert sq.get_radix_classes("u64") == 0
        sq.set_radix_classes("u32", 0x30)
        assert sq.get_radix_classes("u32") == 0x30 and sq.get_radix_classes("f32") == before["f32"]
        sq.set_radix_classes("f32", 0xFFFF)
        assert sq.get_radix_classes("f32") == sq.RADIX_CLASSES_ALL
        with pytest.raises(sq.SquareSortError):
            sq.set_radix_classes("u64", 0x10)
        sq.set_radix_classes("u64", 0)
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "t.json")
            with open(path, "w") as f:
                json.dump({"cutoff_by_log2n": {}, "radix_classes": {"u32": 0x70, "f32": 0x7F0}}, f)
            assert sq.load_tuning(path)
        assert sq.get_radix_classes("u32") == 0x70
    finally:
        for d, m in before.items():
            sq.set_radix_classes(d, m)


def test_radix_choice_and_class_sizes():
    from paper_2407_14801_gb300 import autotune as at

    assert [at.class_size(c) for c in at.RADIX_CLASSES] == [2048, 8192, 16384, 24576, 32768, 40960, 49152, 57344, 65536]
    assert at.choose_radix(1.0, 1.0) and at.choose_radix(1.01, 1.0) and not at.choose_radix(1.1, 1.0)
