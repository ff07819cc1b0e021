"""The tuning table lookup (no GPU): workload classes, the fallbacks to the
nearest tuned class, the batch entry and the defaults when a class or the
whole table is missing."""
import json

from paper_2005_05371_gb300 import autotune


def test_classes():
    assert autotune.size_class(512, 512) == "small"
    assert autotune.size_class(1620, 1620) == "medium"
    assert autotune.size_class(4096, 4096) == "large"
    assert autotune.size_class(999, 1000) == "small" and autotune.size_class(1000, 1000) == "medium"
    assert autotune.key(1620, 1620, "u8", 9, 5, 0.2) == "medium|u8|s>=9|w>=5|d<0.3"
    assert autotune.key(512, 512, "u16", 7, 3, 0.4) == "small|u16|s<=7|w<=3|d>=0.3"
    assert autotune.key(512, 512, "u16", 7, 3, None).endswith("|d?")


def _table(tmp_path, entries):
    p = tmp_path / f"t{len(list(tmp_path.iterdir()))}.json"
    p.write_text(json.dumps({"table": {k: {"knobs": v, "ms": ms} for k, (v, ms) in entries.items()}}))
    return str(p)


def test_choose_from_a_table(tmp_path):
    p = _table(tmp_path, {
        "small|u8|s<=7|w<=3|d<0.1": ([16, 3, 0, 8, 0, 0, 0], 1.0),
        "small|u8|s<=7|w<=3|d<0.3": ([24, 3, 0, 0, 0, 0, 0], 1.1),
        "large|u16|s>=9|w>=5|d>=0.3": ([64, 0, 1, -1, 2, 0, 0], 2.0),
        "large|u16|s<=7|w<=3|d<0.1": ([48, 2, 0, 0, 0, 0, 0], 1.5),
        "batch": ([48, 2, 0, 0, 0, 10, 1], 3.0)})
    assert autotune.choose(512, 512, "u8", 7, 3, 0.05, p) == (16, 3, 0, 8, 0, 0, 0)        # exact class
    assert autotune.choose(512, 512, "u8", 7, 3, None, p) == (24, 3, 0, 0, 0, 0, 0)        # density unknown: middle
    assert autotune.choose(4096, 4096, "u16", 11, 5, 0.4, p) == (64, 0, 1, -1, 2, 0, 0)
    # no entry for the class: the fastest of the same size and dtype
    assert autotune.choose(4096, 4096, "u16", 11, 3, 0.2, p) == (48, 2, 0, 0, 0, 0, 0)
    # nothing of the size: the library's defaults
    assert autotune.choose(1620, 1620, "u8", 9, 5, 0.2, p) == autotune.DEFAULT
    assert autotune.choose_batch(p) == (48, 2, 0, 0, 0, 10, 1)
    q = _table(tmp_path, {"large|u16|s>=9|w>=5|d<0.3": ([40, 3, 0, 0, 0, 0, 0], 2.0)})
    assert autotune.choose_batch(q) == (40, 3, 0, 0, 0, 0, 0)                 # falls back to a large entry
    assert autotune.choose(512, 512, path=str(tmp_path / "absent.json")) == autotune.DEFAULT


def test_shipped_table_is_complete():
    data = json.load(open(autotune.TABLE_PATH))
    tab = data["table"]
    assert data["fields"] == list(autotune.FIELDS)
    assert "batch" in tab
    cases = {k for k in autotune._cases()}
    assert cases <= set(tab), sorted(cases - set(tab))[:5]
    for k, ent in tab.items():
        kn = ent["knobs"]
        assert kn[0] in autotune.REGION_H and kn[1] in autotune.CTAS_PER_SM
        assert kn[2] in (0, 1) and kn[3] in autotune.SMALL_GROWTH and kn[4] in autotune.SELECT_LANES
        if k == "batch":
            assert kn[5] in autotune.BATCH_LAG and kn[6] in (0, 1)
