"""The tuning table lookup (no GPU): size classes, the batch entry and the
defaults when a class or the whole table is missing."""
import json

from paper_2005_05371_gb300 import autotune


def test_size_classes():
    assert autotune.size_class(512, 512) == "small"
    assert autotune.size_class(1620, 1620) == "medium"
    assert autotune.size_class(4096, 4096) == "large"
    assert autotune.size_class(999, 1000) == "small" and autotune.size_class(1000, 1000) == "medium"


def test_choose_from_a_table(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"table": {"small": {"region_h": 16, "ctas_per_sm": 3, "ms": 1.0},
                                       "large": {"region_h": 64, "ctas_per_sm": 0, "ms": 2.0},
                                       "batch": {"region_h": 48, "ctas_per_sm": 2, "ms": 3.0}}}))
    assert autotune.choose(512, 512, str(p)) == (16, 3)
    assert autotune.choose(1620, 1620, str(p)) == (32, 0)          # class missing: the default
    assert autotune.choose(4096, 4096, str(p)) == (64, 0)
    assert autotune.choose_batch(str(p)) == (48, 2)
    q = tmp_path / "nobatch.json"
    q.write_text(json.dumps({"table": {"large": {"region_h": 40, "ctas_per_sm": 3, "ms": 2.0}}}))
    assert autotune.choose_batch(str(q)) == (40, 3)                  # falls back to the large entry
    assert autotune.choose(512, 512, str(tmp_path / "absent.json")) == (32, 0)


def test_shipped_table_is_complete():
    tab = json.load(open(autotune.TABLE_PATH))["table"]
    for cls in ("small", "medium", "large", "batch"):
        ent = tab[cls]
        assert ent["region_h"] in autotune.REGION_H and ent["ctas_per_sm"] in autotune.CTAS_PER_SM
