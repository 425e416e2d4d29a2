"""The histogram tier table (no GPU): snnmap_set_tier_table accepts rows in
increasing size order and refuses malformed ones, and autotune.load_table
installs a table file (and ignores a missing one)."""
import json

import pytest


@pytest.fixture(scope="module")
def P():
    from paper_2609_07577_gb300 import _build
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build here: {e}")
    import paper_2609_07577_gb300 as P
    P.lib()
    yield P
    P.snnmap_set_tier_table([])


def test_table_rows_checked(P):
    P.snnmap_set_tier_table([(1 << 20, 4096, 1 << 15, 1 << 21), (1 << 62, 8192, 1 << 16, 1 << 22)])
    for bad in ([(10, 1, 2, 3), (10, 1, 2, 3)], [(10, -1, 2, 3)], [(20, 1, 2, 3), (10, 1, 2, 3)]):
        with pytest.raises(P.SnnmapError) as e:
            P.snnmap_set_tier_table(bad)
        assert e.value.code == 1
    P.snnmap_set_tier_table([])


def test_load_table(P, tmp_path):
    from paper_2609_07577_gb300 import autotune
    path = tmp_path / "t.json"
    assert autotune.load_table(str(path)) == []
    rows = [[1 << 21, 4096, 1 << 16, 1 << 22], [1 << 62, 8192, 1 << 17, 1 << 23]]
    path.write_text(json.dumps({"rows": rows}))
    assert autotune.load_table(str(path)) == rows
    P.snnmap_set_tier_table([])


def test_candidates_ordered():
    from paper_2609_07577_gb300 import autotune
    assert autotune.CLASSES == sorted(autotune.CLASSES)
    d = autotune.DEFAULTS
    assert d["wwork"] in autotune.CANDIDATES["wwork"] and d["bwork"] in autotune.CANDIDATES["bwork"]
    assert d["gwork"] in autotune.CANDIDATES["gwork"]
