"""The autotuner's table: JSON round trip through rs_tune_save / rs_tune_load (host only), and
rejection of malformed files without touching the table."""
import pytest


@pytest.fixture(scope="module")
def rs():
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    P.lib()
    return P


def test_empty_table_round_trip(rs, tmp_path):
    rs.rs_tune_clear()
    p = tmp_path / "t.json"
    rs.rs_tune_save(p)
    rs.rs_tune_load(p)
    assert rs.rs_tune_count() == 0


def test_load_merges_entries_and_rejects_malformed(rs, tmp_path):
    rs.rs_tune_clear()
    good = tmp_path / "good.json"
    good.write_text('{"rs_tune": 1, "entries": {\n  "cpqr.s8.b8.m43.r46.gscale": 0.5,\n  "sweep.s8.b8.m43.r0.gscale": 1}}\n')
    rs.rs_tune_load(good)
    assert rs.rs_tune_count() == 2
    again = tmp_path / "again.json"
    rs.rs_tune_save(again)
    rs.rs_tune_clear()
    rs.rs_tune_load(again)
    assert rs.rs_tune_count() == 2
    text = again.read_text()
    assert '"cpqr.s8.b8.m43.r46.gscale": 0.5' in text
    bad = tmp_path / "bad.json"
    bad.write_text('{"rs_tune": 1, "entries": {"k": nope}}')
    with pytest.raises(rs.RsError) as e:
        rs.rs_tune_load(bad)
    assert e.value.code == rs.RS_E_INVALID
    assert rs.rs_tune_count() == 2
    with pytest.raises(rs.RsError):
        rs.rs_tune_load(tmp_path / "missing.json")
    rs.rs_tune_clear()
    assert rs.rs_tune_count() == 0
