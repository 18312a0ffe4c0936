"""Autotune cache (host logic): entries round-trip, other keys survive an
update, and a damaged file reads as empty."""
from paper_2501_01677_b300 import autotune as AT


def test_cache_roundtrip_and_update(tmp_path):
    path = str(tmp_path / "sub" / "autotune.json")
    assert AT._load_cache(path) == {}
    e1 = {"shape": {"tile_w": 16, "tile_h": 16, "ctas_per_sm": 4, "lpt": True}, "table": [{"ms": 1.0}]}
    e2 = {"shape": {"tile_w": 8, "tile_h": 8, "ctas_per_sm": None, "lpt": False}, "table": []}
    AT._store_cache(path, "a", e1)
    AT._store_cache(path, "b", e2)
    c = AT._load_cache(path)
    assert c["a"] == e1 and c["b"] == e2
    shape = AT.LaunchShape(**c["b"]["shape"])
    assert shape.tile == (8, 8) and shape.ctas_per_sm is None


def test_damaged_cache_reads_empty(tmp_path):
    path = tmp_path / "autotune.json"
    path.write_text("{not json")
    assert AT._load_cache(str(path)) == {}


def test_candidate_sets():
    assert (16, 16) in AT.TILES and (8, 8) in AT.TILES and (16, 32) in AT.TILES
    assert None in AT.QUEUE_DEPTHS and any(q for q in AT.QUEUE_DEPTHS)
