"""CPU tests of the autotuner's search and cache logic (the GPU timer is replaced
by a deterministic fake)."""
from paper_1902_09171_gb300 import autotune, rcell


def test_search_picks_fastest_and_skips_invalid():
    calls = []

    def fake(prm, cells, tpa):
        calls.append((prm.skin, tpa))
        if prm.skin > 1.9:
            return None  # invalid candidate
        return abs(prm.skin - 1.5) * 10 + abs(tpa - 2) + 1.0

    best, table = autotune.search(lambda s: rcell.params_sc_cu(skin=s), [], fake, (1.0, 1.5, 2.0), (1, 2, 4))
    assert best == {"skin": 1.5, "tpa": 2, "ms_per_step": 1.0}
    assert len(calls) == 9 and len(table) == 6


def test_cache_roundtrip_and_buckets(tmp_path):
    path = str(tmp_path / "c.json")
    assert autotune.load_cache(path) == {}
    k = autotune.key("NVIDIA GB300", 1, 128000)
    assert k == "NVIDIA GB300|pot1|n131072"
    autotune.store(k, {"skin": 1.5, "tpa": 1}, path)
    autotune.store(autotune.key("NVIDIA GB300", 2, 800000), {"skin": 0.3, "tpa": 2}, path)
    c = autotune.load_cache(path)
    assert c[k] == {"skin": 1.5, "tpa": 1} and len(c) == 2
    assert autotune.bucket(1) == "1" and autotune.bucket(5000) == "8192"
