"""Tuning cache host logic (no GPU)."""
import json

from paper_2105_07544_b300 import autotune as at


def test_key_buckets_sizes():
    k1 = at.key("B300", 3_375_000, 23_490_000, "f32", 50, 0)
    k2 = at.key("B300", 3_300_000, 23_000_000, "f32", 50, 0)      # same log2 bucket, w = 7
    k3 = at.key("B300", 6_250_000, 31_240_000, "f32", 50, 0)      # next bucket, w = 5
    assert k1 == k2 and k1 != k3
    assert at.key("B300", 1000, 5000, "bf16", 50, 25) != at.key("B300", 1000, 5000, "f32", 50, 25)


def test_cache_round_trip_and_schema(tmp_path):
    p = tmp_path / "t.json"
    c = at.TuningCache(str(p))
    assert c.get("k") is None
    shapes = dict(sweep_stage_kb=8, sweep_ctas_per_sm=2, spmv_ctas_per_sm=0)
    c.put("k", shapes, 1e-4, 2e-4)
    d = at.TuningCache(str(p))
    assert d.get("k")["shapes"] == shapes and d.get("k")["s_per_iter"] == 1e-4
    data = json.loads(p.read_text())
    data["schema"] = 999
    p.write_text(json.dumps(data))
    assert at.TuningCache(str(p)).get("k") is None          # other schema: ignored


def test_default_path_honours_environment(monkeypatch, tmp_path):
    monkeypatch.setenv("GMRESB3_TUNING_CACHE", str(tmp_path / "x.json"))
    assert at.default_path() == str(tmp_path / "x.json")
