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


def test_batch_key_buckets_and_separates_from_single_system_keys():
    k1 = at.batch_key("B300", 256, 9_300_000, 46_000_000, 16)
    k2 = at.batch_key("B300", 256, 9_700_000, 48_000_000, 16)     # same log2 bucket, w = 5
    assert k1 == k2
    assert k1 != at.batch_key("B300", 256, 9_300_000, 46_000_000, 8)
    assert k1 != at.batch_key("B300", 128, 9_300_000, 46_000_000, 16)
    assert "|batch|" in k1 and k1 != at.key("B300", 9_300_000, 46_000_000, "bf16", 16, 0)


class _FakeBatch:
    """Host stand-in for BatchSolver: records the shapes it is given and counts tuning runs."""

    def __init__(self):
        self.sizes = [1000, 2000]
        self.shapes = None
        self.tuned = 0

    def set_tuning(self, **kw):
        self.shapes = kw

    def autotune(self, B, tol, max_cycles):
        self.tuned += 1
        self.shapes = dict(chunk_tiles=8, sweep_smem_kb=0, sweep_max_stages=8)
        return dict(self.shapes), 0.4, 0.5


def test_tune_batch_times_once_then_hits_the_cache(tmp_path, monkeypatch):
    monkeypatch.setattr(at, "gpu_name", lambda: "FakeGPU")
    c = at.TuningCache(str(tmp_path / "t.json"))
    s1 = _FakeBatch()
    r1 = at.tune_batch(s1, None, nnz=15000, m=16, cache=c)
    assert not r1["cached"] and s1.tuned == 1
    s2 = _FakeBatch()
    r2 = at.tune_batch(s2, None, nnz=15000, m=16, cache=at.TuningCache(str(tmp_path / "t.json")))
    assert r2["cached"] and s2.tuned == 0 and s2.shapes == s1.shapes
    assert r2["key"] == r1["key"]
