"""Host logic of bench.py that needs no GPU: the committed ncu traffic records (a record counts only
while the sources it names are unchanged and the method defaults match, and a record taken on a
smaller workload is scaled by the unit its traffic grows with), the bounded CPU sample of a frame,
and the replica throughput."""
import hashlib
import json
import os
import types

import numpy as np

import bench


def _fake_root(tmp_path, defaults, scales_to=("big",)):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    rec = {"k@big": {"dram_bytes_per_launch": 1000.0, "workload": "small", "scales_to": list(scales_to),
                     "unit": "hits", "units_per_launch": 10, "launch_shape": {"a": 1},
                     "method_defaults": defaults, "sources": ["kernel.cu"], "sources_sha256": h}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return src


def test_traffic_record_scaled_and_invalidated(tmp_path, monkeypatch):
    defaults = {"lmin": 6}
    src = _fake_root(tmp_path, defaults)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    b, note = bench._recorded_traffic("k", "big", defaults, {"hits": 25})
    assert b == 2500.0 and note["capture_workload"] == "small" and "25 / 10" in note["scaled_by"]
    # another workload than the record names, no unit counts, other defaults: no traffic
    assert bench._recorded_traffic("k", "other", defaults, {"hits": 25}) == (None, None)
    assert bench._recorded_traffic("k", "big", defaults, None) == (None, None)
    assert bench._recorded_traffic("k", "big", {"lmin": 5}, {"hits": 25}) == (None, None)
    # a changed source (even one byte) voids the record
    src.write_text("__global__ void k() { }\n")
    assert bench._recorded_traffic("k", "big", defaults, {"hits": 25}) == (None, None)
    assert bench._traffic_fields("k", "big", defaults, {"hits": 25}) == {"traffic": None}


def test_committed_traffic_records_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        recs = json.load(fh)
    assert "tracklets@full_570" in recs
    for key, rec in recs.items():
        for s in rec["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, s)), (key, s)
        assert rec["dram_bytes_per_launch"] > 0


def test_cpu_sample_bounds_each_sector():
    rng = np.random.default_rng(3)
    n = 40000
    f = types.SimpleNamespace(n=n, sector=rng.integers(0, 4, n).astype(np.uint8),
                              w=rng.uniform(-100, 100, n).astype(np.float32))
    m = bench.cpu_sample(f, 2, 1000)
    for s in range(4):
        k = int(np.sum(m & (f.sector == s)))
        if s < 2:
            assert 900 <= k <= 1000  # a window of about 1000 clusters around the sector's median w
        else:
            assert k == 0
    # a sector smaller than the window is taken whole
    assert np.sum(bench.cpu_sample(f, 1, n)) == np.sum(f.sector == 0)


def test_whole_job_value_counts_every_replica():
    assert bench.whole_job_value(2.0e8, 10, 0.8, 1) == 2.0e8 * 10 / 0.8
