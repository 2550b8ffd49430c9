"""bench.py bookkeeping on the host: the DRAM-traffic ratio from a committed
ncu summary applies only to the workload and kernel sources it was captured
on, and every workload line describes its inputs."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_ratio_tied_to_sources(tmp_path, monkeypatch):
    cur = bench.kernel_sources_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(
        "text\ntraffic-per-algorithmic-byte: 1.5 (workload wl_a, sources %s)\n"
        "traffic-per-algorithmic-byte: 9.0 (workload wl_b, sources 0000000000000000)\n"
        "traffic-per-algorithmic-byte: 1.2 (workload wl_small, sources %s, stands for wl_big)\n" % (cur, cur))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the sources are hashed from ROOT: point it back at the repository for them
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: cur)
    assert bench.profiled_traffic_ratio("wl_a")[0] == 1.5
    assert bench.profiled_traffic_ratio("wl_b") is None      # captured on other sources
    assert bench.profiled_traffic_ratio("wl_c") is None      # never captured
    # a small case captured for a workload too large to capture stands in for it
    assert bench.profiled_traffic_ratio("wl_big")[:1] == (1.2,) and bench.profiled_traffic_ratio("wl_big")[2] == "wl_small"


def test_source_hash_is_stable_and_short():
    h = bench.kernel_sources_hash()
    assert h == bench.kernel_sources_hash() and len(h) == 16


def test_workloads_describe_their_inputs():
    for name, w in bench.WORKLOADS.items():
        d = bench.describe(w)
        assert f"R-MAT scale {w['scale']}" in d and f"L={w['L']}" in d, name
        if w.get("weights", "grid14").startswith("lognormal"):
            assert "log-normal" in d
        if w.get("starts") == "maxdeg":
            assert "max-degree" in d


def test_source_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    for f in bench.KERNEL_SOURCES:
        (tmp_path / f).parent.mkdir(parents=True, exist_ok=True)
        (tmp_path / f).write_text('int a = 1;  // one\n/* block */ const char* s = "x // y";\n')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash()
    f0 = tmp_path / bench.KERNEL_SOURCES[0]
    f0.write_text('int a = 1;  // other words\n/* a longer\n   block */   const char* s = "x // y";\n')
    assert bench.kernel_sources_hash() == h0          # comments and layout only
    f0.write_text('int a = 2;  // one\n/* block */ const char* s = "x // y";\n')
    assert bench.kernel_sources_hash() != h0          # code
    f0.write_text('int a = 1;  // one\n/* block */ const char* s = "x // z";\n')
    assert bench.kernel_sources_hash() != h0          # a string literal is code
