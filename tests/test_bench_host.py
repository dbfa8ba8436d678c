"""Host logic of bench.py that needs no GPU: the code-only hash that ties the
recorded ncu counters of the sweep's kernels (DRAM bytes, instructions) to
the code they were captured with.  Comments and blank lines do not change
the hash; code does, and then the bench line reports no counters.  Also:
the recorded hash matches the committed sources (the counters in the line
are those of the code that runs), and the serving stream sizes."""
import os
import shutil

import bench


def _copy_sources(tmp_path, files):
    src = os.path.join(bench.ROOT, "paper_1105_5804_gb300", "csrc")
    dst = tmp_path / "paper_1105_5804_gb300" / "csrc"
    dst.mkdir(parents=True, exist_ok=True)
    for f in files:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_sources_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path, bench.SWEEP_COUNTER_SOURCES)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.sources_hash(bench.SWEEP_COUNTER_SOURCES)
    p = dst / bench.SWEEP_COUNTER_SOURCES[0]
    text = p.read_text()
    first, rest = text.split("\n", 1)
    p.write_text("// a comment line\n\n" + first + "   // a trailing comment\n\n" + rest)
    assert bench.sources_hash(bench.SWEEP_COUNTER_SOURCES) == h0
    p.write_text(text + "\nint one_more_declaration;\n")
    h1 = bench.sources_hash(bench.SWEEP_COUNTER_SOURCES)
    assert h1 != h0
    monkeypatch.setattr(bench, "SWEEP_COUNTER_HASH", h0)
    assert bench.sweep_counters() is None
    monkeypatch.setattr(bench, "SWEEP_COUNTER_HASH", h1)
    assert bench.sweep_counters() == bench.SWEEP_COUNTERS


def test_recorded_counters_belong_to_the_committed_kernels():
    assert bench.sweep_counters() is not None, "sweep kernels changed since their ncu capture"
    assert bench._ccl_traffic(1 << 20) is not None, "labeling kernels changed since their ncu capture"
    for k, (b, wi) in bench.SWEEP_COUNTERS.items():
        assert 0.1 < b < 10 and 0.1 < wi < 10, k


def test_serving_job_counts():
    assert bench.serving_jobs(10) == 200          # at least 200 jobs
    assert bench.serving_jobs(100) == 600         # about six seconds of the stream
    assert bench.serving_jobs(2000) == 2000       # at most 2000
