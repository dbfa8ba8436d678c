"""Host logic of bench.py that needs no GPU: the code-only hash that ties
the recorded DRAM traffic of the labeling kernel to the code it was captured
with.  Comments and blank lines do not change the hash; code does, and then
the bench line reports no traffic."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1105_5804_gb300", "csrc")
    dst = tmp_path / "paper_1105_5804_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.LABEL_TRAFFIC_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_label_sources_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.label_sources_hash()
    p = dst / bench.LABEL_TRAFFIC_SOURCES[0]
    text = p.read_text()
    first, rest = text.split("\n", 1)
    p.write_text("// a comment line\n\n" + first + "   // a trailing comment\n\n" + rest)
    assert bench.label_sources_hash() == h0
    p.write_text(text + "\nint one_more_declaration;\n")
    h1 = bench.label_sources_hash()
    assert h1 != h0
    monkeypatch.setattr(bench, "LABEL_TRAFFIC_SOURCE_HASH", h0)
    assert bench._label_traffic(1 << 20) is None
    monkeypatch.setattr(bench, "LABEL_TRAFFIC_SOURCE_HASH", h1)
    assert bench._label_traffic(1 << 20) == bench.LABEL_TRAFFIC_BYTES_PER_SITE * (1 << 20)
