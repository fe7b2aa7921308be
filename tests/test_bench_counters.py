"""bench.py reports a kernel's ncu counters (executed flops, DRAM traffic)
only while that kernel's sources hash to the digest recorded at the
capture: the recorded digests are well formed, each names existing
sources, and an edit of any one source file changes the digest (checked
on a copy of the sources, with one byte appended to each file in turn)."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_digests_are_recorded_for_every_counted_kernel():
    assert set(bench.COUNTER_DIGEST) == set(bench.COUNTER_SOURCES)
    for kind, digest in bench.COUNTER_DIGEST.items():
        assert len(digest) == 16 and int(digest, 16) >= 0, kind
        assert len(bench.source_digest(kind)) == 16


def test_any_source_edit_changes_the_digest(tmp_path):
    csrc = os.path.join(ROOT, "paper_2107_12027_gb300", "csrc")
    for kind, files in bench.COUNTER_SOURCES.items():
        base = bench.source_digest(kind)
        for f in files:
            d = tmp_path / (kind + "_" + f.replace(".", "_"))
            d.mkdir()
            for g in files:
                shutil.copy(os.path.join(csrc, g), d / g)
            assert bench.source_digest(kind, str(d)) == base
            with open(d / f, "ab") as fh:
                fh.write(b" ")
            assert bench.source_digest(kind, str(d)) != base, (kind, f)
