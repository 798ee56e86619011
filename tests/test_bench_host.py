"""Host logic of bench.py that needs no GPU: the ncu traffic record is keyed by a hash of the
kernel's code (comments and layout left out), and is reported only while that code is unchanged."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _copy_sources(tmp_path):
    src = os.path.join(ROOT, "paper_2310_19855_gb300", "csrc")
    dst = tmp_path / "paper_2310_19855_gb300" / "csrc"
    shutil.copytree(src, dst)
    return dst


@pytest.mark.parametrize("key", sorted(bench.NCU_TRAFFIC))
def test_traffic_record_matches_the_committed_sources(key):
    # every record was taken on the code as committed: a stale hash would report null traffic
    assert bench.ncu_traffic(key) == bench.NCU_TRAFFIC[key]["bytes_per_launch"]


def test_comment_edits_keep_the_hash_and_code_edits_change_it(tmp_path, monkeypatch):
    dst = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    srcs = bench.NCU_TRAFFIC["2:update"]["sources"]
    h0 = bench._source_sha(srcs)
    p = dst / "gi_cache.cu"
    text = p.read_text()
    marker = bench.UPDATE_SECTION[1]
    # a comment line and re-indentation inside the update section: same code
    p.write_text(text.replace(marker, marker + "\n// a note\n/* and a block\n   comment */\n", 1))
    assert bench._source_sha(srcs) == h0
    # one changed token inside the section: new code, the record no longer applies
    i = text.index(marker)
    j = text.index("kUpdThreads", i)
    p.write_text(text[:j] + "kUpdThreads + 0" + text[j + len("kUpdThreads"):])
    assert bench._source_sha(srcs) != h0
    assert bench.ncu_traffic("2:update") is None
    # a change outside the section leaves the update's record alone
    p.write_text(text + "\n// trailing note\nstatic int unrelated_symbol = 0;\n")
    assert bench._source_sha(srcs) == h0
