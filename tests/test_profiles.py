"""The committed ncu summaries: each names the kernel source it was captured
on and that source's hash, which must match the source as committed (the
bench reports a summary's DRAM traffic and instruction counts only while it
does); each gives its capture command, with the clocks left uncontrolled,
and the per-launch figures the bench reads."""
import glob
import hashlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUMMARIES = sorted(p for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))
                   if "source_sha256_16" in open(p).read())


@pytest.mark.parametrize("path", SUMMARIES, ids=[os.path.basename(p) for p in SUMMARIES])
def test_summary_matches_its_kernel_source(path):
    text = open(path).read()
    m = re.search(r"source_sha256_16: (\S+)\s+\((\S+) at capture", text)
    assert m, "no source hash line"
    src = os.path.join(ROOT, m.group(2))
    with open(src, "rb") as f:
        assert hashlib.sha256(f.read()).hexdigest()[:16] == m.group(1), "re-capture after editing " + m.group(2)
    assert re.search(r"traffic_bytes_per_launch: \d+", text)
    assert "ncu " in text and "--clock-control none" in text


def test_bench_reads_the_summaries():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.profile_traffic("paper_1205_0106_gb300/csrc/sweep_v2.cu",
                                 "profiles/sweep_lsm_v2_2p20x252_mixed.md") > 1.0e9
    rl = bench.issue_roofline("paper_1205_0106_gb300/csrc/pathgen.cu", "profiles/pathgen_2p20x252_mixed.md", 6.0e11)
    assert 0.0 < rl["frac"] < 1.0 and rl["pipes_pct_of_peak"]["fma"] > 0.0
    assert bench.profile_traffic("paper_1205_0106_gb300/csrc/sweep_v2.cu", "profiles/pathgen_2p20x252_mixed.md") is None
