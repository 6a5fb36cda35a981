"""The benchmark's measurement bookkeeping on CPU: the per-level ncu counters that feed the
roofline are used only while the kernel sources still hash to the captured version, the
ncu CSV log is parsed into per-metric values, and the launch counts per multigrid level
give the 4 P and 3 P^T applications per A2 iteration that the metric counts."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1008_2042_gb300 import profile_counters as pc  # noqa: E402

NCU_LOG = """==PROF== Connected to process 1 (/usr/bin/python3)
==PROF== Disconnected from process 1
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python3","127.0.0.1","void k_project<0, float, 40>(GeomDev)","1","7","(192, 1, 1)","(20480, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","byte","372,484,608"
"0","1","python3","127.0.0.1","void k_project<0, float, 40>(GeomDev)","1","7","(192, 1, 1)","(20480, 1, 1)","0","10.3","Command line profiler metrics","smsp__thread_inst_executed.sum","inst","23102998157"
"0","1","python3","127.0.0.1","void k_project<0, float, 40>(GeomDev)","1","7","(192, 1, 1)","(20480, 1, 1)","0","10.3","Command line profiler metrics","lts__t_sector_hit_rate.pct","%","86.85"
"""


def test_ncu_csv_log_is_parsed_per_metric(tmp_path):
    log = tmp_path / "counters.csv"
    log.write_text(NCU_LOG)
    m = pc._parse(str(log))
    assert m["dram__bytes_read.sum"] == 372484608.0  # thousands separators removed
    assert m["smsp__thread_inst_executed.sum"] == 23102998157.0
    assert m["lts__t_sector_hit_rate.pct"] == 86.85
    assert m["kernel_name"].startswith("void k_project<0, float, 40>")


@pytest.mark.parametrize("kernel", sorted(pc.KERNEL_SOURCES))
def test_source_hash_follows_every_listed_file(tmp_path, monkeypatch, kernel):
    """Changing any file a kernel is built from (its own units or the internal header)
    changes the hash the counters are tied to; the other kernel's files do not."""
    for name in os.listdir(pc.CSRC):
        shutil.copy(os.path.join(pc.CSRC, name), tmp_path / name)
    monkeypatch.setattr(pc, "CSRC", str(tmp_path))
    base = pc.kernel_sources_sha(kernel)
    for name in pc.KERNEL_SOURCES[kernel] + ("cbct_internal.cuh",):
        original = (tmp_path / name).read_bytes()
        (tmp_path / name).write_bytes(original + b"\n// edited\n")
        assert pc.kernel_sources_sha(kernel) != base, name
        (tmp_path / name).write_bytes(original)
    assert pc.kernel_sources_sha(kernel) == base
    others = {n for k, files in pc.KERNEL_SOURCES.items() if k != kernel for n in files}
    for name in others - set(pc.KERNEL_SOURCES[kernel]):
        (tmp_path / name).write_bytes((tmp_path / name).read_bytes() + b"\n// edited\n")
    assert pc.kernel_sources_sha(kernel) == base


def test_counters_are_used_only_for_the_captured_sources(tmp_path, monkeypatch):
    levels = {"0": {"thread_inst": 1.0, "dram_read_bytes": 2.0, "dram_write_bytes": 3.0}}
    (tmp_path / "profiles").mkdir()
    path = tmp_path / "profiles" / "kernels.json"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    current = pc.kernel_sources_sha("k_project")
    path.write_text(json.dumps({"k_project": {"sources_sha256": current, "levels": levels}}))
    assert bench.stored_counters("k_project") == levels
    path.write_text(json.dumps({"k_project": {"sources_sha256": "0" * 64, "levels": levels}}))
    assert bench.stored_counters("k_project") is None
    assert bench.stored_counters("k_backproject") is None  # no record at all
    path.write_text("not json")
    assert bench.stored_counters("k_project") is None


def test_launches_per_level_count_four_p_and_three_pt_per_iteration():
    """Level 0 is the finest; iterations are given coarsest first (8/17/25)."""
    p, pt = bench.launches_per_level([8, 17, 25])
    assert p == [25 * 4, 17 * 4, 8 * 4]
    assert pt == [25 * 3, 17 * 3, 8 * 3]
    assert (sum(p), sum(pt)) == (200, 150)
