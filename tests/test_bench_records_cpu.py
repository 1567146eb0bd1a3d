"""The bench's hash-tied ncu records: the tracklet kernel's DRAM bytes per
helix step and the double-float kernel's instructions per helix step are
used only while the kernel sources hash to the value recorded with them;
any change of a source turns the bench's figure null."""
import hashlib
import json
import os
import shutil

import pytest

import bench

SRCS = ["paper_2502_09138_gb300/csrc/tracklet.cu", "paper_2502_09138_gb300/csrc/track_math.cuh",
        "paper_2502_09138_gb300/csrc/df64.cuh", "paper_2502_09138_gb300/csrc/tpct_internal.cuh"]


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    for s in SRCS:
        (tmp_path / os.path.dirname(s)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, s), tmp_path / s)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256()
    for s in SRCS:
        h.update((tmp_path / s).read_bytes())
    common = {"sources": SRCS, "sources_sha256": h.hexdigest()}
    (tmp_path / "profiles" / "k_tracklets_traffic.json").write_text(
        json.dumps(dict(common, dram_bytes_per_helix_step=40.0)))
    (tmp_path / "profiles" / "k_tracklets_df_issue.json").write_text(
        json.dumps(dict(common, warp_instructions_per_helix_step=80.0)))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_records_apply_while_the_sources_match(fake_root):
    assert bench.tracklet_traffic(1000) == pytest.approx(40000.0)
    iss = bench.tracklet_issue(1_000_000, 1.0, 2070.0)
    assert iss["warp_instructions"] == pytest.approx(80e6)
    assert iss["issue_frac"] == pytest.approx(80e6 / (152 * 4 * 1e-3 * 2070e6))


def test_records_turn_null_when_a_source_changes(fake_root):
    p = fake_root / SRCS[1]
    p.write_text(p.read_text() + "\n// changed\n")
    assert bench.tracklet_traffic(1000) is None
    assert bench.tracklet_issue(1_000_000, 1.0, 2070.0) is None


def test_committed_records_name_the_committed_sources():
    for name in ("k_tracklets_traffic.json", "k_tracklets_df_issue.json"):
        with open(os.path.join(bench.ROOT, "profiles", name)) as f:
            doc = json.load(f)
        assert doc["sources"] == SRCS
        assert doc["capture"].startswith("ncu ") and "--clock-control none" in doc["capture"]
