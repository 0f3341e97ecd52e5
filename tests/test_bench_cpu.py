"""CPU checks of the bench's roofline bookkeeping: profiled per-launch figures
are used only while the kernel's sources are the profiled ones, the issue-rate
roofline is the profiled instruction count over the launch time against the
GB300's 608 schedulers, and the algorithmic bytes of the fused step kernel are
its G2P and P2G halves without the state round trip."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2303_02346_gb300 import build as b  # noqa: E402


def test_profiled_values_follow_the_kernel_source_group(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    fwd, adj = b.source_hash("mpm_fwd"), b.source_hash("mpm_adj")
    (prof / "x.md").write_text(
        f"traffic_per_launch_full_size: 1000 kernel=g2p2g source_hash={fwd}\n"
        f"instructions_per_launch_full_size: 2000 kernel=g2p2g source_hash={fwd}\n"
        f"traffic_per_launch_full_size: 3000 kernel=adj_fused source_hash={fwd}\n"
        f"traffic_per_launch_full_size: 4000 kernel=p2g_adj source_hash={adj}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("g2p2g") == 1000
    assert bench.profiled_value("g2p2g", "instructions_per_launch_full_size") == 2000
    # an adjoint kernel's figure counts only under the adjoint sources' hash
    assert bench.profiled_traffic("adj_fused") is None
    assert bench.profiled_traffic("p2g_adj") == 4000
    assert bench.profiled_traffic("g2p") is None


def test_issue_roofline_arithmetic(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    fwd = b.source_hash("mpm_fwd")
    # a quarter of 608 schedulers x 2.07 GHz for 1 ms
    (prof / "x.md").write_text(f"instructions_per_launch_full_size: 314640000 kernel=g2p2g source_hash={fwd}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))  # no peaks file: the 2070 MHz maximum clock
    r = bench.issue_roofline("g2p2g", 1.0)
    assert r["peak"] == pytest.approx(152 * 4 * 2.07, abs=0.1)  # G warp-instructions/s
    assert r["achieved"] == pytest.approx(314.6, abs=0.1)
    assert r["frac"] == pytest.approx(0.25, abs=1e-4)
    assert bench.issue_roofline("g2p", 1.0) is None


def test_fused_step_bytes_are_the_two_halves_without_the_round_trip():
    g2p = bench.algorithmic_bytes("g2p", 1, 0, 0), bench.algorithmic_bytes("g2p", 0, 1, 0)
    p2g = bench.algorithmic_bytes("p2g", 1, 0, 0), bench.algorithmic_bytes("p2g", 0, 1, 0)
    fused = bench.algorithmic_bytes("g2p2g", 1, 0, 0), bench.algorithmic_bytes("g2p2g", 0, 1, 0)
    for i in range(2):
        assert fused[i] < g2p[i] + p2g[i]
        assert fused[i] >= max(g2p[i], p2g[i])
    # per active node: the fused kernel gathers one grid and scatters the next
    assert bench.algorithmic_bytes("g2p2g", 0, 0, 1) == (bench.algorithmic_bytes("g2p", 0, 0, 1)
                                                          + bench.algorithmic_bytes("p2g", 0, 0, 1))


def test_profiled_records_are_matched_by_workload(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    fwd = b.source_hash("mpm_fwd")
    (prof / "x.md").write_text(
        f"traffic_per_launch_full_size: 1000 kernel=g2p2g source_hash={fwd} workload=multi_material\n"
        f"traffic_per_launch_full_size: 7000 kernel=g2p2g source_hash={fwd} workload=dam_break\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("g2p2g", "dam_break") == 7000
    assert bench.profiled_traffic("g2p2g", "multi_material") == 1000
    assert bench.profiled_traffic("g2p2g", "batched") is None


def test_step_bytes_are_the_state_round_trip_per_particle_step():
    # forward: state read + write (64 B liquid, 96 B solid) + 6 B of grid;
    # adjoint: three state sizes + 18 B of grid
    assert bench.STEP_BYTES["g2p2g"] == (2 * 64 + 6, 2 * 96 + 6)
    assert bench.STEP_BYTES["adj_fused"] == (3 * 64 + 18, 3 * 96 + 18)
    # the dam-break launch: 1.4M liquid and 0.6M solid particles, 306 MB
    liq, sol = bench.STEP_BYTES["g2p2g"]
    assert 1_400_000 * liq + 600_000 * sol == pytest.approx(306.4e6, rel=1e-4)
