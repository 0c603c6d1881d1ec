"""Host logic of bench.py's roofline object (no GPU): the dominant kernel is
the one with the largest share of the profiled step; achieved = algorithmic
work per launch / mean launch time; frac = achieved / peak; the DRAM traffic
figure is reported only while the kernel sources match the revision it was
captured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _profile(ms_per_kernel, steps=2):
    # [steps, launches]: the dt kernel, then three stages of the kernels
    row = [0.01] + list(ms_per_kernel) * 3
    return {"prof": [row for _ in range(steps)]}


def test_mixed_dominant_sweep_and_alu_fraction():
    ncell = 4096 * 4096
    r = _profile([1.5, 1.4, 0.36])             # x sweep, transposed y sweep, combine
    out = bench._roofline(r, 1, ncell, 6777.0, "measured")
    assert out["kernel"] == "x_sweep" and out["bound"] == "alu"
    tf = 787.0 * ncell / 1.5e-3 / 1e12
    assert out["achieved"] == pytest.approx(tf, rel=1e-3)
    assert out["frac"] == pytest.approx(tf / bench.ALU_PEAK_TFLOPS[1], rel=1e-3)
    comb = out["kernels"]["stage_combine"]
    assert comb["bound"] == "hbm"
    gbs = bench.KERNEL_BYTES[1][2][1] * ncell / 0.36e-3 / 1e9
    assert comb["hbm_gbs"] == pytest.approx(gbs, rel=1e-3)
    total = 0.01 + 3 * (1.5 + 1.4 + 0.36)
    assert out["shares"]["x_sweep"] == pytest.approx(3 * 1.5 / total, abs=1e-3)


def test_combine_dominant_is_reported_against_hbm():
    r = _profile([0.2, 0.2, 1.0])
    out = bench._roofline(r, 1, 4096 * 4096, 6777.0, "measured")
    assert out["kernel"] == "stage_combine" and out["bound"] == "hbm" and out["unit"] == "GB/s"
    assert out["frac"] == pytest.approx(out["achieved"] / 6777.0, abs=1e-4)


def test_traffic_only_for_the_captured_sources(monkeypatch):
    r = _profile([1.5, 1.4, 0.36])
    ncell = 1000
    monkeypatch.setattr(bench, "_kernel_src_sha256", lambda: bench.TRAFFIC_SRC_SHA256)
    out = bench._roofline(r, 1, ncell, 6777.0, "measured")
    assert out["traffic"] == round(bench.TRAFFIC_PER_CELL[(1, "x_sweep")] * ncell)
    monkeypatch.setattr(bench, "_kernel_src_sha256", lambda: "0" * 64)
    assert bench._roofline(r, 1, ncell, 6777.0, "measured")["traffic"] is None



def test_checked_step_tail_is_kept_out_of_the_stage_kernels():
    """Checked steps (eq. (CFL-CD) on the face values) end with a commit copy,
    a transposed-plane restore and the step-end kernel: they get their own
    entry and leave the per-stage kernel averages unchanged."""
    ncell = 4096 * 4096
    row = [0.01] + [1.5, 1.4, 0.36] * 3 + [0.2, 0.001, 0.003]
    out = bench._roofline({"prof": [row, row]}, 1, ncell, 6777.0, "measured")
    assert out["kernel"] == "x_sweep" and out["avg_launch_ms"] == pytest.approx(1.5)
    tail = out["kernels"]["step_end"]
    assert tail["launches_per_step"] == 3
    assert tail["avg_ms_per_step"] == pytest.approx(0.204, abs=1e-4)
    assert tail["share"] == pytest.approx(0.204 / sum(row), abs=1e-3)


def test_cpu_baseline_reports_all_cores_and_one_core(monkeypatch):
    """The bench's oracle baseline (no GPU): all-core steps of the blast and
    the one-core figures (a blast step, one step of each of the first
    problems of the Riemann batch), on shrunk workloads so the test is fast;
    the oracle's thread count is restored afterwards."""
    import oracle
    from paper_1402_5618_gb300 import workloads as W
    real_blast, real_rb = W.blast_2d, W.riemann_batch
    monkeypatch.setattr(bench, "N_GRID", 48)
    monkeypatch.setattr(W, "blast_2d", lambda n, *a, **k: real_blast(min(n, 48), *a, **k))
    monkeypatch.setattr(W, "riemann_batch", lambda *a, **k: real_rb(nprob=8, n_lo=64, n_hi=128))
    cores = oracle.num_threads()
    out = bench._cpu_baseline(0.05)
    assert oracle.num_threads() == cores
    assert out["kind"] == "oracle" and out["cores"] == cores and out["value"] > 0
    sc = out["single_core"]
    assert sc["blast_1024"] > 0 and sc["riemann_batch_256"] > 0 and sc["unit"] == bench.UNIT
