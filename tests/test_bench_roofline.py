"""bench.py's roofline accounting, on the CPU: algorithmic bytes per gate in the
paper's convention (Section 5.2), the FP32 flop counts of the double-float
updates rebuilt from their parts, the per-pass flop sum over a dry-run plan,
the instruction-issue summary and the roofline peak."""

import ctypes

import numpy as np
import pytest

import bench
import qsgen as G
from paper_1601_07195_gb300 import qs


def test_gate_bytes_follow_the_papers_convention():
    n, s = 10, 16
    N = 1 << n
    assert bench.gate_cost(G.gate_u1(3, G.haar_2x2(G.SplitMix64(1)))[0], n, s)[0] == 2 * N * s  # read + write
    assert bench.gate_cost(G.gate_u1(3, G.MAT_T)[0], n, s)[0] == N * s                           # |1> half only
    assert bench.gate_cost(G.gate_cu(1, 3, G.MAT_X)[0], n, s)[0] == N * s                        # control-1 half
    assert bench.gate_cost(G.gate_cu(1, 3, G.mat_cphase(0.3))[0], n, s)[0] == N * s / 2          # one quarter
    assert bench.gate_cost(G.gate_swap(1, 3)[0], n, s)[0] == N * s


def test_double_float_flop_counts_from_their_parts():
    """Per touched amplitude, from df.cuh's building blocks: df_mul = FMUL + 3 FFMA
    (7 flops), TwoSum 6, a sum of k unnormalised products = k df_mul + (k - 1)
    TwoSum + 2 (k - 1) adds."""
    df_mul, two_sum = 7, 6
    dot = lambda k: k * df_mul + (k - 1) * two_sum + 2 * (k - 1)
    cmul = 2 * dot(2)                                  # complex product, per amplitude
    assert bench._DF_FLOPS["general"] == 2 * dot(4)   # 104
    assert bench._DF_FLOPS["real"] == 2 * dot(2)      # 44
    assert bench._DF_FLOPS["diag1"] == cmul           # one complex product on the changed half
    addsig = 1 + two_sum + 2 + 1                      # s*bh, TwoSum, FFMA, add
    assert bench._DF_FLOPS_BALANCED == 2 * (addsig + df_mul)
    assert bench._DF_FLOPS_BALANCED_FREE == (2 * addsig + 2 * (addsig + 2)) / 2
    shear = df_mul + two_sum + 2                       # a + t w, one component
    assert bench._DF_FLOPS_PRP == (cmul + 4 * shear + cmul) / 2
    assert bench._DF_FLOPS_PRP_NZ == (cmul + 4 * shear) / 2


def test_kernel_flops_of_a_dry_run_plan():
    n = 10
    h = ctypes.c_void_p()
    assert qs.load().qs_wrap(ctypes.c_void_p(1 << 30), n, qs.QS_C128, None, ctypes.byref(h)) == qs.QS_OK
    st = qs.State(h.value, n, qs.QS_C128)
    rng = G.SplitMix64(2)
    gates = G.concat([G.gate_u1(0, G.haar_2x2(rng)), G.gate_u1(1, G.haar_2x2(rng)), G.gate_u1(2, G.MAT_T),
                      G.gate_cu(3, 4, G.MAT_X)])
    p = qs.Plan(st, gates, flags=qs.PLAN_DRY_RUN | qs.PLAN_NO_PRP | qs.PLAN_NO_PHASE_RUNS)
    assert p.stats()["passes"] == 1
    N = float(1 << n)
    got = bench.kernel_flops(p.op_counts(0), n, bench._DF_FLOPS)
    p.close()
    assert got == pytest.approx(2 * 104 * N + 44 * N * 0.5)


def test_counters_go_stale_with_the_kernel_source(monkeypatch):
    """Counters from an ncu capture are used only while the kernel's sources hash
    to the value recorded with them; the issue summary is their plain ratio."""
    entry = dict(bench.NCU_COUNTERS["df"], n=26, dram_bytes=2.0e9, warp_inst=1.2e9, ms=1.4)
    entry["sha"] = bench.sources_sha(entry["sources"])
    monkeypatch.setitem(bench.NCU_COUNTERS, "df", entry)
    s = bench.issue_summary("df")
    assert s["frac_of_issue_peak"] == pytest.approx(1.2e9 / 1.4e-3 / (152 * 4 * 2.07e9))
    assert bench.ncu_counters("df")["dram_bytes"] == 2.0e9
    monkeypatch.setitem(bench.NCU_COUNTERS, "df", dict(entry, sha="0" * 16))
    assert bench.issue_summary("df") is None and bench.ncu_counters("df") is None
    assert bench.issue_summary("nonexistent") is None


def test_hbm_peak_prefers_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6679.8}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (6679.8, "measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    assert bench.hbm_peak() == (bench.HBM_FALLBACK_GBS, "fallback")
