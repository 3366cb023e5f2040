"""The benchmark's workload variants (CPU only): the sweep over the number of
areas re-partitions the headline network itself (same buses and branches,
only the partition changes), the default is the headline grid, and a dropped
family masks exactly that family's rows."""
import argparse
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2604_23175_gb300 import synth  # noqa: E402


def _inputs(areas, snapshots=2):
    return bench.workload_inputs(argparse.Namespace(workload=bench.WORKLOAD, areas=areas,
                                                    snapshots=snapshots))


def test_default_is_the_benchmark_grid():
    g, *_ = _inputs(0)
    h = synth.make_grid(bench.WORKLOAD)
    for f in ("from_bus", "to_bus", "r", "x", "b_charge", "area_of_bus"):
        np.testing.assert_array_equal(getattr(g, f), getattr(h, f))


def test_area_sweep_repartitions_the_same_network():
    h = synth.make_grid(bench.WORKLOAD)
    for K in (16, 48):
        g, *_ = _inputs(K)
        assert (g.n_bus, g.n_branch, g.n_area) == (9241, 16049, K)
        for f in ("from_bus", "to_bus", "r", "x", "b_charge"):
            np.testing.assert_array_equal(getattr(g, f), getattr(h, f))
        assert np.bincount(g.area_of_bus, minlength=K).min() > 0


def test_family_mask_drops_one_family():
    g = synth.make_grid("grid300_k4")
    N, L = g.n_bus, g.n_branch
    m = synth.family_mask(g, "Qt", 3)
    assert m.shape == (3, g.n_meas)
    assert np.all(m[:, 3 * N + 3 * L:] == 0) and np.all(m[:, :3 * N + 3 * L] == 1)


def test_oracle_baseline_children_on_a_small_grid():
    """The CPU baseline's worker processes (centralised and multi-area
    oracle) solve their snapshots and agree with each other."""
    argv = ["--workload", "grid300_k4", "--snapshots", "4"]
    wall, outs, x = bench.oracle_run(argv, [[0], [1]])
    assert x.shape == (2, 600) and wall > 0 and all(o["iters"][0] >= 2 for o in outs)
    wall2, outs2, x2 = bench.oracle_run(argv, [[0, 1]], multi=True)
    assert np.max(np.abs(x - x2)) < 1e-9


def test_oracle_baseline_children_use_the_workload_mask():
    """Under random drops the CPU baseline solves the masked problem: its
    estimate equals the oracle's own solve with the same mask and differs
    from the unmasked one."""
    from oracle import wls
    from tests.helpers import net_of
    argv = ["--workload", "grid300_k4", "--snapshots", "3", "--drop", "0.2"]
    _, _, x = bench.oracle_run(argv, [[1]])
    args = bench.parse_from(argv)
    g = bench.workload_grid(args)
    _, Vm, Va, e, sig = bench.workload_inputs(args)
    mask = bench.workload_mask(args, g)
    assert mask is not None and mask.shape == (3, g.n_meas) and mask[1].mean() < 0.85
    net = net_of(g)
    z = wls.measure(net, Vm[1], Va[1]) + e[1]
    ref = wls.gauss_newton(net, z, wls.weights(sig, mask[1]), tol=bench.TOL, max_iter=bench.MAX_ITER)
    full = wls.gauss_newton(net, z, wls.weights(sig), tol=bench.TOL, max_iter=bench.MAX_ITER)
    assert np.max(np.abs(x[0] - np.concatenate([ref.Vm, ref.Va]))) < 1e-12
    assert np.max(np.abs(x[0] - np.concatenate([full.Vm, full.Va]))) > 1e-6


def test_workload_name_is_shared_by_both_arms():
    """The GPU arm and the oracle's reference arm name the same workload: the
    benchmark's own description by default, a variant's flags otherwise."""
    args = bench.parse_from([])
    g = synth.make_grid(bench.WORKLOAD)
    assert bench.workload_desc(args, g, args.snapshots) == bench.WORKLOAD_DESC
    v = bench.parse_from(["--areas", "16", "--drop", "0.1"])
    d = bench.workload_desc(v, g, v.snapshots)
    assert d != bench.WORKLOAD_DESC and "10% rows dropped" in d
    assert bench.workload_desc(args, g, 16) != bench.WORKLOAD_DESC


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle on the host cores, no GPU) prints
    one JSON line with the GPU arm's metric, unit and direction, a
    cpu_baseline describing the run and an e2e entry without copies."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "grid300_k4", "--snapshots", "4", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(s) for s in out.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["n_bus"] == 300 and d["config"]["n_snap"] == 4
    assert d["config"]["workload"] == "grid300_k4 x4 snapshots"


def test_headline_roofline_against_the_derived_alu_peak():
    """The dominant kernel's roofline: achieved FP64 rate over the peak
    derived from SMs, FP64 FMAs per SM cycle and the maximum SM clock, with
    the measured DGEMM as a second denominator."""
    peak, src = bench.fp64_alu_peak_tflops()
    mhz = float(src.split(" x ")[-1].split()[0])
    assert peak == pytest.approx(152 * 2 * 2 * mhz * 1e-6)
    assert 1.0 < peak < 1.5                      # GB300 nominal FP64: 1.25 TFLOP/s
    lo = {"fp64_tflops": 0.05, "avg_launch_ms": 2.9}
    r = bench.headline_roofline(lo, peak, src, 1.1, 1.2e8)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["traffic"] == 1.2e8
    assert r["frac"] == pytest.approx(0.05 / peak) and r["frac_of_measured_dgemm"] == pytest.approx(0.05 / 1.1)
    for k in ("achieved", "peak", "frac", "traffic"):
        assert k in r
