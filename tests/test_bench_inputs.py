"""The benchmark's workload variants (CPU only): the sweep over the number of
areas draws the headline grid itself at 32 areas, and a dropped family masks
exactly that family's rows."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2604_23175_gb300 import synth  # noqa: E402


def _inputs(areas, snapshots=2):
    return bench.workload_inputs(argparse.Namespace(workload=bench.WORKLOAD, areas=areas,
                                                    snapshots=snapshots))


def test_area_sweep_at_32_is_the_benchmark_grid():
    g, *_ = _inputs(32)
    h = synth.make_grid(bench.WORKLOAD)
    for f in ("from_bus", "to_bus", "r", "x", "b_charge", "area_of_bus"):
        np.testing.assert_array_equal(getattr(g, f), getattr(h, f))


def test_area_sweep_keeps_the_network_size():
    for K in (16, 64):
        g, *_ = _inputs(K)
        assert (g.n_bus, g.n_branch, g.n_area) == (9241, 16049, K)
        assert np.bincount(g.area_of_bus, minlength=K).min() > 0


def test_family_mask_drops_one_family():
    g = synth.make_grid("grid300_k4")
    N, L = g.n_bus, g.n_branch
    m = synth.family_mask(g, "Qt", 3)
    assert m.shape == (3, g.n_meas)
    assert np.all(m[:, 3 * N + 3 * L:] == 0) and np.all(m[:, :3 * N + 3 * L] == 1)
