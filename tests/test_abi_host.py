"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
and its host-side symbolic setup matches the oracle's partition and dense
Cholesky (no GPU calls)."""
import os
import re

import numpy as np
import pytest

from oracle import wls
from paper_2604_23175_gb300 import synth
from tests.helpers import net_of, tiny_grid, with_parallel_branches

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mase():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_23175_gb300 import mase as m
    m.load()
    return m


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(mase_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(mase):
    import ctypes
    lib = ctypes.CDLL(mase.LIB_PATH)
    names = _declared_functions()
    assert "mase_create" in names and "mase_solve" in names and "mase_destroy" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_struct_layouts_match_the_library(mase):
    for name, (c_size, py_size) in mase.abi_sizes().items():
        assert c_size == py_size, (name, c_size, py_size)


def test_status_strings_and_defaults(mase):
    assert mase.status_str(0) == "MASE_OK"
    assert mase.status_str(-2) == "MASE_EUNOBSERVABLE"
    o = mase.default_options()
    assert o.precision == mase.MIXED and o.schedule == mase.BATCHED and o.refine == 1 and o.inner_iters == 0
    assert o.autotune == 1 and o.profile == 0 and o.wait_polls == 0


@pytest.mark.parametrize("name", ["grid300_k4", "grid2869_k16", "grid9241_k32"])
def test_setup_counts_match_oracle_partition(mase, name):
    g = synth.make_grid(name)
    info = mase.analyze(g)
    part = wls.partition(net_of(g), g.area_of_bus, g.n_area)
    assert info["n_state"] == 2 * g.n_bus - 1
    assert info["n_meas"] == 3 * g.n_bus + 4 * g.n_branch
    assert info["n_boundary_bus"] == len(part.boundary_buses)
    assert info["n_gamma"] == len(part.gamma_cols)
    nb = max(len(c) for c in part.boundary_cols)
    assert info["max_area_nb"] == nb


@pytest.mark.parametrize("name,slack_b", [("grid300_k4", False), ("grid2869_k16", False),
                                           ("grid2869_k16", True), ("grid9241_k32", False)])
def test_symbolic_setup_selfcheck(mase, name, slack_b):
    g = synth.make_grid(name, slack_on_boundary=slack_b)
    err = mase.selfcheck(g, seed=7)
    assert np.all(err < 1e-12), err


@pytest.mark.parametrize("name,K", [("grid10000_k48", 0), ("grid9241_k32", 16), ("grid9241_k32", 48)])
def test_symbolic_setup_selfcheck_other_partitions(mase, name, K):
    """The 10000-bus grid and the benchmark network split by the partitioner
    into other numbers of areas (the area-count sweep's inputs)."""
    g = synth.make_grid(name)
    if K:
        g = synth.partition_network(g, K)
    err = mase.selfcheck(g, seed=3)
    assert np.all(err < 1e-12), err


def test_selfcheck_parallel_branches(mase):
    """Parallel lines (inside an area, and a tie line in both orientations)
    share gain entries and boundary unknowns."""
    for g in (with_parallel_branches(tiny_grid(14, 3, seed=5)),
              with_parallel_branches(synth.make_grid("grid300_k4"))):
        info = mase.analyze(g)
        assert info["n_meas"] == 3 * g.n_bus + 4 * g.n_branch
        assert np.all(mase.selfcheck(g, 3) < 1e-12)


def test_selfcheck_tiny_and_single_area(mase):
    g = tiny_grid(12, 3, seed=5)
    assert np.all(mase.selfcheck(g, 1) < 1e-12)
    g1 = tiny_grid(10, 1, seed=2)
    info = mase.analyze(g1)
    assert info["n_gamma"] == 0
    assert np.all(mase.selfcheck(g1, 1) < 1e-12)


def test_invalid_inputs_rejected_on_host(mase):
    g = synth.make_grid("grid300_k4")
    bad = synth.Grid(g.n_bus, g.from_bus.copy(), g.to_bus.copy(), g.r, g.x, g.b_charge,
                     g.area_of_bus, g.n_area, 0)
    bad.to_bus[3] = bad.from_bus[3]
    with pytest.raises(mase.MaseError) as e:
        mase.analyze(bad)
    assert e.value.code == mase.MASE_EINVAL
    bad2 = synth.Grid(g.n_bus, g.from_bus, g.to_bus, g.r, g.x, g.b_charge,
                      g.area_of_bus.copy(), g.n_area, 0)
    bad2.area_of_bus[0] = 99
    with pytest.raises(mase.MaseError):
        mase.analyze(bad2)
    bad3 = synth.Grid(g.n_bus, g.from_bus.copy(), g.to_bus, g.r, g.x, g.b_charge,
                      g.area_of_bus, g.n_area, 0)
    bad3.from_bus[0] = g.n_bus
    with pytest.raises(mase.MaseError):
        mase.analyze(bad3)


def test_noalloc_argument_checks_on_host(mase):
    """The binding's size and dtype checks of the no-alloc coordinator step,
    with sizes from the host-only analysis (no GPU): short or FP32 buffers are
    refused before any call into the library."""
    g = synth.make_grid("grid2869_k16")
    info = mase.analyze(g)
    part = wls.partition(net_of(g), g.area_of_bus, g.n_area)
    nbs = [len(c) for c in part.boundary_cols]
    assert info["coord_S_elems"] == sum(n * (n + 1) // 2 for n in nbs)
    assert info["coord_b_elems"] == sum(nbs)
    need = mase.noalloc_sizes(info, 3)
    ok = [np.zeros(n) for n in need]
    mase.check_noalloc_args(need, *ok)
    for i in range(3):
        short = list(ok)
        short[i] = np.zeros(need[i] - 1)
        with pytest.raises(ValueError):
            mase.check_noalloc_args(need, *short)
        f32 = list(ok)
        f32[i] = np.zeros(need[i], dtype=np.float32)
        with pytest.raises(ValueError):
            mase.check_noalloc_args(need, *f32)


def test_array_checks_before_any_library_call(mase):
    """Per-snapshot buffers of another element type or size are refused by
    the binding before it calls the library (which would read or write them
    at the sizes the handle implies).  The handle below is never created: a
    method that reached the library would fail with MaseError instead."""
    import torch
    g = synth.make_grid("grid300_k4")
    S, N, m = 2, g.n_bus, g.n_meas
    mase.check_array("x", np.zeros(S * 2 * N), S * 2 * N, "float64")
    mase.check_array("x", torch.zeros(S, 2 * N, dtype=torch.float64), S * 2 * N, "float64")
    mase.check_array("mask", np.ones((S, m), dtype=np.uint8), S * m, "uint8")
    mase.check_array("x", None, S * 2 * N, "float64")
    for bad in (np.zeros(S * 2 * N - 1), np.zeros(S * 2 * N, dtype=np.float32),
                torch.zeros(S, 2 * N, dtype=torch.float32), [0.0] * (S * 2 * N)):
        with pytest.raises(ValueError):
            mase.check_array("x", bad, S * 2 * N, "float64")
    with pytest.raises(ValueError):
        mase.check_array("mask", np.ones((S, m), dtype=bool), S * m, "uint8")

    est = mase.Estimator.__new__(mase.Estimator)
    est.lib, est.h, est.n_snap, est.n_bus, est.n_meas = mase.load(), None, S, N, m
    x_ok, z_ok = np.zeros((S, 2 * N)), np.zeros((S, m))
    x_short, z_f32 = np.zeros((S, 2 * N - 1)), np.zeros((S, m), dtype=np.float32)
    calls = [lambda: est.solve(x_out=x_short), lambda: est.solve(x0=x_short, x_out=x_ok),
             lambda: est.measure(x_short, z_ok), lambda: est.measure(x_ok, z_f32),
             lambda: est.set_measurements(z_f32), lambda: est.set_measurements(z_ok, np.ones((S, m))),
             lambda: est.warmstart_predict(x_short),
             lambda: est.warmstart_train(z_ok, x_short), lambda: est.warmstart_train(z_f32, x_ok)]
    for call in calls:
        with pytest.raises(ValueError):
            call()
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    with pytest.raises(ValueError):
        mase.Estimator(g, sig[:-1], S)
    with pytest.raises(ValueError):
        mase.Estimator(g, sig, S, z=z_ok[:1])


def test_product_path_fails_loudly_without_its_library_or_gpu(tmp_path):
    """There is no CPU path: the binding raises when the library is absent,
    and the benchmark's own arm exits with an error when no GPU is present."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2604_23175_gb300 import mase\n"
            "mase.LIB_PATH = %r\n"
            "try:\n    mase.load()\nexcept RuntimeError as e:\n    print('raised', e)\n") % (
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), str(tmp_path / "absent.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("raised"), out.stdout + out.stderr
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        return
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode != 0 and "needs a CUDA device" in (out.stdout + out.stderr)
    assert not any(s.startswith("{") for s in out.stdout.splitlines())
