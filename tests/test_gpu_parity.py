"""GPU parity of libmase against the FP64 CPU oracle, through the C ABI.

Bars (from the method's stated accuracy targets): converged state within
1e-6 in |dV| and |dtheta| and J = r^T W r within 1e-8 relative of the oracle's
converged WLS estimate; the FP64 path additionally takes the oracle's
iteration counts (a condensed step equals the centralised step).
"""
import numpy as np
import pytest

from oracle import wls
from paper_2604_23175_gb300 import synth
from tests.helpers import net_of, problem, with_parallel_branches

pytestmark = pytest.mark.gpu

STATE_TOL = 1e-6
J_RTOL = 1e-8


@pytest.fixture(scope="module")
def mase():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_23175_gb300 import mase as m
    m.load()
    return m


def _run(mase, grid, sig, z, mask=None, precision=None, schedule=None, x0=None, tol=1e-8,
         max_iter=20, **kw):
    S = z.shape[0]
    est = mase.Estimator(grid, sig, S, z=z, mask=mask, precision=precision, schedule=schedule, **kw)
    x = np.zeros((S, 2 * grid.n_bus))
    res = est.solve(x0=x0, tol=tol, max_iter=max_iter, x_out=x, check=False)
    est.close()
    return x, res


def _check(net, grid, x, res, z, w, snaps, tol=1e-8, same_iters=False, x0=None):
    N = grid.n_bus
    for s in snaps:
        v0 = (None, None) if x0 is None else (x0[s, :N], x0[s, N:])
        ref = wls.gauss_newton(net, z[s], w if w.ndim == 1 else w[s], Vm0=v0[0], Va0=v0[1],
                               tol=tol, max_iter=30)
        assert ref.converged
        dV = np.max(np.abs(x[s, :N] - ref.Vm))
        dT = np.max(np.abs(x[s, N:] - ref.Va))
        assert dV <= STATE_TOL and dT <= STATE_TOL, (s, dV, dT)
        assert abs(res.J[s] - ref.J) <= J_RTOL * ref.J, (s, res.J[s], ref.J)
        assert res.status[s] == 0
        if same_iters:
            assert res.iters[s] == ref.iters, (s, res.iters[s], ref.iters)


def test_measure_matches_oracle(mase):
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 3, 3100)
    est = mase.Estimator(g, sig, 3, z=z)
    x = np.concatenate([Vm, Va], axis=1)
    out = np.zeros_like(z)
    est.measure(np.ascontiguousarray(x), out)
    est.close()
    for s in range(3):
        h = wls.measure(net, Vm[s], Va[s])
        assert np.max(np.abs(out[s] - h)) <= 1e-11 * max(1.0, np.max(np.abs(h)))


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_parity_parallel_branches(mase, precision):
    """Parallel lines (one inside an area, one tie line doubled in the
    reverse orientation): h(x) and the converged estimates equal the
    oracle's, and FP64 takes its iteration counts."""
    g = with_parallel_branches(synth.make_grid("grid300_k4"))
    net, Vm, Va, z, sig = problem(g, 2, 3250)
    est = mase.Estimator(g, sig, 2, z=z)
    out = np.zeros_like(z)
    est.measure(np.ascontiguousarray(np.concatenate([Vm, Va], axis=1)), out)
    est.close()
    for s in range(2):
        h = wls.measure(net, Vm[s], Va[s])
        assert np.max(np.abs(out[s] - h)) <= 1e-11 * max(1.0, np.max(np.abs(h)))
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=getattr(mase, precision), schedule=mase.BATCHED)
    assert res.rc == mase.MASE_OK, (res.rc, res.status)
    _check(net, g, x, res, z, w, range(2), same_iters=(precision == "FP64"))


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
@pytest.mark.parametrize("schedule", ["PER_AREA", "BATCHED"])
@pytest.mark.parametrize("name", ["grid300_k4", "grid2869_k16"])
def test_parity_small_grids(mase, name, precision, schedule):
    g = synth.make_grid(name)
    net, Vm, Va, z, sig = problem(g, 2, 3200)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=getattr(mase, precision),
                  schedule=getattr(mase, schedule))
    assert res.rc == mase.MASE_OK, res
    _check(net, g, x, res, z, w, range(2), same_iters=(precision == "FP64"))


@pytest.mark.parametrize("precision,schedule", [("MIXED", "BATCHED"), ("FP64", "PER_AREA")])
def test_parity_inner_local_iterations(mase, precision, schedule):
    """Two local Gauss-Newton steps per area with the boundary fixed before each
    condensed step (Eq. local_wls) change the path, not the WLS estimate."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 2, 3270)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=getattr(mase, precision),
                  schedule=getattr(mase, schedule), inner_iters=2)
    assert res.rc == mase.MASE_OK, res
    _check(net, g, x, res, z, w, range(2))


@pytest.mark.parametrize("threads", [128, 256])
def test_parity_fewer_warps_without_graphs(mase, threads):
    """The task lists are scheduled for 16 warps; fewer warps per block must
    give the same estimates (any warp count preserves the topological order),
    and so must stepping without CUDA graphs."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 2, 3260)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED, threads=threads,
                  use_graph=False)
    assert res.rc == mase.MASE_OK, res
    _check(net, g, x, res, z, w, range(2))


@pytest.mark.parametrize("tensor_units", [1, 8, 16])
@pytest.mark.parametrize("name", ["grid300_k4", "grid2869_k16"])
def test_parity_tensor_core_units(mase, name, tensor_units):
    """MIXED with the factorisation's update units on the tensor cores (3xTF32
    MMA) for source panels at least tensor_units wide (1: every unit, in the
    area factors and the coordinator): the oracle's estimates, and the FP32
    units' iteration counts."""
    g = synth.make_grid(name)
    net, Vm, Va, z, sig = problem(g, 3, 3310)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED,
                  tensor_units=tensor_units)
    assert res.rc == mase.MASE_OK, res
    _check(net, g, x, res, z, w, range(3))
    x0, res0 = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED, tensor_units=0)
    assert np.array_equal(res.iters, res0.iters), (res.iters, res0.iters)
    assert np.max(np.abs(x - x0)) <= 1e-8


@pytest.mark.parametrize("refine", [0, 3])
def test_parity_refinement_sweeps(mase, refine):
    """MIXED without the FP64 refinement of the boundary solve (an inexact
    Newton step each iteration) and with three sweeps."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 2, 3250)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED, refine=refine)
    assert res.rc == mase.MASE_OK, res
    _check(net, g, x, res, z, w, range(2))


def test_parity_slack_on_boundary(mase):
    g = synth.make_grid("grid2869_k16", slack_on_boundary=True)
    net, Vm, Va, z, sig = problem(g, 2, 3300)
    w = wls.weights(sig)
    for prec in (mase.FP64, mase.MIXED):
        x, res = _run(mase, g, sig, z, precision=prec, schedule=mase.BATCHED)
        assert res.rc == mase.MASE_OK
        _check(net, g, x, res, z, w, range(2), same_iters=(prec == mase.FP64))
        assert np.all(x[:, g.n_bus + g.slack] == 0.0)


def test_parity_random_row_drops(mase):
    g = synth.make_grid("grid2869_k16")
    S = 4
    net, Vm, Va, z, sig = problem(g, S, 3400)
    mask = synth.make_mask(g, S, 0.10, 3401)
    W = np.stack([wls.weights(sig, mask[s]) for s in range(S)])
    for prec in (mase.FP64, mase.MIXED):
        x, res = _run(mase, g, sig, z, mask=mask, precision=prec, schedule=mase.BATCHED)
        assert res.rc == mase.MASE_OK
        _check(net, g, x, res, z, W, range(S), same_iters=(prec == mase.FP64))


def test_parity_family_mask(mase):
    """Structured masking of a whole flow family (Sec. 5.4 experiment)."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 1, 3450)
    for fam in ("Pf", "Qt"):
        mask = synth.family_mask(g, fam, 1)
        w = wls.weights(sig, mask[0])
        x, res = _run(mase, g, sig, z, mask=mask, precision=mase.MIXED, schedule=mase.BATCHED)
        assert res.rc == mase.MASE_OK
        _check(net, g, x, res, z, w, [0])


def test_start_from_solution_takes_one_step(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 2, 3500)
    w = wls.weights(sig)
    x0 = np.zeros((2, 2 * g.n_bus))
    for s in range(2):
        ref = wls.gauss_newton(net, z[s], w, tol=1e-13, max_iter=30)
        x0[s] = np.concatenate([ref.Vm, ref.Va])
    x, res = _run(mase, g, sig, z, x0=x0, precision=mase.MIXED, schedule=mase.BATCHED)
    assert res.rc == mase.MASE_OK
    assert np.all(res.iters == 1)
    assert np.max(np.abs(x - x0)) < 1e-8


def test_device_pointers_match_host(mase):
    import torch
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 3, 3600)
    xh, rh = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED)
    zd = torch.tensor(z, device="cuda")
    est = mase.Estimator(g, sig, 3, z=zd, precision=mase.MIXED, schedule=mase.BATCHED)
    xd = torch.zeros((3, 2 * g.n_bus), dtype=torch.float64, device="cuda")
    rd = est.solve(tol=1e-8, max_iter=20, x_out=xd)
    est.close()
    assert np.array_equal(rd.iters, rh.iters)
    assert np.max(np.abs(xd.cpu().numpy() - xh)) < 1e-9


def test_unobservable_snapshot_reports_status(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 2, 3700)
    mask = np.ones((2, g.n_meas), dtype=np.uint8)
    mask[1, :] = 0                       # snapshot 1 has no measurements at all
    x, res = _run(mase, g, sig, z, mask=mask, precision=mase.MIXED, schedule=mase.BATCHED)
    assert res.rc == mase.MASE_EUNOBSERVABLE
    assert res.status[0] == mase.SNAP_CONVERGED
    assert res.status[1] == mase.SNAP_NOT_SPD


def test_nonfinite_measurement_reports_status(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 2, 3800)
    z = z.copy()
    z[1, 5] = np.nan
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED)
    assert res.status[0] == mase.SNAP_CONVERGED
    assert res.status[1] == mase.SNAP_NONFINITE
    assert res.rc == mase.MASE_ENONFINITE


def test_max_iter_reports_not_converged(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 1, 3900)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED, max_iter=1)
    assert res.rc == mase.MASE_NOT_CONVERGED
    assert res.status[0] == mase.SNAP_MAX_ITER and res.iters[0] == 1


def test_repeat_solves_and_launch_counts(mase):
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 2, 4000)
    est = mase.Estimator(g, sig, 2, z=z, precision=mase.MIXED, schedule=mase.BATCHED)
    classes = est.info()["local_classes"]
    x1 = np.zeros((2, 2 * g.n_bus))
    x2 = np.zeros_like(x1)
    r1 = est.solve(tol=1e-8, max_iter=20, x_out=x1)
    r2 = est.solve(tol=1e-8, max_iter=20, x_out=x2)
    est.close()
    assert np.array_equal(r1.iters, r2.iters)
    # FP32 atomic accumulation order varies between runs; the converged states
    # agree to within the stopping tolerance
    assert np.max(np.abs(x1 - x2)) < 1e-8
    it = int(r1.iters.max())
    # reset + state-in + per step (one area-kernel launch per autotuned class,
    # boundary, back, bookkeeping) + objective + state-out
    assert r1.launches == 2 + (classes + 3) * it + 2


def test_stage_times_account_for_the_solve(mase):
    """The per-stage device times, the learned-start and start/finish phases
    and the loop's gaps add up to the solve's wall time; with the device-side
    loop (graph) the gaps are small, stepping from the host they hold the
    per-step round trips."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 8, 4100)
    for use_graph, inner in ((True, 0), (False, 0), (True, 2)):
        est = mase.Estimator(g, sig, 8, z=z, precision=mase.MIXED, schedule=mase.BATCHED,
                             use_graph=use_graph, inner_iters=inner)
        est.solve(tol=1e-8, max_iter=10)
        r = est.solve(tol=1e-8, max_iter=10)
        est.close()
        st = np.array(r.stage_ms)
        assert r.rc == mase.MASE_OK and r.steps == int(r.iters.max())
        assert np.all(st[:6] >= 0.0) and st[6] >= -0.01, (inner, st)
        assert st[0] > 0 and st[1] > 0 and st[2] > 0 and st[3] > 0
        assert abs(st.sum() - r.solve_ms) <= 1e-3 * r.solve_ms + 1e-3, (st, r.solve_ms)
        if use_graph:
            assert st[6] <= 0.2 * r.solve_ms, (inner, st)


def test_bounded_wait_gives_up_with_device_status(mase):
    """A dependency wait of the area factorisation that runs out of polls
    (here after one unsatisfied poll) ends the kernel normally with the
    snapshot's status MASE_SNAP_DEVICE and mase_solve returning MASE_EDEVICE;
    the context stays usable and a default handle then solves correctly."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 4, 4200)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED, wait_polls=1)
    assert res.rc == mase.MASE_EDEVICE, (res.rc, res.status)
    assert np.any(res.status == mase.SNAP_DEVICE)
    assert np.all((res.status == mase.SNAP_DEVICE) | (res.status == mase.SNAP_CONVERGED))
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=mase.MIXED, schedule=mase.BATCHED)
    assert res.rc == mase.MASE_OK
    _check(net, g, x, res, z, w, [0])


def _one_area(g):
    return synth.Grid(g.n_bus, g.from_bus, g.to_bus, g.r, g.x, g.b_charge,
                      np.zeros(g.n_bus, dtype=np.int32), 1, g.slack, g.name + "_central")


@pytest.mark.parametrize("precision", ["FP64", "MIXED"])
def test_parity_centralised_one_area(mase, precision):
    """Centralised GPU Gauss-Newton: the whole network as one area (no
    boundary, no coordinator), its gain matrix factored as one sparse
    supernodal Cholesky with vectors and factor in global memory.  The
    paper's "centralized GPU" baseline (Sec. 5.1); same estimates as the
    oracle, and in FP64 the same iteration counts."""
    g = _one_area(synth.make_grid("grid2869_k16"))
    net, Vm, Va, z, sig = problem(g, 2, 4400)
    w = wls.weights(sig)
    x, res = _run(mase, g, sig, z, precision=getattr(mase, precision), schedule=mase.BATCHED)
    assert res.rc == mase.MASE_OK, (res.rc, res.status)
    _check(net, g, x, res, z, w, range(2), same_iters=(precision == "FP64"))


def test_autotuner_reports_a_valid_configuration(mase):
    """With autotune (the default) mase_create measures the launch
    configuration and reports it; the classes cover every area once, each
    within the block-size and shared-memory limits; without autotune one
    launch holds every area.  Both configurations give the oracle's
    estimates (every other parity test also runs tuned handles)."""
    g = synth.make_grid("grid2869_k16")
    net, Vm, Va, z, sig = problem(g, 4, 4500)
    w = wls.weights(sig)
    for tune in (True, False):
        est = mase.Estimator(g, sig, 4, z=z, precision=mase.MIXED, schedule=mase.BATCHED, autotune=tune)
        info = est.info()
        x = np.zeros((4, 2 * g.n_bus))
        res = est.solve(tol=1e-8, max_iter=20, x_out=x)
        est.close()
        assert info["tuned"] == int(tune)
        nc = info["local_classes"]
        assert 1 <= nc <= 3
        assert sum(info["class_areas"][:nc]) == g.n_area
        for c in range(nc):
            assert 64 <= info["class_threads"][c] <= 512 and info["class_threads"][c] % 32 == 0
            assert 0 < info["class_smem"][c] <= 227 * 1024
        if not tune:
            assert nc == 1 and info["class_threads"][0] == 512
        assert info["back_threads"] in (128, 256)
        _check(net, g, x, res, z, w, range(4))
