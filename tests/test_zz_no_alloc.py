"""The allocation-free coordinator entry point (mase_coordinator_noalloc).

It serves callers that cannot call cudaMalloc when they need the coordinator
step: programs whose device memory belongs to another allocator, and
latency-bound loops that must not take the synchronisation an allocation can
imply.  The test feeds it the condensed per-area blocks (S_b, b_hat_b) of a
state x0, computed by the CPU oracle, and compares its boundary step with the
step that the existing entry point mase_solve takes from x0 (one Gauss-Newton
step), on two calls in a row.  This file is named to be collected last.
"""
import numpy as np
import pytest

from oracle import wls
from paper_2604_23175_gb300 import synth
from tests.helpers import net_of, problem

pytestmark = pytest.mark.gpu

# the FP64 path reproduces the exact condensed step; both sides agree far
# inside the state bar used by the parity tests (1e-6)
STEP_RTOL = 1e-9


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


def _condensed_blocks(net, part, z, w, x0):
    """Oracle S_b^k, b_hat_b^k for every area and snapshot, packed as the
    entry point expects: area-major, then snapshot, packed lower column-major."""
    S = z.shape[0]
    N = net.n_bus
    per_area_S = [[] for _ in range(part.n_area)]
    per_area_b = [[] for _ in range(part.n_area)]
    for s in range(S):
        Vm, Va = x0[s, :N], x0[s, N:]
        r = z[s] - wls.measure(net, Vm, Va)
        H = wls.jacobian(net, Vm, Va)
        for k in range(part.n_area):
            Sb, bh = wls.schur_condense(wls.area_blocks(H, w, r, part, k))
            nb = Sb.shape[0]
            per_area_S[k].append(np.concatenate([Sb[c:, c] for c in range(nb)]))
            per_area_b[k].append(bh)
    Sflat = np.concatenate([np.concatenate(v) for v in per_area_S])
    bflat = np.concatenate([np.concatenate(v) for v in per_area_b])
    return Sflat, bflat


def test_coordinator_noalloc_matches_solve_step(mase):
    import torch
    g = synth.make_grid("grid2869_k16")
    S = 2
    net, Vm, Va, z, sig = problem(g, S, 5100)
    w = wls.weights(sig)
    part = wls.partition(net_of(g), g.area_of_bus, g.n_area)
    rng = np.random.Generator(np.random.PCG64(5101))
    x0 = np.concatenate([1.0 + 0.01 * rng.standard_normal((S, g.n_bus)),
                         0.02 * rng.standard_normal((S, g.n_bus))], axis=1)
    x0[:, g.n_bus + g.slack] = 0.0
    est = mase.Estimator(g, sig, S, z=z, precision=mase.FP64, schedule=mase.BATCHED)
    # existing entry point: one Gauss-Newton step from x0
    x1 = np.zeros_like(x0)
    est.solve(x0=np.ascontiguousarray(x0), tol=0.0, max_iter=1, x_out=x1, check=False)
    cols = wls.state_columns(net)
    ref = (x1 - x0)[:, cols][:, part.gamma_cols]
    Sflat, bflat = _condensed_blocks(net, part, z, w, x0)
    Sd = torch.tensor(Sflat, device="cuda")
    bd = torch.tensor(bflat, device="cuda")
    nG = len(part.gamma_cols)
    for call in range(2):
        dx = torch.full((S, nG), float("nan"), dtype=torch.float64, device="cuda")
        est.coordinator_noalloc(Sd, bd, dx)
        got = dx.cpu().numpy()
        err = np.max(np.abs(got - ref))
        assert err <= STEP_RTOL * max(1.0, np.max(np.abs(ref))), (call, err)
    est.close()


def test_coordinator_noalloc_mixed_with_refinement(mase):
    """MIXED handles factor S_Gamma in FP32 and refine the step once in FP64;
    the step then agrees with the FP64 one to the FP32 factor's accuracy."""
    import torch
    g = synth.make_grid("grid2869_k16")
    S = 2
    net, Vm, Va, z, sig = problem(g, S, 5200)
    w = wls.weights(sig)
    part = wls.partition(net_of(g), g.area_of_bus, g.n_area)
    rng = np.random.Generator(np.random.PCG64(5201))
    x0 = np.concatenate([1.0 + 0.01 * rng.standard_normal((S, g.n_bus)),
                         0.02 * rng.standard_normal((S, g.n_bus))], axis=1)
    x0[:, g.n_bus + g.slack] = 0.0
    est = mase.Estimator(g, sig, S, z=z, precision=mase.FP64, schedule=mase.BATCHED)
    x1 = np.zeros_like(x0)
    est.solve(x0=np.ascontiguousarray(x0), tol=0.0, max_iter=1, x_out=x1, check=False)
    est.close()
    cols = wls.state_columns(net)
    ref = (x1 - x0)[:, cols][:, part.gamma_cols]
    Sflat, bflat = _condensed_blocks(net, part, z, w, x0)
    mixed = mase.Estimator(g, sig, S, z=z, precision=mase.MIXED, schedule=mase.BATCHED, refine=1)
    dx = torch.full((S, len(part.gamma_cols)), float("nan"), dtype=torch.float64, device="cuda")
    mixed.coordinator_noalloc(torch.tensor(Sflat, device="cuda"), torch.tensor(bflat, device="cuda"), dx)
    got = dx.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    mixed.close()


def test_coordinator_noalloc_rejects_oversized_request(mase):
    import torch
    g = synth.make_grid("grid9241_k32")
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    # 64 snapshots of the FP64 boundary system need more than the static maximum
    est = mase.Estimator(g, sig, 64, z=None, precision=mase.FP64, schedule=mase.BATCHED)
    nS, nb, ndx = mase.noalloc_sizes(est.info(), 64)
    Sd = torch.zeros(nS, dtype=torch.float64, device="cuda")
    bd = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dx = torch.zeros(ndx, dtype=torch.float64, device="cuda")
    with pytest.raises(mase.MaseError) as e:
        est.coordinator_noalloc(Sd, bd, dx)
    assert e.value.code == mase.MASE_EINVAL
    assert "static maximum" in str(e.value)
    est.close()


def test_coordinator_noalloc_checks_element_counts(mase):
    """Short buffers are refused by the C entry point itself (before any
    device work) and by the binding (with FP32 tensors too)."""
    import ctypes
    import torch
    g = synth.make_grid("grid2869_k16")
    S = 2
    net, Vm, Va, z, sig = problem(g, S, 5300)
    est = mase.Estimator(g, sig, S, z=z, precision=mase.FP64, schedule=mase.BATCHED)
    nS, nb, ndx = mase.noalloc_sizes(est.info(), S)
    Sd = torch.zeros(nS, dtype=torch.float64, device="cuda")
    bd = torch.zeros(nb, dtype=torch.float64, device="cuda")
    dx = torch.zeros(ndx, dtype=torch.float64, device="cuda")
    lib = mase.load()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    for counts in ((nS - 1, nb, ndx), (nS, nb - 1, ndx), (nS, nb, ndx + 1)):
        rc = lib.mase_coordinator_noalloc(est.h, p(Sd), counts[0], p(bd), counts[1], p(dx), counts[2])
        assert rc == mase.MASE_EINVAL
    with pytest.raises(ValueError):
        est.coordinator_noalloc(Sd[:-1], bd, dx)
    with pytest.raises(ValueError):
        est.coordinator_noalloc(Sd.float(), bd, dx)
    est.close()
