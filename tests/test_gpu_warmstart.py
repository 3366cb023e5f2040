"""Learned warm start: GPU training kernels against the FP64 MLP oracle, and
what the trained networks gain over the flat start (through the C ABI)."""
import os
import tempfile

import numpy as np
import pytest

from oracle import mlp as omlp
from oracle import wls
from paper_2604_23175_gb300 import synth
from tests.helpers import net_of, problem

pytestmark = pytest.mark.gpu


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


def _net(dims, seed):
    rng = np.random.default_rng(seed)
    P, flat = [], []
    for i in range(len(dims) - 1):
        W = rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i])
        b = 0.1 * rng.standard_normal(dims[i + 1])
        P.append((W, b))
        flat += [W.ravel(), b]
    return P, np.concatenate(flat)


@pytest.mark.parametrize("dims,batch", [([40, 64, 64, 64, 12], 37), ([100, 512, 512, 512, 30], 16)])
def test_training_kernels_match_oracle_gradients(mase, dims, batch):
    """BF16 weights/activations with FP32 accumulation: loss and every layer's
    gradient within BF16 tolerance of the FP64 oracle's backpropagation."""
    P, flat = _net(dims, 1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((batch, dims[0]))
    T = rng.standard_normal((batch, dims[-1]))
    loss, g = mase.mlp_check(dims, flat, X, T)
    lref, gref = omlp.loss_and_grads(P, X, T)
    assert abs(loss - lref) <= 2e-2 * lref
    off = 0
    for (gw, gb) in gref:
        ref = np.concatenate([gw.ravel(), gb])
        got = g[off:off + ref.size]
        off += ref.size
        assert np.max(np.abs(got - ref)) <= 3e-2 * np.max(np.abs(ref))
        assert got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref)) > 0.999


def _batch(mase, est, g, seed, S, walk=None):
    import torch
    Vm, Va = synth.make_states(g, S, seed, walk_len=walk)
    e = synth.make_noise(g, S, seed + 1)
    xt = torch.tensor(np.concatenate([Vm, Va], 1), device="cuda")
    z = torch.empty((S, g.n_meas), dtype=torch.float64, device="cuda")
    est.measure(xt, z)
    z += torch.tensor(e, device="cuda")
    return z


def test_learned_start_gain_and_parity(mase):
    """Networks trained on estimator-solved snapshots cut Gauss-Newton steps on
    a held-out 64-step walk, and the estimates stay the oracle's."""
    import torch
    g = synth.make_grid("grid2869_k16")
    N, S = g.n_bus, 64
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    est = mase.Estimator(g, sig, S, z=None, precision=mase.MIXED, schedule=mase.BATCHED)
    Z, X = [], []
    for b in range(128):                      # 8192 independent training states
        z = _batch(mase, est, g, 20000 + 7 * b, S, walk=1)
        est.set_measurements(z)
        x = torch.zeros((S, 2 * N), dtype=torch.float64, device="cuda")
        est.solve(tol=1e-8, max_iter=10, x_out=x)
        Z.append(z)
        X.append(x)
    est.warmstart_train(torch.cat(Z), torch.cat(X), epochs=30, batch=256, lr=1e-3)
    # held-out walk, measurements formed by the oracle for the parity check
    net, Vm, Va, zh, _ = problem(g, S, 4242)
    est.set_measurements(torch.tensor(zh, device="cuda"))
    xf = np.zeros((S, 2 * N))
    rf = est.solve(tol=1e-8, max_iter=10, x_out=xf)
    est.set_start_mode(mase.START_LEARNED)
    xl = np.zeros((S, 2 * N))
    rl = est.solve(tol=1e-8, max_iter=10, x_out=xl)
    assert np.all(rl.status == 0)
    assert rl.iters.mean() < rf.iters.mean(), (rl.iters.mean(), rf.iters.mean())
    w = wls.weights(sig)
    for s in (0, 31, 63):
        ref = wls.gauss_newton(net, zh[s], w, tol=1e-8, max_iter=30)
        assert np.max(np.abs(xl[s, :N] - ref.Vm)) <= 1e-6
        assert np.max(np.abs(xl[s, N:] - ref.Va)) <= 1e-6
        assert abs(rl.J[s] - ref.J) <= 1e-8 * ref.J
    # the proposal itself is closer to the estimate than the flat start
    xp = np.zeros((S, 2 * N))
    est.warmstart_predict(xp)
    assert np.sqrt(np.mean((xp[:, :N] - xf[:, :N]) ** 2)) < np.sqrt(np.mean((1.0 - xf[:, :N]) ** 2))
    # save / load round trip reproduces the proposal
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ws.bin")
        est.warmstart_save(path)
        est2 = mase.Estimator(g, sig, S, z=torch.tensor(zh, device="cuda"), precision=mase.MIXED,
                              schedule=mase.BATCHED)
        est2.warmstart_load(path)
        xp2 = np.zeros_like(xp)
        est2.warmstart_predict(xp2)
        est2.close()
    assert np.max(np.abs(xp2 - xp)) == 0.0
    est.close()


def test_learned_start_requires_a_model(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 2, 4300)
    est = mase.Estimator(g, sig, 2, z=z)
    est.set_start_mode(mase.START_LEARNED)
    res = est.solve(tol=1e-8, max_iter=10, check=False)
    assert res.rc == mase.MASE_ENOTREADY
    est.close()
