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


def _bf16_bits_rne(a32):
    """Round-to-nearest-even of FP32 values to BF16, as raw 16-bit patterns."""
    u = np.asarray(a32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def test_adamw_kernel_matches_oracle(mase):
    """The training's AdamW kernel (FP32) against the FP64 oracle update over
    20 steps with a cosine learning-rate schedule and weight decay, on
    parameters and gradients spanning several magnitudes (zero and tiny
    gradients exercise pure decay and eps).  The oracle gets the kernel's
    constants as the FP32 numbers they are.  Bar, with u = 2^-24: a few
    roundings per operation, plus the FP32 bias corrections 1 - beta^t, whose
    rounding is amplified by beta^t / (1 - beta^t)."""
    rng = np.random.default_rng(11)
    n, steps = 4099, 20
    f32 = lambda x: float(np.float32(x))
    b1, b2, eps, wd = f32(0.9), f32(0.999), f32(1e-8), f32(1e-2)
    w0 = (rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 1, n)).astype(np.float32)
    grads = (rng.standard_normal((steps, n)) * 10.0 ** rng.uniform(-9, 1, (1, n))).astype(np.float32)
    grads[:, :7] = 0.0
    lr = (1e-3 * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * np.arange(steps) / (steps - 1))))).astype(np.float32)
    w, m, v, w16 = mase.adamw_check(w0, grads, lr, wd)
    u = 2.0 ** -24
    wr = w0.astype(np.float64)
    mr = np.zeros(n)
    vr = np.zeros(n)
    bw = np.zeros(n)      # error bounds, accumulated along the oracle's trajectory
    bm = np.zeros(n)
    bv = np.zeros(n)
    for t in range(1, steps + 1):
        g = grads[t - 1].astype(np.float64)
        lt = float(lr[t - 1])
        bm = b1 * bm + 3 * u * (b1 * np.abs(mr) + (1 - b1) * np.abs(g))
        bv = b2 * bv + 3 * u * (b2 * vr + (1 - b2) * g * g)
        w_prev = wr.copy()
        mr, vr = omlp.adamw_step(wr, g, mr, vr, t, lt, beta1=b1, beta2=b2, eps=eps, wd=wd)
        step = np.abs(w_prev * (1 - lt * wd) - wr)
        amp = u * (b1 ** t / (1 - b1 ** t) + 0.5 * b2 ** t / (1 - b2 ** t))
        rel_m = bm / np.maximum(np.abs(mr), 1e-300)
        bw = bw + 3 * u * np.abs(w_prev) + step * (8 * u + amp + np.minimum(rel_m, 1.0)) \
            + lt * bm / (1 - b1 ** t) / (np.sqrt(vr / (1 - b2 ** t)) + eps) * (rel_m > 1.0)
    assert np.all(np.abs(w - wr) <= 2 * bw + 1e-30), np.max(np.abs(w - wr) / (bw + 1e-30))
    assert np.all(np.abs(m - mr) <= 2 * bm + 1e-38)
    assert np.all(np.abs(v - vr) <= 2 * bv + 1e-38)
    # the BF16 copy the networks compute with is the FP32 master rounded to nearest even
    assert np.array_equal(w16, _bf16_bits_rne(w))


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


def test_learned_start_trained_under_drops(mase):
    """Networks trained on masked samples (10 % of rows dropped at random per
    sample, the training snapshots solved under their masks) still cut
    Gauss-Newton steps on a held-out walk with fresh random drops, and the
    estimates stay the oracle's for the masked problem."""
    import torch
    g = synth.make_grid("grid2869_k16")
    N, S = g.n_bus, 64
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    est = mase.Estimator(g, sig, S, z=None, precision=mase.MIXED, schedule=mase.BATCHED)
    masks = [torch.tensor(synth.make_mask(g, S, 0.10, 21000 + b), device="cuda") for b in range(4)]
    Z, X, Ms = [], [], []
    for b in range(128):                      # 8192 independent training states
        z = _batch(mase, est, g, 20000 + 7 * b, S, walk=1)
        est.set_measurements(z, masks[b % 4])
        x = torch.zeros((S, 2 * N), dtype=torch.float64, device="cuda")
        r = est.solve(tol=1e-8, max_iter=10, x_out=x, check=False)
        ok = torch.tensor(r.status == 0, device="cuda")
        Z.append(z[ok])
        X.append(x[ok])
        Ms.append(masks[b % 4][ok])
    with pytest.raises(ValueError):
        est.warmstart_train(torch.cat(Z), torch.cat(X), mask=torch.cat(Ms)[:-1])
    est.warmstart_train(torch.cat(Z), torch.cat(X), epochs=30, batch=256, lr=1e-3, mask=torch.cat(Ms))
    net, Vm, Va, zh, _ = problem(g, S, 4343)
    mh = synth.make_mask(g, S, 0.10, 4344)
    est.set_measurements(torch.tensor(zh, device="cuda"), torch.tensor(mh, device="cuda"))
    xf = np.zeros((S, 2 * N))
    rf = est.solve(tol=1e-8, max_iter=15, x_out=xf)
    est.set_start_mode(mase.START_LEARNED)
    xl = np.zeros((S, 2 * N))
    rl = est.solve(tol=1e-8, max_iter=15, x_out=xl)
    assert np.all(rl.status == 0) and np.all(rf.status == 0)
    assert rl.iters.mean() < rf.iters.mean(), (rl.iters.mean(), rf.iters.mean())
    for s in (0, 40):
        ref = wls.gauss_newton(net, zh[s], wls.weights(sig, mh[s]), tol=1e-8, max_iter=30)
        assert np.max(np.abs(xl[s, :N] - ref.Vm)) <= 1e-6
        assert np.max(np.abs(xl[s, N:] - ref.Va)) <= 1e-6
    est.close()


def _edit_model(path, **arrays):
    """Rewrite named float arrays (fm, fsd, om, osd) of a saved warm-start file."""
    raw = bytearray(open(path, "rb").read())
    K, Hd, FS, OS = np.frombuffer(bytes(raw[8:24]), dtype=np.int32)
    off = 24 + 8 * int(K) + 8
    spans = {}
    for name, n in (("fm", FS), ("fsd", FS), ("om", OS), ("osd", OS)):
        spans[name] = (off, int(n))
        off += 4 * int(n)
    for name, fn in arrays.items():
        o, n = spans[name]
        v = np.frombuffer(bytes(raw[o:o + 4 * n]), dtype=np.float32).copy()
        raw[o:o + 4 * n] = fn(v).astype(np.float32).tobytes()
    open(path, "wb").write(bytes(raw))


def test_learned_start_falls_back_to_flat(mase):
    """A proposal that lowers J but leaves one bus at Vm = 0 (its angle column
    of H is then exactly zero, so the factor meets a zero pivot) is solved
    again from the flat start: every snapshot converges to the oracle's
    estimate, and its iteration count includes the failed attempt."""
    import torch
    g = synth.make_grid("grid2869_k16")
    N, S = g.n_bus, 16
    net, Vm, Va, zh, sig = problem(g, S, 4400)
    deg = np.bincount(np.concatenate([g.from_bus, g.to_bus]), minlength=N)
    b = int(np.nonzero((deg >= 3) & (np.arange(N) != g.slack))[0][0])
    mask = np.ones((S, g.n_meas), dtype=np.uint8)
    mask[:, b] = 0                                   # the Vm row of bus b
    for s in range(S):                               # the proposal below is kept
        w = wls.weights(sig, mask[s])
        vp = zh[s, :N].copy()
        vp[b] = 0.0
        assert wls.objective(net, zh[s], w, vp, np.zeros(N)) < \
            wls.objective(net, zh[s], w, np.ones(N), np.zeros(N))
    est = mase.Estimator(g, sig, S, z=torch.tensor(zh, device="cuda"),
                         mask=torch.tensor(mask, device="cuda"), precision=mase.MIXED,
                         schedule=mase.BATCHED)
    xf = np.zeros((S, 2 * N))
    rf = est.solve(tol=1e-8, max_iter=15, x_out=xf)
    assert rf.restarted == 0
    zt = torch.tensor(zh, device="cuda")
    est.warmstart_train(zt, torch.tensor(xf, device="cuda"), epochs=1, batch=8, hidden=64)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ws.bin")
        est.warmstart_save(path)
        # outputs ignore the networks (zero output scale): magnitudes are the
        # measured Vm (the skip row), angles 0; with zero feature means the
        # absent Vm row of bus b reads as 0, so its proposal is Vm = 0
        _edit_model(path, fm=lambda v: v * 0, om=lambda v: v * 0, osd=lambda v: v * 0)
        est.warmstart_load(path)
    xp = np.zeros((S, 2 * N))
    est.warmstart_predict(xp)
    assert np.all(xp[:, b] == 0.0) and np.all(xp[:, N:] == 0.0)
    est.set_start_mode(mase.START_LEARNED)
    xl = np.zeros((S, 2 * N))
    rl = est.solve(tol=1e-8, max_iter=15, x_out=xl)
    assert rl.restarted == S, rl.restarted
    assert np.all(rl.status == 0)
    # the count includes the failed first step; a snapshot that sits at the
    # stopping tolerance may take one step less or more from the flat start
    # on another run (FP32 accumulation order), so the bar allows that step
    assert np.all(rl.iters >= rf.iters), (rl.iters, rf.iters)
    assert np.all(rl.iters >= rf.iters.min() + 1), (rl.iters, rf.iters)
    for s in (0, 9):
        ref = wls.gauss_newton(net, zh[s], wls.weights(sig, mask[s]), tol=1e-8, max_iter=30)
        assert np.max(np.abs(xl[s, :N] - ref.Vm)) <= 1e-6
        assert np.max(np.abs(xl[s, N:] - ref.Va)) <= 1e-6
    est.close()


def test_learned_start_requires_a_model(mase):
    g = synth.make_grid("grid300_k4")
    net, Vm, Va, z, sig = problem(g, 2, 4300)
    est = mase.Estimator(g, sig, 2, z=z)
    est.set_start_mode(mase.START_LEARNED)
    res = est.solve(tol=1e-8, max_iter=10, check=False)
    assert res.rc == mase.MASE_ENOTREADY
    est.close()
