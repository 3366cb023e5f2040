"""Pins of the FP64 MLP oracle: tabulated normal CDF values, central finite
differences, PyTorch CPU autograd in float64 and torch.optim.AdamW."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def _params(dims, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]),
             0.1 * rng.standard_normal(dims[i + 1])) for i in range(len(dims) - 1)]


def test_gelu_tabulated_values():
    # gelu(u) = u * Phi(u); Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457
    np.testing.assert_allclose(mlp.gelu(np.array([0.0, 1.0, -1.0, 8.0, -8.0])),
                               [0.0, 0.841344746068543, -0.158655253931457, 8.0, 0.0],
                               atol=1e-13)
    u = np.linspace(-4, 4, 33)
    fd = (mlp.gelu(u + 1e-6) - mlp.gelu(u - 1e-6)) / 2e-6
    np.testing.assert_allclose(mlp.gelu_grad(u), fd, atol=1e-8)


def test_gradients_match_finite_differences():
    dims = [5, 7, 6, 7, 3]
    P = _params(dims, 1)
    rng = np.random.Generator(np.random.PCG64(2))
    X, Y = rng.standard_normal((4, 5)), rng.standard_normal((4, 3))
    _, grads = mlp.loss_and_grads(P, X, Y)
    eps = 1e-6
    for li, (W, b) in enumerate(P):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _ = mlp.loss_and_grads(P, X, Y)
                flat[idx] = old - eps
                lm, _ = mlp.loss_and_grads(P, X, Y)
                flat[idx] = old
                assert abs((lp - lm) / (2 * eps) - g.reshape(-1)[idx]) < 1e-8


def test_gradients_match_torch_autograd():
    dims = [11, 16, 16, 16, 4]
    P = _params(dims, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    X, Y = rng.standard_normal((9, 11)), rng.standard_normal((9, 4))
    loss, grads = mlp.loss_and_grads(P, X, Y)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in P]
    a = torch.tensor(X)
    for li, (W, b) in enumerate(tp):
        a = a @ W.T + b
        if li + 1 < len(tp):
            a = torch.nn.functional.gelu(a)          # exact erf form
    tl = torch.mean((a - torch.tensor(Y)) ** 2)
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    for (W, b), (gW, gb) in zip(tp, grads):
        np.testing.assert_allclose(W.grad.numpy(), gW, atol=1e-12)
        np.testing.assert_allclose(b.grad.numpy(), gb, atol=1e-12)


def test_adamw_matches_torch():
    rng = np.random.Generator(np.random.PCG64(5))
    p = rng.standard_normal(13)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=3e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 6):
        g = rng.standard_normal(13)
        tp.grad = torch.tensor(g)
        opt.step()
        m, v = mlp.adamw_step(p, g, m, v, t, 3e-3, wd=0.01)
    np.testing.assert_allclose(p, tp.detach().numpy(), atol=1e-14)
