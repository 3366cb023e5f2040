"""Random row-drop masks keep every snapshot observable (CPU, oracle): with
35 % of the rows dropped at random, the oracle's Gauss-Newton converges on
every snapshot within 10 steps (a repair that only counts rows per bus
leaves snapshots that need 14 steps or do not converge in 15), the dropped
fraction stays at its target, no branch loses both flow rows of one kind,
and no leaf bus loses its magnitude row."""
import numpy as np

from oracle import wls
from paper_2604_23175_gb300 import synth
from tests.helpers import problem


def test_masks_keep_snapshots_observable():
    g = synth.make_grid("grid300_k4")
    S = 24
    net, Vm, Va, z, sig = problem(g, S, 6100)
    mask = synth.make_mask(g, S, 0.35, 6101)
    frac = 1.0 - mask.mean(axis=1)
    assert np.all(np.abs(frac - 0.35) < 0.01), frac
    for s in range(S):
        r = wls.gauss_newton(net, z[s], wls.weights(sig, mask[s]), tol=1e-8, max_iter=15)
        assert r.converged and r.iters <= 10, (s, r.iters)


def test_masks_are_deterministic_and_keep_both_row_kinds():
    g = synth.make_grid("grid2869_k16")
    a = synth.make_mask(g, 3, 0.10, 7)
    b = synth.make_mask(g, 3, 0.10, 7)
    assert np.array_equal(a, b)
    p_rows, q_rows = synth._rows_touching_bus_by_kind(g)
    N, L = g.n_bus, g.n_branch
    base = 3 * N
    for s in range(3):
        assert all(a[s][p].any() for p in p_rows)
        assert all(a[s][q].any() for q in q_rows)
        for o in (base, base + L):          # P flows, Q flows: from end | to end
            assert np.all(a[s][o:o + L] | a[s][o + 2 * L:o + 3 * L])
        deg = np.bincount(np.concatenate([g.from_bus, g.to_bus]), minlength=N)
        assert np.all(a[s][:N][deg == 1] == 1)   # leaves keep their magnitude row
        assert abs((1.0 - a[s].mean()) - 0.10) < 2e-4
