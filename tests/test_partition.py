"""The network partitioner used by the area-count sweep (CPU only): it covers
every bus with K connected areas, is deterministic for a seed, and on grids
with planted areas joined by few tie lines it finds a cut no larger than the
planted one."""
from collections import deque

import numpy as np
import pytest

from paper_2604_23175_gb300 import synth


def _connected(grid, k):
    members = set(np.nonzero(grid.area_of_bus == k)[0].tolist())
    adj = {v: [] for v in members}
    for a, b in zip(grid.from_bus.tolist(), grid.to_bus.tolist()):
        if a in members and b in members:
            adj[a].append(b)
            adj[b].append(a)
    start = next(iter(members))
    seen = {start}
    q = deque([start])
    while q:
        v = q.popleft()
        for u in adj[v]:
            if u not in seen:
                seen.add(u)
                q.append(u)
    return len(seen) == len(members)


@pytest.mark.parametrize("name,K", [("grid2869_k16", 6), ("grid2869_k16", 16), ("grid9241_k32", 2),
                                    ("grid9241_k32", 4), ("grid9241_k32", 24)])
def test_partition_covers_connected_and_deterministic(name, K):
    g = synth.make_grid(name)
    p = synth.partition_network(g, K, seed=3)
    assert p.n_area == K and p.area_of_bus.shape == (g.n_bus,)
    assert set(np.unique(p.area_of_bus).tolist()) == set(range(K))
    assert np.array_equal(p.from_bus, g.from_bus) and np.array_equal(p.r, g.r)
    sizes = np.bincount(p.area_of_bus, minlength=K)
    assert sizes.max() <= 2.0 * g.n_bus / K and sizes.min() >= g.n_bus / (4 * K)
    assert all(_connected(p, k) for k in range(K))
    q = synth.partition_network(g, K, seed=3)
    assert np.array_equal(p.area_of_bus, q.area_of_bus)


@pytest.mark.parametrize("name,factor", [("grid300_k4", 1.0), ("grid2869_k16", 1.5)])
def test_partition_finds_planted_areas(name, factor):
    """Areas drawn as separate trees with chords and joined by 2-6 tie lines
    per adjacent pair: with equal planted sizes, splitting into the planted
    count cuts no more branches than the planted partition does; with planted
    sizes varying 3.4x (80-320 buses), the size-balanced split stays within
    1.5x of the planted cut (a split ignoring the structure cuts ~10x more)."""
    g = synth.make_grid(name)
    p = synth.partition_network(g, g.n_area, seed=1)
    assert synth.cut_branches(p) <= factor * synth.cut_branches(g)
