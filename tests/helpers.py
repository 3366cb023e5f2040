"""Shared test helpers: build oracle inputs from the seeded generator.

Measurements are formed with the oracle's measurement functions, so no test
input or expected value ever comes from the CUDA path."""
from __future__ import annotations

import os

import numpy as np

from oracle import wls
from paper_2604_23175_gb300 import synth


def net_of(grid: synth.Grid) -> wls.Net:
    return wls.Net(grid.n_bus, grid.from_bus.astype(np.int64), grid.to_bus.astype(np.int64),
                   grid.r, grid.x, grid.b_charge, grid.slack)


def problem(grid: synth.Grid, n_snap: int = 1, seed: int = 2000, noise: bool = True,
            walk_len=None):
    """(net, Vm_true[S,N], Va_true[S,N], z[S,m], sigma[m]) for a grid."""
    net = net_of(grid)
    Vm, Va = synth.make_states(grid, n_snap, seed, walk_len=walk_len)
    sig = synth.sigma_vector(grid.n_bus, grid.n_branch)
    e = synth.make_noise(grid, n_snap, seed + 1) if noise else np.zeros((n_snap, grid.n_meas))
    z = np.stack([wls.measure(net, Vm[s], Va[s]) for s in range(n_snap)]) + e
    return net, Vm, Va, z, sig


def tiny_grid(n_bus=10, n_area=3, seed=7, slack_on_boundary=False):
    """A hand-sized partitioned grid (ring + chords), for brute-force checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    # contiguous arcs of the ring; with a zero shift bus 0 (the slack) and bus
    # n-1 sit in different areas, so the slack is a boundary bus
    shift = 0 if slack_on_boundary else n_bus // (2 * n_area)
    area = np.array([((i + shift) * n_area // n_bus) % n_area for i in range(n_bus)],
                    dtype=np.int32)
    edges = [(i, (i + 1) % n_bus) for i in range(n_bus)]
    have = {(min(a, b), max(a, b)) for a, b in edges}
    tries = 0
    while len(edges) < n_bus + n_bus // 3 and tries < 10000:
        tries += 1
        a, b = rng.integers(n_bus, size=2)
        k = (int(min(a, b)), int(max(a, b)))
        if a != b and k not in have and area[a] == area[b]:   # chords stay inside an area
            have.add(k)
            edges.append(k)
    f = np.array([e[0] for e in edges], dtype=np.int32)
    t = np.array([e[1] for e in edges], dtype=np.int32)
    L = len(edges)
    return synth.Grid(n_bus, f, t, rng.uniform(0.002, 0.02, L), rng.uniform(0.02, 0.2, L),
                      rng.uniform(0.0, 0.05, L), area, n_area, 0, "tiny")


def with_parallel_branches(grid: synth.Grid) -> synth.Grid:
    """The grid with two branches doubled by parallel lines of other
    impedance: one inside an area, and one tie line whose copy runs in the
    reverse orientation."""
    area = grid.area_of_bus
    f, t = grid.from_bus, grid.to_bus
    tie = int(np.flatnonzero(area[f] != area[t])[0])
    inner = int(np.flatnonzero(area[f] == area[t])[0])
    extra = np.array([inner, tie])
    f2 = np.r_[f, f[inner], t[tie]].astype(np.int32)
    t2 = np.r_[t, t[inner], f[tie]].astype(np.int32)
    return synth.Grid(grid.n_bus, f2, t2, np.r_[grid.r, 1.3 * grid.r[extra]],
                      np.r_[grid.x, 0.9 * grid.x[extra]], np.r_[grid.b_charge, grid.b_charge[extra]],
                      area, grid.n_area, grid.slack, grid.name + "_parallel")


def _gn_one(args):
    net, z, w, x0, tol, max_iter, keep_steps = args
    N = net.n_bus
    v0 = (None, None) if x0 is None else (x0[:N], x0[N:])
    return wls.gauss_newton(net, z, w, Vm0=v0[0], Va0=v0[1], tol=tol, max_iter=max_iter,
                            keep_steps=keep_steps)


def oracle_gn_many(net, z, w, x0=None, tol=1e-8, max_iter=30, keep_steps=False):
    """The oracle's centralised Gauss-Newton for every snapshot of z [S, m],
    in worker processes started with spawn (safe after CUDA is initialised).
    w is one weight vector or one per snapshot."""
    import multiprocessing as mp
    S = z.shape[0]
    ws = [w if w.ndim == 1 else w[s] for s in range(S)] if hasattr(w, "ndim") else [w] * S
    args = [(net, z[s], ws[s], None if x0 is None else x0[s], tol, max_iter, keep_steps)
            for s in range(S)]
    procs = max(1, min(S, os.cpu_count() or 1, 16))
    if procs == 1:
        return [_gn_one(a) for a in args]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gn_one, args)
