"""Seeded synthetic inputs for multi-area WLS state estimation.

This module draws the *inputs* of the method and nothing else: network
topology and branch parameters, the area partition, true states, Gaussian
noise samples, measurement standard deviations and presence masks.  It holds
none of the method's arithmetic (no admittances, no measurement functions):
measurements ``z = h(x_true) + e`` are formed by whoever consumes these arrays
(the CPU oracle in the tests, the library's own measurement kernel in the
benchmark), so both solvers see identical, independently produced inputs.

Shapes follow the paper's benchmark systems (Sec. 5.1, 5.2): PEGASE-2869 has
2869 buses and 4582 branches, giving 2N-1 states; PEGASE-9241 and ACTIVSg10k
are larger siblings.  The real case files are not available, so graphs are
drawn as follows (one reading per choice, all stated here):

* each area is a random recursive tree (bus t attaches to a uniformly drawn
  earlier bus) plus chords that join bus pairs at tree distance 2..6, which
  keeps grid-like small separators;
* the area graph is a ring plus floor(K/2) extra random area pairs (a plain
  ring when ``extra_pairs`` is 0), with a drawn number of tie lines per
  adjacent pair;
* chords are spread over areas in proportion to area size so that the total
  branch count matches the requested one exactly;
* bus labels and branch order are randomly permuted, except that the slack
  is bus 0 (placed in area 0 and kept off the area boundary unless asked);
* branch r ~ U(0.002, 0.02), x ~ U(0.02, 0.2), total line charging
  b ~ U(0, 0.05) p.u.;
* true state Vm ~ U(0.95, 1.05), Va ~ N(0, 0.1) rad, slack Va = 0; a batch of
  snapshots is a random walk dVa ~ N(0, 0.01), dVm ~ N(0, 0.002) started from
  a fresh draw, and long datasets are many independent walks of a fixed length;
* measurement noise sigma is 0.004 p.u. for voltage magnitudes and 0.01 p.u.
  for power rows.

Canonical measurement row order (m = 3N + 4L):
``Vm[N], Pinj[N], Qinj[N], Pf[L], Qf[L], Pt[L], Qt[L]``
where ``f`` rows are measured at the from end of a branch and ``t`` rows at
its to end.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass, field

import numpy as np

SIGMA_V = 0.004
SIGMA_POWER = 0.01

# measurement families in canonical order
FAMILIES = ("Vm", "Pinj", "Qinj", "Pf", "Qf", "Pt", "Qt")


@dataclass
class Grid:
    n_bus: int
    from_bus: np.ndarray      # int32 [L]
    to_bus: np.ndarray        # int32 [L]
    r: np.ndarray             # float64 [L]
    x: np.ndarray             # float64 [L]
    b_charge: np.ndarray      # float64 [L], total line charging
    area_of_bus: np.ndarray   # int32 [N]
    n_area: int
    slack: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_branch(self) -> int:
        return int(self.from_bus.shape[0])

    @property
    def n_meas(self) -> int:
        return 3 * self.n_bus + 4 * self.n_branch

    @property
    def n_state(self) -> int:
        return 2 * self.n_bus - 1


@dataclass(frozen=True)
class GridSpec:
    name: str
    n_bus: int
    n_branch: int            # total branch count (internal + tie lines)
    n_area: int
    area_lo: int
    area_hi: int
    ties_lo: int
    ties_hi: int
    extra_pairs: bool        # ring + floor(K/2) random extra area pairs
    equal_areas: bool = False
    seed: int = 1000


# Workloads named by what they are (sizes from the paper's benchmark systems).
SPECS = {
    # 300-bus grid, 4 areas of 75 buses in a ring, 3 ties per adjacent pair,
    # mean internal degree 2.7 (101 internal branches per area)
    "grid300_k4": GridSpec("grid300_k4", 300, 4 * 101 + 12, 4, 75, 75, 3, 3,
                           False, equal_areas=True, seed=1000),
    # PEGASE-2869-shaped: 2869 buses, 4582 branches, 16 areas of 80..320
    "grid2869_k16": GridSpec("grid2869_k16", 2869, 4582, 16, 80, 320, 2, 6,
                             True, seed=1001),
    # PEGASE-9241-shaped: 9241 buses, 16049 branches, 32 areas of 150..450
    "grid9241_k32": GridSpec("grid9241_k32", 9241, 16049, 32, 150, 450, 2, 6,
                             True, seed=1002),
    # ACTIVSg10k-shaped: 10000 buses, 12706 branches, 48 areas
    "grid10000_k48": GridSpec("grid10000_k48", 10000, 12706, 48, 104, 313, 2, 6,
                              True, seed=1003),
    # stress: 50000 buses at mean degree 2.7, 128 areas of 200..600
    "grid50000_k128": GridSpec("grid50000_k128", 50000, 67500, 128, 200, 600, 2, 6,
                               True, seed=1004),
}


def _area_sizes(rng, spec: GridSpec) -> np.ndarray:
    K, N = spec.n_area, spec.n_bus
    if spec.equal_areas:
        if N % K:
            raise ValueError("equal areas need n_bus divisible by n_area")
        return np.full(K, N // K, dtype=np.int64)
    if not (K * spec.area_lo <= N <= K * spec.area_hi):
        raise ValueError("area size bounds cannot sum to n_bus")
    raw = rng.uniform(spec.area_lo, spec.area_hi, size=K)
    sizes = np.floor(raw * (N / raw.sum())).astype(np.int64)
    sizes = np.clip(sizes, spec.area_lo, spec.area_hi)
    # hand out the remainder one bus at a time, respecting the bounds
    while sizes.sum() != N:
        d = N - sizes.sum()
        k = int(rng.integers(K))
        if d > 0 and sizes[k] < spec.area_hi:
            sizes[k] += 1
        elif d < 0 and sizes[k] > spec.area_lo:
            sizes[k] -= 1
    return sizes


def _area_pairs(rng, K: int, extra: bool) -> list[tuple[int, int]]:
    if K == 1:
        return []
    pairs = {(min(k, (k + 1) % K), max(k, (k + 1) % K)) for k in range(K)}
    if extra and K > 3:
        want = len(pairs) + K // 2
        while len(pairs) < want:
            a, b = rng.integers(K, size=2)
            if a != b:
                pairs.add((int(min(a, b)), int(max(a, b))))
    return sorted(pairs)


def _tree_and_chords(rng, n: int, n_chords: int) -> list[tuple[int, int]]:
    """Random recursive tree on n local nodes plus chords at tree distance 2..6."""
    edges = []
    adj = [[] for _ in range(n)]
    for t in range(1, n):
        p = int(rng.integers(t))
        edges.append((p, t))
        adj[p].append(t)
        adj[t].append(p)
    have = {(min(a, b), max(a, b)) for a, b in edges}
    added, tries = 0, 0
    while added < n_chords:
        tries += 1
        if tries > 200 * (n_chords + 10):
            raise RuntimeError("could not place chords at tree distance 2..6")
        u = int(rng.integers(n))
        d_want = int(rng.integers(2, 7))
        # BFS on the tree only (chords do not change tree distances)
        dist = {u: 0}
        q = deque([u])
        ring = []
        while q:
            a = q.popleft()
            if dist[a] == d_want:
                ring.append(a)
                continue
            for c in adj[a]:
                if c not in dist:
                    dist[c] = dist[a] + 1
                    q.append(c)
        if not ring:
            continue
        v = ring[int(rng.integers(len(ring)))]
        key = (min(u, v), max(u, v))
        if key in have:
            continue
        have.add(key)
        edges.append(key)
        added += 1
    return edges


def make_grid(spec: GridSpec | str, slack_on_boundary: bool = False,
              seed: int | None = None) -> Grid:
    """Draw a partitioned grid of the given shape (seeded, deterministic)."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    rng = np.random.Generator(np.random.PCG64(spec.seed if seed is None else seed))
    K, N = spec.n_area, spec.n_bus
    sizes = _area_sizes(rng, spec)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    pairs = _area_pairs(rng, K, spec.extra_pairs)
    n_ties = [int(rng.integers(spec.ties_lo, spec.ties_hi + 1)) for _ in pairs]
    tot_ties = int(sum(n_ties))
    n_chords = spec.n_branch - tot_ties - (N - K)
    if n_chords < 0:
        raise ValueError("branch count too small for a spanning forest plus ties")
    # spread chords over areas in proportion to size (largest remainder)
    share = n_chords * sizes / sizes.sum()
    ch = np.floor(share).astype(np.int64)
    rem = n_chords - ch.sum()
    order = np.argsort(-(share - ch), kind="stable")
    ch[order[:rem]] += 1

    # local (area-contiguous) labels first; permuted to global labels below
    f_loc, t_loc = [], []
    for k in range(K):
        for a, b in _tree_and_chords(rng, int(sizes[k]), int(ch[k])):
            f_loc.append(starts[k] + a)
            t_loc.append(starts[k] + b)
    slack_loc = 0  # first bus of area 0
    have = {(min(a, b), max(a, b)) for a, b in zip(f_loc, t_loc)}
    forced_slack_tie = slack_on_boundary
    for (ka, kb), nt in zip(pairs, n_ties):
        placed = 0
        while placed < nt:
            u = int(starts[ka] + rng.integers(sizes[ka]))
            v = int(starts[kb] + rng.integers(sizes[kb]))
            if forced_slack_tie and ka == 0:
                u = slack_loc
            elif u == slack_loc or v == slack_loc:
                continue
            key = (min(u, v), max(u, v))
            if key in have:
                continue
            have.add(key)
            f_loc.append(u)
            t_loc.append(v)
            placed += 1
            if forced_slack_tie and ka == 0:
                forced_slack_tie = False
    f_loc = np.asarray(f_loc, dtype=np.int64)
    t_loc = np.asarray(t_loc, dtype=np.int64)
    L = f_loc.shape[0]
    assert L == spec.n_branch, (L, spec.n_branch)

    # random relabelling of buses (slack -> 0) and of branch order/direction
    perm = np.concatenate([[0], 1 + rng.permutation(N - 1)])  # local -> global
    area_loc = np.repeat(np.arange(K), sizes)
    area_of_bus = np.empty(N, dtype=np.int32)
    area_of_bus[perm] = area_loc
    flip = rng.random(L) < 0.5
    fb = np.where(flip, t_loc, f_loc)
    tb = np.where(flip, f_loc, t_loc)
    border = rng.permutation(L)
    from_bus = perm[fb][border].astype(np.int32)
    to_bus = perm[tb][border].astype(np.int32)
    r = rng.uniform(0.002, 0.02, size=L)
    x = rng.uniform(0.02, 0.2, size=L)
    b = rng.uniform(0.0, 0.05, size=L)
    return Grid(N, from_bus, to_bus, r, x, b, area_of_bus, K, 0, spec.name,
                meta={"n_ties": tot_ties, "n_chords": int(n_chords),
                      "area_sizes": sizes.tolist()})


def sigma_vector(n_bus: int, n_branch: int) -> np.ndarray:
    """Per-row standard deviation in canonical row order."""
    s = np.full(3 * n_bus + 4 * n_branch, SIGMA_POWER)
    s[:n_bus] = SIGMA_V
    return s


def make_states(grid: Grid, n_snap: int, seed: int, walk_len: int | None = None):
    """True states (Vm, Va), each [n_snap][N].

    ``walk_len`` None: one random walk of n_snap steps.  Otherwise independent
    walks of ``walk_len`` steps laid end to end (the last one truncated).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    N = grid.n_bus
    L_walk = n_snap if walk_len is None else walk_len
    Vm = np.empty((n_snap, N))
    Va = np.empty((n_snap, N))
    for s in range(n_snap):
        if s % L_walk == 0:
            Vm[s] = rng.uniform(0.95, 1.05, size=N)
            Va[s] = rng.normal(0.0, 0.1, size=N)
        else:
            Vm[s] = Vm[s - 1] + rng.normal(0.0, 0.002, size=N)
            Va[s] = Va[s - 1] + rng.normal(0.0, 0.01, size=N)
        Va[s, grid.slack] = 0.0
    return Vm, Va


def make_noise(grid: Grid, n_snap: int, seed: int) -> np.ndarray:
    """Gaussian measurement noise e [n_snap][m] with the per-row sigma."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sig = sigma_vector(grid.n_bus, grid.n_branch)
    return rng.standard_normal((n_snap, sig.shape[0])) * sig


def _rows_touching_bus_by_kind(grid: Grid):
    """Rows whose function depends on each bus (structure only), split into
    active-power rows (P injections at the bus and its neighbours, P flows on
    incident branches) and reactive or voltage rows (Vm at the bus, Q
    injections, Q flows)."""
    N, L = grid.n_bus, grid.n_branch
    p_rows = [[N + i] for i in range(N)]
    q_rows = [[i, 2 * N + i] for i in range(N)]
    base = 3 * N
    for l in range(L):
        f, t = int(grid.from_bus[l]), int(grid.to_bus[l])
        pf = [base + l, base + 2 * L + l]
        qf = [base + L + l, base + 3 * L + l]
        p_rows[f] += pf + [N + t]
        p_rows[t] += pf + [N + f]
        q_rows[f] += qf + [2 * N + t]
        q_rows[t] += qf + [2 * N + f]
    return ([np.unique(np.asarray(v, dtype=np.int64)) for v in p_rows],
            [np.unique(np.asarray(v, dtype=np.int64)) for v in q_rows])


def rows_touching_bus(grid: Grid):
    """For each bus, the canonical rows whose function depends on that bus
    (structure only: Vm and injections at the bus and its neighbours, flows on
    incident branches).  Used to keep random masks observable."""
    return [np.union1d(p, q) for p, q in zip(*_rows_touching_bus_by_kind(grid))]


def make_mask(grid: Grid, n_snap: int, drop_frac: float, seed: int,
              min_present: int = 4) -> np.ndarray:
    """Presence mask [n_snap][m] (1 = present) dropping ``drop_frac`` of rows
    per snapshot at random, under two metering rules: every branch keeps at
    least one of its two active-power flow rows and one of its two reactive
    flow rows, and every bus with a single branch keeps its voltage-magnitude
    row.  The draw removes exactly round(drop_frac * m) rows subject to those
    rules (leaf magnitude rows are never drawn; a flow pair drawn whole has
    one row, chosen at random, put back and replaced by a fresh draw).  Then
    every bus keeps at least one present active-power row and one present
    reactive/voltage row touching it, and at least ``min_present`` touching
    rows in all (dropped rows restored at random); this restores a handful of
    rows per snapshot.

    The branch rule keeps both halves of the decoupled problem topologically
    observable (each branch joins its ends through a flow row of each kind).
    Without it, random drops leave, a few times per hundred snapshots of a
    sparse 50000-bus network, a tree leaf whose only branch lost both
    reactive flows: its magnitude is then fixed through the neighbour's
    reactive injection, a quadratic relation with two roots, and Gauss-Newton
    from flat start can walk to the spurious low-voltage root (a stationary
    point far from the true state) even though the network is observable.
    The leaf rule: every power row is unchanged when a bus's magnitude
    changes sign and its angle moves by pi, or its angle by 2 pi, so only
    the magnitude row tells those states apart.  A leaf without it is held by
    its one branch alone, and Gauss-Newton from the flat start was seen to
    wander between such equivalent states for 15-17 steps."""
    import scipy.sparse as sp
    rng = np.random.Generator(np.random.PCG64(seed))
    N, L, m = grid.n_bus, grid.n_branch, grid.n_meas
    base = 3 * N
    partner = np.full(m, -1, dtype=np.int64)
    for a0, b0 in ((base, base + 2 * L), (base + L, base + 3 * L)):
        partner[a0:a0 + L] = b0 + np.arange(L)
        partner[b0:b0 + L] = a0 + np.arange(L)
    deg = np.bincount(np.concatenate([grid.from_bus, grid.to_bus]).astype(np.int64), minlength=N)
    keep = np.zeros(m, dtype=bool)
    keep[np.nonzero(deg == 1)[0]] = True     # magnitude rows of leaves (rows 0..N-1)
    drawable = np.nonzero(~keep)[0]
    first = np.concatenate([base + np.arange(L), base + L + np.arange(L)])
    p_rows, q_rows = _rows_touching_bus_by_kind(grid)
    all_rows = [np.union1d(p, q) for p, q in zip(p_rows, q_rows)]

    def incidence(lists):
        cols = np.concatenate(lists)
        rows = np.repeat(np.arange(N), [len(t) for t in lists])
        return sp.csr_matrix((np.ones(len(cols), dtype=np.int32), (rows, cols)), shape=(N, m))

    checks = [(incidence(p_rows), p_rows, 1), (incidence(q_rows), q_rows, 1),
              (incidence(all_rows), all_rows, min_present)]
    k = int(round(drop_frac * m))
    out = np.ones((n_snap, m), dtype=np.uint8)
    for s in range(n_snap):
        row = np.ones(m, dtype=np.uint8)
        row[rng.choice(drawable, size=k, replace=False)] = 0
        for _ in range(64):
            both = first[(row[first] == 0) & (row[partner[first]] == 0)]
            if len(both) == 0:
                break
            back = np.where(rng.random(len(both)) < 0.5, both, partner[both])
            row[back] = 1
            # a fresh row may be drawn only where its pair partner is present
            free = np.nonzero((row == 1) & ~keep & ((partner < 0) | (row[np.maximum(partner, 0)] == 1)))[0]
            row[rng.choice(free, size=len(back), replace=False)] = 0
        else:
            raise RuntimeError("branch metering rule not met")
        for _ in range(8):
            short = False
            for inc, lists, need in checks:
                cnt = inc @ row.astype(np.int32)
                for b in np.nonzero(cnt < need)[0].tolist():
                    dropped = lists[b][row[lists[b]] == 0]
                    take = min(len(dropped), int(need - cnt[b]))
                    if take > 0:
                        row[rng.choice(dropped, size=take, replace=False)] = 1
                    short = True
            if not short:
                break
        out[s] = row
    return out


def family_mask(grid: Grid, family: str, n_snap: int = 1) -> np.ndarray:
    """Mask that removes one whole measurement family (Sec. 5.4 experiment)."""
    N, L = grid.n_bus, grid.n_branch
    offs = {"Vm": (0, N), "Pinj": (N, N), "Qinj": (2 * N, N),
            "Pf": (3 * N, L), "Qf": (3 * N + L, L), "Pt": (3 * N + 2 * L, L),
            "Qt": (3 * N + 3 * L, L)}
    o, c = offs[family]
    row = np.ones(grid.n_meas, dtype=np.uint8)
    row[o:o + c] = 0
    return np.repeat(row[None, :], n_snap, axis=0)


# ---------------------------------------------------------------------------
# partitioning one fixed network into K areas (the paper's K-sweep, Sec. 5.3,
# re-partitions one network; its "tree partitions" are not specified)
# ---------------------------------------------------------------------------
def _adjacency(n: int, f: np.ndarray, t: np.ndarray) -> list[list[int]]:
    nb = [set() for _ in range(n)]
    for a, b in zip(f.tolist(), t.tolist()):
        nb[a].add(b)
        nb[b].add(a)
    return [sorted(s) for s in nb]


def _bfs_far(start: int, member: set, adj) -> tuple[int, list[int]]:
    """BFS inside ``member`` from ``start``: (last node reached, visit order)."""
    seen = {start}
    order = [start]
    q = deque([start])
    while q:
        a = q.popleft()
        for c in adj[a]:
            if c in member and c not in seen:
                seen.add(c)
                order.append(c)
                q.append(c)
    return order[-1], order


def _fiedler(nodes: list[int], adj) -> np.ndarray:
    """Second eigenvector of the graph Laplacian of the subgraph on ``nodes``
    (shift-invert Lanczos near 0)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    loc = {v: i for i, v in enumerate(nodes)}
    r, c = [], []
    for v in nodes:
        for u in adj[v]:
            if u in loc:
                r.append(loc[v])
                c.append(loc[u])
    n = len(nodes)
    A = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))
    Lap = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    if n < 64:
        w, V = np.linalg.eigh(Lap.toarray())
        return V[:, 1]
    w, V = spla.eigsh(Lap.tocsc(), k=2, sigma=-1e-3, which="LM",
                      v0=np.linspace(1.0, 2.0, n))
    return V[:, np.argsort(w)[1]]


def _bisect(nodes: list[int], target: int, adj, rng, tol: int) -> tuple[list[int], list[int]]:
    """Split ``nodes`` along the Fiedler vector of their subgraph: the sweep
    cut with the fewest cut branches among first-part sizes within ``tol`` of
    ``target``, then greedy boundary moves that cut fewer branches while the
    first part stays within the same window."""
    member = set(nodes)
    f = _fiedler(nodes, adj)
    order = [nodes[i] for i in np.argsort(f, kind="stable")]
    pos = {v: i for i, v in enumerate(order)}
    # cut(prefix of length p) updated incrementally along the sweep
    cut = 0
    best_p, best_cut = target, None
    for p_, v in enumerate(order, start=1):
        for u in adj[v]:
            if u in member:
                cut += 1 if pos[u] >= p_ else -1
        if target - tol <= p_ <= target + tol and (best_cut is None or cut < best_cut):
            best_p, best_cut = p_, cut
    side = {v: (0 if pos[v] < best_p else 1) for v in nodes}
    size0 = best_p
    for _ in range(12):
        moved = 0
        cand = [v for v in nodes if any(c in member and side[c] != side[v] for c in adj[v])]
        rng.shuffle(cand)
        for v in cand:
            sv = side[v]
            ext = sum(1 for c in adj[v] if c in member and side[c] != sv)
            inn = sum(1 for c in adj[v] if c in member and side[c] == sv)
            if ext <= inn:
                continue
            new0 = size0 - 1 if sv == 0 else size0 + 1
            if abs(new0 - target) > tol:
                continue
            side[v] = 1 - sv
            size0 = new0
            moved += 1
        if not moved:
            break
    a = [v for v in nodes if side[v] == 0]
    b = [v for v in nodes if side[v] == 1]
    return a, b


def partition_network(grid: Grid, n_area: int, seed: int = 0, imbalance: float = 0.25) -> Grid:
    """The same network split into ``n_area`` connected areas: recursive
    spectral bisection (sweep cut of the Fiedler vector with the fewest cut
    branches among splits within ``imbalance`` of proportional sizes, then
    greedy boundary moves that cut fewer branches), a K-way pass of the same
    greedy moves, and reassignment of any disconnected piece of an area to
    the neighbouring area it shares most branches with.  Deterministic for a
    seed.  Returns a Grid with the same branches and the new partition."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = grid.n_bus
    adj = _adjacency(N, grid.from_bus, grid.to_bus)
    area = np.empty(N, dtype=np.int64)
    stack = [(list(range(N)), n_area, 0)]
    while stack:
        nodes, k, a0 = stack.pop()
        if k == 1:
            area[nodes] = a0
            continue
        k1 = k // 2
        target = int(round(len(nodes) * k1 / k))
        tol = max(1, int(imbalance * len(nodes) * k1 / k))
        left, right = _bisect(nodes, target, adj, rng, tol)
        stack.append((left, k1, a0))
        stack.append((right, k - k1, a0 + k1))
    # K-way greedy refinement with a size band around N / K
    sizes = np.bincount(area, minlength=n_area)
    lo, hi = (1 - 2 * imbalance) * N / n_area, (1 + 2 * imbalance) * N / n_area
    for _ in range(8):
        moved = 0
        for v in rng.permutation(N).tolist():
            av = area[v]
            cnt = {}
            for c in adj[v]:
                cnt[area[c]] = cnt.get(area[c], 0) + 1
            own = cnt.get(av, 0)
            best, gain = av, 0
            for a, c in cnt.items():
                if a != av and c - own > gain and sizes[a] + 1 <= hi and sizes[av] - 1 >= lo:
                    best, gain = a, c - own
            if best != av:
                area[v] = best
                sizes[av] -= 1
                sizes[best] += 1
                moved += 1
        if not moved:
            break
    # connectivity: pieces other than an area's largest join a neighbouring area
    for _ in range(N):
        changed = False
        for k in range(n_area):
            members = set(np.nonzero(area == k)[0].tolist())
            comps = []
            left = set(members)
            while left:
                s = min(left)
                _, order = _bfs_far(s, left, adj)
                comps.append(order)
                left.difference_update(order)
            if len(comps) <= 1:
                continue
            comps.sort(key=len, reverse=True)
            for comp in comps[1:]:
                cnt = {}
                cs = set(comp)
                for v in comp:
                    for c in adj[v]:
                        if c not in cs:
                            cnt[area[c]] = cnt.get(area[c], 0) + 1
                cnt.pop(k, None)
                if cnt:
                    area[comp] = max(sorted(cnt), key=lambda a: cnt[a])
                    changed = True
        if not changed:
            break
    if len(np.unique(area)) != n_area:
        raise RuntimeError("partition lost an area")
    return Grid(N, grid.from_bus, grid.to_bus, grid.r, grid.x, grid.b_charge, area.astype(np.int32),
                n_area, grid.slack, f"{grid.name}_p{n_area}",
                meta={"partitioned_from": grid.name, "seed": seed})


def cut_branches(grid: Grid) -> int:
    """Number of branches whose terminals lie in different areas."""
    return int(np.sum(grid.area_of_bus[grid.from_bus] != grid.area_of_bus[grid.to_bus]))
