"""FP64 oracle: WLS state estimation by Gauss-Newton, centralised and
multi-area (Schur condensation).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain, slow, readable
NumPy/SciPy in float64; no blocking, fusion or reordering beyond what the
equations state.

Model (Sec. 2.1).  State x = (Vm[0..N), Va[0..N)) with the slack angle held
fixed, so n = 2N - 1 unknowns (Sec. 5.2: 5737 states for 2869 buses).
Measurements z = h(x) + e (Eq. meas_model) in the canonical row order
``Vm[N], Pinj[N], Qinj[N], Pf[L], Qf[L], Pt[L], Qt[L]`` (m = 3N + 4L, the full
set whose flow families each hold 4582 of 26935 rows for PEGASE-2869,
Sec. 5.4).  WLS objective J = r^T W r, r = z - h(x), W = diag(w) (Eq. wls);
masked rows carry w = 0 (Sec. 4.1).  Gauss-Newton: G dx = H^T W r,
G = H^T W H (Eq. gn_normal).

Branch model: pi equivalent with series admittance y = 1/(r + jx) = g + jb
and half the total line charging b_c/2 at each end; no taps, no bus shunts.
Injections are positive into the network at the bus.

Readings of points the paper leaves open (each also listed in the design
notes): convergence is max|dx|_inf < tol per snapshot with the last step
applied; flow rows belong to the area of the bus at which they are measured,
bus rows to the bus's area; the slack angle is fixed and removed from every
block, including x_Gamma when the slack is a boundary bus.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class Net:
    """Plain network description (0-based bus indices)."""
    n_bus: int
    from_bus: np.ndarray
    to_bus: np.ndarray
    r: np.ndarray
    x: np.ndarray
    b_charge: np.ndarray
    slack: int = 0

    @property
    def n_branch(self) -> int:
        return int(len(self.from_bus))

    @property
    def n_meas(self) -> int:
        return 3 * self.n_bus + 4 * self.n_branch


def series_admittance(net: Net):
    """g + jb = 1 / (r + jx) per branch."""
    den = net.r ** 2 + net.x ** 2
    return net.r / den, -net.x / den


# ----------------------------------------------------------------------------
# measurement functions h_tau(x; p_i)   (Sec. 2.2, Eq. typed_meas)
# ----------------------------------------------------------------------------

def _end_flow(Vi, Vj, ti, tj, g, b, bh):
    """P and Q leaving bus i into a branch towards j (pi model)."""
    c, s = np.cos(ti - tj), np.sin(ti - tj)
    P = Vi * Vi * g - Vi * Vj * (g * c + b * s)
    Q = -Vi * Vi * (b + bh) - Vi * Vj * (g * s - b * c)
    return P, Q


def branch_flows(net: Net, Vm, Va):
    """(Pf, Qf, Pt, Qt): flows at the from end and at the to end of each branch."""
    g, b = series_admittance(net)
    bh = 0.5 * net.b_charge
    f, t = net.from_bus, net.to_bus
    Pf, Qf = _end_flow(Vm[f], Vm[t], Va[f], Va[t], g, b, bh)
    Pt, Qt = _end_flow(Vm[t], Vm[f], Va[t], Va[f], g, b, bh)
    return Pf, Qf, Pt, Qt


def measure(net: Net, Vm, Va):
    """h(x) in canonical row order (one snapshot)."""
    N = net.n_bus
    Pf, Qf, Pt, Qt = branch_flows(net, Vm, Va)
    Pinj = np.zeros(N)
    Qinj = np.zeros(N)
    np.add.at(Pinj, net.from_bus, Pf)
    np.add.at(Pinj, net.to_bus, Pt)
    np.add.at(Qinj, net.from_bus, Qf)
    np.add.at(Qinj, net.to_bus, Qt)
    return np.concatenate([Vm, Pinj, Qinj, Pf, Qf, Pt, Qt])


# ----------------------------------------------------------------------------
# analytic Jacobian H = dh/dx  (Eq. gn_normal), columns Vm[0..N), Va[0..N)
# ----------------------------------------------------------------------------

def _end_partials(Vi, Vj, ti, tj, g, b, bh):
    """Partials of (P_ij, Q_ij) w.r.t. (Vi, Vj, ti, tj)."""
    c, s = np.cos(ti - tj), np.sin(ti - tj)
    gc_bs = g * c + b * s
    gs_bc = g * s - b * c
    dP = (2 * Vi * g - Vj * gc_bs, -Vi * gc_bs, Vi * Vj * gs_bc, -Vi * Vj * gs_bc)
    dQ = (-2 * Vi * (b + bh) - Vj * gs_bc, -Vi * gs_bc, -Vi * Vj * gc_bs, Vi * Vj * gc_bs)
    return dP, dQ


def jacobian_full(net: Net, Vm, Va) -> sp.csr_matrix:
    """m x 2N Jacobian including the slack-angle column."""
    N, L = net.n_bus, net.n_branch
    g, b = series_admittance(net)
    bh = 0.5 * net.b_charge
    f, t = net.from_bus, net.to_bus
    rows, cols, vals = [], [], []

    def put(r, c, v):
        rows.append(np.asarray(r))
        cols.append(np.asarray(c))
        vals.append(np.asarray(v, dtype=float))

    ar = np.arange(N)
    put(ar, ar, np.ones(N))                                    # Vm rows
    offs = {"Pf": 3 * N, "Qf": 3 * N + L, "Pt": 3 * N + 2 * L, "Qt": 3 * N + 3 * L}
    lb = np.arange(L)
    for end in ("f", "t"):
        i, j = (f, t) if end == "f" else (t, f)
        dP, dQ = _end_partials(Vm[i], Vm[j], Va[i], Va[j], g, b, bh)
        for fam, d in (("P", dP), ("Q", dQ)):
            row_flow = offs[fam + end] + lb
            row_inj = (N if fam == "P" else 2 * N) + i        # injection at bus i
            for row in (row_flow, row_inj):
                put(row, i, d[0])
                put(row, j, d[1])
                put(row, N + i, d[2])
                put(row, N + j, d[3])
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * N + 4 * L, 2 * N))
    return H.tocsr()          # duplicates (injection terms) are summed


def state_columns(net: Net) -> np.ndarray:
    """Columns of the full Jacobian that are unknowns (slack angle removed)."""
    keep = np.ones(2 * net.n_bus, dtype=bool)
    keep[net.n_bus + net.slack] = False
    return np.nonzero(keep)[0]


def jacobian(net: Net, Vm, Va) -> sp.csr_matrix:
    """m x n Jacobian H over the unknowns."""
    return jacobian_full(net, Vm, Va)[:, state_columns(net)].tocsr()


def weights(sigma, mask=None):
    """W = R^{-1} = diag(1/sigma^2); masked rows get weight 0 (Sec. 4.1)."""
    w = 1.0 / np.asarray(sigma, dtype=float) ** 2
    if mask is not None:
        w = w * (np.asarray(mask) != 0)
    return w


def objective(net: Net, z, w, Vm, Va) -> float:
    """J = r^T W r (Eq. wls).  The paper prints 0.5 * r^T W r as its objective."""
    r = z - measure(net, Vm, Va)
    return float(r @ (w * r))


# ----------------------------------------------------------------------------
# centralised Gauss-Newton   (Eq. gn_normal)
# ----------------------------------------------------------------------------

@dataclass
class GNResult:
    Vm: np.ndarray
    Va: np.ndarray
    iters: int
    converged: bool
    J: float
    steps: list


def flat_start(net: Net):
    return np.ones(net.n_bus), np.zeros(net.n_bus)


def _apply_step(net: Net, Vm, Va, dx):
    cols = state_columns(net)
    full = np.zeros(2 * net.n_bus)
    full[cols] = dx
    return Vm + full[:net.n_bus], Va + full[net.n_bus:]


def gauss_newton(net: Net, z, w, Vm0=None, Va0=None, tol=1e-8, max_iter=10,
                 keep_steps=False) -> GNResult:
    """Centralised WLS Gauss-Newton for one snapshot.

    Each iteration forms G = H^T W H and H^T W r and solves G dx = H^T W r with
    a sparse direct solver; x <- x + dx; stops once max|dx| < tol (the step
    that met the test is applied) or after max_iter steps.
    """
    Vm, Va = flat_start(net) if Vm0 is None else (np.array(Vm0, float), np.array(Va0, float))
    steps = []
    W = sp.diags(w)
    for it in range(1, max_iter + 1):
        r = z - measure(net, Vm, Va)
        H = jacobian(net, Vm, Va)
        G = (H.T @ W @ H).tocsc()
        rhs = H.T @ (w * r)
        dx = spla.spsolve(G, rhs)
        Vm, Va = _apply_step(net, Vm, Va, dx)
        if keep_steps:
            steps.append(dx)
        if np.max(np.abs(dx)) < tol:
            return GNResult(Vm, Va, it, True, objective(net, z, w, Vm, Va), steps)
    return GNResult(Vm, Va, max_iter, False, objective(net, z, w, Vm, Va), steps)


# ----------------------------------------------------------------------------
# multi-area decomposition   (Sec. 2.3, Sec. 3)
# ----------------------------------------------------------------------------

@dataclass
class Partition:
    """Boundary sets and selectors of a K-area partition."""
    n_area: int
    area_of_bus: np.ndarray
    boundary_buses: np.ndarray          # ascending global bus ids
    gamma_cols: np.ndarray              # x_Gamma -> column of the unknown vector
    rows: list                          # per area: canonical rows it owns
    internal_cols: list                 # per area: unknown columns x_i^k
    boundary_cols: list                 # per area: unknown columns x_b^k
    E: list                             # per area: E_k as index array into x_Gamma


def variable_columns(net: Net, buses) -> np.ndarray:
    """Unknown-vector columns of the (Vm, Va) of the given buses, Vm then Va
    per bus, slack angle omitted."""
    N = net.n_bus
    col_of = -np.ones(2 * N, dtype=np.int64)
    col_of[state_columns(net)] = np.arange(2 * N - 1)
    out = []
    for bus in buses:
        out.append(col_of[bus])
        if bus != net.slack:
            out.append(col_of[N + bus])
    return np.asarray(out, dtype=np.int64)


def partition(net: Net, area_of_bus, n_area: int) -> Partition:
    """Boundary buses are the terminals of cut branches (Sec. 2.3).

    Area k keeps its own buses; its local boundary set is its own boundary
    buses together with the far terminals of its tie lines, the overlap that
    lets every row it owns be evaluated locally.  Bus rows belong to the
    bus's area, a flow row to the area of the bus at which it is measured.
    """
    A = np.asarray(area_of_bus)
    N, L = net.n_bus, net.n_branch
    f, t = net.from_bus, net.to_bus
    cut = A[f] != A[t]
    is_bnd = np.zeros(N, dtype=bool)
    is_bnd[f[cut]] = True
    is_bnd[t[cut]] = True
    bbus = np.nonzero(is_bnd)[0]
    gamma_cols = variable_columns(net, bbus)
    pos_in_gamma = {int(c): k for k, c in enumerate(gamma_cols)}
    rows, icols, bcols, E = [], [], [], []
    for k in range(n_area):
        own = np.nonzero(A == k)[0]
        far = set(t[cut & (A[f] == k)].tolist()) | set(f[cut & (A[t] == k)].tolist())
        own_b = [b for b in own if is_bnd[b]]
        loc_b = sorted(set(own_b) | far)
        intern = [b for b in own if not is_bnd[b]]
        icols.append(variable_columns(net, intern))
        bc = variable_columns(net, loc_b)
        bcols.append(bc)
        E.append(np.asarray([pos_in_gamma[int(c)] for c in bc], dtype=np.int64))
        lb = np.arange(L)
        rr = [own, N + own, 2 * N + own,
              3 * N + lb[A[f] == k], 3 * N + L + lb[A[f] == k],
              3 * N + 2 * L + lb[A[t] == k], 3 * N + 3 * L + lb[A[t] == k]]
        rows.append(np.sort(np.concatenate(rr)))
    return Partition(n_area, A, bbus, gamma_cols, rows, icols, bcols, E)


@dataclass
class AreaBlocks:
    Gii: np.ndarray
    Gib: np.ndarray
    Gbb: np.ndarray
    bi: np.ndarray
    bb: np.ndarray


def area_blocks(H: sp.csr_matrix, w, r, part: Partition, k: int) -> AreaBlocks:
    """Local normal-equation blocks of area k (Eq. block_normal):
    G_ii = Hi^T W Hi, G_ib = Hi^T W Hb, G_bb = Hb^T W Hb, b = H_k^T W r."""
    rows = part.rows[k]
    Hk = H[rows]
    Hi = Hk[:, part.internal_cols[k]].toarray()
    Hb = Hk[:, part.boundary_cols[k]].toarray()
    wk, rk = w[rows], r[rows]
    return AreaBlocks(Hi.T @ (wk[:, None] * Hi), Hi.T @ (wk[:, None] * Hb),
                      Hb.T @ (wk[:, None] * Hb), Hi.T @ (wk * rk), Hb.T @ (wk * rk))


def schur_condense(blk: AreaBlocks):
    """S_b = G_bb - G_bi G_ii^{-1} G_ib and b_hat = b_b - G_bi G_ii^{-1} b_i
    (Eq. schur_defs), via a Cholesky factor of G_ii."""
    if blk.Gii.shape[0] == 0:
        return blk.Gbb.copy(), blk.bb.copy()
    Lc = np.linalg.cholesky(blk.Gii)
    Y = np.linalg.solve(Lc, blk.Gib)           # L^{-1} G_ib
    c = np.linalg.solve(Lc, blk.bi)            # L^{-1} b_i
    return blk.Gbb - Y.T @ Y, blk.bb - Y.T @ c


def multi_area_step(net: Net, part: Partition, z, w, Vm, Va, return_parts=False):
    """One boundary-condensed Gauss-Newton step (Sec. 3).

    Per area: blocks (Eq. block_normal), condensation (Eq. schur_defs);
    coordinator: S_Gamma = sum_k E_k^T S_b^k E_k, b_Gamma likewise
    (Eq. global_assembly), Cholesky solve; scatter dx_b^k = E_k dx_Gamma
    (Eq. Ek_select); interior recovery by Eq. backsub.
    """
    r = z - measure(net, Vm, Va)
    H = jacobian(net, Vm, Va)
    nG = len(part.gamma_cols)
    S_G = np.zeros((nG, nG))
    b_G = np.zeros(nG)
    blocks, conds = [], []
    for k in range(part.n_area):
        blk = area_blocks(H, w, r, part, k)
        Sb, bh = schur_condense(blk)
        Ek = part.E[k]
        S_G[np.ix_(Ek, Ek)] += Sb
        np.add.at(b_G, Ek, bh)
        blocks.append(blk)
        conds.append((Sb, bh))
    LG = np.linalg.cholesky(S_G)
    dxG = np.linalg.solve(LG.T, np.linalg.solve(LG, b_G))
    dx = np.zeros(2 * net.n_bus - 1)
    dx[part.gamma_cols] = dxG
    for k in range(part.n_area):
        blk = blocks[k]
        dxb = dxG[part.E[k]]
        if blk.Gii.shape[0]:
            dxi = np.linalg.solve(blk.Gii, blk.bi - blk.Gib @ dxb)
            dx[part.internal_cols[k]] = dxi
    if return_parts:
        return dx, dict(S_G=S_G, b_G=b_G, blocks=blocks, conds=conds, H=H, r=r)
    return dx


def multi_area_gauss_newton(net: Net, part: Partition, z, w, Vm0=None, Va0=None,
                            tol=1e-8, max_iter=10, keep_steps=False) -> GNResult:
    """Gauss-Newton whose every step is the boundary-condensed step."""
    Vm, Va = flat_start(net) if Vm0 is None else (np.array(Vm0, float), np.array(Va0, float))
    steps = []
    for it in range(1, max_iter + 1):
        dx = multi_area_step(net, part, z, w, Vm, Va)
        Vm, Va = _apply_step(net, Vm, Va, dx)
        if keep_steps:
            steps.append(dx)
        if np.max(np.abs(dx)) < tol:
            return GNResult(Vm, Va, it, True, objective(net, z, w, Vm, Va), steps)
    return GNResult(Vm, Va, max_iter, False, objective(net, z, w, Vm, Va), steps)


def gain_and_gradient(net: Net, z, w, Vm, Va):
    """Centralised G = H^T W H (dense) and H^T W r, for small checks."""
    H = jacobian(net, Vm, Va)
    r = z - measure(net, Vm, Va)
    Hd = H.toarray()
    return Hd.T @ (w[:, None] * Hd), Hd.T @ (w * r)
