"""Every element of the oracle's vector-Jacobian products, built from its
exact forward-mode derivatives (dual numbers), for element-wise comparison
with the hand-written adjoint.

Ubar = J^T W has the elements Ubar[v, q] = sum_i W_i (J e_{v,q})_i. The
right-hand side at a cell depends only on cells at most REACH cells away
along each axis (the WENO5 faces of a cell read cells i-3..i+3; the viscous
faces read two cells on each side and the nodal gradients two more across,
which stays inside that box), so J e_{v,q} vanishes outside the box of
radius REACH around q. Unit perturbations of one field at cells that lie at
least 2 REACH + 1 apart along every axis (one colour class) therefore have
disjoint footprints: one JVP direction carries all of them, and the sum of
W (J e) over the box around q recovers Ubar[v, q] alone. For one RK3 step the
same holds with the reach of three stages. Periodic axes whose length is
not a multiple of the spacing are not compressed.
"""
import numpy as np

from oracle.xfo import KDIR

REACH = 3


def _spacing(case, reach):
    s = []
    for d in range(3):
        n = case.n[d]
        if d >= case.dim:
            s.append(1)
            continue
        sp = 2 * reach + 1
        periodic = case.bc[d][0] == 1
        if sp >= n or (periodic and n % sp != 0):
            # try the next spacings that divide n, else no compression
            cand = [k for k in range(sp, n) if n % k == 0] if periodic else []
            sp = cand[0] if cand else n
        s.append(sp)
    return s


def box_sum(case, a, reach):
    """Per cell q: the sum of the per-cell array ``a`` over the box of radius
    ``reach`` around q (periodic axes wrapped, the others clipped)."""
    nx, ny, nz = case.n
    x = np.asarray(a, dtype=np.float64).reshape(nz, ny, nx)
    for d in range(case.dim):
        ax = 2 - d
        periodic = case.bc[d][0] == 1
        out = np.zeros_like(x)
        lo, hi = -reach, reach
        if periodic and 2 * reach + 1 > case.n[d]:
            lo, hi = 0, case.n[d] - 1      # the box wraps round: every cell once
        for sh in range(lo, hi + 1):
            r = np.roll(x, sh, axis=ax)
            if not periodic and sh != 0:
                sl = [slice(None)] * 3
                sl[ax] = slice(0, sh) if sh > 0 else slice(sh, None)
                r[tuple(sl)] = 0.0
            out += r
        x = out
    return x.reshape(-1)


def _colours(case, cells, spacing):
    nx, ny, nz = case.n
    k, j, i = np.unravel_index(np.asarray(cells), (nz, ny, nx))
    return (i % spacing[0]) * spacing[1] * spacing[2] + (j % spacing[1]) * spacing[2] + (k % spacing[2])


def vjp(case, W, jvp, cells=None, reach=REACH):
    """Ubar[v, q] for every field v and every cell q in ``cells`` (default:
    all), from ``jvp(V) -> J V`` ([k, n_v, cells] -> same) over batches of
    at most KDIR directions."""
    nv, ncell = case.n_v, case.cells
    cells = np.arange(ncell) if cells is None else np.asarray(cells)
    spacing = _spacing(case, reach)
    col = _colours(case, cells, spacing)
    dirs = [(v, c) for v in range(nv) for c in np.unique(col)]
    Ubar = np.full((nv, ncell), np.nan)
    for b0 in range(0, len(dirs), KDIR):
        batch = dirs[b0:b0 + KDIR]
        V = np.zeros((len(batch), nv, ncell))
        for k, (v, c) in enumerate(batch):
            V[k, v, cells[col == c]] = 1.0
        JV = jvp(V)
        for k, (v, c) in enumerate(batch):
            s = np.sum(W * JV[k], axis=0)
            q = cells[col == c]
            Ubar[v, q] = box_sum(case, s, reach)[q]
    return Ubar


def reach_of(o):
    """Stencil reach of the oracle's right-hand side: one cell more for
    WENO7's eight-cell faces."""
    return REACH + (1 if o.p.weno == 7 else 0)


def rhs_vjp(o, U, T, W, cells=None):
    """Every element of (dL/dU)^T W of the oracle's right-hand side."""
    def jvp(V):
        return o.rhs_jvp(U, V, T.copy())[1]
    return vjp(o.case, W, jvp, cells, reach=reach_of(o))


def step_vjp(o, U, T, dt, W, cells=None):
    """Every element of (dU^{n+1}/dU^n)^T W of one fixed-dt SSP-RK3 step."""
    def jvp(V):
        return o.rk3_jvp(U, V, T.copy(), dt, 1)[1]
    return vjp(o.case, W, jvp, cells, reach=3 * reach_of(o))
