"""Near-ties of the LLF maxima, located on the oracle's side.

Eq. 14 splits each characteristic field with alpha_n = max over the face's
stencil of |lambda_n| at each cell's own state (lambda in {u_d - c, u_d, u_d + c}).
The maximum is not differentiable where two stencil cells tie: the adjoint
passes the derivative of alpha to the first maximal cell. Where the tied
values come from states that differ only in their last bits (the saturated
tanh tails of a shock-bubble interface), the GPU and the oracle, whose sound
speeds agree only to a few ulp, can pick different cells. The derivative then
moves between cells whose states are equal to round-off, so each cell's
adjoint can differ while the sum over the tied cells does not.

``tie_groups`` scans a state for such faces and returns the groups of cells
that can receive a moved derivative: per face and eigenvalue family, the
cells whose |lambda| lies within ``rel`` of the stencil maximum, when there
is more than one such cell, their states are not bitwise equal and the
maximum is not zero (|u| at 0 has derivative 0). Groups that share a cell
are merged.

A second kind of kink sits at |u| = 0: in gas at rest the velocity of a
stage state is round-off (or exactly zero on one side only), so the two
sides can disagree on its sign and on the stencil's arg-max. With
``abs_rel`` given, a face also counts as tied when its maximum lies within
``abs_rel`` of the family's largest |lambda| over the grid of zero, all
stencil cells within that distance of the maximum forming the group (one
cell alone included: its sign is in doubt).

How far a moved derivative reaches is bounded by the stencil's variation:
alpha multiplies half the difference of the two one-sided reconstructions
of the characteristic variable l_n . U over the stencil (Eq. 14-15), which
vanishes with the variation of U there. With ``min_var`` given, ties whose
stencil varies by no more than that (per field, relative to the field's
largest value; the momentum rows share the momentum scale) are left out:
a flip there moves the adjoint by about that fraction of its scale.
"""
import numpy as np

from oracle.xfo import Oracle


def _sound_speed_and_velocity(o, U, T):
    c = o.case
    P, T1, _ = o.cons_to_prim(U, T.copy())
    dim, N = c.dim, c.n_species
    rho, p = P[0], P[1 + dim]
    Y = np.vstack([P[2 + dim:], 1.0 - P[2 + dim:].sum(axis=0)])
    cs = np.empty(c.cells)
    for k in range(c.cells):
        _, cv, cp, _, _ = o.thermo(T1[k], Y[:, k])
        cs[k] = np.sqrt(cp / cv * p[k] / rho[k])
    return P[1:1 + dim], cs


def _padded_map(n, G, bc):
    """Interior index and normal-velocity sign of padded positions -G..n+G-1."""
    idx = np.arange(-G, n + G)
    out = idx.copy()
    sign = np.ones(n + 2 * G)
    lo, hi = bc
    for k, i in enumerate(idx):
        if i < 0:
            side, j = lo, i
            if side == 1:
                out[k] = i % n
            elif side == 0:
                out[k] = 0
            else:
                out[k], sign[k] = -1 - i, -1.0
        elif i >= n:
            side = hi
            if side == 1:
                out[k] = i % n
            elif side == 0:
                out[k] = n - 1
            else:
                out[k], sign[k] = 2 * n - 1 - i, -1.0
    return out, sign


class _DSU:
    def __init__(self):
        self.p = {}

    def find(self, a):
        self.p.setdefault(a, a)
        while self.p[a] != a:
            self.p[a] = self.p[self.p[a]]
            a = self.p[a]
        return a

    def union(self, a, b):
        self.p[self.find(a)] = self.find(b)


def _field_scale(case, U):
    sc = np.max(np.abs(U), axis=1)
    sc[1:1 + case.dim] = np.max(sc[1:1 + case.dim])
    return np.maximum(sc, 1e-300)


def tie_groups(case, U, T, rel=1e-13, weno=5, oracle=None, min_var=0.0, abs_rel=0.0):
    """Groups (sets of flat interior cell indices) of LLF near-ties in state U."""
    o = oracle or Oracle(case)
    G = 4 if weno == 7 else 3
    u, cs = _sound_speed_and_velocity(o, U, T)
    Us = U / _field_scale(case, U)[:, None]
    nz, ny, nx = case.n[2], case.n[1], case.n[0]
    cell = np.arange(case.cells).reshape(nz, ny, nx)
    dsu = _DSU()
    for d in range(case.dim):
        ax = 2 - d
        idx, sign = _padded_map(case.n[d], G, case.bc[d])
        cid = np.moveaxis(cell, ax, -1)[..., idx]
        ud = np.moveaxis(u[d].reshape(nz, ny, nx), ax, -1)[..., idx] * sign
        cc = np.moveaxis(cs.reshape(nz, ny, nx), ax, -1)[..., idx]
        win_c = np.lib.stride_tricks.sliding_window_view(cid, 2 * G, axis=-1)
        for lam in (np.abs(ud - cc), np.abs(ud), np.abs(ud + cc)):
            win = np.lib.stride_tricks.sliding_window_view(lam, 2 * G, axis=-1)
            mx = win.max(axis=-1, keepdims=True)
            floor = abs_rel * lam.max()
            noise = mx[..., 0] <= floor
            near = (mx - win) <= np.maximum(rel * mx, floor)
            cand = ((near.sum(axis=-1) > 1) & (mx[..., 0] > 0.0)) | (noise & (floor > 0.0))
            for pos in zip(*np.nonzero(cand)):
                cells = np.unique(win_c[pos][near[pos]])
                if not noise[pos]:
                    if cells.size < 2:
                        continue
                    Uc = U[:, cells]
                    if np.all(Uc == Uc[:, :1]):
                        continue
                if min_var > 0.0:
                    Uw = Us[:, win_c[pos]]
                    if np.max(Uw.max(axis=1) - Uw.min(axis=1)) <= min_var:
                        continue
                dsu.find(int(cells[0]))
                for a in cells[1:]:
                    dsu.union(int(cells[0]), int(a))
    groups = {}
    for a in list(dsu.p):
        groups.setdefault(dsu.find(a), set()).add(a)
    return list(groups.values())


def dilate(case, cells, radius):
    """Cells within ``radius`` (per axis, periodic axes wrapped, others
    clipped) of any cell in ``cells``: the reach of a change at those cells
    through ``radius`` cells of stencil."""
    nz, ny, nx = case.n[2], case.n[1], case.n[0]
    m = np.zeros((nz, ny, nx), dtype=bool)
    m.reshape(-1)[list(cells)] = True
    for d in range(case.dim):
        ax = 2 - d
        periodic = case.bc[d][0] == 1
        out = m.copy()
        for s in range(1, radius + 1):
            for sh in (s, -s):
                r = np.roll(m, sh, axis=ax)
                if not periodic:
                    sl = [slice(None)] * 3
                    sl[ax] = slice(0, sh) if sh > 0 else slice(sh, None)
                    r[tuple(sl)] = False
                out |= r
        m = out
    return set(np.nonzero(m.reshape(-1))[0].tolist())
