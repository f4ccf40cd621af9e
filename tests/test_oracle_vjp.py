"""The compressed construction of the oracle's full vector-Jacobian products
(tests/oracle_vjp.py) against one JVP per unit direction, and the stencil
reach it relies on. These products are what the element-wise adjoint tests
compare the CUDA adjoint with; they use the oracle alone."""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

import oracle_vjp as ov

CASES = {
    "sbi2d_n4_64x32": (lambda: cases.shock_bubble(2, (64, 32), 4, 1.5, 0.2, seed=0), {}),
    "smooth2d_n3_periodic": (lambda: cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3), {}),
    "sbi3d_n5": (lambda: cases.config(2, n=(12, 8, 8)), {}),
    "tube1d_n2": (lambda: cases.shock_tube(0, n=64), {}),
    "sbi2d_n4_weno7": (lambda: cases.config(4, n=(24, 14)), {"weno": 7}),
}


def _sample_cells(case, rng, k=6):
    corners = [0, case.cells - 1, case.n[0] - 1]
    return np.unique(np.concatenate([corners, rng.integers(0, case.cells, size=k)]))


def _direct(o, U, T, W, q, step_dt=None):
    nv = o.case.n_v
    out = np.zeros(nv)
    for v0 in range(0, nv, 8):
        vs = list(range(v0, min(nv, v0 + 8)))
        V = np.zeros((len(vs), nv, o.case.cells))
        for k, v in enumerate(vs):
            V[k, v, q] = 1.0
        if step_dt is None:
            JV = o.rhs_jvp(U, V, T.copy())[1]
        else:
            JV = o.rk3_jvp(U, V, T.copy(), step_dt, 1)[1]
        for k, v in enumerate(vs):
            out[v] = np.sum(W * JV[k])
    return out, JV


@pytest.mark.parametrize("name", list(CASES))
def test_compressed_rhs_vjp_equals_unit_directions(name):
    make, kw = CASES[name]
    case = make()
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    rng = np.random.default_rng(3)
    W = rng.normal(size=U.shape)
    Ub = ov.rhs_vjp(o, U, T, W)
    scale = np.max(np.abs(Ub), axis=1)
    reach = ov.reach_of(o)
    nx, ny, nz = case.n
    for q in _sample_cells(case, rng):
        d, JV = _direct(o, U, T, W, q)
        assert np.all(np.abs(d - Ub[:, q]) <= 1e-13 * scale)
        # the footprint stays inside the box of the stencil reach (periodic
        # axes measured the short way round)
        sup = np.nonzero(np.any(JV != 0.0, axis=(0, 1)))[0]
        kq, jq, iq = np.unravel_index(q, (nz, ny, nx))
        ks, js, is_ = np.unravel_index(sup, (nz, ny, nx))
        for a, (cq, cs) in enumerate(((iq, is_), (jq, js), (kq, ks))):
            dist = np.abs(cs - cq)
            if case.bc[a][0] == 1:
                dist = np.minimum(dist, case.n[a] - dist)
            assert dist.max(initial=0) <= reach


def test_compressed_step_vjp_equals_unit_directions():
    case = cases.shock_bubble(2, (64, 32), 4, 1.5, 0.2, seed=0)
    o = Oracle(case)
    U, T = o.prim_to_cons()
    dt = 0.9 * o.dt(U, T.copy())
    rng = np.random.default_rng(4)
    W = rng.normal(size=U.shape)
    patch = np.array([j * 64 + i for j in range(0, 4) for i in range(6, 14)])
    Ub = ov.step_vjp(o, U, T, dt, W, cells=patch)
    scale = np.nanmax(np.abs(Ub), axis=1)
    for q in patch[[0, 5, 17, 31]]:
        d, _ = _direct(o, U, T, W, q, step_dt=dt)
        assert np.all(np.abs(d - Ub[:, q]) <= 1e-13 * scale)
