"""Edge cases of the CUDA path against the oracle: the smallest grids each
scheme accepts (n = 3 per axis, 4 with WENO7) under every boundary
condition, where the ghost layers wrap or mirror the whole interior; strongly
anisotropic boxes; the smallest and largest species counts; a single-cell
thick slab in 3D. RHS and one RK3 step at the 1e-11 bar."""
import dataclasses

import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import field_err, gpu_rhs, gpu_steps

pytestmark = pytest.mark.gpu

BCS = {"periodic": cases.BC_PERIODIC, "symmetric": cases.BC_SYMMETRIC,
       "transmissive": cases.BC_TRANSMISSIVE}


def _case(dim, n, N, bc, seed=0, viscous=True):
    c = cases.smooth_periodic(dim, n, N, seed=seed, amp=0.3, viscous=viscous)
    b = tuple((bc, bc) if a < dim else (cases.BC_TRANSMISSIVE,) * 2 for a in range(3))
    return dataclasses.replace(c, bc=b)


def _check(case, **kw):
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    R, _, st = o.rhs(U, T.copy())
    Rg, _, stg = gpu_rhs(case, U, T, **kw)
    assert st == stg == 0
    assert np.max(field_err(Rg, R, case.dim)) <= 1e-11
    U1, T1 = U.copy(), T.copy()
    o.step(U1, T1, 0.0)
    Ug, _, stg, _ = gpu_steps(case, U, T, 1, **kw)
    assert stg == 0
    assert np.max(field_err(Ug, U1, case.dim)) <= 1e-11


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("weno", [5, 6, 7])
def test_smallest_grid(dim, bc, weno):
    n0 = 4 if weno == 7 else 3
    _check(_case(dim, (n0,) * dim, 3, BCS[bc], seed=dim), weno=weno)


@pytest.mark.parametrize("n", [(3, 64), (64, 3), (61, 3, 5), (3, 5, 33), (40, 12, 1 + 2)])
def test_anisotropic_boxes(n):
    _check(_case(len(n), n, 3, cases.BC_PERIODIC, seed=len(n) + 7))


@pytest.mark.parametrize("N", [2, 5])
def test_species_count_extremes_3d(N):
    _check(_case(3, (11, 9, 7), N, cases.BC_SYMMETRIC, seed=N))


def test_inviscid_smallest_3d():
    _check(_case(3, (3, 3, 3), 4, cases.BC_PERIODIC, seed=4, viscous=False))
