"""The hand-written adjoint against every element of the oracle's exact
vector-Jacobian product (dual-number JVPs, tests/oracle_vjp.py), per field at
1e-10 of the field's largest adjoint value.

RHS (xf_rhs_adjoint): every cell of the grid. One RK3 step
(xf_step_rk3_adjoint and the taped xf_step_rk3_adjoint_tape): a 16 x 8 patch
of the 64 x 32 differentiated shock-bubble case (shock, bubble and symmetry
plane inside it), or every cell of the small cases.

Kinks of the LLF maxima (Eq. 14): where the stencil maximum of |lambda| is
shared by cells whose states differ only in their last bits (the saturated
tanh tails of the bubble interface ahead of the shock), the GPU and the
oracle may hand alpha's derivative to different cells of the tie
(tests/llf_ties.py locates them on the oracle's side). For the RHS such cells
are compared as groups: the sum of the adjoint over each group of tied cells
must match at 1e-10, and every other cell matches on its own.

A step adds the kink of |u| at 0: after the first stage the gas at rest holds
velocities of round-off size (or exactly zero on one side), whose signs the
two sides need not share. On the unperturbed shock-bubble state that reaches
every cell of the patch (the bubble sits in gas at rest), so there the test
checks that every element above 1e-10 lies within the reach of such a kink
or tie and reports how many do. A perturbed shock-bubble state (a smooth
seeded 1e-3 perturbation of density, velocity and pressure, which leaves no
tie and no gas at rest at any stage, asserted) is compared on every cell of
the patch at 1e-10.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

import llf_ties
import oracle_vjp
from gpu_util import dev, gpu_solver

pytestmark = pytest.mark.gpu

TOL = 1e-10
MIN_VAR = 1e-13   # ties on stencils flatter than this move the adjoint by less than TOL
N_SBI, MA, RADIUS = (64, 32), 1.5, 0.2


def perturbed(case):
    return cases.with_smooth_perturbation(case, seed=0, amp=1e-3)


def _sbi64():
    return cases.shock_bubble(2, N_SBI, 4, MA, RADIUS, seed=0, name="sbi2d_n4_64x32")


RHS_CASES = {
    "sbi2d_n4_64x32": (_sbi64, {}),
    "sbi2d_n4_64x32_perturbed": (lambda: perturbed(_sbi64()), {}),
    "sbi2d_n3_visc": (lambda: cases.config(1, n=(20, 12)), {}),
    "sbi3d_n5_visc": (lambda: cases.config(2, n=(12, 8, 8)), {}),
    "tube1d_n2": (lambda: cases.shock_tube(0, n=64), {}),
    "smooth2d_n3_periodic": (lambda: cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3), {}),
    "smooth1d_n4_inviscid": (lambda: cases.smooth_periodic(1, (40,), 4, seed=2, amp=0.3,
                                                           viscous=False), {}),
    "sbi2d_n4_cu6": (lambda: cases.config(4, n=(24, 14)), {"weno": 6}),
    "sbi2d_n4_weno7": (lambda: cases.config(4, n=(24, 14)), {"weno": 7}),
    "sbi2d_n4_dsm": (lambda: cases.with_binary_diffusion(cases.config(4, n=(24, 14)), seed=1),
                     {"diffusion": 1}),
    # two species: the Wilke and D_sm sums over a single pair
    "smooth2d_n2_periodic_visc": (lambda: cases.smooth_periodic(2, (14, 12), 2, seed=9, amp=0.3),
                                  {}),
    "smooth2d_n2_periodic_dsm": (lambda: cases.with_binary_diffusion(
        cases.smooth_periodic(2, (14, 12), 2, seed=11, amp=0.3), seed=4), {"diffusion": 1}),
}


def _scale(Ub):
    return np.maximum(np.nanmax(np.abs(Ub), axis=1), 1e-300)


def compare(Ub_gpu, Ub_or, cells, groups=(), skip=()):
    """Per-field max error over ``cells`` outside the tie groups and ``skip``
    (each cell on its own), and over the tie groups (sums over each group);
    both relative to the field's largest oracle value."""
    scale = _scale(Ub_or[:, cells])
    flagged = set().union(*groups) if groups else set()
    alone = np.array([q for q in cells if q not in flagged and q not in skip], dtype=int)
    diff = Ub_gpu - Ub_or
    err_alone = np.max(np.abs(diff[:, alone]), axis=1) / scale if alone.size else np.zeros(1)
    err_groups = np.zeros(1)
    for g in groups:
        g = np.array(sorted(g))
        err_groups = np.maximum(err_groups, np.abs(diff[:, g].sum(axis=1)) / scale)
    err_cells_in_groups = (np.max(np.abs(diff[:, sorted(flagged)]), axis=1) / scale
                           if flagged else np.zeros(1))
    return err_alone, err_groups, err_cells_in_groups


@pytest.mark.parametrize("name", list(RHS_CASES))
def test_rhs_adjoint_elementwise(name):
    import torch
    make, kw = RHS_CASES[name]
    case = make()
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    rng = np.random.default_rng(31)
    W = rng.normal(size=U.shape)
    cells = np.arange(case.cells)
    if case.dim == 3:
        cells = cells[cells < 3 * case.n[0] * case.n[1]]   # the three lowest z planes
    Ub_or = oracle_vjp.rhs_vjp(o, U, T, W, cells=cells)
    groups = llf_ties.tie_groups(case, U, T, 1e-13, weno=kw.get("weno", 5), oracle=o,
                                 min_var=MIN_VAR)
    groups = [g for g in groups if g & set(cells.tolist())]
    s = gpu_solver(case, **kw)
    s.set_state(dev(U), dev(T))
    Ub = torch.zeros((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.rhs_adjoint(dev(U), dev(W), Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    # groups reaching beyond the compared cells cannot be summed whole
    whole = [g for g in groups if g <= set(cells.tolist())]
    partial = set().union(*[g for g in groups if not g <= set(cells.tolist())]) if groups else set()
    alone, grp, in_grp = compare(Ub.cpu().numpy(), Ub_or, cells, whole, skip=partial)
    print(f"\n{name}: tie groups {len(groups)} ({sum(len(g) for g in groups)} cells); "
          f"cells alone {alone.max():.2e}, group sums {grp.max():.2e}, "
          f"single cells in groups {in_grp.max():.2e}")
    assert np.all(alone <= TOL), alone
    assert np.all(grp <= TOL), grp


PATCH = np.array([j * N_SBI[0] + i for j in range(0, 8) for i in range(6, 22)])


def _stages(o, U, T, dt):
    """Stage states U1, U2 of Eq. 16 from the oracle's right-hand side."""
    L0 = o.rhs(U, T.copy())[0]
    U1 = U + dt * L0
    L1 = o.rhs(U1, T.copy())[0]
    U2 = 0.75 * U + 0.25 * (U1 + dt * L1)
    return U1, U2


def step_tie_reach(case, o, U, T, dt, weno=5, rel=1e-11):
    """Cells of U^n that a near-tie at one of the step's stage states can
    reach: the tied cells of U^n itself, those of U1 widened by one stencil
    reach and those of U2 by two. The stage states of the two sides agree to
    about 1e-13, so ties within 1e-11 cover every flip; in the stage states
    maxima at round-off velocities (|u| near 0 in gas at rest) count too."""
    r = oracle_vjp.REACH + (1 if weno == 7 else 0)
    U1, U2 = _stages(o, U, T, dt)
    out = set()
    for k, S in enumerate((U, U1, U2)):
        for g in llf_ties.tie_groups(case, S, T, rel, weno=weno, oracle=o, min_var=MIN_VAR,
                                     abs_rel=1e-13 if k else 0.0):
            out |= llf_ties.dilate(case, g, k * r) if k else g
    return out


STEP_CASES = {
    "sbi2d_n4_64x32": (_sbi64, PATCH),
    "sbi2d_n4_64x32_perturbed": (lambda: perturbed(_sbi64()), PATCH),
    "tube1d_n2": (lambda: cases.shock_tube(0, n=64), None),
    "smooth2d_n3_periodic": (lambda: cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3),
                             None),
}


_STEP_ORACLE = {}


def step_oracle_side(name):
    """Inputs, the oracle's step VJP on the compared cells and the tie reach
    of one step case (shared by the recomputing and the taped reverse)."""
    if name not in _STEP_ORACLE:
        make, patch = STEP_CASES[name]
        case = make()
        o = Oracle(case)
        U, T = o.prim_to_cons()
        dt = 0.5 * o.dt(U, T.copy())
        W = np.random.default_rng(32).normal(size=U.shape)
        cells = np.arange(case.cells) if patch is None else patch
        Ub_or = oracle_vjp.step_vjp(o, U, T, dt, W, cells=cells)
        _STEP_ORACLE[name] = (case, U, T, dt, W, cells, Ub_or, step_tie_reach(case, o, U, T, dt))
    return _STEP_ORACLE[name]


@pytest.mark.parametrize("taped", [False, True], ids=["recomputing", "taped"])
@pytest.mark.parametrize("name", list(STEP_CASES))
def test_step_adjoint_elementwise(name, taped):
    import torch
    case, U, T, dt, W, cells, Ub_or, reach = step_oracle_side(name)
    if name.endswith("perturbed") or name.startswith("smooth"):
        assert not reach, "a case compared on every cell holds no near-tie"
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    Ub = dev(W).clone()
    if taped:
        U1, U2 = torch.empty_like(Ub), torch.empty_like(Ub)
        s.step_tape(dt, U1, U2)
        s.set_state(dev(U), dev(T))
        s.step_adjoint_tape(dt, U1, U2, Ub)
    else:
        s.step_adjoint(dt, Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    Ub = Ub.cpu().numpy()
    skip = reach & set(cells.tolist())
    alone, _, _ = compare(Ub, Ub_or, cells, skip=skip)
    cell_err = np.max(np.abs(Ub[:, cells] - Ub_or[:, cells]) / _scale(Ub_or[:, cells])[:, None],
                      axis=0)
    off = set(cells[cell_err > TOL].tolist())
    print(f"\n{name} ({'taped' if taped else 'recomputing'}): {len(cells)} cells, "
          f"{len(skip)} within a stage tie's reach; {len(off)} above {TOL:g} "
          f"(largest {cell_err.max():.2e}); cells outside the reach {alone.max():.2e}")
    assert np.all(alone <= TOL), alone
    assert off <= skip, sorted(off - skip)
