"""The hand-written adjoint against exact forward-mode derivatives of the
oracle (dual numbers) and against central finite differences of the CUDA
forward path.

<w, J^T-product(v)> identities: for random directions V and weights W,
sum(Ubar * V_k) computed by xf_rhs_adjoint (Ubar = J^T W) must equal
sum(W * (J V_k)) from the oracle's dual-number JVP, to 1e-10 of the largest
product. Directions vanish on the cells of the state's LLF near-ties
(tests/llf_ties.py), where the two sides may hand the maximum's derivative
to different cells of a tie; test_gpu_adjoint_elementwise.py compares those
cells as groups.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

import llf_ties
from gpu_util import dev, gpu_solver

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "sbi2d_n4_visc": cases.config(4, n=(24, 14)),
        "sbi2d_n3_visc": cases.config(1, n=(20, 12)),
        "smooth2d_n3_periodic": cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3),
        "sbi3d_n5_visc": cases.config(2, n=(12, 8, 8)),
        "tube1d_n2": cases.shock_tube(0, n=64),
        "smooth1d_n4_inviscid": cases.smooth_periodic(1, (40,), 4, seed=2, amp=0.3, viscous=False),
    }


CASES = _cases()
TOL = 1e-10


def _dirs(rng, U, k, rel=1.0):
    """k random directions scaled per field like U."""
    sc = np.max(np.abs(U), axis=1, keepdims=True) + 1e-3
    return rng.normal(size=(k,) + U.shape) * sc * rel


def _off_ties(case, U, T, V, weno=5):
    """V with every cell of an LLF near-tie of U (within 1e-13) set to zero:
    the shock-bubble states hold such ties where the tanh tails of the
    bubble interface make cells' |u -+ c| differ in the last bits, and which
    of them receives alpha's one-sided derivative is decided by round-off
    that the GPU and the oracle need not share. Returns V and the count."""
    tied = set().union(*llf_ties.tie_groups(case, U, T, 1e-13, weno=weno) or [set()])
    V = V.copy()
    V[..., sorted(tied)] = 0.0
    return V, len(tied)


def _dot_check(lhs, rhs, tol):
    lhs, rhs = np.asarray(lhs), np.asarray(rhs)
    assert np.all(np.abs(lhs - rhs) <= tol * (np.abs(rhs) + np.abs(lhs)).max()), (lhs, rhs)


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_adjoint_matches_oracle_jvp(name):
    import torch
    case = CASES[name]
    o = Oracle(case)
    U, T = o.prim_to_cons()
    rng = np.random.default_rng(11)
    V, _ = _off_ties(case, U, T, _dirs(rng, U, 8))
    R, JV, _, st = o.rhs_jvp(U, V, T.copy())
    W = rng.normal(size=U.shape)
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    Ub = torch.zeros((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.rhs_adjoint(dev(U), dev(W), Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, TOL)
    s.close()


PERTURBED = {
    "sbi2d_n4_visc_perturbed": cases.with_smooth_perturbation(cases.config(4, n=(24, 14))),
    "sbi3d_n5_visc_perturbed": cases.with_smooth_perturbation(cases.config(2, n=(12, 8, 8))),
}


@pytest.mark.parametrize("name,tol", [("smooth2d_n3_periodic", 1e-10),
                                      ("smooth1d_n4_inviscid", 1e-10),
                                      ("tube1d_n2", 1e-10),
                                      ("sbi2d_n4_visc_perturbed", 1e-10),
                                      ("sbi3d_n5_visc_perturbed", 1e-10),
                                      ("sbi2d_n4_visc", 1e-5),
                                      ("sbi3d_n5_visc", 1e-5)])
def test_step_adjoint_matches_oracle_jvp(name, tol):
    """Reverse of one RK3 step against the oracle's exact JVP, a round-off
    identity (1e-10) wherever the step is differentiable. The unperturbed
    shock-bubble states are not: after the first stage their gas at rest
    holds velocities of round-off size whose signs the GPU and the oracle
    need not share (the kink of |u| at 0 in the LLF maxima; on the 64 x 32
    workload about half of the cells of a patch disagree in sign), which
    moves the kink's one-sided derivative; they are held to 1e-5, and their
    smoothly perturbed versions (no gas at rest, no tie) to 1e-10."""
    import torch
    case = PERTURBED[name] if name in PERTURBED else CASES[name]
    o = Oracle(case)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    rng = np.random.default_rng(12)
    V = _dirs(rng, U, 8)
    U1, JV, _, _ = o.rk3_jvp(U, V, T.copy(), dt, 1)
    W = rng.normal(size=U.shape)
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    Ub = dev(W).clone()
    s.step_adjoint(dt, Ub)
    torch.cuda.synchronize()
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, tol)
    s.close()


def test_rhs_adjoint_accumulates_and_matches_gpu_fd():
    """Central differences of the CUDA RHS itself. A smooth random field:
    uniform regions (as in the shock-bubble state) hold exact ties in the LLF
    maxima, where the RHS has a kink. Per-cell random directions excite the
    WENO weights' curvature, so the difference step is 1e-7 (its truncation
    error scales as h^2: 5.5e-6 relative at 1e-6, 5.5e-8 at 1e-7)."""
    import torch
    case = CASES["smooth2d_n3_periodic"]
    U, T = Oracle(case).prim_to_cons()
    rng = np.random.default_rng(13)
    V = _dirs(rng, U, 1)[0]
    W = rng.normal(size=U.shape)
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    h = 1e-7
    Rp, Rm = torch.empty_like(dev(U)), torch.empty_like(dev(U))
    s.rhs(dev(U + h * V), Rp)
    s.rhs(dev(U - h * V), Rm)
    fd = np.sum(W * (Rp.cpu().numpy() - Rm.cpu().numpy()) / (2 * h))
    Ub = dev(np.ones_like(U))  # accumulates on top of this
    s.rhs_adjoint(dev(U), dev(W), Ub)
    adj = np.sum((Ub.cpu().numpy() - 1.0) * V)
    assert abs(adj - fd) <= 1e-6 * abs(fd)
    s.close()


def test_objective_and_primitive_adjoints_match_fd():
    import torch
    case = CASES["sbi2d_n4_visc"]
    s = gpu_solver(case)
    P = case.prim.copy()
    rng = np.random.default_rng(14)
    dP = rng.normal(size=P.shape) * (np.max(np.abs(P), axis=1, keepdims=True) + 1e-3) * 1e-2

    def J_of(Pv):
        s.set_primitive(dev(Pv))
        U = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
        s.get_state(U)
        Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
        Ub = torch.empty_like(U)
        s.objective_mixing(U, 2, Jd, Ub)
        torch.cuda.synchronize()
        return Jd.item(), U, Ub

    J0, U, Ub = J_of(P)
    Pb = torch.empty_like(U)
    s.set_primitive_adjoint(dev(P), Ub, Pb)
    adj = float(np.sum(Pb.cpu().numpy() * dP))
    h = 1e-5
    fd = (J_of(P + h * dP)[0] - J_of(P - h * dP)[0]) / (2 * h)
    assert J0 > 0
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    s.close()



DSM_CASES = {
    "sbi2d_n4_visc_dsm": cases.with_binary_diffusion(cases.config(4, n=(24, 14)), seed=1),
    "smooth2d_n3_periodic_dsm": cases.with_binary_diffusion(
        cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3), seed=2),
    "sbi3d_n5_visc_dsm": cases.with_binary_diffusion(cases.config(2, n=(12, 8, 8)), seed=3),
}


@pytest.mark.parametrize("name", list(DSM_CASES))
def test_rhs_adjoint_with_mixture_diffusion_matches_oracle_jvp(name):
    """The mixture-averaged D_sm of Eq. 26 reversed (binary fits through the
    temperature and the pressure, the regularised mole fractions) against the
    oracle's dual-number JVP of the same model."""
    import torch
    case = DSM_CASES[name]
    o = Oracle(case, diffusion=1)
    U, T = o.prim_to_cons()
    rng = np.random.default_rng(15)
    V, _ = _off_ties(case, U, T, _dirs(rng, U, 8))
    R, JV, _, st = o.rhs_jvp(U, V, T.copy())
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, diffusion=1)
    s.set_state(dev(U), dev(T))
    Ub = torch.zeros((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.rhs_adjoint(dev(U), dev(W), Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, TOL)
    s.close()


def test_step_adjoint_with_mixture_diffusion_matches_oracle_jvp():
    import torch
    case = DSM_CASES["smooth2d_n3_periodic_dsm"]
    o = Oracle(case, diffusion=1)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    rng = np.random.default_rng(16)
    V = _dirs(rng, U, 8)
    U1, JV, _, _ = o.rk3_jvp(U, V, T.copy(), dt, 1)
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, diffusion=1)
    s.set_state(dev(U), dev(T))
    Ub = dev(W).clone()
    s.step_adjoint(dt, Ub)
    torch.cuda.synchronize()
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, 1e-10)
    s.close()


def _rarefaction(n=120, uabs=2.0):
    """Two species pulled apart at |u| = 2 from p = 0.4: the centre goes near
    vacuum and the positivity blend acts there."""
    rng = np.random.default_rng(0)
    sp = cases._draw_species(rng, np.array([0.028, 0.004]))
    x = cases._centres(n, 0.0, 1.0)
    left = x < 0.5
    Y = np.stack([np.where(left, 1.0, 0.0), np.where(left, 0.0, 1.0)])
    prim = cases._pack(1, np.ones(n), [np.where(left, -uabs, uabs)], np.full(n, 0.4), Y)
    return cases.Case("rarefaction", 1, (n, 1, 1), (0.0,) * 3, (1.0,) * 3,
                      ((0, 0), (0, 0), (0, 0)), sp, cases.R_U * 300 / 0.028, 1.0, 1.0,
                      False, 0.5, prim)


@pytest.mark.parametrize("name,tol", [("rarefaction", 1e-8), ("sbi2d_n4_visc", 1e-5)])
def test_step_adjoint_with_positivity_blend_matches_oracle_jvp(name, tol):
    """Reverse of one RK3 step with the positivity-preserving blend (Eq. 17-20)
    against the oracle's exact JVP of its blended step. On the rarefaction
    the blend acts (theta < 1 at the centre faces, checked); near vacuum
    theta is ill-conditioned, hence 1e-8. The shock-bubble state carries the
    kinks of its gas at rest (as for the unblended step, hence 1e-5); its
    post-shock gas holds none of the bubble species (their partial densities
    are zero, the implied last one round-off), so the blend binds there on
    round-off-sized species fluxes, and which side's theta binds is decided
    by round-off alone. The directions vanish on every cell such a decision
    can reach within the step: the cells with a partial density at or below
    1e-12 of their density, widened by one cell (the faces beside them) and
    three stencil reaches (the three stages). No perturbed shock-bubble
    state is used: setting that gas in motion makes those fluxes round-off
    on both sides everywhere in it."""
    import torch
    case = _rarefaction() if name == "rarefaction" else CASES[name]
    o = Oracle(case, positivity=True)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    if name == "rarefaction":
        Ub_, Tb_ = U.copy(), T.copy()
        Up_, Tp_ = U.copy(), T.copy()
        Oracle(case).step(Ub_, Tb_, dt)
        o.step(Up_, Tp_, dt)
        assert np.max(np.abs(Ub_ - Up_)) > 1e-6 * np.max(np.abs(U))   # the blend acts
    rng = np.random.default_rng(17)
    V = _dirs(rng, U, 8, rel=1e-3)
    if name != "rarefaction":
        dim = case.dim
        partial = np.vstack([U[dim + 2:], U[:1] - U[dim + 2:].sum(axis=0)])
        trace = set(np.nonzero(np.any(partial <= 1e-12 * U[0], axis=0))[0].tolist())
        reach = llf_ties.dilate(case, trace, 1 + 3 * 3)
        assert 0 < len(reach) < case.cells
        V[..., sorted(reach)] = 0.0
    U1, JV, _, _ = o.rk3_jvp(U, V, T.copy(), dt, 1)
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, positivity=True)
    s.set_state(dev(U), dev(T))
    Ub = dev(W).clone()
    s.step_adjoint(dt, Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, tol)
    s.close()



@pytest.mark.parametrize("weno", [6, 7])
@pytest.mark.parametrize("name", ["smooth2d_n3_periodic", "sbi2d_n4_visc", "sbi3d_n5_visc",
                                  "smooth1d_n4_inviscid"])
def test_rhs_adjoint_with_cu6_and_weno7_matches_oracle_jvp(name, weno):
    """The reverse of the WENO-CU6 and WENO7 reconstructions (indicators,
    weights, candidates; CU6's beta_6 and tau) inside the face adjoint,
    against the oracle's dual-number JVP of the same scheme."""
    import torch
    case = CASES[name]
    o = Oracle(case, weno=weno)
    U, T = o.prim_to_cons()
    rng = np.random.default_rng(18 + weno)
    V, _ = _off_ties(case, U, T, _dirs(rng, U, 8), weno=weno)
    R, JV, _, st = o.rhs_jvp(U, V, T.copy())
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, weno=weno)
    s.set_state(dev(U), dev(T))
    Ub = torch.zeros((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.rhs_adjoint(dev(U), dev(W), Ub)
    torch.cuda.synchronize()
    assert s.status() == 0
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, TOL)
    s.close()


@pytest.mark.parametrize("weno", [6, 7])
def test_step_adjoint_with_cu6_and_weno7_matches_oracle_jvp(weno):
    import torch
    case = CASES["smooth2d_n3_periodic"]
    o = Oracle(case, weno=weno)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    rng = np.random.default_rng(20 + weno)
    V = _dirs(rng, U, 8)
    U1, JV, _, _ = o.rk3_jvp(U, V, T.copy(), dt, 1)
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, weno=weno)
    s.set_state(dev(U), dev(T))
    Ub = dev(W).clone()
    s.step_adjoint(dt, Ub)
    torch.cuda.synchronize()
    Ubar = Ub.cpu().numpy()
    lhs = [np.sum(Ubar * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    _dot_check(lhs, rhs, 1e-10)
    s.close()
