"""The taped SSP-RK3 step and its adjoint (xf_step_rk3_tape,
xf_step_rk3_adjoint_tape): the stage states the step writes are those of
Eq. 16 built from the oracle's RHS; the step itself is bitwise the plain step;
the taped reverse passes the same dot tests against the oracle's dual-number
JVP as the recomputing reverse and equals it up to the order of atomic adds,
for every option of the path (the blended rarefaction included, whose binding
partial density is decided on round-off-sized fluxes: the taped reverse must
see bitwise the forward step's fields); and the checkpointed gradient is the
same either way."""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, field_err, gpu_solver

pytestmark = pytest.mark.gpu


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


def _smooth():
    return cases.smooth_periodic(2, (14, 12), 3, seed=5, amp=0.3)


# (case, options, dot-test tolerance): smooth states are round-off identities;
# the unperturbed shock-bubble states carry the kinks of their gas at rest
# (see the step-adjoint tests), their perturbed versions none; the
# rarefaction is blended near vacuum
SETUPS = {
    "weno5": (_smooth, {}, 1e-10),
    "weno_cu6": (_smooth, {"weno": 6}, 1e-10),
    "weno7": (_smooth, {"weno": 7}, 1e-10),
    "mixture_diffusion": (lambda: cases.with_binary_diffusion(_smooth(), seed=2),
                          {"diffusion": 1}, 1e-10),
    "positivity": (_rarefaction, {"positivity": True}, 1e-8),
    "sbi2d_n4_visc": (lambda: cases.config(4, n=(24, 14)), {}, 1e-5),
    "sbi3d_n5_visc": (lambda: cases.config(2, n=(12, 8, 8)), {}, 1e-5),
    "sbi2d_n4_visc_perturbed": (
        lambda: cases.with_smooth_perturbation(cases.config(4, n=(24, 14))), {}, 1e-10),
    "sbi3d_n5_visc_perturbed": (
        lambda: cases.with_smooth_perturbation(cases.config(2, n=(12, 8, 8))), {}, 1e-10),
}


def _setup(name):
    make, kw, tol = SETUPS[name]
    case = make()
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    return case, kw, tol, o, U, T, dt


def _empty(case):
    import torch
    return torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", list(SETUPS))
def test_tape_holds_the_stage_states_of_eq16(name):
    """U1 = U + dt L(U) and U2 = 3/4 U + 1/4 (U1 + dt L(U1)) with the
    oracle's L, to the one-step parity bar (not with the blend: L(U), a plain
    RHS, does not blend); the step's result bitwise that of xf_step_rk3 from
    the same state."""
    import torch
    case, kw, _, o, U, T, dt = _setup(name)
    blend = kw.get("positivity", False)
    if not blend:
        R0, T0, st0 = o.rhs(U, T.copy())
        U1o = U + dt * R0
        R1, _, st1 = o.rhs(U1o, T0.copy())
        U2o = 0.75 * U + 0.25 * (U1o + dt * R1)
        assert st0 == st1 == 0
    s = gpu_solver(case, **kw)
    s.set_state(dev(U), dev(T))
    U1, U2 = _empty(case), _empty(case)
    s.step_tape(dt, U1, U2)
    Ut = _empty(case)
    s.get_state(Ut)
    s.set_state(dev(U), dev(T))
    s.step(dt)
    Up = _empty(case)
    s.get_state(Up)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    assert torch.equal(Ut, Up)
    if blend:
        return
    assert np.max(field_err(U1.cpu().numpy(), U1o, case.dim)) <= 1e-11
    assert np.max(field_err(U2.cpu().numpy(), U2o, case.dim)) <= 1e-11


@pytest.mark.parametrize("name", list(SETUPS))
def test_tape_adjoint_matches_oracle_jvp_and_the_recomputing_adjoint(name):
    import torch
    case, kw, tol, o, U, T, dt = _setup(name)
    rng = np.random.default_rng(31)
    V = rng.normal(size=(8,) + U.shape) * (np.max(np.abs(U), axis=1, keepdims=True) + 1e-3)
    if kw.get("positivity"):
        V = V * 1e-3
    _, JV, _, _ = o.rk3_jvp(U, V, T.copy(), dt, 1)
    W = rng.normal(size=U.shape)
    s = gpu_solver(case, **kw)
    s.set_state(dev(U), dev(T))
    U1, U2 = _empty(case), _empty(case)
    s.step_tape(dt, U1, U2)
    s.set_state(dev(U), dev(T))
    Ub_tape = dev(W).clone()
    s.step_adjoint_tape(dt, U1, U2, Ub_tape)
    # both reverses leave the warm start at U2's temperature, from the same
    # chain of Newton solves as the forward step
    Tt = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(None, Tt)
    s.set_state(dev(U), dev(T))
    Ub_rec = dev(W).clone()
    s.step_adjoint(dt, Ub_rec)
    Tr = torch.empty_like(Tt)
    s.get_state(None, Tr)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    assert torch.equal(Tt, Tr)
    # equal up to the order of the atomic adds
    a, b = Ub_tape.cpu().numpy(), Ub_rec.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    lhs = [np.sum(a * V[k]) for k in range(8)]
    rhs = [np.sum(W * JV[k]) for k in range(8)]
    lhs, rhs = np.asarray(lhs), np.asarray(rhs)
    assert np.all(np.abs(lhs - rhs) <= tol * (np.abs(rhs) + np.abs(lhs)).max()), (lhs, rhs)


def test_checkpointed_gradient_is_the_same_with_and_without_the_tape():
    """J(P0) of the differentiated workload's form (shock-bubble, 4 species,
    fixed dt, checkpoints) on a small grid: the taped backward pass gives the
    recomputing one's gradient to round-off."""
    import torch
    from paper_2403_05910_b300.autodiff import mixing_after_steps
    c = cases.shock_bubble(2, (48, 24), 4, 1.5, 0.2, seed=0, name="sbi2d_n4_adjoint")
    s = gpu_solver(c)
    s.set_primitive(dev(c.prim))
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.compute_dt(d)
    dt = 0.9 * d.item()
    grads, Js = [], []
    for tape in (True, False):
        P0 = dev(c.prim).requires_grad_(True)
        J = mixing_after_steps(P0, s, dt, 30, 7, 2, tape=tape)
        J.backward()
        grads.append(P0.grad.cpu().numpy())
        Js.append(J.item())
    assert s.status() == 0
    s.close()
    assert Js[0] == Js[1]
    g0, g1 = grads
    assert np.max(np.abs(g0 - g1)) <= 1e-10 * np.max(np.abs(g1))
    assert np.max(np.abs(g1)) > 0.0


def test_tape_argument_errors():
    import torch
    from paper_2403_05910_b300.xf import XFError
    case = _smooth()
    s = gpu_solver(case)
    U, T = Oracle(case).prim_to_cons()
    s.set_state(dev(U), dev(T))
    U1 = _empty(case)
    Ub = dev(U).clone()
    with pytest.raises(XFError):
        s.step_tape(1e-3, U1, U1)            # stage buffers must differ
    with pytest.raises(XFError):
        s.step_tape(0.0, U1, _empty(case))   # fixed dt only
    with pytest.raises(XFError):
        s.step_adjoint_tape(-1.0, U1, U1, Ub)
    with pytest.raises(XFError):
        s.step_adjoint_tape(1e-3, U, U1, Ub)   # a host stage state
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()


@pytest.mark.parametrize("name", ["positivity", "sbi2d_n4_visc"])
def test_flux_tape_gives_the_taped_step_and_adjoint(name):
    """xf_step_rk3_tape_flux is bitwise the plain step and its flux tape
    holds every stage's unblended convective face fluxes; the reverse that
    reads them (xf_step_rk3_adjoint_tape_flux) equals the taped reverse that
    recomputes them, up to the order of the atomic adds, with the blend on."""
    import torch
    make, kw = SETUPS[name][0], dict(SETUPS[name][1])
    kw["positivity"] = True
    case = make()
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    dt = 0.5 * o.dt(U, T.copy())
    W = np.random.default_rng(33).normal(size=U.shape)
    s = gpu_solver(case, **kw)
    n = s.tape_flux_len()
    assert n == 3 * case.n_v * sum(
        int(np.prod([case.n[a] + (a == d) for a in range(3)])) for d in range(case.dim))
    s.set_state(dev(U), dev(T))
    U1, U2 = _empty(case), _empty(case)
    Fh = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    s.step_tape(dt, U1, U2, Fhat=Fh)
    Uf = _empty(case)
    s.get_state(Uf)
    s.set_state(dev(U), dev(T))
    s.step(dt)
    Up = _empty(case)
    s.get_state(Up)
    assert torch.equal(Uf, Up)
    assert torch.isfinite(Fh).all()
    s.set_state(dev(U), dev(T))
    Ub_flux = dev(W).clone()
    s.step_adjoint_tape(dt, U1, U2, Ub_flux, Fhat=Fh)
    s.set_state(dev(U), dev(T))
    Ub_tape = dev(W).clone()
    s.step_adjoint_tape(dt, U1, U2, Ub_tape)
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    a, b = Ub_flux.cpu().numpy(), Ub_tape.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_checkpointed_gradient_with_the_blend_is_the_same_with_the_flux_tape():
    """The checkpointed gradient of the differentiated workload's form with
    the positivity blend: the taped backward pass (stage states and flux
    tape kept by the segment re-runs) gives the recomputing one's gradient."""
    import torch
    from paper_2403_05910_b300.autodiff import mixing_after_steps
    c = cases.shock_bubble(2, (48, 24), 4, 1.5, 0.2, seed=0, name="sbi2d_n4_adjoint")
    s = gpu_solver(c, positivity=True)
    s.set_primitive(dev(c.prim))
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.compute_dt(d)
    dt = 0.9 * d.item()
    grads, Js = [], []
    for tape in (True, False):
        P0 = dev(c.prim).requires_grad_(True)
        J = mixing_after_steps(P0, s, dt, 12, 5, 2, tape=tape)
        J.backward()
        grads.append(P0.grad.cpu().numpy())
        Js.append(J.item())
    assert s.status() == 0
    s.close()
    assert Js[0] == Js[1]
    g0, g1 = grads
    assert np.max(np.abs(g0 - g1)) <= 1e-10 * np.max(np.abs(g1))
