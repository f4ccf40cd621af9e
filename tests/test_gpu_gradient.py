"""The differentiated 2D shock-bubble workload on its 64x32 sub-grid version:
4 species, 200 fixed-dt RK3 steps with a checkpoint every 20 steps, objective
J = sum Y_3 (1 - Y_3) dV at the final time. The adjoint gradient (through
torch.autograd, all derivatives in the library's kernels) is checked against
central finite differences (h = 1e-6 relative) of the CUDA forward path, for
the shock Mach number, the bubble radius and density-field directions, and
against the oracle's exact forward-mode derivative (dual numbers) over the
same 200 steps along 8 tangents of the initial state, on the workload, on
its smoothly perturbed version and on a smooth periodic field.

Ma and r enter through the seeded input generator (Eq. 32-33); their chain
rule dJ/dMa = sum Pbar0 . dP0/dMa uses generator differences (input
construction, not the solver path). Density directions live on the bubble
interface, where the state is not uniform: uniform regions hold exact ties in
the LLF maxima, where J has a kink.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, gpu_solver

pytestmark = pytest.mark.gpu

N_GRID = (64, 32)
STEPS, EVERY = 200, 20
MA0, R0 = 1.5, 0.2
SPECIES = 2  # the third species (0-based)


def _case(Ma, r):
    return cases.shock_bubble(2, N_GRID, 4, Ma, r, seed=0, name="sbi2d_n4_adjoint")


def _frozen_dt():
    import torch
    c = _case(MA0, R0)
    s = gpu_solver(c)
    s.set_primitive(dev(c.prim))
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.compute_dt(d)
    torch.cuda.synchronize()
    s.close()
    return 0.9 * d.item()


def _J(P, solver, dt):
    import torch
    solver.set_primitive(dev(P))
    for _ in range(STEPS):
        solver.step(dt)
    U = torch.empty((solver.nv, solver.cells), dtype=torch.float64, device="cuda")
    solver.get_state(U)
    Jd = torch.zeros(1, dtype=torch.float64, device="cuda")
    Ub = torch.empty_like(U)
    solver.objective_mixing(U, SPECIES, Jd, Ub)
    torch.cuda.synchronize()
    assert solver.status() == 0
    return Jd.item()


def test_mixing_gradient_matches_finite_differences():
    import torch
    from paper_2403_05910_b300.autodiff import mixing_after_steps
    dt = _frozen_dt()
    c0 = _case(MA0, R0)
    s = gpu_solver(c0)
    P0 = dev(c0.prim).requires_grad_(True)
    J = mixing_after_steps(P0, s, dt, STEPS, EVERY, SPECIES)
    J.backward()
    Pbar = P0.grad.cpu().numpy()
    J0 = J.item()
    assert J0 == pytest.approx(_J(c0.prim, s, dt), rel=1e-13)

    def rel(a, b):
        return abs(a - b) / max(abs(a), abs(b))

    # shock Mach number and bubble radius through the generator
    for name, f in (("Ma", lambda h: _case(MA0 + h, R0).prim),
                    ("r", lambda h: _case(MA0, R0 + h).prim)):
        base = MA0 if name == "Ma" else R0
        hg = 1e-7 * base
        dP = (f(hg) - f(-hg)) / (2 * hg)
        adj = float(np.sum(Pbar * dP))
        h = 1e-6 * base
        fd = (_J(f(h), s, dt) - _J(f(-h), s, dt)) / (2 * h)
        assert rel(adj, fd) <= 1e-6, (name, adj, fd)

    # density-field directions supported on the interface (fixed u, p, Y)
    rng = np.random.default_rng(21)
    Y3 = c0.prim[6]  # rows: rho, u, v, p, Y_1, Y_2, Y_3
    w = Y3 * (1.0 - Y3)
    for _ in range(2):
        d = np.zeros_like(c0.prim)
        d[0] = rng.normal(size=c0.cells) * w * c0.prim[0]
        adj = float(np.sum(Pbar * d))
        h = 1e-6
        fd = (_J(c0.prim + h * d, s, dt) - _J(c0.prim - h * d, s, dt)) / (2 * h)
        assert rel(adj, fd) <= 1e-6, ("rho", adj, fd)
    s.close()


def _objective_tangent(case, U, dU, species=SPECIES):
    """dJ of J = sum Y_s (1 - Y_s) dV along the tangents dU [k, n_v, cells]
    (Y_s = (rho Y_s) / rho, the species row after the momentum and energy rows)."""
    row = case.dim + 2 + species
    dV = float(np.prod(case.dx[:case.dim]))
    Y = U[row] / U[0]
    dY = (dU[:, row] - Y * dU[:, 0]) / U[0]
    return np.sum((1.0 - 2.0 * Y) * dY, axis=1) * dV


def _gpu_gradient_U0(case, U0, T0, dt, steps, every):
    """dJ/dU0 of `steps` fixed-dt steps from (U0, T0) through the checkpointed
    reverse (torch.autograd over the C-ABI calls)."""
    import torch
    from paper_2403_05910_b300.autodiff import RK3Steps, MixingObjective
    s = gpu_solver(case)
    s.set_state(dev(U0), dev(T0))
    U = dev(U0).requires_grad_(True)
    J = MixingObjective.apply(RK3Steps.apply(U, s, dt, steps, every), s, SPECIES)
    J.backward()
    torch.cuda.synchronize()
    assert s.status() == 0
    s.close()
    return J.item(), U.grad.cpu().numpy()


def _interface_directions(c0, o, rng, k):
    """Tangents of U0 for perturbations of the primitive fields supported on
    the bubble interface (weight Y_3 (1 - Y_3)), each mapped to conserved
    variables through the oracle's EOS by central differences."""
    Y3 = c0.prim[6]
    w = Y3 * (1.0 - Y3)
    out = []
    for row in [0, 0, 0, 3, 1, 6][:k]:       # rho (three), p, u, Y_3
        d = np.zeros_like(c0.prim)
        d[row] = rng.normal(size=c0.cells) * w * (np.max(np.abs(c0.prim[row])) if row != 6 else 1.0)
        h = 1e-7
        Up = o.prim_to_cons(c0.prim + h * d)[0]
        Um = o.prim_to_cons(c0.prim - h * d)[0]
        out.append((Up - Um) / (2 * h))
    return out


def test_mixing_gradient_matches_the_oracle_jvp():
    """The 200-step checkpointed gradient dJ/dU0 of the differentiated
    workload against the oracle's exact forward-mode derivative over the
    same 200 fixed-dt steps, along 8 tangents of U0: the generator's Ma and
    r directions (Eq. 32-33 through the oracle's EOS) and six perturbations
    supported on the bubble interface (density three times, pressure,
    velocity, Y_3). Both sides start from the oracle's U0 and T0 and use the
    same dt.

    The gas at rest around the bubble holds velocities of round-off size
    after the first stage, whose signs the two sides need not share: |u| in
    the LLF maxima has its kink there. Tangents that set that gas in motion
    at once (the pressure and velocity perturbations) pass through the kink
    and are held to 1e-7; the others to 1e-10. The smoothly perturbed
    workload below has no gas at rest and holds every direction to 1e-10."""
    c0 = _case(MA0, R0)
    o = Oracle(c0)
    U0, T0 = o.prim_to_cons()
    dt = 0.9 * o.dt(U0, T0.copy())
    V = []
    for f, base in ((lambda h: _case(MA0 + h, R0).prim, MA0), (lambda h: _case(MA0, R0 + h).prim, R0)):
        hg = 1e-7 * base
        V.append((o.prim_to_cons(f(hg))[0] - o.prim_to_cons(f(-hg))[0]) / (2 * hg))
    V += _interface_directions(c0, o, np.random.default_rng(22), 6)
    V = np.asarray(V)
    UT, JV, _, st = o.rk3_jvp(U0, V, T0.copy(), dt, STEPS)
    assert st == 0
    dJ_or = _objective_tangent(c0, UT, JV)
    J_gpu, G = _gpu_gradient_U0(c0, U0, T0, dt, STEPS, EVERY)
    dJ_gpu = np.array([np.sum(G * V[k]) for k in range(len(V))])
    err = np.abs(dJ_gpu - dJ_or) / np.max(np.abs(dJ_or))
    print("\n200-step gradient vs oracle JVP, per direction:", np.array2string(err, precision=2))
    tol = np.array([1e-10] * 5 + [1e-7, 1e-7, 1e-10])   # Ma, r, rho x3, p, u, Y_3
    assert np.all(err <= tol), (dJ_gpu, dJ_or)


def test_perturbed_workload_gradient_matches_the_oracle_jvp():
    """The differentiated workload with a smooth seeded 1e-3 perturbation of
    density, velocity and pressure (no gas at rest, so no kink of |u| at 0
    and no tie of the LLF maxima along the run): the 200-step checkpointed
    gradient against the oracle's exact JVP to 1e-10 along the six interface
    tangents and two random per-cell tangents."""
    c0 = cases.with_smooth_perturbation(_case(MA0, R0))
    o = Oracle(c0)
    U0, T0 = o.prim_to_cons()
    dt = 0.9 * o.dt(U0, T0.copy())
    rng = np.random.default_rng(24)
    V = _interface_directions(c0, o, rng, 6)
    V += list(rng.normal(size=(2,) + U0.shape) * np.max(np.abs(U0), axis=1, keepdims=True))
    V = np.asarray(V)
    UT, JV, _, st = o.rk3_jvp(U0, V, T0.copy(), dt, STEPS)
    assert st == 0
    dJ_or = _objective_tangent(c0, UT, JV)
    _, G = _gpu_gradient_U0(c0, U0, T0, dt, STEPS, EVERY)
    dJ_gpu = np.array([np.sum(G * V[k]) for k in range(len(V))])
    err = np.abs(dJ_gpu - dJ_or) / np.max(np.abs(dJ_or))
    print("\nperturbed 200-step gradient vs oracle JVP, per direction:",
          np.array2string(err, precision=2))
    assert np.all(err <= 1e-10), (dJ_gpu, dJ_or)


def test_smooth_field_gradient_matches_the_oracle_jvp_in_random_directions():
    """The same 200-step checkpointed gradient on a smooth periodic 4-species
    field (no kinks anywhere), along 8 random per-cell tangents of U0."""
    c = cases.smooth_periodic(2, (32, 16), 4, seed=3, amp=0.3)
    o = Oracle(c)
    U0, T0 = o.prim_to_cons()
    dt = 0.5 * o.dt(U0, T0.copy())
    rng = np.random.default_rng(23)
    V = rng.normal(size=(8,) + U0.shape) * (np.max(np.abs(U0), axis=1, keepdims=True) + 1e-3)
    UT, JV, _, st = o.rk3_jvp(U0, V, T0.copy(), dt, STEPS)
    assert st == 0
    dJ_or = _objective_tangent(c, UT, JV)
    _, G = _gpu_gradient_U0(c, U0, T0, dt, STEPS, EVERY)
    dJ_gpu = np.array([np.sum(G * V[k]) for k in range(8)])
    err = np.abs(dJ_gpu - dJ_or) / np.max(np.abs(dJ_or))
    print("\nsmooth 200-step gradient vs oracle JVP, per direction:",
          np.array2string(err, precision=2))
    assert np.all(err <= 1e-10), (dJ_gpu, dJ_or)
