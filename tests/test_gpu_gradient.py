"""The differentiated 2D shock-bubble workload on its 64x32 sub-grid version:
4 species, 200 fixed-dt RK3 steps with a checkpoint every 20 steps, objective
J = sum Y_3 (1 - Y_3) dV at the final time. The adjoint gradient (through
torch.autograd, all derivatives in the library's kernels) is checked against
central finite differences (h = 1e-6 relative) of the CUDA forward path, for
the shock Mach number, the bubble radius and density-field directions.

Ma and r enter through the seeded input generator (Eq. 32-33); their chain
rule dJ/dMa = sum Pbar0 . dP0/dMa uses generator differences (input
construction, not the solver path). Density directions live on the bubble
interface, where the state is not uniform: uniform regions hold exact ties in
the LLF maxima, where J has a kink.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases

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
