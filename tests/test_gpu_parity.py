"""Parity of the CUDA path (through the C-ABI) with the CPU oracle, element by
element, on seeded inputs that span several thread blocks with ragged tails.

Tolerances (per-field metric max|gpu - ref| / max|ref|):
1e-11 after one RK3 step and for one RHS evaluation, 1e-8 after ten steps.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle, FLAG_NONPHYS, FLAG_NEWTON

from gpu_util import field_err, gpu_rhs, gpu_steps, gpu_solver, dev

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-11
TOL_1 = 1e-11
TOL_10 = 1e-8


def _cases():
    out = {
        "tube1d_n2": cases.shock_tube(0, n=400),
        "tube1d_n2_ragged": cases.shock_tube(3, n=301),
        "sbi2d_n3_visc": cases.config(1, n=(96, 48)),
        "sbi2d_n4_visc": cases.config(4, n=(70, 35)),
        "sbi3d_n5_visc": cases.config(2, n=(40, 20, 20)),
        "sbi2d_n5_inviscid": cases.shock_bubble(2, (61, 37), 5, 2.2, 0.2, seed=4, viscous=False),
        "smooth2d_n3_periodic": cases.smooth_periodic(2, (33, 29), 3, seed=5, amp=0.3),
        "smooth3d_n2_periodic": cases.smooth_periodic(3, (17, 14, 12), 2, seed=6, amp=0.3),
        "smooth1d_n5_periodic": cases.smooth_periodic(1, (53,), 5, seed=7, amp=0.3),
    }
    return out


CASES = _cases()


def _oracle(case, **kw):
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    return o, U, T


@pytest.mark.parametrize("name", list(CASES))
def test_from_primitive(name):
    import torch
    case = CASES[name]
    o, U, T = _oracle(case)
    s = gpu_solver(case)
    s.set_primitive(dev(case.prim))
    Ug = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    Tg = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(Ug, Tg)
    torch.cuda.synchronize()
    assert np.max(field_err(Ug.cpu().numpy(), U, case.dim)) <= 1e-14
    assert np.max(np.abs(Tg.cpu().numpy() - T) / T) <= 1e-14
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_rhs(name):
    case = CASES[name]
    o, U, T = _oracle(case)
    R, To, st = o.rhs(U, T.copy())
    Rg, Tg, stg = gpu_rhs(case, U, T)
    err = field_err(Rg, R, case.dim)
    assert np.max(err) <= TOL_RHS, err
    assert np.max(np.abs(Tg - To) / To) <= 1e-13
    assert stg == st


@pytest.mark.parametrize("name", list(CASES))
def test_one_step(name):
    case = CASES[name]
    o, U, T = _oracle(case)
    U1, T1 = U.copy(), T.copy()
    dt, st = o.step(U1, T1, 0.0)
    Ug, Tg, stg, dts = gpu_steps(case, U, T, 1)
    assert dts[0] == pytest.approx(dt, rel=1e-13)
    err = field_err(Ug, U1, case.dim)
    assert np.max(err) <= TOL_1, err
    assert np.max(np.abs(Tg - T1) / T1) <= 1e-11
    assert stg == st


@pytest.mark.parametrize("name", ["tube1d_n2", "sbi2d_n3_visc", "sbi3d_n5_visc",
                                  "smooth2d_n3_periodic", "sbi2d_n5_inviscid"])
def test_ten_steps(name):
    case = CASES[name]
    o, U, T = _oracle(case)
    U1, T1 = U.copy(), T.copy()
    for _ in range(10):
        o.step(U1, T1, 0.0)
    Ug, Tg, stg, dts = gpu_steps(case, U, T, 10)
    err = field_err(Ug, U1, case.dim)
    assert np.max(err) <= TOL_10, err


def test_fixed_dt_matches():
    case = CASES["sbi2d_n4_visc"]
    o, U, T = _oracle(case)
    U1, T1 = U.copy(), T.copy()
    dt = 2.5e-4
    for _ in range(3):
        o.step(U1, T1, dt)
    Ug, Tg, stg, dts = gpu_steps(case, U, T, 3, dt=dt)
    assert all(d == dt for d in dts)
    assert np.max(field_err(Ug, U1, case.dim)) <= 1e-10


def test_uniform_state_rhs_vanishes():
    case = cases.uniform_state(3, (9, 8, 7), 4, seed=3, viscous=True)
    o, U, T = _oracle(case)
    Rg, Tg, st = gpu_rhs(case, U, T)
    assert st == 0
    scale = np.max(np.abs(U), axis=1)[:, None] * 9
    assert np.max(np.abs(Rg) / scale) <= 1e-13


def test_shock_tube_to_t_end():
    """Config-1 workload in full: 400 cells to t = 0.2 with the last step clipped."""
    import torch
    case = cases.config(0)
    o, U, T = _oracle(case)
    U1, T1 = U.copy(), T.copy()
    n_or, st = o.run_to(U1, T1, 0.2)
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    dtd = torch.zeros(1, dtype=torch.float64, device="cuda")
    t, n = 0.0, 0
    while t < 0.2:
        s.compute_dt(dtd)
        dt = float(dtd.item())
        if t + dt >= 0.2:
            dt = 0.2 - t
        s.step(dt)
        t += dt
        n += 1
        if 0.2 - t <= 1e-14 * 0.2:
            break
    Ug = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.get_state(Ug)
    torch.cuda.synchronize()
    assert n == n_or
    assert s.status() == 0
    err = field_err(Ug.cpu().numpy(), U1, case.dim)
    assert np.max(err) <= 1e-8, err


def test_nonphysical_state_is_flagged():
    case = CASES["sbi2d_n3_visc"]
    o, U, T = _oracle(case)
    U = U.copy()
    U[0, 100] = -1.0      # negative density
    U[1, 777] = np.nan    # NaN momentum
    R, _, st = o.rhs(U, T.copy())
    Rg, Tg, stg = gpu_rhs(case, U, T)
    assert st & FLAG_NONPHYS and stg & FLAG_NONPHYS


def test_newton_cap_is_flagged():
    case = CASES["sbi2d_n4_visc"]
    o, U, T = _oracle(case, newton_max=1)
    R, _, st = o.rhs(U, np.full_like(T, 300.0))
    Rg, Tg, stg = gpu_rhs(case, U, np.full_like(T, 300.0), newton_max=1)
    assert st & FLAG_NEWTON and stg & FLAG_NEWTON


@pytest.mark.parametrize("dt", [0.0, 2.0e-4])
def test_graph_steps_are_bitwise_single_steps(dt):
    """xf_step_rk3_n (one step captured per temperature-buffer parity, replayed)
    against the same number of xf_step_rk3 calls: state and warm start bit for
    bit, over both parities, after a change of step size and with the
    positivity blend (which reads the stage dt inside the graph)."""
    import torch
    case = cases.multicomponent_diffusion(n=200)
    U, T = Oracle(case, diffusion=1).prim_to_cons()
    out = []
    for graph in (False, True):
        s = gpu_solver(case, diffusion=1, positivity=True)
        s.set_state(dev(U), dev(T))
        for n, d in ((5, dt), (4, dt), (3, 0.5 * dt)):
            if graph:
                s.steps(n, d)
            else:
                for _ in range(n):
                    s.step(d)
        Uo = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
        To = torch.empty(case.cells, dtype=torch.float64, device="cuda")
        s.get_state(Uo, To)
        torch.cuda.synchronize()
        assert s.status() == 0
        out.append((Uo.cpu().numpy(), To.cpu().numpy()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
