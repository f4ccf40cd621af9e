"""The other reconstructions REC of Eq. 15 on the GPU: WENO-CU6 (ref. 34,
weno = 6) and WENO7-JS (ref. 36, weno = 7, 8-cell stencil and 4 ghost
layers). Parity with the oracle's same scheme on the RHS, one step and ten
steps; the design order on the advected density wave; and the entry points
that need one scheme (a batch) refuse a mix. Their adjoints are checked in
test_gpu_adjoint.py.

Tolerances as for WENO5: 1e-11 for one RHS and one step, 1e-8 after ten steps
(per-field max |gpu - ref| / max |ref|).
"""
import math

import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, field_err, gpu_rhs, gpu_solver, gpu_steps

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "tube1d_n2": cases.shock_tube(0, n=400),
        "tube1d_n2_ragged": cases.shock_tube(3, n=301),
        "sbi2d_n3_visc": cases.config(1, n=(96, 48)),
        "sbi3d_n5_visc": cases.config(2, n=(40, 20, 20)),
        "sbi2d_n5_inviscid": cases.shock_bubble(2, (61, 37), 5, 2.2, 0.2, seed=4, viscous=False),
        "smooth2d_n3_periodic": cases.smooth_periodic(2, (33, 29), 3, seed=5, amp=0.3),
    }


CASES = _cases()


WENOS = [6, 7]


def _oracle(case, weno, **kw):
    o = Oracle(case, weno=weno, **kw)
    U, T = o.prim_to_cons()
    return o, U, T


@pytest.mark.parametrize("weno", WENOS)
@pytest.mark.parametrize("name", list(CASES))
def test_rhs(name, weno):
    case = CASES[name]
    o, U, T = _oracle(case, weno)
    R, To, st = o.rhs(U, T.copy())
    Rg, Tg, stg = gpu_rhs(case, U, T, weno=weno)
    assert np.max(field_err(Rg, R, case.dim)) <= 1e-11
    assert stg == st == 0
    # and it is a different scheme from WENO5 on these states
    R5, _, _ = Oracle(case).rhs(U, T.copy())
    assert np.max(field_err(R5, R, case.dim)) > 1e-8


@pytest.mark.parametrize("weno", WENOS)
@pytest.mark.parametrize("name,steps,tol", [("tube1d_n2", 1, 1e-11), ("sbi2d_n3_visc", 1, 1e-11),
                                            ("sbi3d_n5_visc", 1, 1e-11), ("tube1d_n2", 10, 1e-8),
                                            ("sbi2d_n5_inviscid", 10, 1e-8),
                                            ("smooth2d_n3_periodic", 10, 1e-8)])
def test_steps(name, steps, tol, weno):
    case = CASES[name]
    o, U, T = _oracle(case, weno)
    U1, T1 = U.copy(), T.copy()
    dts = []
    for _ in range(steps):
        dt, st = o.step(U1, T1, 0.0)
        assert st == 0
        dts.append(dt)
    Ug, Tg, stg, dtg = gpu_steps(case, U, T, steps, weno=weno)
    assert stg == 0
    assert np.max(np.abs(np.array(dtg) - dts) / np.array(dts)) <= tol
    assert np.max(field_err(Ug, U1, case.dim)) <= tol


@pytest.mark.parametrize("weno", WENOS)
def test_with_positivity_blend(weno):
    """The scheme feeding the blend of Eq. 17-20 (one step, shock-bubble state)."""
    case = cases.config(4, n=(48, 24))
    o, U, T = _oracle(case, weno, positivity=True)
    U1, T1 = U.copy(), T.copy()
    o.step(U1, T1, 0.0)
    Ug, _, st, _ = gpu_steps(case, U, T, 1, weno=weno, positivity=True)
    assert st == 0
    assert np.max(field_err(Ug, U1, case.dim)) <= 1e-11


@pytest.mark.parametrize("weno,ns,power,order", [(6, (40, 80, 160), 2.0, 5.5),
                                                (7, (20, 40, 80), 7.0 / 3.0, 6.0)])
def test_design_order_density_wave(weno, ns, power, order):
    """rho = 1 + 0.2 sin(2 pi x) advected to t = 0.1 with dt ~ dx^power (RK3
    below the spatial error): the L1 error of the CUDA path falls at the
    oracle's rate (CU6: 5.98, 5.98; WENO7: 6.2, 6.3)."""
    errs = []
    for n in ns:
        c = cases.density_wave(n)
        U, T = Oracle(c).prim_to_cons()
        dt0 = 0.4 * (1.0 / n) ** power
        steps = int(math.ceil(0.1 / dt0))
        Ug, _, st, _ = gpu_steps(c, U, T, steps, dt=0.1 / steps, weno=weno)
        assert st == 0
        x = cases._centres(n, 0.0, 1.0)
        errs.append(np.mean(np.abs(Ug[0] - (1.0 + 0.2 * np.sin(2 * np.pi * (x - 0.1))))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= order, (errs, orders)


@pytest.mark.parametrize("weno", WENOS)
def test_batch_needs_one_scheme(weno):
    """One batch shares one reconstruction: mixing schemes is refused."""
    import ctypes as C
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import XF_ERR_ARG, Grid, Opts, Thermo, lib, structs
    c2 = cases.config(1, n=(20, 10))
    g5, t5, o5, k5 = structs(c2)
    g6, t6, o6, k6 = structs(c2, weno=weno)
    G, Th, O = (Grid * 2)(g5, g6), (Thermo * 2)(t5, t6), (Opts * 2)(o5, o6)
    h = C.c_void_p()
    assert lib.xf_batch_create(2, G, Th, O, C.byref(h)) == XF_ERR_ARG


def test_weno7_needs_four_cells_per_axis():
    from paper_2403_05910_b300.xf import XFError
    case = cases.shock_tube(0, n=3)
    gpu_solver(case, weno=5).close()
    with pytest.raises(XFError):
        gpu_solver(case, weno=7)


@pytest.mark.parametrize("weno", [5, 6, 7])
def test_all_options_together(weno):
    """Each reconstruction with the positivity blend and the mixture-averaged
    diffusion at once (2D and 3D shock-bubble states): one step and ten."""
    for case, steps, tol in ((cases.with_binary_diffusion(cases.config(4, n=(40, 20)), seed=5), 10, 1e-8),
                             (cases.with_binary_diffusion(cases.config(2, n=(20, 12, 12)), seed=6), 1, 1e-11)):
        kw = {"weno": weno, "positivity": True, "diffusion": 1}
        o, U, T = _oracle(case, weno, positivity=True, diffusion=1)
        U1, T1 = U.copy(), T.copy()
        for _ in range(steps):
            _, st = o.step(U1, T1, 0.0)
            assert st == 0
        Ug, _, stg, _ = gpu_steps(case, U, T, steps, **kw)
        assert stg == 0
        assert np.max(field_err(Ug, U1, case.dim)) <= tol, case.name



@pytest.mark.parametrize("weno", WENOS)
def test_batch_with_scheme_is_bitwise_single_grid(weno):
    """The batched persistent form with CU6 or WENO7 (and the blend on):
    every instance bit for bit equal to stepping it alone."""
    from paper_2403_05910_b300.xf import Batch
    cs = cases.batch(11, count=5, scale=4)
    ins = [Oracle(c).prim_to_cons() for c in cs]
    b = Batch(cs, weno=weno, positivity=True)
    for i, (U, T) in enumerate(ins):
        b.set_state(i, dev(U), dev(T))
    for _ in range(2):
        b.step(0.0)
    import torch
    got = []
    for i, c in enumerate(cs):
        Ug = torch.empty((c.n_v, c.cells), dtype=torch.float64, device="cuda")
        Tg = torch.empty(c.cells, dtype=torch.float64, device="cuda")
        b.get_state(i, Ug, Tg)
        got.append((Ug, Tg))
    torch.cuda.synchronize()
    assert b.status() == 0
    b.close()
    for c, (U, T), (Ug, Tg) in zip(cs, ins, got):
        Up, Tp, st, _ = gpu_steps(c, U, T, 2, weno=weno, positivity=True)
        assert st == 0
        assert np.array_equal(Ug.cpu().numpy(), Up), c.name
        assert np.array_equal(Tg.cpu().numpy(), Tp), c.name
