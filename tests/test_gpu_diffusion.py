"""Mixture-averaged species diffusion (Eq. 25-26, xf_opts.diffusion = 1) on
the GPU: parity with the oracle's model on the RHS, one step and ten steps,
including the 1D multicomponent diffusion case of Sec. IV.B (Table IV,
synthetic species); conservation over a long run of that case; the batched
form with the model. Its adjoint is checked in test_gpu_adjoint.py.

Tolerances as for the rest of the path: 1e-11 for one RHS and one step,
1e-8 after ten steps (per-field max |gpu - ref| / max |ref|).
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, field_err, gpu_rhs, gpu_solver, gpu_steps

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "diffusion1d_n4": cases.multicomponent_diffusion(n=200),
        "diffusion1d_n4_ragged": cases.multicomponent_diffusion(n=173, seed=3),
        "sbi2d_n3_visc": cases.with_binary_diffusion(cases.config(1, n=(96, 48)), seed=1),
        "sbi3d_n5_visc": cases.with_binary_diffusion(cases.config(2, n=(40, 20, 20)), seed=2),
        "smooth2d_n4_periodic": cases.with_binary_diffusion(
            cases.smooth_periodic(2, (33, 29), 4, seed=5, amp=0.3), seed=3),
    }


CASES = _cases()


def _oracle(case, **kw):
    o = Oracle(case, diffusion=1, **kw)
    U, T = o.prim_to_cons()
    return o, U, T


@pytest.mark.parametrize("name", list(CASES))
def test_rhs(name):
    """The diffusion case starts at rest in uniform pressure: its convective
    RHS is pure round-off of O(rho c / dx) terms, which would swamp the small
    diffusive rates in a per-field relative metric, so its RHS is compared
    with the convective operator off (the steps below run the full path)."""
    case = CASES[name]
    kw = {"convective": False} if name.startswith("diffusion1d") else {}
    o, U, T = _oracle(case, **kw)
    R, To, st = o.rhs(U, T.copy())
    Rg, Tg, stg = gpu_rhs(case, U, T, diffusion=1, **kw)
    assert stg == st == 0
    assert np.max(field_err(Rg, R, case.dim)) <= 1e-11
    # the model changes the species rows against the common-D model
    R0, _, _ = Oracle(case, **kw).rhs(U, T.copy())
    sl = slice(2 + case.dim, None)
    assert np.max(np.abs(R0[sl] - R[sl])) > 1e-6 * np.max(np.abs(R[sl]))


@pytest.mark.parametrize("name,steps,tol,weno", [("diffusion1d_n4", 1, 1e-11, 5),
                                                 ("sbi2d_n3_visc", 1, 1e-11, 5),
                                                 ("sbi3d_n5_visc", 1, 1e-11, 5),
                                                 ("diffusion1d_n4", 10, 1e-8, 5),
                                                 ("diffusion1d_n4", 10, 1e-8, 6),
                                                 ("sbi2d_n3_visc", 10, 1e-8, 5),
                                                 ("smooth2d_n4_periodic", 10, 1e-8, 5)])
def test_steps(name, steps, tol, weno):
    """The diffusion case starts at rest: its momentum after a step is
    round-off of the pressure balance, so momentum is measured against the
    mass scale (rho a_ref) there."""
    case = CASES[name]
    o, U, T = _oracle(case, weno=weno)
    U1, T1 = U.copy(), T.copy()
    dts = []
    for _ in range(steps):
        dt, st = o.step(U1, T1, 0.0)
        assert st == 0
        dts.append(dt)
    Ug, Tg, stg, dtg = gpu_steps(case, U, T, steps, diffusion=1, weno=weno)
    assert stg == 0
    assert np.max(np.abs(np.array(dtg) - dts) / np.array(dts)) <= tol
    floor = np.max(np.abs(U1[0])) if name.startswith("diffusion1d") else 0.0
    assert np.max(field_err(Ug, U1, case.dim, mom_floor=floor)) <= tol


def test_diffusion_case_conserves_over_a_long_run():
    """20000 CFL steps of the periodic diffusion case on the GPU: every
    partial density and the energy keep their totals to round-off, momentum
    stays at round-off of the mass, and the CH4 variance falls."""
    case = CASES["diffusion1d_n4"]
    U, T = Oracle(case, diffusion=1).prim_to_cons()
    Ug, _, st, _ = gpu_steps(case, U, T, 20000, diffusion=1)
    assert st == 0
    scale = np.abs(U).sum(axis=1)
    scale[1] = scale[0]
    drift = np.abs(Ug.sum(axis=1) - U.sum(axis=1)) / scale
    assert np.max(drift) <= 1e-11, drift

    def ch4(V):
        return (V[0] - V[3:].sum(0)) / V[0]
    assert np.var(ch4(Ug)) < 0.9 * np.var(ch4(U))


def test_model_needs_binary_fits():
    with pytest.raises(ValueError):
        gpu_solver(cases.config(1, n=(24, 12)), diffusion=1)   # no binary fits



def test_batch_with_mixture_diffusion_is_bitwise_single_grid():
    """The batched persistent form with the mixture-averaged model (instances
    with their own binary fits): bit for bit equal to stepping alone."""
    import torch
    from paper_2403_05910_b300.xf import Batch
    cs = [cases.with_binary_diffusion(c, seed=k) for k, c in enumerate(cases.batch(12, count=5, scale=4))]
    ins = [Oracle(c).prim_to_cons() for c in cs]
    b = Batch(cs, diffusion=1)
    for i, (U, T) in enumerate(ins):
        b.set_state(i, dev(U), dev(T))
    for _ in range(2):
        b.step(0.0)
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
        Up, Tp, st, _ = gpu_steps(c, U, T, 2, diffusion=1)
        assert st == 0
        assert np.array_equal(Ug.cpu().numpy(), Up), c.name
        assert np.array_equal(Tg.cpu().numpy(), Tp), c.name
