"""Parity at the full workload sizes, in the launch configuration bench.py uses.

The CUDA path runs the whole grid; the oracle runs windows of it. A cell's RHS
depends on cells at most 3 away along each axis (6-point WENO stencil, 4-point
viscous faces with +-2 tangential derivatives), so one RHS needs a margin of 3
and one RK3 step (three stages) a margin of 9. Where a window reaches the
domain edge it keeps the domain's boundary condition; elsewhere its margin
makes the window's own (transmissive) boundary irrelevant to its core cells.
"""
import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import dev, gpu_solver

pytestmark = pytest.mark.gpu


def _window(case, U, T, lo, hi, margin):
    """Sub-case of cells [lo, hi) (+ margin, clipped at the domain) and its arrays.

    Returns (sub-case, U_w, T_w, core slices into the window)."""
    d = case.dim
    nn = case.n
    dx = case.dx
    wlo, whi, bc, core = [], [], [], []
    for a in range(3):
        if a >= d:
            wlo.append(0); whi.append(1); bc.append((0, 0)); core.append(slice(0, 1))
            continue
        a0 = max(lo[a] - margin, 0)
        a1 = min(hi[a] + margin, nn[a])
        wlo.append(a0); whi.append(a1)
        bc.append((case.bc[a][0] if a0 == 0 else cases.BC_TRANSMISSIVE,
                   case.bc[a][1] if a1 == nn[a] else cases.BC_TRANSMISSIVE))
        core.append(slice(lo[a] - a0, hi[a] - a0))
    n_w = tuple(whi[a] - wlo[a] for a in range(3))
    nv = case.n_v
    Ug = U.reshape(nv, nn[2], nn[1], nn[0])
    Tg = T.reshape(nn[2], nn[1], nn[0])
    sl = (slice(wlo[2], whi[2]), slice(wlo[1], whi[1]), slice(wlo[0], whi[0]))
    Uw = np.ascontiguousarray(Ug[(slice(None),) + sl].reshape(nv, -1))
    Tw = np.ascontiguousarray(Tg[sl].reshape(-1))
    sub = cases.Case(case.name + "_win", d, n_w,
                     tuple(case.lo[a] + wlo[a] * dx[a] if a < d else case.lo[a] for a in range(3)),
                     tuple(case.lo[a] + whi[a] * dx[a] if a < d else case.hi[a] for a in range(3)),
                     tuple(bc), case.species, case.a_ref2, case.rho_ref, case.L_ref,
                     case.viscous, case.cfl, np.zeros((nv, 1)))
    return sub, Uw, Tw, (core[2], core[1], core[0]), sl


def _windows(case, w):
    """Window cores: domain corners, boundary faces, the shock and the bubble."""
    nn = case.n[:case.dim]
    rng = np.random.default_rng(17)
    xs = int(case.params["x_shock"] / case.dx[0])
    xc = int(0.5 / case.dx[0])
    picks = [
        [0] * case.dim,                                  # corner at the symmetry planes
        [nn[0] - w] + [nn[a] - w for a in range(1, case.dim)],  # far corner (outflow)
        [max(xs - w // 2, 0)] + [0] * (case.dim - 1),    # shock on the symmetry plane
        [xc - w // 2] + [int(0.15 / case.dx[1]) - w // 2] * (case.dim - 1),  # bubble edge
        [int(rng.integers(0, nn[a] - w)) for a in range(case.dim)],
    ]
    out = []
    for p in picks:
        lo = [min(max(p[a], 0), nn[a] - w) for a in range(case.dim)] + [0] * (3 - case.dim)
        hi = [lo[a] + w if a < case.dim else 1 for a in range(3)]
        out.append((lo, hi))
    return out


_INPUTS = {}


def _full_inputs(case):
    """U, T of a full-size case (cached: the conversion of 33.5 M cells takes
    the oracle a while and several tests share it)."""
    key = (case.name, case.n)
    if key not in _INPUTS:
        _INPUTS[key] = Oracle(case).prim_to_cons()
    return _INPUTS[key]


def _rel(pairs, dim):
    """Parity metric over all sampled windows: per field, the largest
    |gpu - oracle| over every window divided by the largest |oracle| over every
    window (momentum rows share one scale)."""
    nv = pairs[0][1].shape[0]
    diff = np.max([np.max(np.abs(g.reshape(nv, -1) - r.reshape(nv, -1)), axis=1) for g, r in pairs], axis=0)
    sc = np.max([np.max(np.abs(r.reshape(nv, -1)), axis=1) for _, r in pairs], axis=0)
    sc[1:1 + dim] = np.max(sc[1:1 + dim])
    return diff / np.maximum(sc, 1e-300)


@pytest.mark.parametrize("cfg,w", [(1, 24), (2, 12)])
def test_fullsize_rhs_windows(cfg, w):
    import torch
    case = cases.config(cfg)
    U, T = _full_inputs(case)
    s = gpu_solver(case)
    Ud = dev(U)
    s.set_state(Ud, dev(T))
    R = torch.empty_like(Ud)
    s.rhs(Ud, R)
    torch.cuda.synchronize()
    assert s.status() == 0
    Rg = R.cpu().numpy().reshape(case.n_v, case.n[2], case.n[1], case.n[0])
    s.close()
    del Ud, R
    pairs = []
    for lo, hi in _windows(case, w):
        sub, Uw, Tw, core, sl = _window(case, U, T, lo, hi, 3)
        Rw, _, st = Oracle(sub).rhs(Uw, Tw)
        ref = Rw.reshape(case.n_v, sub.n[2], sub.n[1], sub.n[0])[(slice(None),) + core]
        got = Rg[(slice(None),) + tuple(slice(l, h) for l, h in zip(lo[::-1], hi[::-1]))]
        pairs.append((got, ref))
    err = _rel(pairs, case.dim)
    assert np.max(err) <= 1e-11, err


@pytest.mark.parametrize("cfg,w,dt", [(1, 20, 2e-4), (2, 10, 1e-4)])
def test_fullsize_one_step_windows(cfg, w, dt):
    import torch
    case = cases.config(cfg)
    U, T = _full_inputs(case)
    s = gpu_solver(case)
    s.set_state(dev(U), dev(T))
    s.step(dt)
    Uo = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    s.get_state(Uo)
    torch.cuda.synchronize()
    assert s.status() == 0
    Ug = Uo.cpu().numpy().reshape(case.n_v, case.n[2], case.n[1], case.n[0])
    s.close()
    del Uo
    pairs = []
    for lo, hi in _windows(case, w):
        sub, Uw, Tw, core, sl = _window(case, U, T, lo, hi, 9)
        o = Oracle(sub)
        Uw = Uw.copy()
        o.step(Uw, Tw, dt)
        ref = Uw.reshape(case.n_v, sub.n[2], sub.n[1], sub.n[0])[(slice(None),) + core]
        got = Ug[(slice(None),) + tuple(slice(l, h) for l, h in zip(lo[::-1], hi[::-1]))]
        pairs.append((got, ref))
    err = _rel(pairs, case.dim)
    assert np.max(err) <= 1e-11, err


@pytest.mark.parametrize("kw,margin", [({"weno": 6}, 3), ({"weno": 7}, 4),
                                       ({"diffusion": 1}, 3), ({"positivity": True}, 3)])
def test_fullsize_variants_rhs_windows(kw, margin):
    """The other options of the path on the bench's 512x256x256 workload, in
    the launch configuration of bench.py's variants leg: one RHS per option,
    compared on the sampled windows (WENO7's 8-cell stencil needs a margin of
    4; the blend does not act in a plain RHS, which must equal the unblended
    one). The binary diffusion fits come from their own RNG, so the inputs are
    the bench's."""
    import torch
    base = cases.config(2)
    case = cases.with_binary_diffusion(base) if kw.get("diffusion") else base
    U, T = _full_inputs(base)
    s = gpu_solver(case, **kw)
    Ud = dev(U)
    s.set_state(Ud, dev(T))
    R = torch.empty_like(Ud)
    s.rhs(Ud, R)
    torch.cuda.synchronize()
    assert s.status() == 0
    Rg = R.cpu().numpy().reshape(case.n_v, case.n[2], case.n[1], case.n[0])
    s.close()
    del Ud, R
    pairs = []
    for lo, hi in _windows(case, 12):
        sub, Uw, Tw, core, sl = _window(case, U, T, lo, hi, margin)
        Rw, _, st = Oracle(sub, **kw).rhs(Uw, Tw)
        ref = Rw.reshape(case.n_v, sub.n[2], sub.n[1], sub.n[0])[(slice(None),) + core]
        got = Rg[(slice(None),) + tuple(slice(l, h) for l, h in zip(lo[::-1], hi[::-1]))]
        pairs.append((got, ref))
    err = _rel(pairs, case.dim)
    assert np.max(err) <= 1e-11, err
