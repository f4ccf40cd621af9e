"""Helpers shared by the GPU tests: run the CUDA path through the C-ABI and
compare with the oracle field by field."""
import numpy as np


def field_err(gpu, ref, dim=None, mom_floor=0.0):
    """Per-field max |gpu - ref| / max |ref| (the parity metric).

    With ``dim`` given, the momentum rows 1..dim share one scale, the largest
    momentum magnitude: a component that vanishes in exact arithmetic (v in a
    y-uniform planar shock) carries only round-off of the momentum flux and
    has no scale of its own. ``mom_floor`` bounds that scale from below, for
    states at rest whose momentum is round-off altogether."""
    ref = np.asarray(ref)
    gpu = np.asarray(gpu).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    scale = np.max(np.abs(ref), axis=1)
    if dim:
        scale[1:1 + dim] = max(np.max(scale[1:1 + dim]), mom_floor)
    scale = np.maximum(scale, 1e-300)
    return np.max(np.abs(gpu - ref), axis=1) / scale


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_solver(case, **kw):
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import Solver
    return Solver(case, **kw)


def gpu_rhs(case, U, T, **kw):
    import torch
    s = gpu_solver(case, **kw)
    Ud, Td = dev(U), dev(T)
    s.set_state(Ud, Td)
    R = torch.empty_like(Ud)
    s.rhs(Ud, R)
    torch.cuda.synchronize()
    st = s.status()
    T_out = torch.empty_like(Td)
    s.get_state(None, T_out)
    torch.cuda.synchronize()
    out = R.cpu().numpy(), T_out.cpu().numpy(), st
    s.close()
    return out


def gpu_steps(case, U, T, steps, dt=0.0, **kw):
    """Run ``steps`` RK3 steps (dt <= 0: CFL); returns (U, T, status, dts)."""
    import torch
    s = gpu_solver(case, **kw)
    s.set_state(dev(U), dev(T))
    dtd = torch.zeros(1, dtype=torch.float64, device="cuda")
    dts = []
    for _ in range(steps):
        s.step(dt, dtd)
        dts.append(float(dtd.item()))
    Uo = torch.empty((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    To = torch.empty(case.cells, dtype=torch.float64, device="cuda")
    s.get_state(Uo, To)
    torch.cuda.synchronize()
    st = s.status()
    s.close()
    return Uo.cpu().numpy(), To.cpu().numpy(), st, dts
