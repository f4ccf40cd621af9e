"""The allocation-free RHS entry point against the regular one.

xf_rhs_static serves callers that may not allocate device memory (a host whose
device memory all belongs to its own pool or caching allocator, or a loop where
an allocation would stall the device): its scratch is one fixed array inside
the library. This file is collected last so that a failure here stops a
first-failure run only after every other test has run. It passes alone in a
fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import field_err, gpu_rhs, dev

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-11  # the RHS parity tolerance of the other GPU tests


def _inputs(case):
    o = Oracle(case)
    U, T = o.prim_to_cons()
    return U, T


def _static_rhs(case, U, T):
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import rhs_static
    Ud, Td = dev(U), dev(T)
    R = torch.full_like(Ud, float("nan"))
    flags = rhs_static(case, Ud, R, Td)
    torch.cuda.synchronize()
    return R.cpu().numpy(), flags


def test_two_calls_in_a_row_match_the_regular_entry_point():
    # two different grids back to back: the second call must not see stale
    # scratch from the first (status word and accumulators are cleared per call)
    first = cases.config(1, n=(96, 48))                  # 2D, 3 species, viscous
    second = cases.config(2, n=(24, 16, 12))              # 3D, 5 species, viscous
    for case in (first, second):
        U, T = _inputs(case)
        R_ref, _, st_ref = gpu_rhs(case, U, T)
        R, st = _static_rhs(case, U, T)
        err = field_err(R, R_ref, case.dim)
        assert np.max(err) <= TOL_RHS, (case.name, err)
        assert st == st_ref == 0


def test_oversize_grid_is_rejected_with_a_clear_message():
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300 import xf
    import torch
    case = cases.config(2, n=(64, 64, 64))
    cap = xf.rhs_static_capacity_bytes()
    assert cap == 32 * 1024 * 1024
    U = torch.zeros((case.n_v, case.cells), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    g, t, o, keep = xf.structs(case)
    code = xf.lib.xf_rhs_static(C.byref(g), C.byref(t), C.byref(o), xf.ptr(U), None, xf.ptr(R),
                                None, xf.stream_ptr())
    assert code == xf.XF_ERR_ARG
    msg = xf.lib.xf_last_error().decode()
    assert "needs" in msg and str(cap) in msg
