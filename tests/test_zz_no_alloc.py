"""The allocation-free RHS entry point against the regular one.

xf_rhs_static serves callers that may not allocate device memory (a host whose
device memory all belongs to its own pool or caching allocator, or a loop where
an allocation would stall the device): its scratch is one fixed array inside
the library. It launches the same kernels as xf_rhs on the same inputs, so its
results must be bitwise those of xf_rhs. This file is collected last so that a
failure here stops a first-failure run only after every other test has run. It
passes alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle

from gpu_util import gpu_rhs, dev

pytestmark = pytest.mark.gpu


def _inputs(case, **kw):
    o = Oracle(case, **kw)
    U, T = o.prim_to_cons()
    return U, T


def _static_rhs(case, U, T, **kw):
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import rhs_static
    Ud, Td = dev(U), dev(T)
    R = torch.full_like(Ud, float("nan"))
    flags = rhs_static(case, Ud, R, Td, **kw)
    torch.cuda.synchronize()
    return R.cpu().numpy(), flags


def _two_in_a_row(first, second, **kw):
    """Two different grids back to back: the second call must not see stale
    scratch from the first (status word and accumulators are cleared per call)."""
    for case in (first, second):
        U, T = _inputs(case, diffusion=kw.get("diffusion", 0))
        R_ref, _, st_ref = gpu_rhs(case, U, T, **kw)
        R, st = _static_rhs(case, U, T, **kw)
        assert np.array_equal(R, R_ref), case.name
        assert st == st_ref == 0


def test_two_calls_in_a_row_match_the_regular_entry_point():
    _two_in_a_row(cases.config(1, n=(96, 48)),          # 2D, 3 species, viscous
                  cases.config(2, n=(24, 16, 12)))      # 3D, 5 species, viscous


def test_weno7_four_ghost_layers_match_the_regular_entry_point():
    _two_in_a_row(cases.config(2, n=(20, 16, 12)), cases.config(1, n=(64, 40)), weno=7)


def test_mixture_averaged_diffusion_matches_the_regular_entry_point():
    # the mixture-averaged model stores N more per-cell fields in the scratch
    _two_in_a_row(cases.with_binary_diffusion(cases.config(2, n=(20, 16, 12)), seed=1),
                  cases.with_binary_diffusion(cases.config(1, n=(80, 40)), seed=2),
                  diffusion=1)


def test_repeated_calls_allocate_no_device_memory():
    """After a first call (which may load the library's kernels, and with them
    the array, on this device), further calls leave the device's free memory
    and the torch allocator's statistics unchanged."""
    import torch
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300.xf import rhs_static
    case = cases.config(2, n=(24, 16, 12))
    U, T = _inputs(case)
    Ud, Td = dev(U), dev(T)
    R = torch.empty_like(Ud)
    rhs_static(case, Ud, R, Td)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        rhs_static(case, Ud, R, Td, flags=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0


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


def test_host_pointers_are_rejected_with_their_own_message():
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300 import xf
    case = cases.config(1, n=(32, 16))
    U = np.zeros((case.n_v, case.cells))
    R = np.zeros_like(U)
    g, t, o, keep = xf.structs(case)
    code = xf.lib.xf_rhs_static(C.byref(g), C.byref(t), C.byref(o),
                                U.ctypes.data_as(C.c_void_p), None, R.ctypes.data_as(C.c_void_p),
                                None, xf.stream_ptr())
    assert code == xf.XF_ERR_ARG
    assert "device pointers" in xf.lib.xf_last_error().decode()
