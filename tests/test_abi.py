"""The C-ABI library loads and exports every entry point declared in include/
(CPU only: no compute call runs). Argument validation returns XF_ERR_ARG
before any device work, so it is checked here as well."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(xf_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2403_05910_b300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2403_05910_b300 import build
    build.build()
    from paper_2403_05910_b300 import xf
    assert set(xf.EXPORTS) == _declared()


def test_argument_errors_need_no_device():
    from paper_2403_05910_b300 import build, cases
    build.build()
    from paper_2403_05910_b300 import xf
    c = cases.shock_tube(0, n=16)
    good = xf.structs(c)
    h = C.c_void_p()
    # a bad option, a bad grid and a bad species count are all rejected up front
    for bad in (4, 8):
        g, t, o, keep = xf.structs(c)
        o.weno = bad
        assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    g.n[0] = 2
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    t.n_species = 6
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    g.bc[0][0], g.bc[0][1] = xf.BC_PERIODIC, xf.BC_TRANSMISSIVE
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    # a grid whose padded block would exceed the 2^31-cell index range, a
    # zero-sized axis and an out-of-range dimension
    g, t, o, keep = xf.structs(c)
    g.dim, g.n[0], g.n[1], g.n[2] = 3, 2048, 1024, 1024
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    g.n[0] = 0
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    g.dim = 4
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    # WENO7 needs four cells per axis; the mixture-averaged model needs fits
    g, t, o, keep = xf.structs(cases.shock_tube(0, n=3))
    o.weno = 7
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    g, t, o, keep = xf.structs(c)
    o.viscous, o.diffusion = 1, 1
    t.mu_coef, t.kappa_coef = keep[3].ctypes.data_as(C.POINTER(C.c_double)), keep[4].ctypes.data_as(C.POINTER(C.c_double))
    assert xf.lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)) == xf.XF_ERR_ARG
    assert xf.lib.xf_step_rk3(None, 0.0, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_rhs(None, None, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_step_rk3_tape(None, 1e-3, None, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_step_rk3_host(None, None, None, None, None, 0.0, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_rcp(None, None, None, 16, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_rcp(None, None, None, -1, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_exp(None, None, None, 16, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_exp(None, None, None, -1, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_log(None, None, None, 16, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_probe_log(None, None, None, -1, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_step_rk3_adjoint_tape(None, 1e-3, None, None, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_tape_flux_len(None) == -1
    assert xf.lib.xf_step_rk3_tape_flux(None, 1e-3, None, None, None, None) == xf.XF_ERR_ARG
    assert xf.lib.xf_step_rk3_adjoint_tape_flux(None, 1e-3, None, None, None, None,
                                                None) == xf.XF_ERR_ARG
    assert xf.lib.xf_status_str(xf.XF_ERR_NEWTON).decode().startswith("temperature")
    del good
