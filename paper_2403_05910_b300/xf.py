"""ctypes binding of the C-ABI library ``libxf.so`` (include/xf.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C-ABI. Device memory and streams come from PyTorch. There
is no CPU fallback: if the library cannot be loaded, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxf.so")

(XF_OK, XF_ERR_ARG, XF_ERR_CUDA, XF_ERR_NONPHYS, XF_ERR_NEWTON, XF_ERR_EIGEN, XF_ERR_TIMEOUT,
 XF_ERR_OOM) = range(8)
FLAG_NONPHYS, FLAG_NEWTON, FLAG_EIGEN, FLAG_TIMEOUT = 1, 2, 4, 8
BC_TRANSMISSIVE, BC_PERIODIC, BC_SYMMETRIC = 0, 1, 2


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("bc", (C.c_int * 2) * 3)]


class Thermo(C.Structure):
    _fields_ = [("n_species", C.c_int), ("W", C.POINTER(C.c_double)), ("T_lo", C.c_double),
                ("T_hi", C.c_double), ("cp_coef", C.POINTER(C.c_double)),
                ("h_off", C.POINTER(C.c_double)), ("mu_coef", C.POINTER(C.c_double)),
                ("kappa_coef", C.POINTER(C.c_double)), ("lewis", C.c_double),
                ("a_ref2", C.c_double), ("rho_ref", C.c_double), ("L_ref", C.c_double),
                ("dbin_coef", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("cfl", C.c_double), ("weno", C.c_int), ("split", C.c_int), ("viscous", C.c_int),
                ("convective", C.c_int), ("newton_max", C.c_int), ("newton_rtol", C.c_double),
                ("weno_eps", C.c_double), ("positivity", C.c_int), ("pos_eps", C.c_double),
                ("diffusion", C.c_int)]


# every symbol declared in include/xf.h
EXPORTS = ["xf_create", "xf_destroy", "xf_nv", "xf_cells", "xf_set_state", "xf_set_primitive",
           "xf_get_state", "xf_rhs", "xf_compute_dt", "xf_step_rk3", "xf_step_rk3_n",
           "xf_step_rk3_host",
           "xf_get_status",
           "xf_clear_status", "xf_status_str", "xf_last_error", "xf_profile_enable",
           "xf_profile_read", "xf_probe_fp64", "xf_probe_rcp", "xf_probe_exp", "xf_probe_log", "xf_rhs_static", "xf_rhs_static_capacity_bytes",
           "xf_batch_create", "xf_batch_destroy", "xf_batch_size", "xf_batch_set_primitive",
           "xf_batch_set_state", "xf_batch_get_state", "xf_batch_step_rk3", "xf_batch_autotune",
           "xf_batch_config", "xf_batch_get_status", "xf_barrier_probe", "xf_batch_uses_graph",
           "xf_batch_num_candidates", "xf_rhs_adjoint", "xf_step_rk3_adjoint",
           "xf_step_rk3_tape", "xf_step_rk3_adjoint_tape", "xf_tape_flux_len",
           "xf_step_rk3_tape_flux", "xf_step_rk3_adjoint_tape_flux", "xf_objective_mixing",
           "xf_set_primitive_adjoint"]
PROF_SLOTS = 10
PROF_NAMES = ["prim", "dt", "grad", "face_x", "face_y", "face_z", "update", "face_adj", "prim_adj",
              "spare"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libxf.so is not built ({LIB_PATH}); run paper_2403_05910_b300/build.py")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    L.xf_create.argtypes = [C.POINTER(Grid), C.POINTER(Thermo), C.POINTER(Opts), C.POINTER(vp)]
    L.xf_destroy.argtypes = [vp]
    L.xf_destroy.restype = None
    L.xf_nv.argtypes = [vp]
    L.xf_cells.argtypes = [vp]
    L.xf_cells.restype = C.c_int64
    L.xf_set_state.argtypes = [vp, vp, vp, vp]
    L.xf_set_primitive.argtypes = [vp, vp, vp]
    L.xf_get_state.argtypes = [vp, vp, vp, vp]
    L.xf_rhs.argtypes = [vp, vp, vp, vp]
    L.xf_compute_dt.argtypes = [vp, vp, vp]
    L.xf_step_rk3.argtypes = [vp, C.c_double, vp, vp]
    L.xf_step_rk3_n.argtypes = [vp, C.c_int, C.c_double, vp]
    L.xf_step_rk3_host.argtypes = [vp, vp, vp, vp, vp, C.c_double, vp, vp]
    L.xf_get_status.argtypes = [vp, C.POINTER(C.c_uint32), vp]
    L.xf_clear_status.argtypes = [vp, vp]
    L.xf_status_str.argtypes = [C.c_int]
    L.xf_status_str.restype = C.c_char_p
    L.xf_last_error.restype = C.c_char_p
    L.xf_profile_enable.argtypes = [vp, C.c_int]
    L.xf_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.xf_probe_fp64.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_double)]
    L.xf_probe_rcp.argtypes = [vp, vp, vp, C.c_int64, vp]
    L.xf_probe_exp.argtypes = [vp, vp, vp, C.c_int64, vp]
    L.xf_probe_log.argtypes = [vp, vp, vp, C.c_int64, vp]
    L.xf_rhs_static.argtypes = [C.POINTER(Grid), C.POINTER(Thermo), C.POINTER(Opts), vp, vp, vp,
                                C.POINTER(C.c_uint32), vp]
    L.xf_rhs_static_capacity_bytes.restype = C.c_int64
    L.xf_rhs_adjoint.argtypes = [vp, vp, vp, vp, vp]
    L.xf_step_rk3_adjoint.argtypes = [vp, C.c_double, vp, vp]
    L.xf_step_rk3_tape.argtypes = [vp, C.c_double, vp, vp, vp]
    L.xf_step_rk3_adjoint_tape.argtypes = [vp, C.c_double, vp, vp, vp, vp]
    L.xf_tape_flux_len.argtypes = [vp]
    L.xf_tape_flux_len.restype = C.c_int64
    L.xf_step_rk3_tape_flux.argtypes = [vp, C.c_double, vp, vp, vp, vp]
    L.xf_step_rk3_adjoint_tape_flux.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp]
    L.xf_objective_mixing.argtypes = [vp, vp, C.c_int, vp, vp, vp]
    L.xf_set_primitive_adjoint.argtypes = [vp, vp, vp, vp, vp]
    L.xf_batch_create.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(Thermo), C.POINTER(Opts),
                                  C.POINTER(vp)]
    L.xf_batch_destroy.argtypes = [vp]
    L.xf_batch_destroy.restype = None
    L.xf_batch_size.argtypes = [vp]
    L.xf_batch_uses_graph.argtypes = [vp]
    L.xf_batch_set_primitive.argtypes = [vp, C.c_int, vp, vp]
    L.xf_batch_set_state.argtypes = [vp, C.c_int, vp, vp, vp]
    L.xf_batch_get_state.argtypes = [vp, C.c_int, vp, vp, vp]
    L.xf_batch_step_rk3.argtypes = [vp, C.c_double, vp]
    L.xf_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float), vp]
    L.xf_batch_config.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]
    L.xf_batch_get_status.argtypes = [vp, C.c_int, C.POINTER(C.c_uint32), vp]
    L.xf_barrier_probe.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_uint32)]
    return L


lib = _load()


class XFError(RuntimeError):
    def __init__(self, code, what=""):
        msg = lib.xf_status_str(code).decode()
        if code == XF_ERR_CUDA:
            msg += ": " + lib.xf_last_error().decode()
        super().__init__(f"{what}: {msg}" if what else msg)
        self.code = code


def check(code, what=""):
    if code != XF_OK:
        raise XFError(code, what)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def structs(case, viscous=None, convective=True, cfl=None, newton_max=50, newton_rtol=1e-13,
            weno_eps=1e-6, positivity=False, pos_eps=1e-13, weno=5, diffusion=0):
    """(Grid, Thermo, Opts, keepalive) from a generator ``Case``. ``weno``: 5
    for WENO5-JS, 6 for WENO-CU6, 7 for WENO7-JS. ``diffusion``: 0 for a
    common D = kappa/(rho c_p Le), 1 for the mixture-averaged D_sm of Eq. 26
    (the species need binary diffusion fits)."""
    g = Grid()
    g.dim = case.dim
    for a in range(3):
        g.n[a] = case.n[a]
        g.lo[a] = case.lo[a]
        g.hi[a] = case.hi[a]
        g.bc[a][0], g.bc[a][1] = case.bc[a]
    sp = case.species
    keep = [np.ascontiguousarray(sp.W, dtype=np.float64),
            np.ascontiguousarray(sp.cp_coef, dtype=np.float64),
            np.ascontiguousarray(sp.h_off, dtype=np.float64),
            np.ascontiguousarray(sp.mu_coef, dtype=np.float64),
            np.ascontiguousarray(sp.kappa_coef, dtype=np.float64)]
    t = Thermo()
    t.n_species = sp.n
    t.W, t.cp_coef, t.h_off, t.mu_coef, t.kappa_coef = (_dptr(k) for k in keep)
    t.T_lo, t.T_hi = sp.T_lo, sp.T_hi
    t.lewis = sp.lewis
    t.a_ref2, t.rho_ref, t.L_ref = case.a_ref2, case.rho_ref, case.L_ref
    if sp.dbin_coef is not None:
        keep.append(np.ascontiguousarray(sp.dbin_coef, dtype=np.float64))
        t.dbin_coef = _dptr(keep[-1])
    elif diffusion:
        raise ValueError("the mixture-averaged model needs binary diffusion fits")
    o = Opts()
    o.cfl = case.cfl if cfl is None else cfl
    o.weno = int(weno)
    o.split = 0
    o.viscous = int(case.viscous if viscous is None else viscous)
    o.convective = int(convective)
    o.newton_max = newton_max
    o.newton_rtol = newton_rtol
    o.weno_eps = weno_eps
    o.positivity = int(positivity)
    o.pos_eps = pos_eps
    o.diffusion = int(diffusion)
    return g, t, o, keep


def stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def ptr(x):
    """Raw address of a torch tensor or numpy array (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(x.data_ptr())


class Solver:
    """One grid's solver state behind an ``xf_handle``.

    Arguments are torch float64 tensors (CUDA, or CPU for the host-or-device
    entry points) or numpy arrays where the C-ABI accepts host memory.
    """

    def __init__(self, case, **kw):
        g, t, o, keep = structs(case, **kw)
        self.case = case
        self.nv = case.n_v
        self.cells = case.cells
        self.positivity = bool(kw.get("positivity", False))
        h = C.c_void_p()
        check(lib.xf_create(C.byref(g), C.byref(t), C.byref(o), C.byref(h)), "xf_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.xf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, U, T=None, stream=None):
        check(lib.xf_set_state(self.h, ptr(U), ptr(T), stream_ptr(stream)), "xf_set_state")

    def set_primitive(self, P, stream=None):
        check(lib.xf_set_primitive(self.h, ptr(P), stream_ptr(stream)), "xf_set_primitive")

    def get_state(self, U=None, T=None, stream=None):
        check(lib.xf_get_state(self.h, ptr(U), ptr(T), stream_ptr(stream)), "xf_get_state")

    def rhs(self, U, dUdt, stream=None):
        check(lib.xf_rhs(self.h, ptr(U), ptr(dUdt), stream_ptr(stream)), "xf_rhs")

    def compute_dt(self, dt_dev, stream=None):
        check(lib.xf_compute_dt(self.h, ptr(dt_dev), stream_ptr(stream)), "xf_compute_dt")

    def step(self, dt=0.0, dt_dev=None, stream=None):
        check(lib.xf_step_rk3(self.h, float(dt), ptr(dt_dev), stream_ptr(stream)), "xf_step_rk3")

    def step_host(self, U_in, T_in, U_out, T_out=None, dt=0.0, dt_dev=None, stream=None):
        """One RK3 step of a host-resident state (pinned host buffers overlap
        the copies with compute); U_out may be U_in."""
        check(lib.xf_step_rk3_host(self.h, ptr(U_in), ptr(T_in), ptr(U_out), ptr(T_out),
                                   float(dt), ptr(dt_dev), stream_ptr(stream)), "xf_step_rk3_host")

    def steps(self, n, dt=0.0, stream=None):
        """n RK3 steps replayed from a captured CUDA graph (dt <= 0: CFL)."""
        check(lib.xf_step_rk3_n(self.h, int(n), float(dt), stream_ptr(stream)), "xf_step_rk3_n")

    def status(self, stream=None):
        f = C.c_uint32(0)
        code = lib.xf_get_status(self.h, C.byref(f), stream_ptr(stream))
        if code == XF_ERR_CUDA:
            check(code, "xf_get_status")
        return f.value

    def clear_status(self, stream=None):
        check(lib.xf_clear_status(self.h, stream_ptr(stream)), "xf_clear_status")

    def rhs_adjoint(self, U, dUdt_bar, U_bar, stream=None):
        """U_bar += (dL/dU)^T dUdt_bar at U (device tensors)."""
        check(lib.xf_rhs_adjoint(self.h, ptr(U), ptr(dUdt_bar), ptr(U_bar), stream_ptr(stream)),
              "xf_rhs_adjoint")

    def step_adjoint(self, dt, U_bar, stream=None):
        """Reverse of one fixed-dt RK3 step from the current state (U_bar in/out)."""
        check(lib.xf_step_rk3_adjoint(self.h, float(dt), ptr(U_bar), stream_ptr(stream)),
              "xf_step_rk3_adjoint")

    def step_tape(self, dt, U1, U2, stream=None, Fhat=None):
        """One fixed-dt RK3 step that also writes its stage states U1, U2 (and,
        with Fhat, the unblended convective face fluxes of its stages)."""
        if Fhat is None:
            check(lib.xf_step_rk3_tape(self.h, float(dt), ptr(U1), ptr(U2), stream_ptr(stream)),
                  "xf_step_rk3_tape")
        else:
            check(lib.xf_step_rk3_tape_flux(self.h, float(dt), ptr(U1), ptr(U2), ptr(Fhat),
                                            stream_ptr(stream)), "xf_step_rk3_tape_flux")

    def step_adjoint_tape(self, dt, U1, U2, U_bar, stream=None, Fhat=None):
        """step_adjoint with the stage states of step_tape given (U_bar in/out),
        and with its flux tape when Fhat is given."""
        if Fhat is None:
            check(lib.xf_step_rk3_adjoint_tape(self.h, float(dt), ptr(U1), ptr(U2), ptr(U_bar),
                                               stream_ptr(stream)), "xf_step_rk3_adjoint_tape")
        else:
            check(lib.xf_step_rk3_adjoint_tape_flux(self.h, float(dt), ptr(U1), ptr(U2),
                                                    ptr(Fhat), ptr(U_bar), stream_ptr(stream)),
                  "xf_step_rk3_adjoint_tape_flux")

    def tape_flux_len(self):
        """Doubles of one step's flux tape (step_tape with Fhat)."""
        return int(lib.xf_tape_flux_len(self.h))

    def objective_mixing(self, U, species, J_dev, U_bar, stream=None):
        check(lib.xf_objective_mixing(self.h, ptr(U), int(species), ptr(J_dev), ptr(U_bar),
                                      stream_ptr(stream)), "xf_objective_mixing")

    def set_primitive_adjoint(self, P, U_bar, P_bar, stream=None):
        check(lib.xf_set_primitive_adjoint(self.h, ptr(P), ptr(U_bar), ptr(P_bar), stream_ptr(stream)),
              "xf_set_primitive_adjoint")

    def profile(self, on=True):
        check(lib.xf_profile_enable(self.h, int(on)), "xf_profile_enable")

    def profile_read(self):
        """{kernel class: (total ms, launches)} since the last read."""
        ms = (C.c_double * PROF_SLOTS)()
        n = (C.c_int64 * PROF_SLOTS)()
        check(lib.xf_profile_read(self.h, ms, n), "xf_profile_read")
        return {PROF_NAMES[k]: (ms[k], n[k]) for k in range(PROF_SLOTS) if n[k]}


def probe_fp64(iters=20000, blocks_per_sm=8):
    """Measured FP64 FMA throughput (TFLOP/s) of the current device."""
    t = C.c_double(0.0)
    check(lib.xf_probe_fp64(int(iters), int(blocks_per_sm), C.byref(t)), "xf_probe_fp64")
    return t.value


def probe_rcp(x, y, ref, stream=None):
    """y = the kernels' reciprocal of x, ref = 1.0 / x (device float64 tensors)."""
    check(lib.xf_probe_rcp(ptr(x), ptr(y), ptr(ref), int(x.numel()), stream_ptr(stream)),
          "xf_probe_rcp")


def probe_exp(x, y, ref, stream=None):
    """y = the kernels' exponential of x, ref = CUDA's exp(x) (device float64 tensors)."""
    check(lib.xf_probe_exp(ptr(x), ptr(y), ptr(ref), int(x.numel()), stream_ptr(stream)),
          "xf_probe_exp")


def probe_log(x, y, ref, stream=None):
    """y = the kernels' logarithm of x, ref = CUDA's log(x) (device float64 tensors)."""
    check(lib.xf_probe_log(ptr(x), ptr(y), ptr(ref), int(x.numel()), stream_ptr(stream)),
          "xf_probe_log")


def rhs_static(case, U, dUdt, T=None, flags=True, stream=None, **kw):
    """dUdt = L(U) through the allocation-free entry point (no handle, no
    device allocation; scratch is the library's fixed device array). Returns
    the status bits when ``flags`` is true (that synchronises the stream)."""
    g, t, o, keep = structs(case, **kw)
    f = C.c_uint32(0)
    check(lib.xf_rhs_static(C.byref(g), C.byref(t), C.byref(o), ptr(U), ptr(T), ptr(dUdt),
                            C.byref(f) if flags else None, stream_ptr(stream)), "xf_rhs_static")
    return f.value if flags else None


def rhs_static_capacity_bytes():
    return int(lib.xf_rhs_static_capacity_bytes())


class Batch:
    """Many 2D instances advanced together (xf_batch_*)."""

    def __init__(self, case_list, **kw):
        self.cases = list(case_list)
        n = len(self.cases)
        gs, ts, os_ = (Grid * n)(), (Thermo * n)(), (Opts * n)()
        self._keep = []
        for i, c in enumerate(self.cases):
            g, t, o, keep = structs(c, **kw)
            gs[i], ts[i], os_[i] = g, t, o
            self._keep.append(keep)
        self._structs = (gs, ts, os_)
        h = C.c_void_p()
        check(lib.xf_batch_create(n, gs, ts, os_, C.byref(h)), "xf_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.xf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitive(self, i, P, stream=None):
        check(lib.xf_batch_set_primitive(self.h, i, ptr(P), stream_ptr(stream)), "xf_batch_set_primitive")

    def set_state(self, i, U, T=None, stream=None):
        check(lib.xf_batch_set_state(self.h, i, ptr(U), ptr(T), stream_ptr(stream)), "xf_batch_set_state")

    def get_state(self, i, U=None, T=None, stream=None):
        check(lib.xf_batch_get_state(self.h, i, ptr(U), ptr(T), stream_ptr(stream)), "xf_batch_get_state")

    def step(self, dt=0.0, stream=None):
        check(lib.xf_batch_step_rk3(self.h, float(dt), stream_ptr(stream)), "xf_batch_step_rk3")

    def uses_graph(self):
        return bool(lib.xf_batch_uses_graph(self.h))

    def autotune(self, steps=1, stream=None, report=False):
        """Pick the fastest launch shape; returns its index (and, with
        ``report``, the ms per step of every candidate)."""
        k = C.c_int(0)
        nc = lib.xf_batch_num_candidates()
        ms = (C.c_float * nc)()
        check(lib.xf_batch_autotune(self.h, int(steps), C.byref(k), ms, stream_ptr(stream)),
              "xf_batch_autotune")
        return (k.value, list(ms)) if report else k.value

    def config(self, choice=-1):
        bt, tw, th = C.c_int(), C.c_int(), C.c_int()
        check(lib.xf_batch_config(self.h, int(choice), C.byref(bt), C.byref(tw), C.byref(th)),
              "xf_batch_config")
        return bt.value, tw.value, th.value

    def status(self, i=-1, stream=None):
        f = C.c_uint32(0)
        code = lib.xf_batch_get_status(self.h, int(i), C.byref(f), stream_ptr(stream))
        if code == XF_ERR_CUDA:
            check(code, "xf_batch_get_status")
        return f.value


def barrier_probe(timeout_cycles, extra_arrivals):
    """Status bits of one bounded grid barrier (see xf_barrier_probe)."""
    f = C.c_uint32(0)
    code = lib.xf_barrier_probe(int(timeout_cycles), int(extra_arrivals), C.byref(f))
    if code == XF_ERR_CUDA:
        check(code, "xf_barrier_probe")
    return f.value
