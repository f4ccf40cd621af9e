"""ctypes binding of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Wraps ``libxfo.so`` (``xfo.h``) with numpy in/out arrays. Inputs come from the
seeded generators; nothing here computes any part of the method itself.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

MAXN = 8
KDIR = 8
FLAG_NONPHYS, FLAG_NEWTON, FLAG_EIGEN = 1, 2, 4


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int64 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", (C.c_int * 2) * 3), ("N", C.c_int), ("W", C.c_double * MAXN),
        ("T_lo", C.c_double), ("T_hi", C.c_double), ("cp", (C.c_double * 5) * MAXN),
        ("h_off", C.c_double * MAXN), ("mu", (C.c_double * 4) * MAXN),
        ("kap", (C.c_double * 4) * MAXN), ("lewis", C.c_double), ("a_ref2", C.c_double),
        ("rho_ref", C.c_double), ("L_ref", C.c_double), ("cfl", C.c_double),
        ("viscous", C.c_int), ("convective", C.c_int), ("newton_max", C.c_int),
        ("newton_rtol", C.c_double), ("weno_eps", C.c_double), ("threads", C.c_int),
        ("positivity", C.c_int), ("weno", C.c_int), ("pos_eps", C.c_double),
        ("diffusion", C.c_int), ("dbin", ((C.c_double * 4) * MAXN) * MAXN),
    ]


_lib = None


def load(path):
    """Open an oracle library at ``path`` with the argument types of xfo.h."""
    L = C.CDLL(path)
    P = C.POINTER(Params)
    dp = C.POINTER(C.c_double)
    up = C.POINTER(C.c_uint32)
    L.xfo_prim_to_cons.argtypes = [P, dp, dp, dp]
    L.xfo_cons_to_prim.argtypes = [P, dp, dp, dp, up]
    L.xfo_rhs.argtypes = [P, dp, dp, dp, up]
    L.xfo_dt.argtypes = [P, dp, dp, up]
    L.xfo_dt.restype = C.c_double
    L.xfo_step_rk3.argtypes = [P, dp, dp, C.c_double, up]
    L.xfo_step_rk3.restype = C.c_double
    L.xfo_run_to.argtypes = [P, dp, dp, C.c_double, C.c_int, up]
    L.xfo_thermo.argtypes = [P, C.c_double, dp, dp, dp, dp, dp, dp]
    L.xfo_temperature.argtypes = [P, C.c_double, dp, C.c_double, C.POINTER(C.c_int), up]
    L.xfo_temperature.restype = C.c_double
    L.xfo_eigen.argtypes = [P, C.c_int, dp, dp, C.c_double, C.c_double, dp, dp, dp, dp, up]
    L.xfo_flux.argtypes = [P, C.c_int, dp, C.c_double, dp, up]
    L.xfo_weno5.argtypes = [dp]
    L.xfo_weno5.restype = C.c_double
    L.xfo_weno_cu6.argtypes = [dp, C.c_double]
    L.xfo_weno_cu6.restype = C.c_double
    L.xfo_species_diffusion.argtypes = [P, C.c_double, C.c_double, dp, dp]
    L.xfo_weno7.argtypes = [dp, C.c_double]
    L.xfo_weno7.restype = C.c_double
    L.xfo_cu6_beta6.argtypes = [dp]
    L.xfo_cu6_beta6.restype = C.c_double
    L.xfo_transport.argtypes = [P, C.c_double, C.c_double, dp, dp, dp, dp]
    L.xfo_rhs_jvp.argtypes = [P, dp, dp, dp, dp, dp, up]
    L.xfo_rk3_jvp.argtypes = [P, dp, dp, dp, C.c_double, C.c_int, up]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def params(case, viscous=None, convective=True, threads=0, newton_max=50,
           newton_rtol=1e-13, weno_eps=1e-6, positivity=False, pos_eps=1e-13,
           weno=5, diffusion=0) -> Params:
    """Build the oracle parameter block from a generator ``Case``.
    ``diffusion``: 0 for D = kappa/(rho c_p Le) for every species, 1 for the
    mixture-averaged D_sm of Eq. 26 (needs ``species.dbin_coef``)."""
    sp = case.species
    p = Params()
    p.dim = case.dim
    for a in range(3):
        p.n[a] = case.n[a]
        p.lo[a] = case.lo[a]
        p.hi[a] = case.hi[a]
        p.bc[a][0], p.bc[a][1] = case.bc[a]
    p.N = sp.n
    for s in range(sp.n):
        p.W[s] = sp.W[s]
        p.h_off[s] = sp.h_off[s]
        for j in range(5):
            p.cp[s][j] = sp.cp_coef[s, j]
        for j in range(4):
            p.mu[s][j] = sp.mu_coef[s, j]
            p.kap[s][j] = sp.kappa_coef[s, j]
    p.T_lo, p.T_hi = sp.T_lo, sp.T_hi
    p.lewis = sp.lewis
    p.a_ref2, p.rho_ref, p.L_ref = case.a_ref2, case.rho_ref, case.L_ref
    p.cfl = case.cfl
    p.viscous = int(case.viscous if viscous is None else viscous)
    p.convective = int(convective)
    p.newton_max = newton_max
    p.newton_rtol = newton_rtol
    p.weno_eps = weno_eps
    p.threads = threads
    p.positivity = int(positivity)
    p.pos_eps = pos_eps
    p.weno = int(weno)
    p.diffusion = int(diffusion)
    if diffusion:
        if sp.dbin_coef is None:
            raise ValueError("the mixture-averaged model needs binary diffusion fits")
        for s in range(sp.n):
            for t in range(sp.n):
                for j in range(4):
                    p.dbin[s][t][j] = sp.dbin_coef[s, t, j]
    return p


class Oracle:
    """Stateless helpers around one parameter block."""

    def __init__(self, case, library=None, **kw):
        """``library``: an oracle library opened with ``load`` (default: the
        built oracle/libxfo.so)."""
        self.case = case
        self.p = params(case, **kw)
        self.nv = case.n_v
        self.cells = case.cells
        self.L = lib() if library is None else library

    def prim_to_cons(self, prim=None):
        prim = np.ascontiguousarray(self.case.prim if prim is None else prim, dtype=np.float64)
        U = np.zeros_like(prim)
        T = np.zeros(self.cells)
        assert self.L.xfo_prim_to_cons(C.byref(self.p), _p(prim), _p(U), _p(T)) == 0
        return U, T

    def cons_to_prim(self, U, T):
        U = np.ascontiguousarray(U, dtype=np.float64)
        T = np.array(T, dtype=np.float64)
        P = np.zeros_like(U)
        st = C.c_uint32(0)
        assert self.L.xfo_cons_to_prim(C.byref(self.p), _p(U), _p(T), _p(P), C.byref(st)) == 0
        return P, T, st.value

    def rhs(self, U, T):
        """Returns (dU/dt, recovered T, status)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        T = np.array(T, dtype=np.float64)
        R = np.zeros_like(U)
        st = C.c_uint32(0)
        assert self.L.xfo_rhs(C.byref(self.p), _p(U), _p(T), _p(R), C.byref(st)) == 0
        return R, T, st.value

    def dt(self, U, T):
        U = np.ascontiguousarray(U, dtype=np.float64)
        T = np.array(T, dtype=np.float64)
        st = C.c_uint32(0)
        return self.L.xfo_dt(C.byref(self.p), _p(U), _p(T), C.byref(st))

    def step(self, U, T, dt=0.0):
        """One RK3 step in place; returns (dt used, status)."""
        st = C.c_uint32(0)
        d = self.L.xfo_step_rk3(C.byref(self.p), _p(U), _p(T), float(dt), C.byref(st))
        return d, st.value

    def run_to(self, U, T, t_end, max_steps=100000):
        st = C.c_uint32(0)
        n = self.L.xfo_run_to(C.byref(self.p), _p(U), _p(T), float(t_end), int(max_steps),
                              C.byref(st))
        return n, st.value

    def eigen(self, d, UL, UR, TL, TR):
        nv = self.nv
        L = np.zeros((nv, nv)); R = np.zeros((nv, nv)); lam = np.zeros(nv); c2 = np.zeros(1)
        st = C.c_uint32(0)
        assert self.L.xfo_eigen(C.byref(self.p), d, _p(np.ascontiguousarray(UL)),
                                _p(np.ascontiguousarray(UR)), TL, TR, _p(L), _p(R), _p(lam),
                                _p(c2), C.byref(st)) == 0
        return L, R, lam, c2[0], st.value

    def flux(self, d, U1, T):
        F = np.zeros(self.nv)
        st = C.c_uint32(0)
        assert self.L.xfo_flux(C.byref(self.p), d, _p(np.ascontiguousarray(U1, dtype=np.float64)),
                               float(T), _p(F), C.byref(st)) == 0
        return F

    def thermo(self, T, Y):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        e, cv, cp = np.zeros(1), np.zeros(1), np.zeros(1)
        es, hs = np.zeros(MAXN), np.zeros(MAXN)
        self.L.xfo_thermo(C.byref(self.p), float(T), _p(Y), _p(e), _p(cv), _p(cp), _p(es), _p(hs))
        return e[0], cv[0], cp[0], es[:len(Y)], hs[:len(Y)]

    def temperature(self, e, Y, T0):
        it = C.c_int(0)
        st = C.c_uint32(0)
        T = self.L.xfo_temperature(C.byref(self.p), float(e),
                                   _p(np.ascontiguousarray(Y, dtype=np.float64)), float(T0),
                                   C.byref(it), C.byref(st))
        return T, it.value, st.value

    def transport(self, T, rho, Y):
        mu, ka, D = np.zeros(1), np.zeros(1), np.zeros(1)
        self.L.xfo_transport(C.byref(self.p), float(T), float(rho),
                             _p(np.ascontiguousarray(Y, dtype=np.float64)), _p(mu), _p(ka), _p(D))
        return mu[0], ka[0], D[0]

    def species_diffusion(self, T, rho, Y):
        """Per-species D_s (dimensionless) of the selected diffusion model."""
        Ds = np.zeros(self.case.n_species)
        rc = self.L.xfo_species_diffusion(C.byref(self.p), float(T), float(rho),
                                          _p(np.ascontiguousarray(Y, dtype=np.float64)), _p(Ds))
        assert rc == 0
        return Ds

    def rhs_jvp(self, U, V, T):
        """V: [k <= KDIR, n_v*cells] tangents; returns (dU/dt, J V[k], T, status)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        k = V.shape[0]
        Vp = np.zeros((KDIR, U.size))
        Vp[:k] = V.reshape(k, -1)
        T = np.array(T, dtype=np.float64)
        R = np.zeros_like(U)
        JV = np.zeros_like(Vp)
        st = C.c_uint32(0)
        assert self.L.xfo_rhs_jvp(C.byref(self.p), _p(U), _p(Vp), _p(T), _p(R), _p(JV),
                                  C.byref(st)) == 0
        return R, JV[:k].reshape((k,) + U.shape), T, st.value

    def rk3_jvp(self, U, V, T, dt, steps):
        """March ``steps`` fixed-dt RK3 steps with tangents; returns (U, V, T, status)."""
        U = np.array(U, dtype=np.float64)
        k = V.shape[0]
        Vp = np.zeros((KDIR, U.size))
        Vp[:k] = V.reshape(k, -1)
        T = np.array(T, dtype=np.float64)
        st = C.c_uint32(0)
        assert self.L.xfo_rk3_jvp(C.byref(self.p), _p(U), _p(Vp), _p(T), float(dt), int(steps),
                                  C.byref(st)) == 0
        return U, Vp[:k].reshape((k,) + U.shape), T, st.value


def weno5(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().xfo_weno5(_p(f))


def weno_cu6(f, eps=1e-6) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().xfo_weno_cu6(_p(f), eps)


def weno7(f, eps=1e-6) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().xfo_weno7(_p(f), eps)


def cu6_beta6(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().xfo_cu6_beta6(_p(f))
