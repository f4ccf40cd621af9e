"""Pins of the oracle's mixture transport (Eq. 22 Wilke rule, Eq. 29 fits) and
of its CFL time step (the multi-dimensional reading of Eq. 17), each against
something other than the oracle's own formulas:

* Eq. 29 fits placed through seeded (ln T, ln mu) nodes must give back the
  node values in a pure species (this also fixes Wilke's Phi_ss = 1);
* Wilke's interaction factors, recovered from binary-mixture viscosities,
  must obey the reciprocity Phi_ts = Phi_st (mu_t/mu_s)(W_s/W_t), which any
  swapped ratio inside Phi breaks, and must predict a third binary and the
  ternary mixtures;
* relabelling the species changes nothing;
* the time step of a calorically perfect gas, whose sound speed and
  diffusivities are closed forms, is the convective or the viscous limit of
  the reading, whichever binds.

The last test plants plausible mistakes in copies of the oracle source and
checks that each one fails at least one of these pins. None needs a GPU.
"""
import math
import os
import subprocess

import numpy as np
import pytest
from scipy.optimize import least_squares

from paper_2403_05910_b300 import cases
from oracle import build as obuild
from oracle.xfo import Oracle, load

R_U = cases.R_U
RHO_REF, A_REF2, L_REF = 1.2, 101325.0 / 1.2, 0.05
MU_SCALE = RHO_REF * math.sqrt(A_REF2) * L_REF              # mu* = mu / MU_SCALE
KA_SCALE = RHO_REF * math.sqrt(A_REF2) ** 3 * L_REF        # kappa* = kappa / KA_SCALE
T_NODES = np.array([250.0, 600.0, 1500.0, 3500.0])


def _node_fit(lnT, lnv):
    """Coefficients of the cubic in ln T through four (ln T, ln value) nodes."""
    return np.linalg.solve(np.vander(lnT, 4, increasing=True), lnv)


def _species(W, seed=0):
    """Constant c_p/R per species (distinct) and Eq. 29 fits through seeded
    node values mu_n[s, k] = mu_s(T_NODES[k]), kappa_n likewise."""
    rng = np.random.default_rng(seed)
    N = len(W)
    cp = np.zeros((N, 5))
    mu, ka = np.zeros((N, 4)), np.zeros((N, 4))
    mu_n, ka_n = np.zeros((N, 4)), np.zeros((N, 4))
    for s in range(N):
        cp[s, 0] = rng.uniform(2.5, 4.5)
        mu_n[s] = np.sort(rng.uniform(1e-5, 1e-4, 4))
        ka_n[s] = np.sort(rng.uniform(1e-2, 2e-1, 4))
        mu[s] = _node_fit(np.log(T_NODES), np.log(mu_n[s]))
        ka[s] = _node_fit(np.log(T_NODES), np.log(ka_n[s]))
    sp = cases.Species(W=np.asarray(W, dtype=np.float64), cp_coef=cp, h_off=np.zeros(N),
                       mu_coef=mu, kappa_coef=ka)
    return sp, mu_n, ka_n


def _case(sp, dim=1, n=(4, 1, 1), hi=(1.0, 1.0, 1.0), prim=None, L_ref=L_REF, cfl=0.5):
    nv = dim + 2 + sp.n - 1
    if prim is None:
        prim = np.zeros((nv, int(np.prod(n))))
    return cases.Case("pin", dim, n, (0.0,) * 3, hi, ((1, 1),) * 3, sp, A_REF2, RHO_REF,
                      L_ref, True, cfl, prim)


def _Y_from_X(X, W):
    m = np.asarray(X) * np.asarray(W)
    return m / m.sum()


W3 = np.array([0.004, 0.028, 0.131])   # distinct molar masses


# ---------------------------------------------------------------- the pins --

def check_eq29_pure_species(library=None):
    """A pure species returns its own Eq. 29 values at the nodes: the fit is
    evaluated as a cubic in ln T, exponentiated, scaled to dimensionless
    units, and Wilke's rule gives mu = mu_s when X_s = 1 (Phi_ss = 1)."""
    sp, mu_n, ka_n = _species(W3, seed=1)
    o = Oracle(_case(sp), library=library)
    for s in range(sp.n):
        Y = np.eye(sp.n)[s]
        cpR = sp.cp_coef[s, 0]
        for k, T in enumerate(T_NODES):
            mu, ka, D = o.transport(T, 0.7, Y)
            assert mu * MU_SCALE == pytest.approx(mu_n[s, k], rel=1e-11)
            assert ka * KA_SCALE == pytest.approx(ka_n[s, k], rel=1e-11)
            # Lewis number one: D = kappa/(rho c_p) with c_p = (c_p/R) R_s
            cp_star = cpR * R_U / sp.W[s] / A_REF2
            assert D == pytest.approx(ka_n[s, k] / KA_SCALE / (0.7 * cp_star), rel=1e-11)


def _binary_phis(o, s, t, T, W, which):
    """Wilke factors (Phi_st, Phi_ts) recovered from the mixture value at
    three molar compositions of the s-t binary, together with the pure values
    and the misfit of a fourth composition."""
    N = len(W)

    def mix(xs):
        X = np.zeros(N)
        X[s], X[t] = xs, 1.0 - xs
        return o.transport(T, 1.0, _Y_from_X(X, W))[which]

    a_s, a_t = mix(1.0), mix(0.0)
    xs_fit = np.array([0.2, 0.5, 0.8])
    m_fit = np.array([mix(x) for x in xs_fit])

    def model(ph, xs):
        P, Q = ph
        return xs * a_s / (xs + (1 - xs) * P) + (1 - xs) * a_t / ((1 - xs) + xs * Q)

    # the fit is not convex: start from a grid and keep the best solution
    sol = min((least_squares(lambda ph: model(ph, xs_fit) / m_fit - 1.0, [P0, Q0],
                             bounds=(1e-6, np.inf), xtol=1e-15, ftol=1e-15, gtol=1e-15)
               for P0 in (0.1, 0.5, 2.0, 8.0) for Q0 in (0.1, 0.5, 2.0, 8.0)),
              key=lambda r: r.cost)
    misfit = abs(model(sol.x, 0.35) / mix(0.35) - 1.0)
    return sol.x[0], sol.x[1], a_s, a_t, misfit


def check_wilke_reciprocity(library=None):
    """Phi_ts / Phi_st = (a_t / a_s)(W_s / W_t) for mu and for kappa, on every
    pair of three species with distinct molar masses and coefficients; the
    recovered factors then predict a fourth binary composition and the
    ternary mixture value Sum_s X_s a_s / Sum_t X_t Phi_st."""
    sp, _, _ = _species(W3, seed=2)
    o = Oracle(_case(sp), library=library)
    W = sp.W
    for T in (420.0, 2100.0):
        for which in (0, 1):
            phi = np.ones((3, 3))
            pure = np.zeros(3)
            for s, t in ((0, 1), (0, 2), (1, 2)):
                P, Q, a_s, a_t, misfit = _binary_phis(o, s, t, T, W, which)
                assert misfit <= 1e-12
                assert Q / P == pytest.approx((a_t / a_s) * (W[s] / W[t]), rel=1e-10)
                phi[s, t], phi[t, s] = P, Q
                pure[s], pure[t] = a_s, a_t
            for X in ([0.2, 0.3, 0.5], [0.6, 0.1, 0.3], [0.05, 0.9, 0.05]):
                X = np.asarray(X)
                pred = sum(X[s] * pure[s] / (phi[s] @ X) for s in range(3))
                got = o.transport(T, 1.0, _Y_from_X(X, W))[which]
                assert got == pytest.approx(pred, rel=1e-11)


def check_relabelling(library=None):
    """Reordering the species (tables and mass fractions together) leaves mu,
    kappa and D unchanged."""
    sp, _, _ = _species(np.array([0.004, 0.028, 0.032, 0.131]), seed=3)
    o = Oracle(_case(sp), library=library)
    rng = np.random.default_rng(4)
    for _ in range(20):
        perm = rng.permutation(sp.n)
        spp = cases.Species(W=sp.W[perm], cp_coef=sp.cp_coef[perm], h_off=sp.h_off[perm],
                            mu_coef=sp.mu_coef[perm], kappa_coef=sp.kappa_coef[perm])
        op = Oracle(_case(spp), library=library)
        Y = rng.dirichlet(np.ones(sp.n))
        T = rng.uniform(300.0, 3000.0)
        a = o.transport(T, 0.9, Y)
        b = op.transport(T, 0.9, Y[perm])
        assert np.allclose(a, b, rtol=1e-14, atol=0.0)


def _dt_case(mu, kappa, lewis, L_ref):
    """Calorically perfect pure gas (species 1 of a binary) on a 2D periodic
    8 x 4 grid with dx = 1/8, dy = 1/4: a left half at rest and a right half
    moving diagonally, hotter and lighter."""
    sp = cases.Species(W=np.array([0.028, 0.004]), cp_coef=np.array([[3.5, 0, 0, 0, 0],
                                                                      [2.5, 0, 0, 0, 0]]),
                       h_off=np.zeros(2), mu_coef=np.array([[math.log(mu), 0, 0, 0]] * 2),
                       kappa_coef=np.array([[math.log(kappa), 0, 0, 0]] * 2), lewis=lewis)
    nx, ny = 8, 4
    i = np.tile(np.arange(nx), ny)
    right = i >= nx // 2
    rho = np.where(right, 0.6, 1.0)
    u = np.where(right, 0.3, 0.0)
    v = np.where(right, -0.2, 0.0)
    p = np.where(right, 1.4, 1.0)
    prim = np.stack([rho, u, v, p, np.ones(nx * ny)])
    return _case(sp, dim=2, n=(nx, ny, 1), hi=(1.0, 1.0, 1.0), prim=prim, L_ref=L_ref,
                 cfl=0.6), rho, u, v, p


def _dt_closed_form(case, rho, u, v, p, mu, kappa, lewis):
    """The reading of Eq. 17 with every ingredient in closed form: for a
    calorically perfect gas c^2 = gamma p / rho with gamma = c_p/(c_p - R)."""
    cpR = 3.5
    gamma = cpR / (cpR - 1.0)
    R = R_U / 0.028 / case.a_ref2                      # dimensionless R_s [1/K]
    c = np.sqrt(gamma * p / rho)
    dx, dy = case.dx[0], case.dx[1]
    conv = case.cfl / np.max((np.abs(u) + c) / dx + (np.abs(v) + c) / dy)
    a_ref = math.sqrt(case.a_ref2)
    mu_s = mu / (case.rho_ref * a_ref * case.L_ref)
    ka_s = kappa / (case.rho_ref * a_ref ** 3 * case.L_ref)
    nu = np.max(np.maximum.reduce([4.0 * mu_s / (3.0 * rho), ka_s / (rho * (cpR - 1.0) * R),
                                   ka_s / (rho * cpR * R * lewis)]))
    visc = case.cfl * min(dx, dy) ** 2 / (2 * 2 * nu)
    return conv, visc


def check_dt(library=None):
    """dt = CFL / max_cells Sum_d (|u_d| + c)/dx_d, capped viscously at
    CFL dx_min^2 / (2 dim max(4 mu/(3 rho), kappa/(rho c_v), D)); each of the
    three viscous terms is made to bind in turn, and a long domain scale keeps
    the viscous cap inactive."""
    binding = set()
    for mu, kappa, lewis, L_ref in ((2e-5, 1e-4, 1.0, 1e-7),     # 4 mu / 3 rho binds
                                    (2e-5, 5e-1, 1.0, 1e-7),     # kappa / (rho c_v) binds
                                    (2e-5, 5e-1, 0.3, 1e-7),     # D = kappa/(rho c_p Le) binds
                                    (2e-5, 3e-2, 1.0, 0.05)):    # convective limit binds
        case, rho, u, v, p = _dt_case(mu, kappa, lewis, L_ref)
        o = Oracle(case, library=library)
        U, T = o.prim_to_cons()
        dt = o.dt(U, T.copy())
        conv, visc = _dt_closed_form(case, rho, u, v, p, mu, kappa, lewis)
        assert dt == pytest.approx(min(conv, visc), rel=1e-13)
        binding.add("visc" if visc < conv else "conv")
    assert binding == {"visc", "conv"}


PINS = [check_eq29_pure_species, check_wilke_reciprocity, check_relabelling, check_dt]


@pytest.mark.parametrize("pin", PINS, ids=[f.__name__ for f in PINS])
def test_transport_and_dt_pins(pin):
    pin()


# ------------------------------------------------------- planted mistakes --

MUTANTS = [
    ("W ratio swapped in the quarter power of Phi",
     "std::pow(th.W[t] / th.W[s], 0.25)", "std::pow(th.W[s] / th.W[t], 0.25)"),
    ("property ratio swapped in Phi", "sqrt(al[s] / al[t])", "sqrt(al[t] / al[s])"),
    ("W ratio swapped in the prefactor of Phi",
     "std::pow(1.0 + th.W[s] / th.W[t], -0.5)", "std::pow(1.0 + th.W[t] / th.W[s], -0.5)"),
    ("mass fractions in place of molar fractions",
     "X[s] = (q.Y[s] / th.W[s]) / ysw;", "X[s] = q.Y[s];"),
    ("bracket of Phi not squared", "ph * br * br", "ph * br"),
    ("Eq. 29 coefficients in reverse order",
     "lm = lm + p.mu[s][j] * pw;", "lm = lm + p.mu[s][3 - j] * pw;"),
    ("viscosity scaled with a_ref^2", "wilke(mus) / (p.rho_ref * a_ref * p.L_ref)",
     "wilke(mus) / (p.rho_ref * p.a_ref2 * p.L_ref)"),
    ("D with c_v in place of c_p", "q.D = q.kap / (q.rho * q.cp * p.lewis);",
     "q.D = q.kap / (q.rho * q.cv * p.lewis);"),
    ("viscous cap without its 2 dim", "(2.0 * L.dim * numax)", "(2.0 * numax)"),
    ("convective rate as a max over directions",
     "s += (std::fabs(q.u[a]) + q.c) / L.dx[a];",
     "s = std::max(s, (std::fabs(q.u[a]) + q.c) / L.dx[a]);"),
    ("thermal diffusivity with c_p", "q.kap / (q.rho * q.cv)", "q.kap / (q.rho * q.cp)"),
    ("viscous diffusivity without 4/3", "4.0 * q.mu / (3.0 * q.rho)", "q.mu / q.rho"),
]


def test_planted_mistakes_are_caught(tmp_path):
    """Each plausible mistake, planted in a copy of the oracle source and
    compiled on the CPU, fails at least one pin above."""
    src = open(os.path.join(os.path.dirname(obuild.__file__), "xfo.cpp")).read()
    procs, libs = [], []
    for k, (what, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, what
        path = tmp_path / f"mut{k}.cpp"
        path.write_text(src.replace(old, new))
        out = str(tmp_path / f"libmut{k}.so")
        procs.append(subprocess.Popen(["g++", *obuild.FLAGS, "-I", os.path.dirname(obuild.__file__),
                                       "-o", out, str(path)]))
        libs.append(out)
    assert all(p.wait() == 0 for p in procs)
    for (what, _, _), out in zip(MUTANTS, libs):
        L = load(out)
        caught = []
        for pin in PINS:
            try:
                pin(L)
            except (AssertionError, ValueError):   # a failed check, or a fit with no solution
                caught.append(pin.__name__)
        assert caught, f"planted mistake not caught: {what}"
