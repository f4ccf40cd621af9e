"""Pin of the oracle's multicomponent Roe-averaged face state (the reading of
Sec. II.C, Eq. 14-15, "multicomponent Roe average", ref. 37 only cited)
against a property the mathematics fixes.

For a mixture of calorically perfect species (constant c_p,s, so different
ratios of specific heats), the face state read as sqrt(rho)-weighted u, H, Y_s
and T, Gamma = R(Y)/c_v(Y) and phi_s = R_s T - Gamma (e_s(T) - |u|^2/2) is an
exact Roe matrix: R diag(lambda) L (U_R - U_L) = F(U_R) - F(U_L) for any two
states, to round-off. With one gas the temperature drops out of phi (R T -
Gamma c_v T = 0), so the single-gas pin cannot see how T and Y are averaged;
with several species it can. With c_p,s(T) varying, the same reading is a
consistent linearisation: the Roe residual relative to the flux jump falls
like the square of the jump.

The last test plants plausible mistakes in the face state (arithmetic means
in place of the sqrt(rho) weights, phi without its kinetic term, Gamma from
c_p) in copies of the oracle source and checks that the pin catches each.
None needs a GPU.
"""
import math
import os
import subprocess

import numpy as np

from paper_2403_05910_b300 import cases
from oracle import build as obuild
from oracle.xfo import Oracle, load


def _case(sp, dim):
    nv = dim + 2 + sp.n - 1
    return cases.Case("pt", dim, (4, 4, 4)[:dim] + (1,) * (3 - dim), (0.0,) * 3, (1.0,) * 3,
                      ((0, 0),) * 3, sp, cases.R_U * 300.0 / 0.028, 1.0, 1.0, False, 0.5,
                      np.zeros((nv, 4 ** dim)))


def _state(o, rng):
    """A random mixture state: rho, T, Dirichlet mass fractions and a velocity
    up to three sound speeds per axis."""
    c = o.case
    N = c.n_species
    rho = rng.uniform(0.1, 10.0)
    T = rng.uniform(150.0, 5000.0)
    Y = rng.dirichlet(np.ones(N))
    e, cv, cp, _, _ = o.thermo(T, Y)
    Rm = sum(Y[s] * cases.R_U / c.species.W[s] for s in range(N)) / c.a_ref2
    u = rng.uniform(-3.0, 3.0, size=c.dim) * math.sqrt(cp / cv * Rm * T) / math.sqrt(c.dim)
    U = np.zeros(c.n_v)
    U[0] = rho
    U[1:1 + c.dim] = rho * u
    U[1 + c.dim] = rho * (e + 0.5 * float(np.dot(u, u)))
    U[2 + c.dim:] = rho * Y[:-1]
    return U, T


def check_roe_property_mixtures(library=None, trials=12):
    """R diag(lambda) L (U_R - U_L) = F(U_R) - F(U_L) for calorically perfect
    mixtures of 2 to 5 species with distinct molar masses and c_p, in 1-3D."""
    rng = np.random.default_rng(47)
    worst = 0.0
    for dim in (1, 2, 3):
        for N in (2, 3, 5):
            W = rng.choice(cases.W_SET, size=N, replace=N > len(cases.W_SET))
            sp = cases._draw_species(rng, np.array(W, dtype=float), True)
            o = Oracle(_case(sp, dim), library=library)
            for _ in range(trials):
                UL, TL = _state(o, rng)
                UR, TR = _state(o, rng)
                d = int(rng.integers(0, dim))
                L, R, lam, c2, st = o.eigen(d, UL, UR, TL, TR)
                lhs = R @ np.diag(lam) @ L @ (UR - UL)
                rhs = o.flux(d, UR, TR) - o.flux(d, UL, TL)
                err = float(np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs)))
                worst = max(worst, err)
                assert err <= 1e-12, (dim, N, err)
    return worst


def test_roe_property_calorically_perfect_mixtures():
    assert check_roe_property_mixtures() <= 1e-12


def _on_line(o, UL, TL, UR, TR, eps):
    """The state a fraction eps of the way from L to R in (rho, u, T, Y)."""
    c = o.case
    dim = c.dim

    def prim(U, T):
        rho = U[0]
        return rho, U[1:1 + dim] / rho, T, np.append(U[2 + dim:] / rho, 1 - np.sum(U[2 + dim:] / rho))
    a, b = prim(UL, TL), prim(UR, TR)
    rho, u, T, Y = (x + eps * (y - x) for x, y in zip(a, b))
    e = o.thermo(T, Y)[0]
    U = np.zeros(c.n_v)
    U[0] = rho
    U[1:1 + dim] = rho * u
    U[1 + dim] = rho * (e + 0.5 * float(u @ u))
    U[2 + dim:] = rho * Y[:-1]
    return U, T


def test_roe_residual_vanishes_at_second_order_thermally_perfect():
    """With c_p,s(T) varying no closed-form exact Roe matrix exists; the face
    state is a consistent linearisation: the residual of the Roe property,
    relative to the flux jump, falls like the square of the jump."""
    rng = np.random.default_rng(53)
    for dim in (1, 3):
        for N in (2, 4):
            W = rng.choice(cases.W_SET, size=N)
            sp = cases._draw_species(rng, np.array(W, dtype=float), False)
            o = Oracle(_case(sp, dim))
            for _ in range(3):
                UL, TL = _state(o, rng)
                UR, TR = _state(o, rng)
                TL, TR = rng.uniform(300.0, 3500.0, size=2)   # inside the fits' range
                UL, TL = _on_line(o, UL, TL, UL, TL, 0.0)
                UR, TR = _on_line(o, UR, TR, UR, TR, 0.0)
                d = int(rng.integers(0, dim))
                res = []
                for eps in (0.02, 0.01):
                    Ue, Te = _on_line(o, UL, TL, UR, TR, eps)
                    L, R, lam, c2, st = o.eigen(d, UL, Ue, TL, Te)
                    lhs = R @ np.diag(lam) @ L @ (Ue - UL)
                    rhs = o.flux(d, Ue, Te) - o.flux(d, UL, TL)
                    res.append(float(np.max(np.abs(lhs - rhs)) / np.max(np.abs(rhs))))
                if res[0] < 1e-12:
                    continue                                  # round-off only
                assert math.log2(res[0] / res[1]) >= 1.7, (dim, N, res)


MUTANTS = [
    ("arithmetic mean of T", "S T = ta * qa.T + tb * qb.T;", "S T = 0.5 * (qa.T + qb.T);"),
    ("arithmetic mean of Y", "Y[s] = ta * qa.Y[s] + tb * qb.Y[s];",
     "Y[s] = 0.5 * (qa.Y[s] + qb.Y[s]);"),
    ("arithmetic mean of H", "S H = ta * qa.H + tb * qb.H;", "S H = 0.5 * (qa.H + qb.H);"),
    ("phi without its kinetic term",
     "phi[s] = th.Rs[s] * T - Gam * (th.e_s(s, T) - 0.5 * q2);",
     "phi[s] = th.Rs[s] * T - Gam * th.e_s(s, T);"),
    ("Gamma from c_p", "S Gam = Rbar / cv;", "S Gam = Rbar / (cv + Rbar);"),
]


def test_planted_face_state_mistakes_are_caught(tmp_path):
    """Each plausible mistake in the face state, planted in a copy of the
    oracle source and compiled on the CPU, fails the mixture Roe pin."""
    src = open(os.path.join(os.path.dirname(obuild.__file__), "xfo.cpp")).read()
    procs, libs = [], []
    for k, (what, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, what
        path = tmp_path / f"roe{k}.cpp"
        path.write_text(src.replace(old, new))
        out = str(tmp_path / f"libroe{k}.so")
        procs.append(subprocess.Popen(["g++", *obuild.FLAGS, "-I", os.path.dirname(obuild.__file__),
                                       "-o", out, str(path)]))
        libs.append(out)
    assert all(p.wait() == 0 for p in procs)
    for (what, _, _), out in zip(MUTANTS, libs):
        try:
            check_roe_property_mixtures(load(out), trials=4)
        except AssertionError:
            continue
        raise AssertionError(f"planted mistake not caught: {what}")
