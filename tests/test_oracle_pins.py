"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check ties one part of the oracle to something other than itself: closed
forms, algebraic identities, brute-force differences, exact solutions and
conservation. None of them needs a GPU.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2403_05910_b300 import cases
from oracle.xfo import Oracle, weno5, FLAG_NEWTON


def _rand_species(rng, N, cal_perfect=False):
    W = np.array(rng.choice(cases.W_SET, size=N))
    return cases._draw_species(rng, W, cal_perfect)


def _case_for(sp, dim=3, viscous=False):
    """A 1-cell-sized case wrapper carrying the species tables (for point checks)."""
    nv = dim + 2 + sp.n - 1
    return cases.Case("pt", dim, (4, 4, 4)[:dim] + (1,) * (3 - dim), (0.0,) * 3, (1.0,) * 3,
                      ((0, 0),) * 3, sp, cases.R_U * 300.0 / 0.028, 1.0, 1.0, viscous, 0.5,
                      np.zeros((nv, 4 ** dim)))


def _state(o, rho, u, T, Y):
    """Conserved vector of one state from (rho, u, T, Y) with the oracle's e(T, Y)."""
    c = o.case
    e = o.thermo(T, Y)[0]
    U = np.zeros(c.n_v)
    U[0] = rho
    U[1:1 + c.dim] = rho * np.asarray(u)
    U[1 + c.dim] = rho * (e + 0.5 * float(np.dot(u, u)))
    U[2 + c.dim:] = rho * np.asarray(Y[:-1])
    return U


def _random_state(o, rng):
    c = o.case
    N = c.n_species
    rho = rng.uniform(0.1, 10.0)
    T = rng.uniform(150.0, 5000.0)
    Y = rng.dirichlet(np.ones(N))
    e, cv, cp, _, _ = o.thermo(T, Y)
    Rm = sum(Y[s] * cases.R_U / c.species.W[s] for s in range(N)) / c.a_ref2
    cs = math.sqrt(cp / cv * Rm * T)
    u = rng.uniform(-3.0, 3.0, size=c.dim) * cs / math.sqrt(c.dim)
    return _state(o, rho, u, T, Y), T


# ------------------------------------------------------------------ WENO5 --

def test_weno5_constant_and_linear():
    rng = np.random.default_rng(1)
    for _ in range(200):
        a = rng.uniform(-5, 5)
        assert weno5(np.full(5, a)) == pytest.approx(a, rel=1e-15, abs=1e-15)
        b = rng.uniform(-5, 5)
        f = a + b * np.arange(-2, 3)
        # linear data: beta_0 = beta_1 = beta_2, so the weights are the linear
        # weights and the result is the optimal 5-point combination
        lin = (2 * f[0] - 13 * f[1] + 47 * f[2] + 27 * f[3] - 3 * f[4]) / 60.0
        assert weno5(f) == pytest.approx(lin, rel=1e-14, abs=1e-14)


def test_weno5_picks_smooth_stencil_at_a_jump():
    # a jump between f_0 and f_1: only the left stencil is smooth, so the result
    # is its candidate q_0 = (2 f_-2 - 7 f_-1 + 11 f_0)/6 = 0 up to O(eps^2)
    assert abs(weno5(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))) < 1e-10


def test_weno5_fifth_order_flux_difference():
    """(F_{i+1/2} - F_{i-1/2})/dx -> f'(x_i) at fifth order on smooth data."""
    errs = []
    for n in (20, 40, 80):
        h = 1.0 / n
        x = np.arange(-3, n + 3) * h
        f = 2.0 + np.sin(2 * np.pi * x)
        Fh = np.array([weno5(f[i - 2:i + 3]) for i in range(2, n + 3)])  # faces i+1/2
        d = (Fh[1:] - Fh[:-1]) / h
        ex = 2 * np.pi * np.cos(2 * np.pi * x[3:n + 3])
        errs.append(np.max(np.abs(d - ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 4.5, (errs, orders)


# --------------------------------------------------------------- thermo ---

def test_bernstein_range_and_conversion():
    rng = np.random.default_rng(2)
    tau = np.linspace(0, 1, 101)
    for _ in range(50):
        b = rng.uniform(0, 1, 5)
        a = cases.bernstein_to_monomial(b)
        mono = sum(a[j] * tau ** j for j in range(5))
        bern = 2.5 + 2 * sum(b[j] * math.comb(4, j) * tau ** j * (1 - tau) ** (4 - j) for j in range(5))
        assert np.allclose(mono, bern, rtol=1e-13, atol=1e-13)
        assert mono.min() >= 2.5 - 1e-12 and mono.max() <= 4.5 + 1e-12


def test_enthalpy_derivative_is_cp_and_e_is_h_minus_RT():
    rng = np.random.default_rng(3)
    sp = _rand_species(rng, 4)
    o = Oracle(_case_for(sp))
    R = cases.R_U / sp.W / o.case.a_ref2
    for T in (120.0, 199.0, 201.0, 850.0, 3999.0, 4001.0, 5500.0):
        for s in range(4):
            Y = np.zeros(4); Y[s] = 1.0
            h = 1e-3
            hp = o.thermo(T + h, Y)[4][s]
            hm = o.thermo(T - h, Y)[4][s]
            e, cv, cp, es, hs = o.thermo(T, Y)
            assert (hp - hm) / (2 * h) == pytest.approx(cp, rel=1e-8)
            assert es[s] == pytest.approx(hs[s] - R[s] * T, rel=1e-13, abs=1e-13 * abs(hs[s]) + 1e-300)
            assert cp - cv == pytest.approx(R[s], rel=1e-13)
            assert 2.5 - 1e-12 <= cp / R[s] <= 4.5 + 1e-12


def test_newton_closed_form_calorically_perfect():
    rng = np.random.default_rng(4)
    sp = _rand_species(rng, 3, cal_perfect=True)
    o = Oracle(_case_for(sp))
    R = cases.R_U / sp.W / o.case.a_ref2
    a0 = sp.cp_coef[:, 0]
    for _ in range(100):
        Y = rng.dirichlet(np.ones(3))
        Ttrue = rng.uniform(50, 6000)
        # e = sum Y_s R_s ((a0_s - 1) T - a0_s T_lo + h_off_s) for a constant c_p
        e = float(np.sum(Y * R * ((a0 - 1) * Ttrue - a0 * sp.T_lo + sp.h_off)))
        T, it, st = o.temperature(e, Y, 300.0)
        assert st == 0
        assert T == pytest.approx(Ttrue, rel=1e-13)


def test_newton_polynomial_residual_and_initial_guess():
    rng = np.random.default_rng(5)
    sp = _rand_species(rng, 5)
    o = Oracle(_case_for(sp))
    R = cases.R_U / sp.W / o.case.a_ref2
    for _ in range(100):
        Y = rng.dirichlet(np.ones(5))
        Ttrue = rng.uniform(60, 6000)
        e = o.thermo(Ttrue, Y)[0]
        Ts = []
        for T0 in (100.0, 300.0, 3000.0, 8000.0):
            T, it, st = o.temperature(e, Y, T0)
            assert st == 0 and it < 50
            Ts.append(T)
        scale = float(np.sum(Y * R)) * Ttrue
        assert abs(o.thermo(Ts[0], Y)[0] - e) <= 1e-12 * scale
        assert np.ptp(Ts) <= 1e-12 * Ttrue
        assert Ts[0] == pytest.approx(Ttrue, rel=1e-11)


def test_newton_flags_non_convergence():
    rng = np.random.default_rng(6)
    sp = _rand_species(rng, 3)
    c = _case_for(sp)
    from oracle.xfo import Oracle as O
    o = O(c, newton_max=1)
    Y = np.array([0.3, 0.3, 0.4])
    e = o.thermo(1500.0, Y)[0]
    T, it, st = o.temperature(e, Y, 300.0)
    assert st & FLAG_NEWTON


# ---------------------------------------------------------- eigensystem ---

@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_eigen_LR_identity(N):
    rng = np.random.default_rng(10 + N)
    n_states = 10000 // 4
    worst = 0.0
    for dim in (1, 2, 3):
        sp = _rand_species(rng, N)
        o = Oracle(_case_for(sp, dim))
        for _ in range(n_states // 3 + 1):
            UL, TL = _random_state(o, rng)
            UR, TR = _random_state(o, rng)
            d = int(rng.integers(0, dim))
            L, R, lam, c2, st = o.eigen(d, UL, UR, TL, TR)
            if st:
                continue
            worst = max(worst, np.max(np.abs(L @ R - np.eye(o.nv))))
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_sound_speed_identity(dim):
    """c^2 from the eigen formula equals (c_p/c_v) p / rho at a single state."""
    rng = np.random.default_rng(20 + dim)
    for N in (2, 3, 5):
        sp = _rand_species(rng, N)
        o = Oracle(_case_for(sp, dim))
        for _ in range(200):
            U, T = _random_state(o, rng)
            _, _, _, c2, st = o.eigen(0, U, U, T, T)
            rho = U[0]
            Y = np.append(U[2 + dim:] / rho, 1 - np.sum(U[2 + dim:] / rho))
            e, cv, cp, _, _ = o.thermo(T, Y)
            Rm = sum(Y[s] * cases.R_U / sp.W[s] for s in range(N)) / o.case.a_ref2
            p = rho * Rm * T
            assert c2 == pytest.approx(cp / cv * p / rho, rel=1e-13)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_eigenvectors_of_flux_jacobian(dim):
    """A r_k = lambda_k r_k and l_k A = lambda_k l_k with A = dF/dU from central
    differences of the oracle's own physical flux at a cell state."""
    rng = np.random.default_rng(30 + dim)
    for N in (2, 4):
        sp = _rand_species(rng, N)
        o = Oracle(_case_for(sp, dim))
        for _ in range(10):
            U, T = _random_state(o, rng)
            d = int(rng.integers(0, dim))
            nv = o.nv
            A = np.zeros((nv, nv))
            for j in range(nv):
                h = 1e-6 * max(abs(U[j]), 1e-3 * abs(U[0]), 1e-8)
                Up = U.copy(); Up[j] += h
                Um = U.copy(); Um[j] -= h
                A[:, j] = (o.flux(d, Up, T) - o.flux(d, Um, T)) / (2 * h)
            L, R, lam, c2, st = o.eigen(d, U, U, T, T)
            scale = np.max(np.abs(A)) * np.max(np.abs(R))
            for k in range(nv):
                res = A @ R[:, k] - lam[k] * R[:, k]
                assert np.max(np.abs(res)) <= 1e-7 * scale
                resl = L[k] @ A - lam[k] * L[k]
                assert np.max(np.abs(resl)) <= 1e-7 * np.max(np.abs(A)) * np.max(np.abs(L))


def test_roe_property_single_calorically_perfect_gas():
    """For one calorically perfect gas the sqrt(rho)-weighted face state is the
    classic Roe average: R diag(lambda) L (U_R - U_L) = F(U_R) - F(U_L)."""
    rng = np.random.default_rng(40)
    for dim in (1, 2, 3):
        sp = _rand_species(rng, 2, cal_perfect=True)
        o = Oracle(_case_for(sp, dim))
        for _ in range(50):
            N = 2
            ULs, TL = _random_state(o, rng)
            URs, TR = _random_state(o, rng)
            # force a single species (Y_1 = 1)
            for U, T in ((ULs, TL), (URs, TR)):
                rho = U[0]
                u = U[1:1 + dim] / rho
                Unew = _state(o, rho, u, T, np.array([1.0, 0.0]))
                U[:] = Unew
            d = int(rng.integers(0, dim))
            L, R, lam, c2, st = o.eigen(d, ULs, URs, TL, TR)
            lhs = R @ np.diag(lam) @ L @ (URs - ULs)
            rhs = o.flux(d, URs, TR) - o.flux(d, ULs, TL)
            assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.max(np.abs(rhs)))


# -------------------------------------------------------------- WENO-CU6 --

def _beta6_from_definition():
    """Jiang-Shu indicator of the degree-5 polynomial whose cell averages on
    cells i-2..i+3 are f (dx = 1): sum_l int_{cell i} (p^(l))^2, derived here."""
    import sympy as sp
    x = sp.symbols("x")
    f = sp.symbols("f0:6")
    c = sp.symbols("c0:6")
    p = sum(c[k] * x ** k for k in range(6))
    half = sp.Rational(1, 2)
    sol = sp.solve([sp.integrate(p, (x, j - half, j + half)) - f[j + 2] for j in range(-2, 4)], c)
    p = p.subs(sol)
    beta = sum(sp.integrate(sp.diff(p, x, l) ** 2, (x, -half, half)) for l in range(1, 6))
    terms = [(m, Fraction(int(cf.p), int(cf.q))) for m, cf in sp.Poly(beta, *f).terms()]

    def exact(*v):
        """beta_6 of the (binary-exact) inputs in rational arithmetic"""
        fv = [Fraction(float(a)) for a in v]
        tot = Fraction(0)
        for m, cf in terms:
            t = cf
            for a, e in zip(fv, m):
                t *= a ** e
            tot += t
        return float(tot)
    return exact


def test_cu6_beta6_matches_its_definition():
    """Against the indicator derived above, evaluated exactly: on mean-free data
    of any scale, and on small variations about an offset (smooth data), where
    evaluating the quadratic form on raw values would lose most digits to
    cancellation."""
    from oracle.xfo import cu6_beta6
    b6 = _beta6_from_definition()
    rng = np.random.default_rng(41)
    for _ in range(200):
        f = rng.normal(size=6) * 10 ** rng.uniform(-2, 2)
        assert cu6_beta6(f) == pytest.approx(b6(*f), rel=1e-12, abs=0.0)
    for _ in range(200):
        f = rng.uniform(-3, 3) + rng.normal(size=6) * 10 ** rng.uniform(-7, -1)
        assert cu6_beta6(f) == pytest.approx(b6(*f), rel=1e-12, abs=0.0)


def test_cu6_constant_and_linear():
    from oracle.xfo import weno_cu6
    rng = np.random.default_rng(42)
    for _ in range(100):
        a, b = rng.uniform(-5, 5, size=2)
        assert weno_cu6(np.full(6, a)) == pytest.approx(a, rel=1e-15, abs=1e-15)
        f = a + b * np.arange(-2, 4)
        # linear data: tau_6 = 0, so the weights are (1, 9, 9, 1)/20 and the
        # result is the 6-point central reconstruction
        central = (f[0] - 8 * f[1] + 37 * f[2] + 37 * f[3] - 8 * f[4] + f[5]) / 60.0
        assert weno_cu6(f) == pytest.approx(central, rel=1e-13, abs=1e-13)


def test_cu6_sixth_order_flux_difference():
    from oracle.xfo import weno_cu6
    errs = []
    for n in (20, 40, 80):
        h = 1.0 / n
        x = np.arange(-3, n + 4) * h
        f = 2.0 + np.sin(2 * np.pi * x)
        Fh = np.array([weno_cu6(f[i - 2:i + 4]) for i in range(2, n + 3)])
        d = (Fh[1:] - Fh[:-1]) / h
        ex = 2 * np.pi * np.cos(2 * np.pi * x[3:n + 3])
        errs.append(np.max(np.abs(d - ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 5.5, (errs, orders)


def test_cu6_picks_smooth_stencils_at_a_jump():
    from oracle.xfo import weno_cu6
    # jump between f_i and f_{i+1}: the flat stencil {i-2, i-1, i} (beta_0 = 0)
    # outweighs every stencil that crosses the jump by ~1/eps, so the value
    # stays O(eps) away from the upwind one (0) instead of the central 1/2
    for eps in (1e-6, 1e-10):
        v = weno_cu6(np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]), eps)
        assert 0.0 <= v < 10 * eps, (eps, v)
        w = weno_cu6(np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0]), eps)
        assert 0.0 <= 1.0 - w < 10 * eps, (eps, w)


# ---------------------------------------------------------------- WENO7 --

def _weno7_parts():
    """Candidates, 7-point upwind value and Jiang-Shu indicators of the cubics
    on {i-3+k .. i+k} (cell averages f_0..f_6 = f_{i-3..i+3}, dx = 1), derived
    here from their definitions."""
    import sympy as sp
    x = sp.symbols("x")
    f = sp.symbols("f0:7")
    half = sp.Rational(1, 2)

    def poly_on(cells):
        c = sp.symbols("c0:%d" % len(cells))
        p = sum(c[k] * x ** k for k in range(len(cells)))
        sol = sp.solve([sp.integrate(p, (x, j - half, j + half)) - f[j + 3] for j in cells], c)
        return p.subs(sol)

    betas = []
    for k in range(4):
        p = poly_on(list(range(-3 + k, 1 + k)))
        b = sp.expand(sum(sp.integrate(sp.diff(p, x, l) ** 2, (x, -half, half)) for l in range(1, 4)))
        betas.append([(m, Fraction(int(cf.p), int(cf.q))) for m, cf in sp.Poly(b, *f).terms()])
    full = sp.expand(poly_on(list(range(-3, 4))).subs(x, half))
    return betas, sp.lambdify(f, full, "math")


def _exact_form(terms, v):
    fv = [Fraction(float(a)) for a in v]
    tot = Fraction(0)
    for m, cf in terms:
        t = cf
        for a, e in zip(fv, m):
            t *= a ** e
        tot += t
    return tot


def test_weno7_weights_follow_the_indicators():
    """With the indicators computed exactly from their definition, the weights
    d_k/(eps + beta_k)^2 (d = (1, 12, 18, 4)/35) and the cubic candidates give
    the oracle's value; probes both smooth data about an offset and rough data."""
    from oracle.xfo import weno7
    betas, _ = _weno7_parts()
    d = [Fraction(1, 35), Fraction(12, 35), Fraction(18, 35), Fraction(4, 35)]
    cand = [(-3, 13, -23, 25, 0, 0, 0), (0, 1, -5, 13, 3, 0, 0), (0, 0, -1, 7, 7, -1, 0),
            (0, 0, 0, 3, 13, -5, 1)]
    rng = np.random.default_rng(43)
    eps = Fraction(1, 10 ** 6)
    for scale in (1e-4, 1e-2, 1.0, 10.0):
        for _ in range(40):
            f = rng.uniform(-2, 2) + rng.normal(size=7) * scale
            fv = [Fraction(float(a)) for a in f]
            al = [d[k] / (eps + _exact_form(betas[k], f)) ** 2 for k in range(4)]
            q = [sum(Fraction(c) * a for c, a in zip(cand[k], fv)) / 12 for k in range(4)]
            ref = float(sum(a * b for a, b in zip(al, q)) / sum(al))
            assert weno7(f) == pytest.approx(ref, rel=1e-12, abs=1e-14 * np.max(np.abs(f)))


def test_weno7_exact_for_cubics_and_seventh_order():
    """Cell averages of a cubic: every candidate is exact, so is the scheme.
    Smooth data with eps far above every indicator (weights at their linear
    values): the flux difference converges at seventh order, which fixes the
    linear weights. (With eps = 1e-6 the Jiang-Shu weights lose order at the
    extrema in the max norm, as WENO-JS schemes do.)"""
    from oracle.xfo import weno7
    rng = np.random.default_rng(44)
    for _ in range(50):
        c = rng.normal(size=4)
        P = lambda t: c[0] * t + c[1] * t ** 2 / 2 + c[2] * t ** 3 / 3 + c[3] * t ** 4 / 4
        avg = np.array([P(j + 0.5) - P(j - 0.5) for j in range(-3, 4)])
        exact = c[0] + c[1] * 0.5 + c[2] * 0.25 + c[3] * 0.125
        assert weno7(avg) == pytest.approx(exact, rel=1e-12, abs=1e-12)
    errs = []
    for n in (20, 40, 80):
        h = 1.0 / n
        x = np.arange(-4, n + 5) * h
        f = 2.0 + np.sin(2 * np.pi * x)
        Fh = np.array([weno7(f[i - 3:i + 4], 1e6) for i in range(3, n + 5)])
        dd = (Fh[1:] - Fh[:-1]) / h
        ex = 2 * np.pi * np.cos(2 * np.pi * x[4:n + 5])
        errs.append(np.max(np.abs(dd - ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 6.5, (errs, orders)


def test_weno7_picks_the_smooth_stencil_at_a_jump():
    from oracle.xfo import weno7
    for eps in (1e-6, 1e-10):
        v = weno7(np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0]), eps)
        assert 0.0 <= v < 10 * eps ** 2 * 1e6, (eps, v)
        w = weno7(np.array([1.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0]), eps)
        assert 0.0 <= 1.0 - w < 10 * eps ** 2 * 1e6, (eps, w)
