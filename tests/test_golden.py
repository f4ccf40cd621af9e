"""The synthetic inputs against the values the paper prints for its worked
cases (fixtures under tests/golden/, each citing its section): the 1D
multicomponent diffusion case of Sec. IV.B (Eq. 30, Table IV) and the
shock-bubble set-up of Sec. VI.A (Eq. 32-33). CPU only."""
import math
import os

import numpy as np
import pytest

from paper_2403_05910_b300 import cases

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ATM = 101325.0


def _read(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                vals[line[0]] = [float(x) for x in line[1:]]
    return {k: (v[0] if len(v) == 1 else np.array(v)) for k, v in vals.items()}


def test_table4_rows_are_mass_fractions():
    g = _read("sec4b_table4_multicomponent_diffusion.txt")
    for side in ("Y_fuel", "Y_oxidizer"):
        assert g[side].shape == (4,)
        assert np.all(g[side] >= 0.0)
        assert g[side].sum() == pytest.approx(1.0, abs=1e-12)


def test_diffusion_case_follows_sec4b_and_table4():
    """Domain, resolution, pressure, velocity and the Eq. 30 profiles of T and
    Y_k between the Table IV end states (f(x) = 1 - exp(-((x - x0)/d)^2)/2,
    the reading with the exponent's square restored)."""
    g = _read("sec4b_table4_multicomponent_diffusion.txt")
    assert cases.DIFF_T == (g["T_fuel_K"], g["T_oxidizer_K"])
    assert np.array_equal(np.array(cases.DIFF_Y[0]), g["Y_fuel"])
    assert np.array_equal(np.array(cases.DIFF_Y[1]), g["Y_oxidizer"])
    c = cases.multicomponent_diffusion()
    n = int(g["cells"])
    assert c.n == (n, 1, 1) and c.dim == 1
    assert c.L_ref == g["length_m"]
    assert c.bc[0] == (cases.BC_PERIODIC, cases.BC_PERIODIC)
    # dimensionless p = p / (rho_ref a_ref^2) with a_ref^2 = p0 / rho_ref
    assert c.rho_ref * c.a_ref2 == pytest.approx(g["p_atm"] * ATM, rel=1e-15)
    assert np.all(c.prim[2] == 1.0) and np.all(c.prim[1] == g["u_m_s"])
    x = (np.arange(n) + 0.5) * g["length_m"] / n
    f = 1.0 - 0.5 * np.exp(-((x - g["x0_m"]) / g["d_m"]) ** 2)
    T = g["T_oxidizer_K"] + (g["T_fuel_K"] - g["T_oxidizer_K"]) * f
    assert np.max(np.abs(c.params["T"] - T)) <= 1e-12 * g["T_oxidizer_K"]
    Y = g["Y_oxidizer"][:, None] + (g["Y_fuel"] - g["Y_oxidizer"])[:, None] * f[None, :]
    Yc = np.vstack([c.prim[3:], 1.0 - c.prim[3:].sum(axis=0)])
    assert np.max(np.abs(Yc - Y)) <= 1e-14
    # the state recovered from the generated primitives is the printed one:
    # T = p / (rho R_mix) in kelvin
    Rmix = cases.R_U * np.sum(Yc / np.array(cases.DIFF_W)[:, None], axis=0)
    T_rec = c.prim[2] * c.rho_ref * c.a_ref2 / (c.prim[0] * c.rho_ref * Rmix)
    assert np.max(np.abs(T_rec - T)) <= 1e-11 * g["T_oxidizer_K"]


def test_shock_bubble_set_up_follows_sec6a():
    """Pre-shock T0 and p0, the Eq. 32 interface offset zeta (the bubble gas's
    molar fraction is zeta far outside and 1 - zeta at the centre), the shock
    at 1.25 r ahead of the bubble centre, and the pre-shock temperature
    recovered from the generated state; at the paper's Ma the post-shock
    state is the one of Eq. 33."""
    g = _read("sec6a_shock_bubble_setup.txt")
    assert cases.T0_SBI == g["T0_K"]
    assert cases.P0_SBI == g["p0_atm"] * ATM
    assert cases.ZETA == g["zeta"]
    Ma, r, nx, ny = g["Ma_paper"], 0.15, 256, 128
    c = cases.shock_bubble(2, (nx, ny), 3, Ma, r, seed=0)
    assert c.params["x_shock"] == pytest.approx(0.5 + g["shock_x_over_r"] * r, abs=1e-15)
    W = c.species.W
    Y = np.vstack([c.prim[4:6], 1.0 - c.prim[4:6].sum(axis=0)]).reshape(3, ny, nx)
    X = (Y / W[:, None, None]) / np.sum(Y / W[:, None, None], axis=0)
    xs = (np.arange(nx) + 0.5) * 2.0 / nx
    ys = (np.arange(ny) + 0.5) * 1.0 / ny
    far = (xs[None, :] > 1.5) & (ys[:, None] > 0.8)       # pre-shock, far from the bubble
    assert np.max(np.abs(X[2][far] - g["zeta"])) <= 1e-12
    j0, i0 = 0, int(np.argmin(np.abs(xs - 0.5)))           # bubble centre (on the symmetry plane)
    assert abs(X[2][j0, i0] - (1.0 - g["zeta"])) <= 1e-4
    # pre-shock temperature from the generated state (dimensional T = p / (rho R))
    rho, p = c.prim[0].reshape(ny, nx), c.prim[3].reshape(ny, nx)
    Rmix = cases.R_U * np.sum(Y / W[:, None, None], axis=0)
    T = p * c.rho_ref * c.a_ref2 / (rho * c.rho_ref * Rmix)
    assert np.max(np.abs(T[far] - g["T0_K"])) <= 1e-10 * g["T0_K"]
    # Eq. 33 at the paper's Ma with the ambient gamma
    gm = c.params["gamma_amb"]
    r1, u1, p1 = c.params["post"]
    assert r1 == pytest.approx((gm + 1) * Ma ** 2 / (2 + (gm - 1) * Ma ** 2), rel=1e-15)
    assert u1 == pytest.approx(Ma * math.sqrt(gm) * (1 - 1 / r1), rel=1e-15)
    assert p1 == pytest.approx(1 + 2 * gm / (gm + 1) * (Ma ** 2 - 1), rel=1e-15)
