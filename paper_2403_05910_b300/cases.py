"""Seeded synthetic inputs for the multicomponent RHS/RK3 hot path.

This module is the one place both sides draw their inputs from: the CUDA path
(through the C-ABI binding) and the CPU oracle (``oracle/``) consume the same
species tables, grid descriptions and primitive fields built here. It holds
none of the method's arithmetic -- no equation of state, no temperature solve,
no flux, no transport mixing rule. Each side turns the primitive fields
(rho, u, p, Y) into conserved variables with its own equation of state.

What it generates (the workloads of the XFluids paper, arXiv 2403.05910):

* the 1D two-species inviscid shock tube (Sod states, 400 cells);
* 2D and 3D inert shock-bubble interactions (Sec. VI.A): a planar shock with
  the frozen-gamma Rankine-Hugoniot post-shock state of Eq. 33 and a bubble
  whose interface follows the tanh profile of Eq. 32 in molar fraction;
* a batched ensemble of uneven 2D shock-bubble instances;
* the 1D multicomponent diffusion case (Sec. IV.B, Table IV) with seeded
  binary diffusion fits for the mixture-averaged model of Eq. 25-26;
* small smooth periodic fields used by the tests, and smooth seeded
  perturbations of any case.

Species data is synthetic (no thermochemistry tables exist offline):
c_p/R(T) is a degree-4 polynomial in tau = (T - T_lo)/(T_hi - T_lo), drawn in
Bernstein form so that 2.5 <= c_p/R <= 4.5 on [200, 4000] K, and the
transport fits follow the form of Eq. 29, ln(eta) = sum_n a_n (ln T)^(n-1).

Nondimensionalisation (the paper is silent; this is the project's reading):
rho* = rho/rho_ref, u* = u/a_ref, p* = p/(rho_ref a_ref^2), x* = x/L_ref;
temperatures stay in kelvin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R_U = 8.314462618          # J/(mol K), universal gas constant (Eq. 7)
T_LO, T_HI = 200.0, 4000.0  # K, range of the c_p polynomials
BC_TRANSMISSIVE, BC_PERIODIC, BC_SYMMETRIC = 0, 1, 2
W_SET = (0.004, 0.028, 0.032, 0.131)  # kg/mol, the molar-mass pool
P0_SBI = 101325.0           # Pa, pre-shock pressure (Sec. VI.A)
T0_SBI = 295.0              # K, pre-shock temperature (Sec. VI.A)
H_SBI = 0.05                # m, domain height used as L_ref for shock-bubble cases
ZETA = 1.0e-4               # Eq. 32 interface offset


@dataclass
class Species:
    """Per-species tables, all in SI / kelvin.

    cp_coef[s, j]: c_p/R_s = sum_j cp_coef[s, j] * tau**j, tau in [0, 1].
    h_off[s]: h_s/R_s at T_lo (K).
    mu_coef[s, n], kappa_coef[s, n]: ln(mu [Pa s]) and ln(kappa [W/(m K)])
    as cubic polynomials in ln(T) (Eq. 29 with four terms).
    dbin_coef[s, t, n] (optional, symmetric in s, t): ln(p D_st [Pa m^2/s]) as
    a cubic polynomial in ln(T), the binary diffusion coefficients of Eq. 25
    in the fit form of Eq. 29 (p D_st depends on T only).
    """
    W: np.ndarray
    cp_coef: np.ndarray
    h_off: np.ndarray
    mu_coef: np.ndarray
    kappa_coef: np.ndarray
    T_lo: float = T_LO
    T_hi: float = T_HI
    lewis: float = 1.0
    dbin_coef: np.ndarray = None

    @property
    def n(self) -> int:
        return int(self.W.shape[0])


@dataclass
class Case:
    """One workload: grid, species, reference scales and primitive fields.

    ``prim`` is SoA ``[n_v, nz*ny*nx]`` with i fastest and rows
    (rho, u_1..u_dim, p, Y_1..Y_{N-1}), all dimensionless.
    """
    name: str
    dim: int
    n: tuple
    lo: tuple
    hi: tuple
    bc: tuple                 # ((lo, hi),) * 3
    species: Species
    a_ref2: float
    rho_ref: float
    L_ref: float
    viscous: bool
    cfl: float
    prim: np.ndarray
    params: dict = field(default_factory=dict)

    @property
    def n_species(self) -> int:
        return self.species.n

    @property
    def n_v(self) -> int:
        return self.dim + 2 + self.species.n - 1

    @property
    def cells(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def dx(self) -> tuple:
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(3))


# ---------------------------------------------------------------- species ---

def bernstein_to_monomial(b: np.ndarray) -> np.ndarray:
    """c_p/R = 2.5 + 2 * sum_j b_j B_{j,4}(tau)  ->  monomial coefficients in tau.

    Bernstein weights b_j in [0, 1] keep c_p/R inside [2.5, 4.5] on tau in [0, 1]
    because the Bernstein basis is non-negative and sums to one.
    """
    a = np.zeros(5)
    for j in range(5):
        for m in range(j, 5):
            a[m] += 2.0 * b[j] * math.comb(4, j) * math.comb(4 - j, m - j) * (-1.0) ** (m - j)
    a[0] += 2.5
    return a


def _draw_species(rng: np.random.Generator, W: np.ndarray, calorically_perfect=False) -> Species:
    """Draw per-species tables in a fixed order: for each species s in turn,
    5 Bernstein weights, then mu(300 K), three mu slopes, the Eucken-like factor
    of kappa(300 K) and three kappa slopes.

    Transport reading: mu_s(300 K) ~ U[1.5, 3]e-5 Pa s; kappa_s(300 K) =
    mu_s(300 K) * R_s * f_s with f_s ~ U[3.75, 5.75] (the range a modified Eucken
    factor c_p/R + 1.25 spans for 2.5 <= c_p/R <= 4.5).
    """
    N = W.shape[0]
    cp = np.zeros((N, 5))
    mu = np.zeros((N, 4))
    ka = np.zeros((N, 4))
    L = math.log(300.0)
    for s in range(N):
        b = rng.uniform(0.0, 1.0, size=5)
        if calorically_perfect:
            cp[s, 0] = 2.5 + 2.0 * b[0]
        else:
            cp[s] = bernstein_to_monomial(b)
        mu300 = rng.uniform(1.5e-5, 3.0e-5)
        m2, m3, m4 = rng.uniform(0.6, 0.8), rng.uniform(-5e-3, 5e-3), rng.uniform(-5e-4, 5e-4)
        f = rng.uniform(3.75, 5.75)
        k2, k3, k4 = rng.uniform(0.7, 0.9), rng.uniform(-5e-3, 5e-3), rng.uniform(-5e-4, 5e-4)
        k300 = mu300 * (R_U / W[s]) * f
        mu[s] = [math.log(mu300) - (m2 * L + m3 * L * L + m4 * L ** 3), m2, m3, m4]
        ka[s] = [math.log(k300) - (k2 * L + k3 * L * L + k4 * L ** 3), k2, k3, k4]
    return Species(W=W.astype(np.float64), cp_coef=cp, h_off=np.zeros(N), mu_coef=mu, kappa_coef=ka)


def draw_binary_diffusion(rng: np.random.Generator, W: np.ndarray) -> np.ndarray:
    """ln(p D_st) fits (Eq. 25 in the form of Eq. 29) for every pair s < t, in
    that order: D_st(300 K, 1 atm) = 2e-5 m^2/s * (0.0145 kg/mol / W_st)^(1/2)
    * U[0.8, 1.25] (the Chapman-Enskog scaling with the reduced mass
    W_st = W_s W_t/(W_s + W_t)), a temperature exponent U[1.6, 1.8] and small
    curvature terms. The diagonal holds the self-diffusion fit of the same
    form (unused by the mixture rule of Eq. 26)."""
    N = W.shape[0]
    c = np.zeros((N, N, 4))
    L = math.log(300.0)
    for s in range(N):
        for t in range(s, N):
            Wst = W[s] * W[t] / (W[s] + W[t])
            D300 = 2.0e-5 * math.sqrt(0.0145 / Wst) * rng.uniform(0.8, 1.25)
            e1, e2, e3 = rng.uniform(1.6, 1.8), rng.uniform(-5e-3, 5e-3), rng.uniform(-5e-4, 5e-4)
            row = [math.log(P0_SBI * D300) - (e1 * L + e2 * L * L + e3 * L ** 3), e1, e2, e3]
            c[s, t] = row
            c[t, s] = row
    return c


def with_binary_diffusion(case: "Case", seed: int = 0) -> "Case":
    """Copy of ``case`` whose species carry seeded binary diffusion fits (an
    RNG of their own, so every other input stays as drawn)."""
    import dataclasses
    rng = np.random.default_rng([seed, 25])
    sp = dataclasses.replace(case.species, dbin_coef=draw_binary_diffusion(rng, case.species.W))
    return dataclasses.replace(case, species=sp, name=case.name + "_dsm")


def constant_transport(sp: Species, mu: float, kappa: float) -> Species:
    """Copy of ``sp`` whose mu_s and kappa_s are the same constants for every species."""
    N = sp.n
    m = np.zeros((N, 4)); m[:, 0] = math.log(mu)
    k = np.zeros((N, 4)); k[:, 0] = math.log(kappa)
    return Species(W=sp.W.copy(), cp_coef=sp.cp_coef.copy(), h_off=sp.h_off.copy(),
                   mu_coef=m, kappa_coef=k, T_lo=sp.T_lo, T_hi=sp.T_hi, lewis=sp.lewis)


def _cp_over_R_bernstein_at(sp: Species, s: int, T: float) -> float:
    """c_p/R of species s at T from its monomial table (used only to size the
    initial shock of Eq. 33; the solver sides evaluate their own thermo)."""
    tau = min(max((T - sp.T_lo) / (sp.T_hi - sp.T_lo), 0.0), 1.0)
    return float(sum(sp.cp_coef[s, j] * tau ** j for j in range(5)))


# ------------------------------------------------------------------- grids ---

def _centres(n, lo, hi):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx


def _pack(dim, rho, vel, p, Y):
    """Stack primitive fields into the SoA [n_v, cells] layout (i fastest)."""
    rows = [rho.ravel()] + [vel[a].ravel() for a in range(dim)] + [p.ravel()]
    rows += [Y[s].ravel() for s in range(Y.shape[0] - 1)]
    return np.ascontiguousarray(np.stack(rows).astype(np.float64))


# --------------------------------------------------------- the workloads ---

def shock_tube(seed: int = 0, n: int = 400, calorically_perfect: bool = False,
               W=None) -> Case:
    """1D two-species inviscid shock tube on [0, 1]: left (rho, u, p, Y1) =
    (1, 0, 1, 1), right (0.125, 0, 0.1, Y2 = 1), interface at x = 0.5, CFL 0.5,
    t_end 0.2, transmissive ends.

    Draw order: the two molar masses from {4, 28, 32, 131} g/mol (with
    replacement), then the species tables. Reference scales: a_ref^2 =
    R_u * 300 K / 0.028 kg/mol (a 28 g/mol gas sits at 300 K where p/rho = 1),
    rho_ref = 1 kg/m^3, L_ref = 1 m.
    """
    rng = np.random.default_rng(seed)
    if W is None:
        W = np.array(rng.choice(W_SET, size=2), dtype=np.float64)
    else:
        W = np.asarray(W, dtype=np.float64)
    sp = _draw_species(rng, W, calorically_perfect)
    x = _centres(n, 0.0, 1.0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    u = np.zeros(n)
    Y = np.stack([np.where(left, 1.0, 0.0), np.where(left, 0.0, 1.0)])
    prim = _pack(1, rho, [u], p, Y)
    return Case("shock_tube_1d", 1, (n, 1, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0),
                ((BC_TRANSMISSIVE,) * 2, (BC_TRANSMISSIVE,) * 2, (BC_TRANSMISSIVE,) * 2),
                sp, R_U * 300.0 / 0.028, 1.0, 1.0, False, 0.5, prim,
                {"t_end": 0.2})


def _sbi_species(rng, N, bubble_W=None):
    """Molar masses for a shock-bubble case: species 1, 2 = 28, 32 g/mol
    (ambient pair), species 3 = 4 or 131 g/mol (drawn unless given), species
    4..N drawn from the pool; then the species tables."""
    W = [0.028, 0.032]
    W.append(bubble_W if bubble_W is not None else float(rng.choice([0.004, 0.131])))
    for _ in range(3, N):
        W.append(float(rng.choice(W_SET)))
    W = np.array(W)
    return _draw_species(rng, W)


def shock_bubble(dim: int, n: tuple, N: int, Ma: float, r: float, seed: int = 0,
                 rng=None, viscous: bool = True, perturb: float = 0.0,
                 bubble_W=None, cfl: float = 0.4, name: str = "shock_bubble") -> Case:
    """Inert shock-bubble interaction (Sec. VI.A, Eq. 32-33), dimensionless.

    Domain [0, 2] x [0, 1] (x [0, 1]) in units of H = 0.05 m; bubble centre
    (0.5, 0, 0) on the symmetry plane(s); planar shock at x_s = 0.5 - 1.25 r moving
    in +x; pre-shock p0 = 1 atm, T0 = 295 K; ambient gas = 0.767/0.233 mass mix of
    species 1/2; bubble gas = species 3 (N = 3) or species 3..N with Dirichlet(1)
    mass fractions. Interface: X_amb = ((1 - 2 zeta) tanh(xi d) + 1)/2 with
    zeta = 1e-4 and xi = 2/(3 dx) (three cells thick). Post-shock state from
    Eq. 33 with the ambient gamma at T0. ``perturb`` scales a seeded density
    perturbation rho *= 1 + perturb * eta * 4 X (1 - X), eta ~ U[-1, 1] per
    cell, at fixed p, u, Y. BCs: transmissive in x, symmetric in y and z.
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    sp = _sbi_species(rng, N, bubble_W)
    W = sp.W
    # ambient and bubble compositions (mass fractions)
    Y_amb = np.zeros(N); Y_amb[0], Y_amb[1] = 0.767, 0.233
    Y_bub = np.zeros(N)
    if N == 3:
        Y_bub[2] = 1.0
    else:
        Y_bub[2:] = rng.dirichlet(np.ones(N - 2))
    x_amb = (Y_amb / W) / np.sum(Y_amb / W)
    x_bub = (Y_bub / W) / np.sum(Y_bub / W)
    R_amb = R_U * np.sum(Y_amb / W)
    rho0 = P0_SBI / (R_amb * T0_SBI)
    a_ref2 = P0_SBI / rho0
    # Eq. 33, frozen gamma of the ambient mixture at T0
    cp_amb = sum(Y_amb[s] * R_U / W[s] * _cp_over_R_bernstein_at(sp, s, T0_SBI) for s in range(N))
    g = cp_amb / (cp_amb - R_amb)
    rho1 = (g + 1.0) * Ma * Ma / (2.0 + (g - 1.0) * Ma * Ma)          # rho'/rho0
    c0 = math.sqrt(g)                                                   # c0/a_ref
    u1 = Ma * c0 * (1.0 - 1.0 / rho1)                                   # u'/a_ref
    p1 = 1.0 + 2.0 * g / (g + 1.0) * (Ma * Ma - 1.0)                    # p'/p0

    lo = (0.0, 0.0, 0.0)
    hi = (2.0, 1.0, 1.0 if dim == 3 else 1.0)
    nn = tuple(list(n) + [1] * (3 - len(n)))
    xs = [_centres(nn[a], lo[a], hi[a]) if a < dim else np.zeros(1) for a in range(3)]
    Z, Yg, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    dx = (hi[0] - lo[0]) / nn[0]
    xc = 0.5
    d = np.sqrt((X - xc) ** 2 + Yg ** 2 + (Z ** 2 if dim == 3 else 0.0)) - r
    xi = 2.0 / (3.0 * dx)
    Xa = ((1.0 - 2.0 * ZETA) * np.tanh(xi * d) + 1.0) / 2.0
    Xs = Xa[None] * x_amb[:, None, None, None] + (1.0 - Xa[None]) * x_bub[:, None, None, None]
    Ycell = Xs * W[:, None, None, None]
    Ycell = Ycell / Ycell.sum(axis=0, keepdims=True)
    Rcell = np.sum(Ycell / W[:, None, None, None], axis=0)      # R_mix / R_U
    rho = (np.sum(Y_amb / W) / Rcell)                           # rho*/ at p0, T0
    p = np.ones_like(rho)
    u = np.zeros_like(rho)
    post = X < xc - 1.25 * r
    rho = np.where(post, rho1, rho)
    p = np.where(post, p1, p)
    u = np.where(post, u1, u)
    Ycell = np.where(post[None], Y_amb[:, None, None, None], Ycell)
    if perturb != 0.0:
        eta = rng.uniform(-1.0, 1.0, size=rho.shape)
        Xi = np.where(post, 1.0, Xa)
        rho = rho * (1.0 + perturb * eta * 4.0 * Xi * (1.0 - Xi))
    vel = [u] + [np.zeros_like(u) for _ in range(dim - 1)]
    prim = _pack(dim, rho, vel, p, Ycell)
    bc = ((BC_TRANSMISSIVE, BC_TRANSMISSIVE), (BC_SYMMETRIC, BC_SYMMETRIC),
          (BC_SYMMETRIC, BC_SYMMETRIC))
    return Case(name, dim, nn, lo, hi, bc, sp, a_ref2, rho0, H_SBI, viscous, cfl, prim,
                {"Ma": Ma, "r": r, "gamma_amb": g, "x_shock": xc - 1.25 * r,
                 "post": (rho1, u1, p1)})


def config(i: int, seed: int = 0, n=None) -> Case:
    """The five named workloads (index 0..4), optionally on a reduced grid ``n``.

    0: 1D shock tube, 400 cells, 2 species, inviscid, to t = 0.2.
    1: 2D shock-bubble, 1024x512, 3 species, Ma 1.22, r = 0.15, viscous, 200 steps.
    2: 3D shock-bubble, 512x256x256, 5 species, Ma ~ U[1.2, 2.0], r = 0.2,
       1% interface density perturbation, viscous, 100 steps.
    3: the batched ensemble (see ``batch``); this returns its first instance.
    4: 2D shock-bubble, 512x256, 4 species, differentiated, 200 steps, dt frozen.
    """
    if i == 0:
        return shock_tube(seed, n=400 if n is None else n[0])
    if i == 1:
        c = shock_bubble(2, n or (1024, 512), 3, 1.22, 0.15, seed=seed, name="sbi2d_n3")
        c.params["steps"] = 200
        return c
    if i == 2:
        rng = np.random.default_rng(seed)
        sp_rng = np.random.default_rng(rng.integers(2 ** 31))
        Ma = float(rng.uniform(1.2, 2.0))
        c = shock_bubble(3, n or (512, 256, 256), 5, Ma, 0.2, rng=sp_rng, perturb=0.01,
                         name="sbi3d_n5")
        c.params["steps"] = 100
        return c
    if i == 3:
        return batch(seed)[0]
    if i == 4:
        c = shock_bubble(2, n or (512, 256), 4, 1.5, 0.2, seed=seed, name="sbi2d_n4_adjoint")
        c.params["steps"] = 200
        c.params["checkpoint_every"] = 20
        return c
    raise ValueError(f"no workload {i}")


def batch(seed: int = 0, count: int = 64, scale: int = 1) -> list:
    """The batched ensemble: ``count`` 2D viscous shock-bubble instances.

    Per instance, drawn from one generator in this order: k ~ U{2..12} giving
    nx = 64 k // scale, ny = nx / 2; N ~ U{3, 4, 5}; Ma ~ U[1.1, 2.5];
    r ~ U[0.1, 0.25]; a child seed for the species tables.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        k = int(rng.integers(2, 13))
        N = int(rng.integers(3, 6))
        Ma = float(rng.uniform(1.1, 2.5))
        r = float(rng.uniform(0.1, 0.25))
        child = int(rng.integers(2 ** 31))
        nx = max(16, 64 * k // scale)
        c = shock_bubble(2, (nx, nx // 2), N, Ma, r, seed=child, name=f"batch{b}")
        c.params["steps"] = 100
        out.append(c)
    return out


# ------------------------------------------------------------ test inputs ---

# species of the multicomponent diffusion case (Table IV order); the molar
# masses of O2, N2, H2O and CH4 (kg/mol), the thermo and transport synthetic
DIFF_W = (0.032, 0.028, 0.018, 0.016)
DIFF_T = (320.0, 1350.0)                        # K, fuel / oxidizer side (Table IV)
DIFF_Y = ((0.195, 0.591, 0.0, 0.214),           # fuel side
          (0.142, 0.758, 0.1, 0.0))             # oxidizer side


def multicomponent_diffusion(n: int = 200, seed: int = 0, length: float = 0.05,
                             d: float = 0.0025, x0: float = 0.025) -> Case:
    """1D multicomponent diffusion (Sec. IV.B, Eq. 30, Table IV) with synthetic
    species data: a periodic domain of ``length`` metres on ``n`` cells,
    p = 1 atm, u = 0, and T, Y_k = oxidizer value + (fuel - oxidizer) f(x) with
    f(x) = 1 - 0.5 exp(-(x - x0)^2/d^2) (reading: the printed exponent lost its
    square). Binary diffusion fits are drawn (``draw_binary_diffusion``): the
    case is meant for the mixture-averaged diffusion model of Eq. 26.
    Scales: L_ref = length, rho_ref = the fuel-side density, a_ref^2 = p/rho_ref."""
    rng = np.random.default_rng(seed)
    W = np.array(DIFF_W)
    sp = _draw_species(rng, W)
    sp.dbin_coef = draw_binary_diffusion(np.random.default_rng([seed, 25]), W)
    x = _centres(n, 0.0, length)
    f = 1.0 - 0.5 * np.exp(-((x - x0) / d) ** 2)
    Tf, To = DIFF_T
    Yf, Yo = np.array(DIFF_Y[0]), np.array(DIFF_Y[1])
    T = To + (Tf - To) * f
    Y = Yo[:, None] + (Yf - Yo)[:, None] * f[None, :]
    rho = P0_SBI / (R_U * np.sum(Y / W[:, None], axis=0) * T)
    rho_ref = P0_SBI / (R_U * np.sum(Yf / W) * Tf)
    a_ref2 = P0_SBI / rho_ref
    prim = _pack(1, rho / rho_ref, [np.zeros(n)], np.ones(n), Y)
    return Case("diffusion1d_n4", 1, (n, 1, 1), (0.0,) * 3, (1.0,) * 3,
                ((BC_PERIODIC, BC_PERIODIC), (0, 0), (0, 0)), sp, a_ref2, rho_ref, length,
                True, 0.5, prim, {"T": T, "f": f})


def uniform_state(dim: int, n: tuple, N: int, seed: int = 0, bc=BC_PERIODIC,
                  viscous: bool = True) -> Case:
    """A uniform random state (rho, u, p, Y) on a small box."""
    rng = np.random.default_rng(seed)
    sp = _draw_species(rng, np.array(rng.choice(W_SET, size=N)))
    nn = tuple(list(n) + [1] * (3 - len(n)))
    cells = nn[0] * nn[1] * nn[2]
    rho = rng.uniform(0.5, 2.0)
    vel = rng.uniform(-0.5, 0.5, size=dim)
    p = rng.uniform(0.5, 2.0)
    Y = rng.dirichlet(np.ones(N))
    prim = np.zeros((dim + 2 + N - 1, cells))
    prim[0] = rho
    prim[1:1 + dim] = vel[:, None]
    prim[1 + dim] = p
    prim[2 + dim:] = Y[:N - 1, None]
    bcs = tuple((bc, bc) if a < dim else (BC_TRANSMISSIVE, BC_TRANSMISSIVE) for a in range(3))
    return Case("uniform", dim, nn, (0.0,) * 3, (1.0,) * 3, bcs, sp,
                R_U * 300.0 / 0.028, 1.0, 1.0, viscous, 0.5, np.ascontiguousarray(prim))


def with_smooth_perturbation(case: Case, seed: int = 0, amp: float = 1e-3) -> Case:
    """Copy of ``case`` whose density and pressure are multiplied by
    1 + amp g and whose velocity components are shifted by amp g, each g a
    fresh seeded sum of six plane waves (wave numbers U[0.5, 3] per unit
    length of the unit cube the grid is mapped to, amplitudes U[-1, 1],
    phases U[0, 2 pi], divided by six). Mass fractions are unchanged. Such a
    state has no uniform region and no gas at rest, so no two stencil cells
    share an LLF maximum by round-off."""
    import dataclasses
    rng = np.random.default_rng([seed, 77])
    P = case.prim.copy()
    nx, ny, nz = case.n
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny,
                          (np.arange(nx) + 0.5) / nx, indexing="ij")

    def field_():
        g = np.zeros_like(x)
        for _ in range(6):
            k = rng.uniform(0.5, 3.0, 3)
            g += rng.uniform(-1, 1) * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z)
                                             + rng.uniform(0, 2 * np.pi))
        return g.reshape(-1) / 6

    d = case.dim
    P[0] *= 1 + amp * field_()
    for a in range(d):
        P[1 + a] += amp * field_()
    P[1 + d] *= 1 + amp * field_()
    return dataclasses.replace(case, prim=P, name=case.name + "_perturbed")


def smooth_periodic(dim: int, n: tuple, N: int, seed: int = 0, amp: float = 0.1,
                    viscous: bool = True, species=None, modes: int = 2) -> Case:
    """Random smooth periodic fields on [0, 1]^dim: each primitive is a base value
    plus a few seeded Fourier modes of relative amplitude ``amp``; mass fractions
    are a positive softmax-like mix so that they stay on the simplex."""
    rng = np.random.default_rng(seed)
    sp = species or _draw_species(rng, np.array(rng.choice(W_SET, size=N)))
    nn = tuple(list(n) + [1] * (3 - len(n)))
    xs = [_centres(nn[a], 0.0, 1.0) if a < dim else np.zeros(1) for a in range(3)]
    Z, Yg, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    coords = [X, Yg, Z]

    def field_():
        f = np.zeros_like(X)
        for _ in range(modes):
            kv = rng.integers(1, 3, size=dim)
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * kv[a] * coords[a] for a in range(dim)) + ph
            f += rng.uniform(-1, 1) * np.sin(arg)
        return f / modes

    rho = 1.0 + amp * field_()
    vel = [0.3 * rng.uniform(-1, 1) + amp * field_() for _ in range(dim)]
    p = 1.0 + amp * field_()
    w = np.stack([np.exp(amp * 5 * field_()) * rng.uniform(0.5, 1.5) for _ in range(N)])
    Y = w / w.sum(axis=0, keepdims=True)
    prim = _pack(dim, rho, vel, p, Y)
    bcs = tuple((BC_PERIODIC, BC_PERIODIC) if a < dim else (BC_TRANSMISSIVE, BC_TRANSMISSIVE)
                for a in range(3))
    return Case("smooth_periodic", dim, nn, (0.0,) * 3, (1.0,) * 3, bcs, sp,
                R_U * 300.0 / 0.028, 1.0, 1.0, viscous, 0.5, prim)


def density_wave(n: int, N: int = 2, seed: int = 0, amp: float = 0.2) -> Case:
    """rho = 1 + amp sin(2 pi x), u = 1, p = 1 on a periodic [0, 1], with every
    species given the same molar mass and c_p table (a W-identical mix), so that
    the exact solution is pure advection of the initial profile."""
    rng = np.random.default_rng(seed)
    sp1 = _draw_species(rng, np.array([0.028]))
    sp = Species(W=np.full(N, 0.028), cp_coef=np.repeat(sp1.cp_coef, N, axis=0),
                 h_off=np.zeros(N), mu_coef=np.repeat(sp1.mu_coef, N, axis=0),
                 kappa_coef=np.repeat(sp1.kappa_coef, N, axis=0))
    x = _centres(n, 0.0, 1.0)
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    u = np.ones(n)
    p = np.ones(n)
    Y = np.stack([np.full(n, 1.0 / N)] * N)
    Y[0] = 0.5 + 0.25 * np.sin(2 * np.pi * x)
    Y[1:] = (1.0 - Y[0]) / (N - 1)
    prim = _pack(1, rho, [u], p, Y)
    return Case("density_wave", 1, (n, 1, 1), (0.0,) * 3, (1.0,) * 3,
                ((BC_PERIODIC,) * 2, (0, 0), (0, 0)), sp, R_U * 300.0 / 0.028, 1.0, 1.0,
                False, 0.5, prim)
