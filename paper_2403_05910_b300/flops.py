"""Algorithmic FP64 operation counts of one RHS stage (roofline numerators).

Counted from the operations the method needs as the kernels evaluate them:
an add, multiply, divide, square root, exp or log counts 1, a fused
multiply-add counts 2 (the convention of the FP64 peak). Library expansions
of divide / sqrt / exp / log into several FP64 instructions are NOT counted,
so achieved rates computed from these numbers are lower bounds on the FP64
pipe's occupancy. d = dimension, N = species count, n_v = d + N + 1.
"""

WENO5 = 68          # one WENO5-JS reconstruction (smoothness, weights, candidates)
# one reconstruction of each scheme in its plain form (indicators as quadratic
# forms of the stencil values, weights, candidates, normalisation)
RECON = {5: WENO5, 6: 156, 7: 178}
NEWTON_ITER = 35    # one Newton temperature iteration on mixture coefficients
NEWTON_ITERS = 3    # nominal iterations per cell with the warm start


# Eigenvalue work of the LLF maxima that belongs to the cells, not the faces:
# per stencil cell u_n - c, u_n + c and u_n/2 (6 cells x 3), and the halving
# of the three maxima (3). Primitive recovery evaluates the per-cell part once
# per cell and axis (LLF_CELL), so the face count leaves all of it out.
LLF_FACE_MOVED = 6 * 3 + 3


def face_convective(d: int, N: int, weno: int = 5) -> int:
    """Roe state + PER projection + LLF maxima + 2 reconstructions per field +
    back-projection. The projection is counted for the 6-cell stencil (the
    two extra cells of WENO7 are not counted: a lower bound)."""
    nv = d + N + 1
    return 218 - LLF_FACE_MOVED + 71 * d + 103 * N + 2 * RECON[weno] * nv


def llf_cell(d: int) -> int:
    """Per cell: c/2, and per axis u/2, |u/2 - c/2|, |u/2 + c/2|."""
    return 1 + 3 * d


def face_positivity(d: int, N: int) -> int:
    """Blend of Eq. 17-20: both cells' physical fluxes, the LF flux, theta
    over the 2N one-sided partial densities (the blend itself is rare)."""
    nv = d + N + 1
    return 7 * nv + 8 + 16 * N


def face_viscous(d: int, N: int, diffusion: int = 0) -> int:
    """4th-order face values / derivatives, stress, heat and diffusion fluxes
    (diffusion = 1: a face value of D_sm per species and its own product)."""
    return 41 + 11 * d + 5 * d * d + 38 * N + (6 * N if diffusion else 0)


def face(d: int, N: int, viscous: bool, weno: int = 5, positivity: bool = False,
         diffusion: int = 0) -> int:
    return (face_convective(d, N, weno) + (face_viscous(d, N, diffusion) if viscous else 0) +
            (face_positivity(d, N) if positivity else 0))


def prim_cell(d: int, N: int, viscous: bool, diffusion: int = 0) -> int:
    """Primitive recovery (Newton, EOS, sound speed) + mixture transport
    (diffusion = 1 adds the binary fits, one exp per pair, and Eq. 26)."""
    base = 21 + 24 * N + NEWTON_ITERS * NEWTON_ITER + 24 + llf_cell(d)
    dsm = (11 * N * (N - 1) // 2 + N * (N + 6)) if (viscous and diffusion) else 0
    return base + ((7 + 31 * N + 13 * N * N) if viscous else 0) + dsm


def grad_cell(d: int, viscous: bool) -> int:
    return 5 * d * d if viscous else 0


def update_cell(d: int, N: int) -> int:
    nv = d + N + 1
    return nv * (3 * d + 3)


def per_cell_stage(case, weno: int = 5, positivity: bool = False, diffusion: int = 0) -> dict:
    """Flops of one stage over the whole grid, split by kernel class."""
    d, N, vis = case.dim, case.n_species, bool(case.viscous)
    n = case.n
    cells = case.cells
    ghosts = 4 if weno == 7 else 3
    pcells = 1
    for a in range(3):
        pcells *= (n[a] + 2 * ghosts) if a < d else 1
    nfaces = [((n[0] + (a == 0)) * (n[1] + (a == 1)) * (n[2] + (a == 2))) for a in range(d)]
    out = {
        "prim": prim_cell(d, N, vis, diffusion) * pcells,
        "grad": grad_cell(d, vis) * pcells,
        "face": face(d, N, vis, weno, positivity, diffusion) * sum(nfaces),
        "update": update_cell(d, N) * cells,
    }
    out["total"] = sum(out.values())
    return out


def hbm_bytes_per_cell_stage(case, stage: int) -> int:
    """Minimal traffic of one stage: read U^(s), read U^n (stages 2, 3), write
    U^(s+1), read + write T (the Newton warm start)."""
    nv = case.n_v
    return 8 * (nv + (nv if stage > 0 else 0) + nv + 2)
