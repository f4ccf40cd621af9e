"""torch.autograd bindings of the adjoint (argument marshalling only).

Every derivative is computed by the library's kernels through the C-ABI:
``xf_set_primitive_adjoint`` (EOS), ``xf_step_rk3_adjoint`` or its taped form
(one SSP-RK3 step, Eq. 16, with the hand-written RHS adjoint) and
``xf_objective_mixing``. The
functions here only move device buffers between those calls:

* ``FromPrimitive``: primitive fields P (rho, u, p, Y) -> conserved U.
* ``RK3Steps``: ``steps`` fixed-dt SSP-RK3 steps. The forward pass keeps a
  checkpoint (U and the Newton warm start T) every ``every`` steps; the
  backward pass re-runs each segment from its checkpoint to regain the
  step-start states, then walks the segment's steps in reverse. With ``tape``
  the re-run also keeps every step's two intermediate stage states
  (``xf_step_rk3_tape``, 2 ``every`` extra states per segment) and the reverse
  steps take them (``xf_step_rk3_adjoint_tape``) instead of recomputing them.
  With the positivity-preserving blend the re-run also keeps every step's
  flux tape (``xf_step_rk3_tape_flux``: the unblended convective face fluxes
  of its three stages), which the reverse of the blend reads instead of
  recomputing them.
* ``MixingObjective``: J = sum Y_s (1 - Y_s) dV of one species.

The time step is frozen (a fixed dt), so the discrete map is differentiable
except at the documented kinks (LLF maxima ties, |u| at 0).
"""
from __future__ import annotations

import torch

from .xf import Solver


def _empty_state(solver: Solver, device):
    return torch.empty((solver.nv, solver.cells), dtype=torch.float64, device=device)


class FromPrimitive(torch.autograd.Function):
    @staticmethod
    def forward(ctx, P, solver):
        P = P.contiguous()
        solver.set_primitive(P)
        U = _empty_state(solver, P.device)
        solver.get_state(U)
        ctx.solver = solver
        ctx.save_for_backward(P)
        return U

    @staticmethod
    def backward(ctx, Ubar):
        (P,) = ctx.saved_tensors
        Pbar = torch.empty_like(P)
        ctx.solver.set_primitive_adjoint(P, Ubar.contiguous(), Pbar)
        return Pbar, None


class RK3Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt, steps, every, tape=True):
        U0 = U0.contiguous()
        dev = U0.device
        # keep the solver's current Newton warm start (e.g. the exact T that
        # FromPrimitive left behind)
        T0 = torch.empty(solver.cells, dtype=torch.float64, device=dev)
        solver.get_state(None, T0)
        solver.set_state(U0, T0)
        ck_U, ck_T = [], []
        for k in range(steps):
            if k % every == 0:
                U = _empty_state(solver, dev)
                T = torch.empty(solver.cells, dtype=torch.float64, device=dev)
                solver.get_state(U, T)
                ck_U.append(U)
                ck_T.append(T)
            solver.step(dt)
        Un = _empty_state(solver, dev)
        solver.get_state(Un)
        ctx.solver, ctx.dt, ctx.steps, ctx.every, ctx.tape = solver, dt, steps, every, tape
        ctx.ck = (ck_U, ck_T)
        return Un

    @staticmethod
    def backward(ctx, Ubar):
        s, dt, steps, every = ctx.solver, ctx.dt, ctx.steps, ctx.every
        ck_U, ck_T = ctx.ck
        Ub = Ubar.contiguous().clone()
        dev = Ub.device
        for seg in reversed(range(len(ck_U))):
            start = seg * every
            n = min(every, steps - start)
            s.set_state(ck_U[seg], ck_T[seg])
            states = []
            for _ in range(n):
                U = _empty_state(s, dev)
                T = torch.empty(s.cells, dtype=torch.float64, device=dev)
                s.get_state(U, T)
                if ctx.tape:
                    U1, U2 = _empty_state(s, dev), _empty_state(s, dev)
                    Fh = (torch.empty(s.tape_flux_len(), dtype=torch.float64, device=dev)
                          if s.positivity else None)
                    s.step_tape(dt, U1, U2, Fhat=Fh)
                    states.append((U, T, U1, U2, Fh))
                else:
                    s.step(dt)
                    states.append((U, T))
            for st in reversed(states):
                s.set_state(st[0], st[1])
                if ctx.tape:
                    s.step_adjoint_tape(dt, st[2], st[3], Ub, Fhat=st[4])
                else:
                    s.step_adjoint(dt, Ub)
        return Ub, None, None, None, None, None


class MixingObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, solver, species):
        U = U.contiguous()
        J = torch.zeros(1, dtype=torch.float64, device=U.device)
        Ubar = torch.empty_like(U)
        solver.objective_mixing(U, species, J, Ubar)
        ctx.save_for_backward(Ubar)
        return J[0]

    @staticmethod
    def backward(ctx, gJ):
        (Ubar,) = ctx.saved_tensors
        return Ubar * gJ, None, None


def mixing_after_steps(P0, solver, dt, steps, every, species, tape=True):
    """J(P0): primitive fields -> EOS -> ``steps`` RK3 steps -> mixing measure."""
    U0 = FromPrimitive.apply(P0, solver)
    UT = RK3Steps.apply(U0, solver, dt, steps, every, tape)
    return MixingObjective.apply(UT, solver, species)
