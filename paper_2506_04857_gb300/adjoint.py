"""Discrete adjoint of the AF MHD time stepper behind torch.autograd.

AFSteps runs n SSP-RK3 steps through libaf, records every step's dt and keeps
a checkpoint of the state every `checkpoint_every` steps.  It also records,
from the limiter counters, whether every positivity limiter stayed inactive.
Its backward pass recomputes each segment from its checkpoint (with the
recorded dt), keeping every step's stage states, and applies
af_adjoint_step_stages in reverse, so gradients are those of
the discrete scheme with dt held fixed, or, with dt_sensitivity=True, with
every step's dt differentiated as the function of its state that af_step
forms (dt = cfl / (max varrho_1/dx + max varrho_2/dy), a subgradient at the
maximising DoFs).  When every positivity limiter stayed inactive and the
shock sensor is off (kappa = 0), the transpose is that of the smooth branch.
Otherwise the backward pass records, while it recomputes a segment (bitwise
the forward steps), every stage's limiter coefficients (af_record_coeffs) and
applies af_adjoint_step_frozen: the gradient along the branch the forward pass
took, with theta^s, theta_ij, the face theta and the scaling-limiter theta*,
theta** held at their recorded values.

magnetic_energy is the objective of the adjoint workload: the total magnetic
energy dx dy sum_cells sum_{l,m} w_l w_m |B(U^{l,m})|^2 / 2 on the 3x3 Simpson
nodes of every cell (corners, faces, and the bi-parabola centre value).
"""
from __future__ import annotations

from typing import List

import torch

from . import (AF_BC_PERIODIC, AF_OK, AFError, Solver, af_adjoint_step_frozen, af_adjoint_step_stages,
               af_coeff_len, af_get_params, af_get_stage, af_get_state, af_last_error, af_record_coeffs,
               af_set_state, af_stage, af_status, af_step)

# counters of the positivity limiters (and of non-admissible states)
LIMITER_COUNTERS = ("src_limited", "lambda_lt1", "face_theta_lt1", "shrink", "point_limited", "center_limited",
                    "nonadmissible")


def _counters(solver):
    rc, cnt = af_status(solver.ctx)
    if rc != AF_OK:
        raise AFError(rc, af_last_error(solver.ctx))
    return cnt


def magnetic_energy(U: List[torch.Tensor], dx: float, dy: float, bc: int = AF_BC_PERIODIC) -> torch.Tensor:
    """Total magnetic energy of a state on the 3x3 Simpson nodes of every cell."""
    A, X, Y, Cn = U
    ny, nx = A.shape[1], A.shape[2]

    def right(t):   # value at index i+1 along x (cells -> their right face / corner)
        return torch.roll(t, -1, dims=2) if bc == AF_BC_PERIODIC else t[:, :, 1:]

    def up(t):
        return torch.roll(t, -1, dims=1) if bc == AF_BC_PERIODIC else t[:, 1:, :]

    XL = X[:, :ny, :nx]
    XR = right(X)[:, :ny, :nx]
    YD = Y[:, :ny, :nx]
    YU = up(Y)[:, :ny, :nx]
    C00 = Cn[:, :ny, :nx]
    C10 = right(Cn)[:, :ny, :nx]
    C01 = up(Cn)[:, :ny, :nx]
    C11 = up(right(Cn))[:, :ny, :nx]
    Uc = 2.25 * A - 0.25 * ((XL + XR) + (YD + YU)) - 0.0625 * ((C00 + C10) + (C01 + C11))
    w = (1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)
    nodes = [[C00, YD, C10], [XL, Uc, XR], [C01, YU, C11]]   # nodes[m][l]
    J = 0.0
    for m in range(3):
        for l in range(3):
            B = nodes[m][l][4:7]
            J = J + (w[l] * w[m] * 0.5) * (B * B).sum()
    return J * dx * dy


class AFSteps(torch.autograd.Function):
    """out = U after n steps of solver from U0 (four CUDA float64 tensors)."""

    @staticmethod
    def forward(ctx, solver: Solver, nsteps: int, checkpoint_every: int, dt_sensitivity: bool, *U0):
        ctx.solver = solver
        ctx.dt_sensitivity = bool(dt_sensitivity)
        ctx.nsteps = nsteps
        ctx.every = max(1, int(checkpoint_every))
        dts = torch.empty(max(nsteps, 1), dtype=torch.float64, device=U0[0].device)
        checkpoints = []
        af_set_state(solver.ctx, [u.detach() for u in U0])
        before = _counters(solver)
        for n in range(nsteps):
            if n % ctx.every == 0:
                checkpoints.append(af_get_state(solver.ctx))
            af_step(solver.ctx, dts[n:n + 1])
        out = af_get_state(solver.ctx)
        after = _counters(solver)
        ctx.inactive = all(after[k] == before[k] for k in LIMITER_COUNTERS)
        ctx.smooth = ctx.inactive and af_get_params(solver.ctx)["kappa"] == 0.0
        ctx.dts = dts
        ctx.checkpoints = checkpoints
        return tuple(out)

    @staticmethod
    def backward(ctx, *grads):
        s = ctx.solver
        L = af_coeff_len(s.ctx)
        lam = [g.contiguous() if g is not None else torch.zeros_like(t)
               for g, t in zip(grads, ctx.checkpoints[0] if ctx.checkpoints else grads)]
        for seg in reversed(range(len(ctx.checkpoints))):
            n0 = seg * ctx.every
            n1 = min(ctx.nsteps, n0 + ctx.every)
            states = []   # per step: U^n and the stage states U1, U2 (and U3 = U^{n+1})
            af_set_state(s.ctx, ctx.checkpoints[seg])
            for n in range(n0, n1):
                Un = af_get_state(s.ctx)
                dt = ctx.dts[n:n + 1]
                co = None
                if not ctx.smooth:   # the limited branch: this step's limiter coefficients
                    co = torch.empty(3 * L, dtype=torch.float64, device=Un[0].device)
                    af_record_coeffs(s.ctx, co)
                af_stage(s.ctx, 0, dt)
                U1 = af_get_stage(s.ctx)
                af_stage(s.ctx, 1, dt)
                U2 = af_get_stage(s.ctx)
                af_stage(s.ctx, 2, dt)
                U3 = af_get_stage(s.ctx) if ctx.dt_sensitivity else None
                if co is not None:
                    af_record_coeffs(s.ctx, None)
                states.append((Un, U1, U2, U3, co))
            for n in reversed(range(n0, n1)):
                Un, U1, U2, U3, co = states[n - n0]
                af_set_state(s.ctx, Un)
                if co is None:
                    lam = af_adjoint_step_stages(s.ctx, ctx.dts[n:n + 1], U1, U2, lam, U3=U3,
                                                 dt_sensitivity=ctx.dt_sensitivity)
                else:
                    lam = af_adjoint_step_frozen(s.ctx, ctx.dts[n:n + 1], U1, U2, co, lam, U3=U3,
                                                 dt_sensitivity=ctx.dt_sensitivity)
        return (None, None, None, None) + tuple(lam)


def af_steps(solver: Solver, U0: List[torch.Tensor], nsteps: int, checkpoint_every: int = 20,
             dt_sensitivity: bool = False):
    """Differentiable n-step solve (see AFSteps)."""
    return list(AFSteps.apply(solver, nsteps, checkpoint_every, dt_sensitivity, *U0))
