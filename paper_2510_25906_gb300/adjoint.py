"""Differentiation of the residual and of SSP-RK3 trajectories (FP64).

``ResidualFunction`` exposes hfv_residual / hfv_residual_vjp to
torch.autograd with the cell classes frozen (the detector, tagging and Harten
decisions of Sec. 2.5 taken at the forward state).  ``rk3_gradient`` carries
an objective through several SSP-RK3 steps and back: the forward sweep keeps
one checkpoint per step (the state and the three stages' classes), the
backward sweep recomputes the stages of one step from its checkpoint and
applies the transposed stage updates, so the memory is one state per step,
not three stages' operators.  The step size of each step is the forward
sweep's (CFL from the state at the start of the step) and is held fixed.
"""
from __future__ import annotations

import numpy as np

from . import hfv as H


def _torch():
    import torch
    return torch


class ResidualFunction:
    """R = ResidualFunction.apply(U, scheme): the FP64 residual of U
    (contiguous CUDA FP64 [nv, n]); its backward is hfv_residual_vjp with the
    classes of the forward evaluation."""

    _fn = None

    @classmethod
    def apply(cls, U, scheme):
        """The residual of U under `scheme` (an FP64 hfv.Scheme), recorded
        for autograd."""
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, U, sch):
                    c = torch.empty(sch.n_cells, dtype=torch.uint8, device=U.device)
                    R = sch.residual(U.detach().contiguous(), class_out=c)
                    ctx.save_for_backward(U.detach().contiguous(), c)
                    ctx.sch = sch
                    return R

                @staticmethod
                def backward(ctx, gR):
                    U, c = ctx.saved_tensors
                    return ctx.sch.residual_vjp(U, c, gR.contiguous()), None

            cls._fn = _F
        return cls._fn.apply(U, scheme)


def _stages(sch, U, dt, classes=None):
    """The three stages of one SSP-RK3 step (Shu-Osher form); returns
    (U1, U2, U3, [c1, c2, c3]).  With classes given they are forced."""
    torch = _torch()
    out_cls = []
    Ws = [U]
    for k, (a, b) in enumerate(((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))):
        Us = Ws[-1]
        c = torch.empty(sch.n_cells, dtype=torch.uint8, device=U.device)
        if classes is None:
            R = sch.residual(Us, class_out=c)
        else:
            c.copy_(classes[k])
            R = sch.residual(Us, forced=c)
        out_cls.append(c)
        Ws.append(a * U + b * (Us + dt * R))
    return Ws[1], Ws[2], Ws[3], out_cls


def rk3_gradient(sch, U0, steps: int, dJdU, cfl: float = 0.5, dt: float | None = None):
    """J(U_N) after `steps` SSP-RK3 steps from U0 and dJ/dU0.

    dJdU(U_N) -> (J, dJ/dU_N) gives the objective and its gradient.  dt:
    fixed step, or None for each step's CFL step from its starting state.
    Returns (J, dJ/dU0, U_N, dts)."""
    U = U0.detach().clone().contiguous()
    ckpt = []
    dts = []
    for _ in range(steps):
        h = float(dt) if dt is not None else float(sch.compute_dt(U, cfl)[0].item())
        # hfv_step_classes: the step, with its stages' classes as the checkpoint
        U3, cls = sch.step_classes(U, h)
        ckpt.append((U, cls, h))
        dts.append(h)
        U = U3
    J, lam = dJdU(U)
    lam = lam.contiguous()
    for U, cls, h in reversed(ckpt):
        sch.step_vjp(U, cls, h, lam)       # the transposed stages, in the library
    return J, lam, U, dts


def density_square_integral(vol):
    """J(U) = sum_c |V_c| rho_c^2 and its gradient (the objective of the
    adjoint workload)."""
    torch = _torch()

    def f(U):
        v = torch.as_tensor(vol, device=U.device)
        J = float((v * U[0] * U[0]).sum().item())
        g = torch.zeros_like(U)
        g[0] = 2.0 * v * U[0]
        return J, g
    return f
