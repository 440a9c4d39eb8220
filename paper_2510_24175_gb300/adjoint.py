"""Differentiable RK2 rollouts: a torch.autograd.Function over the C ABI.

forward: advances the state nsteps CFL steps with mhd_step, keeping a copy of
the state every k steps (checkpoints) and recording each step's dt and c_h on
the device (mhd_step_record: no host round trip per step; the record is read
once, when the forward pass ends).  k = 0 keeps every step's input state and
its first Runge-Kutta stage instead (two states per step in device memory:
7.5 GB for 200 steps of a 512^2 FP64 grid), and the backward pass then runs
only adjoint steps (mhd_adjoint_step_stage1), no forward recomputation.
backward (k > 0): for each k-step segment, last first, recomputes the segment's
states from its checkpoint with the recorded dt and c_h (mhd_step with
explicit dt, ch: bitwise the same states), keeping each recomputed step's
first Runge-Kutta stage (mhd_get_stage1), then applies the discrete adjoint
of one step with dt and c_h frozen from the last step of the segment to the
first: mhd_adjoint_step_stage1 with the kept stage, and for the segment's
last step, which is not recomputed, mhd_adjoint_step (which recomputes only
that step's first stage).  Every step of the method runs in the CUDA
library; torch holds the tensors.
"""
from __future__ import annotations

import torch

from . import MHD, MHD_FLAG_ADJOINT, Config


class MHDRollout(torch.autograd.Function):
    """U_N = MHDRollout.apply(U0, solver, nsteps, k).

    U0: conservative state, float64 CUDA tensor (9, nz, ny, nx); solver: an
    ``MHD`` created with ``MHD_FLAG_ADJOINT``; k: checkpoint interval, or 0 to
    keep every step's state and first stage (no recomputation)."""

    @staticmethod
    def forward(ctx, U0, solver: MHD, nsteps: int, k: int):
        assert solver.config.flags & MHD_FLAG_ADJOINT, "solver needs MHD_FLAG_ADJOINT"
        assert k >= 0
        solver.set_state(U0.detach().contiguous())
        ckpts, stage1 = [], []
        rec = torch.empty((max(nsteps, 1), 4), dtype=torch.float64, device=U0.device)
        for n in range(nsteps):
            if k == 0 or n % k == 0:
                ckpts.append(solver.get_state())
            solver.step()
            solver.step_record(rec[n])
            if k == 0:
                stage1.append(solver.get_stage1())
        UN = solver.get_state()
        solver.step_info()  # one synchronisation: raises if the device flagged a fault
        rec = rec.cpu().numpy()
        dts = [float(x) for x in rec[:nsteps, 1]]
        chs = [float(x) for x in rec[:nsteps, 2]]
        ctx.solver, ctx.nsteps, ctx.k = solver, nsteps, k
        ctx.ckpts, ctx.stage1, ctx.dts, ctx.chs = ckpts, stage1, dts, chs
        return UN

    @staticmethod
    def backward(ctx, gUN):
        solver, nsteps, k = ctx.solver, ctx.nsteps, ctx.k
        lam = gUN.contiguous().clone()
        if k == 0:  # every step's state and first stage were kept
            for n in reversed(range(nsteps)):
                out = torch.empty_like(lam)
                solver.adjoint_step_stage1(ctx.ckpts[n], ctx.stage1[n], lam, out, ctx.dts[n],
                                           ctx.chs[n])
                lam = out
            return lam, None, None, None
        nseg = len(ctx.ckpts)
        for s in reversed(range(nseg)):
            n0 = s * k
            n1 = min(n0 + k, nsteps)
            solver.set_state(ctx.ckpts[s])
            states, stage1 = [ctx.ckpts[s]], []
            for n in range(n0, n1 - 1):
                solver.step(ctx.dts[n], ctx.chs[n])
                stage1.append(solver.get_stage1())
                states.append(solver.get_state())
            for i in reversed(range(n1 - n0)):
                n = n0 + i
                out = torch.empty_like(lam)
                if i < len(stage1):
                    solver.adjoint_step_stage1(states[i], stage1[i], lam, out, ctx.dts[n],
                                               ctx.chs[n])
                else:
                    solver.adjoint_step(states[i], lam, out, ctx.dts[n], ctx.chs[n])
                lam = out
        return lam, None, None, None


def rollout_solver(problem) -> MHD:
    """An adjoint-capable FP64 solver for a Problem."""
    return MHD(Config.from_problem(problem, precision=0, flags=MHD_FLAG_ADJOINT))

