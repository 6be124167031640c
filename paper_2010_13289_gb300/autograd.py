"""torch.autograd.Function wrapper of an SSP-RK3 rollout with the frozen-branch adjoint.

Forward: nsteps tenom_rk3_step calls at a fixed dt (dt does not depend on the state, so
no derivative flows through it), keeping the state every `checkpoint_every` steps.
Backward: for each segment, last first, the forward is recomputed from its checkpoint with
tenom_rk3_step_record (stage states and cutoff flags taped), then the segment is reversed
step by step with tenom_rk3_step_adjoint_tape.  Device memory: the checkpoints plus one
segment's tapes (checkpoint_every x (state + 2 stage states + 3 flag sets)).
"""
import math

import torch


class Rk3Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt, nsteps, checkpoint_every):
        dt_dev = torch.tensor([float(dt)], dtype=torch.float64, device="cuda")
        U = U0.detach().clone().contiguous()
        ckpts = []
        for n in range(nsteps):
            if n % checkpoint_every == 0:
                ckpts.append(U.clone())
            solver.rk3_step(U, dt_dev)
        ctx.solver = solver
        ctx.dt_dev = dt_dev
        ctx.nsteps = nsteps
        ctx.every = checkpoint_every
        ctx.ckpts = ckpts
        return U

    @staticmethod
    def backward(ctx, grad):
        S = ctx.solver
        dt_dev = ctx.dt_dev
        Ubar = grad.detach().contiguous().clone()
        nseg = len(ctx.ckpts)
        out = S.tensor()
        for seg in reversed(range(nseg)):
            n0 = seg * ctx.every
            n1 = min(ctx.nsteps, n0 + ctx.every)
            U = ctx.ckpts[seg].clone()
            states, tapes = [], []
            for _ in range(n0, n1):
                states.append(U.clone())
                tape = S.new_tape()
                S.rk3_step_record(U, dt_dev, tape)
                tapes.append(tape)
            for k in reversed(range(n1 - n0)):
                S.rk3_step_adjoint(states[k], dt_dev, Ubar, tape=tapes[k], out=out)
                Ubar, out = out, Ubar
            del states, tapes
        return Ubar, None, None, None, None


def rollout(U0, solver, dt, nsteps, checkpoint_every=20):
    """U(nsteps) from U0 with a differentiable (frozen-branch adjoint) backward."""
    return Rk3Rollout.apply(U0, solver, dt, nsteps, checkpoint_every)
