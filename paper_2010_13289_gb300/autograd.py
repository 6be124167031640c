"""torch.autograd.Function wrapper of an SSP-RK3 rollout with the frozen-branch adjoint.

Forward: nsteps tenom_rk3_step calls at a fixed dt (dt does not depend on the state, so
no derivative flows through it), keeping the state every `checkpoint_every` steps.
Backward: for each segment, last first, the forward is recomputed from its checkpoint with
the stage states and, per stage, either the linearisation (tenom_rk3_step_record_lin; the
reverse reads the frozen linear reconstructions) or only the cutoff flags
(tenom_rk3_step_record; the reverse rebuilds them) taped; then the segment is reversed step
by step.  Device memory: the checkpoints plus one segment's tapes, checkpoint_every x
(state + 2 stage states + 3 linearisations or flag sets).  tape="auto" takes the
linearisation when one segment of it fits in half the free device memory.
"""
import math

import torch


class Rk3Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, solver, dt, nsteps, checkpoint_every, tape):
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
        ctx.linear = _use_linear(solver, min(checkpoint_every, nsteps), tape)
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
                tape = S.new_tape(linear=ctx.linear)
                S.rk3_step_record(U, dt_dev, tape)
                tapes.append(tape)
            for k in reversed(range(n1 - n0)):
                S.rk3_step_adjoint(states[k], dt_dev, Ubar, tape=tapes[k], out=out)
                Ubar, out = out, Ubar
            del states, tapes
        return Ubar, None, None, None, None, None


def _use_linear(solver, steps, tape):
    if tape in ("linear", "flags"):
        return tape == "linear"
    if tape != "auto":
        raise ValueError("tape must be 'auto', 'linear' or 'flags'")
    free, _ = torch.cuda.mem_get_info()
    need = steps * (solver.tape_bytes(linear=True) + 8 * solver.nv * math.prod(solver.shape))
    return need <= free // 2


def rollout(U0, solver, dt, nsteps, checkpoint_every=20, tape="auto"):
    """U(nsteps) from U0 with a differentiable (frozen-branch adjoint) backward."""
    return Rk3Rollout.apply(U0, solver, dt, nsteps, checkpoint_every, tape)
