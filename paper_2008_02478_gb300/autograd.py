"""``torch.autograd.Function`` over an RK4 trajectory of the LLG equation with
checkpointed recomputation.

Forward: n_steps RK4 steps of the library (boris_llg_step), keeping the state
every ``ckpt`` steps.  Backward: for each segment, newest first, the states of
the segment are recomputed from its checkpoint and the library's discrete
adjoint of one RK4 step (boris_llg_step_backward) is applied step by step in
reverse, accumulating dL/dMs and dL/dKu.  Memory: n_steps/ckpt checkpoints
plus ckpt states of one segment.
"""
from __future__ import annotations

import torch

from .binding import LLGParams, Plan


def _params(base: LLGParams, Ms_map, Ku_map) -> LLGParams:
    p = LLGParams(**{k: getattr(base, k) for k in base.__dataclass_fields__})
    p.Ms_map = Ms_map
    p.Ku_map = Ku_map
    return p


class BorisTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, Ms_map, Ku_map, plan: Plan, base: LLGParams, n_steps: int, dt: float, ckpt: int = 50):
        prm = _params(base, Ms_map.detach().contiguous(), Ku_map.detach().contiguous())
        m = m0.detach().clone().contiguous()
        ckpts = [m.clone()]
        for s in range(n_steps):
            plan.llg_step(m, prm, dt)
            if (s + 1) % ckpt == 0 and s + 1 < n_steps:
                ckpts.append(m.clone())
        ctx.plan, ctx.base, ctx.n_steps, ctx.dt, ctx.ckpt = plan, base, n_steps, dt, ckpt
        ctx.save_for_backward(prm.Ms_map, prm.Ku_map, *ckpts)
        return m

    @staticmethod
    def backward(ctx, g_out):
        Ms_map, Ku_map, *ckpts = ctx.saved_tensors
        plan, n_steps, dt, ckpt = ctx.plan, ctx.n_steps, ctx.dt, ctx.ckpt
        prm = _params(ctx.base, Ms_map, Ku_map)
        g = g_out.contiguous().clone()
        g_next = torch.empty_like(g)
        gMs = torch.zeros_like(Ms_map)
        gKu = torch.zeros_like(Ku_map)
        nseg = len(ckpts)
        for seg in range(nseg - 1, -1, -1):
            start = seg * ckpt
            end = min(n_steps, start + ckpt)
            states = [ckpts[seg].clone()]
            m = ckpts[seg].clone()
            for _ in range(start, end - 1):
                plan.llg_step(m, prm, dt)
                states.append(m.clone())
            for s in range(end - start - 1, -1, -1):
                plan.llg_step_backward(states[s], prm, dt, g, g_next, gMs, gKu)
                g, g_next = g_next, g
        return g, gMs, gKu, None, None, None, None, None


def trajectory(m0, Ms_map, Ku_map, plan: Plan, base: LLGParams, n_steps: int, dt: float, ckpt: int = 50):
    """Differentiable final state of n_steps RK4 steps from m0 (w.r.t. m0, Ms_map, Ku_map)."""
    return BorisTrajectory.apply(m0, Ms_map, Ku_map, plan, base, n_steps, dt, ckpt)
