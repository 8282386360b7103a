"""Differentiable PFC rollouts: psi_T = S^n(psi_0; r) with gradients through the hand-written
adjoint step (pfc_step_adjoint).

The forward pass runs the plan's fused steps and keeps a checkpoint every `every` steps. The
backward pass walks the segments from last to first: it recomputes one segment from its
checkpoint, then applies the adjoint step to its states in reverse,
    lam_n = A lam_{n+1} - 3 psi_n^2 (B lam_{n+1}),
    dL/dr += < lam_{n+1}, d psi_{n+1} / dr >   (accumulated in FP64 on the device).
Where the plan has the fused adjoint (pfc_step_record / pfc_adjoint_segment), the recompute
records the segment in the plan's internal layout and the adjoint runs over the record with lam
kept in that layout; otherwise the segment's real states are kept and pfc_step_adjoint is
applied step by step. The result is dL/dpsi_0 = lam_0 and dL/dr. Memory: ceil(n / every)
checkpoints plus one segment. All arithmetic runs in the library's kernels; this module only
orders calls.
"""
from __future__ import annotations

import torch

from .binding import Plan


class PFCRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi0: torch.Tensor, r: torch.Tensor, plan: Plan, nsteps: int, every: int):
        if every < 1:
            raise ValueError("every must be >= 1")
        plan.set_r(float(r))
        x = psi0.detach().clone().contiguous()
        ckpts = []
        done = 0
        while done < nsteps:
            ckpts.append(x.clone())
            k = min(every, nsteps - done)
            plan.step(x, k)
            done += k
        ctx.plan, ctx.nsteps, ctx.every, ctx.ckpts, ctx.r = plan, nsteps, every, ckpts, float(r)
        ctx.r_shape, ctx.r_dtype = r.shape, r.dtype
        return x

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        plan = ctx.plan
        plan.set_r(ctx.r)
        lam = grad_out.detach().to(plan.real_dtype).contiguous().clone()
        dr = torch.zeros(1, dtype=torch.float64, device=lam.device)
        starts = list(range(0, ctx.nsteps, ctx.every))
        nbytes = plan.record_bytes(ctx.every)
        record = None
        if nbytes is not None:
            record = torch.empty(nbytes + 256, dtype=torch.uint8, device=lam.device)
            off = (-record.data_ptr()) % 256
            record = record[off:off + nbytes]
        for start, ck in reversed(list(zip(starts, ctx.ckpts))):
            k = min(ctx.every, ctx.nsteps - start)
            x = ck.clone()
            if record is not None:
                plan.step_record(x, k, record)
                plan.adjoint_segment(record, k, lam, dr)
                continue
            traj = [ck]
            for _ in range(k - 1):
                plan.step(x, 1)
                traj.append(x.clone())
            for n in reversed(range(k)):
                plan.step_adjoint(traj[n], lam, lam, dr)
        grad_r = dr.reshape(()).to(ctx.r_dtype).reshape(ctx.r_shape)
        return lam, grad_r, None, None, None


def rollout(psi0: torch.Tensor, r: torch.Tensor, plan: Plan, nsteps: int, every: int = 20):
    """psi after nsteps semi-implicit steps from psi0 with operator parameter r (single field);
    differentiable with respect to psi0 and r, with checkpoints every `every` steps."""
    return PFCRollout.apply(psi0, r, plan, nsteps, every)
