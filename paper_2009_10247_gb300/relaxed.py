"""torch.autograd.Function over liblp's relaxed fixpoint (lp_relaxed_* in include/lp.h).

Forward and backward both run in liblp's kernels; this module allocates the checkpoint and
scratch buffers with torch and marshals arguments.
"""
import torch

from .lp import Program


class RelaxedFixpoint(torch.autograd.Function):
    """v_T of the relaxed fixpoint for weights (float [n_rules]) and v0 (float [n', b])."""

    @staticmethod
    def forward(ctx, weights, v0, prog: Program, steps: int, tau: float, ckpt_every: int):
        weights = weights.detach().contiguous().float()
        v0 = v0.detach().contiguous().float()
        b = v0.shape[1]
        ck, sc = prog.relaxed_workspace(b, steps, ckpt_every)
        ckpt = torch.empty(ck, dtype=torch.float32, device=v0.device)
        vT = torch.empty_like(v0)
        prog.relaxed_forward(weights, v0, b, steps, tau, ckpt_every, ckpt, vT)
        ctx.prog, ctx.steps, ctx.tau, ctx.ckpt_every, ctx.scratch_floats = prog, steps, tau, ckpt_every, sc
        ctx.save_for_backward(weights, ckpt)
        ctx.v0_shape = v0.shape
        return vT

    @staticmethod
    def backward(ctx, gT):
        weights, ckpt = ctx.saved_tensors
        gT = gT.contiguous().float()
        scratch = torch.empty(ctx.scratch_floats, dtype=torch.float32, device=gT.device)
        dw = torch.empty_like(weights)
        dv0 = torch.empty(ctx.v0_shape, dtype=torch.float32, device=gT.device)
        ctx.prog.relaxed_backward(weights, gT, ctx.v0_shape[1], ctx.steps, ctx.tau, ctx.ckpt_every, ckpt, scratch,
                                  dw, dv0)
        return dw, dv0, None, None, None, None


def relaxed_fixpoint(prog: Program, weights, v0, steps: int, tau: float, ckpt_every: int = 8):
    """Differentiable v_T (see RelaxedFixpoint)."""
    return RelaxedFixpoint.apply(weights, v0, prog, steps, tau, ckpt_every)
