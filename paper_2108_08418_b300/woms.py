"""Differentiable unrolled weighted offset min-sum (autograd over the CUDA adjoint).

`woms_loss(code, llr, synd, target, alpha, beta, ckpt_every)` returns the mean
binary cross-entropy of the decoder's final posteriors against the target
bits; its backward runs the library's hand-written adjoint kernels (segment
recomputation from checkpoints every `ckpt_every` iterations).  alpha and beta
are float32 CUDA tensors [T][2]: per iteration, per check-degree class, the
scale and the offset of the min-sum check messages.
"""
from __future__ import annotations

import torch

from . import Code, qkdrec_woms_backward, qkdrec_woms_forward, qkdrec_woms_workspace_size


class WeightedMinSumLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, beta, code: Code, llr, synd, target, ckpt_every: int):
        alpha = alpha.detach().contiguous()
        beta = beta.detach().contiguous()
        F = llr.numel() // code.n
        ws = torch.empty(qkdrec_woms_workspace_size(code, F, alpha.shape[0], ckpt_every), dtype=torch.uint8,
                         device=llr.device)
        loss, _ = qkdrec_woms_forward(code, llr, synd, target, alpha, beta, ckpt_every, ws)
        ctx.save_for_backward(alpha, beta, llr, synd, target)
        ctx.code, ctx.ckpt_every, ctx.ws = code, ckpt_every, ws
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        alpha, beta, llr, synd, target = ctx.saved_tensors
        ga, gb = qkdrec_woms_backward(ctx.code, llr, synd, target, alpha, beta, ctx.ckpt_every, ctx.ws)
        return grad_out * ga, grad_out * gb, None, None, None, None, None


def woms_loss(code: Code, llr, synd, target, alpha, beta, ckpt_every: int = 5):
    return WeightedMinSumLoss.apply(alpha, beta, code, llr, synd, target, ckpt_every)
