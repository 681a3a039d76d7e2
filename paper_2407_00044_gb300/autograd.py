"""Autograd layer over the Stream-K GEMM: forward C = A @ B through
``sk_gemm``; backward dA = dC @ B^T and dB = A^T @ dC through
``sk_gemm_backward`` (one grouped launch reading the transposed operands
in place)."""
from __future__ import annotations

import torch

from . import api


class SkMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, config=None):
        ctx.save_for_backward(A, B)
        ctx.config = config
        return api.gemm(A, B, config=config)

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous().to(A.dtype)
        dA, dB = api.gemm_backward(A, B, dC, need_dA=ctx.needs_input_grad[0],
                                   need_dB=ctx.needs_input_grad[1], config=ctx.config)
        return dA, dB, None


def sk_matmul(A: torch.Tensor, B: torch.Tensor, config=None) -> torch.Tensor:
    return SkMatmul.apply(A, B, config)
