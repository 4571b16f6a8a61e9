"""Reverse-mode differentiation of the maintained programs through
``torch.autograd.Function``.

The forward pass builds a LINVIEW program on the device (which keeps every
intermediate view resident: the squarings P_h of A^k, or the iterates T_i of
T_{i+1} = A T_i + B); the backward pass runs the library's adjoint on those
views (linview_adjoint_power / linview_adjoint_iteration_seed).  Both passes
run in the CUDA library; this module only marshals tensors.  The program
(and with it the views the backward pass reads) lives as long as the autograd
graph that holds it, so backward may run more than once.

Adjoints:
  A^k by repeated squaring, P_{2h} = P_h P_h:  Gbar_h = Gbar_{2h} P_h^T + P_h^T Gbar_{2h},
  starting from Gbar_k = dL/dA^k; dL/dA = Gbar_1 (= sum_j (A^T)^j G (A^T)^(k-1-j)).
  T_k of T_i = A T_{i-1} + B:  G_k = dL/dT_k, G_i = A^T G_{i+1};
  dL/dA = sum_i G_i T_{i-1}^T, dL/dB = sum_i G_i, dL/dT_0 = A^T G_1.
"""
from __future__ import annotations

import torch
from torch.autograd.function import once_differentiable

from .linview import Program


def _prec(t):
    if t.dtype == torch.float64:
        return "f64"
    if t.dtype == torch.float32:
        return "f32"
    raise TypeError(f"float32 or float64 expected, got {t.dtype}")


def _cuda(t):
    if not t.is_cuda:
        raise ValueError("CUDA tensors expected (there is no CPU path)")
    return t.detach().contiguous()


class MatrixPower(torch.autograd.Function):
    """A -> A^k (k a power of two), by the exponential model's squarings."""

    @staticmethod
    def forward(ctx, A, k):
        A = _cuda(A)
        prog = Program("power", [A], k=int(k), r_max=1, precision=_prec(A))
        out = prog.read_view(int(k).bit_length() - 1)
        ctx.prog = prog
        return out

    @staticmethod
    @once_differentiable
    def backward(ctx, G):
        dA = None
        if ctx.needs_input_grad[0]:
            dA = torch.empty_like(G, memory_format=torch.contiguous_format)
            ctx.prog.adjoint_power(G.contiguous(), dA)
        return dA, None


class GeneralIteration(torch.autograd.Function):
    """(A, B, T_0) -> T_k with T_i = A T_{i-1} + B (Section 4.3)."""

    @staticmethod
    def forward(ctx, A, B, T0, k):
        A, B, T0 = _cuda(A), _cuda(B), _cuda(T0)
        prog = Program("iteration", [A, B, T0], k=int(k), r_max=1, precision=_prec(A))
        out = prog.read_view(int(k))  # view k = T_k
        ctx.prog = prog
        return out

    @staticmethod
    @once_differentiable
    def backward(ctx, G):
        G = G.contiguous()
        n, p = G.shape
        need_a, need_b, need_t = ctx.needs_input_grad[:3]
        dA = G.new_empty((n, n)) if need_a else None
        dB = G.new_empty((n, p)) if need_b else None
        dT0 = G.new_empty((n, p)) if need_t else None
        if need_a or need_b or need_t:
            ctx.prog.adjoint_iteration_seed(G, dA=dA, dB=dB, dT0=dT0)
        return dA, dB, dT0, None


def matrix_power(A, k):
    return MatrixPower.apply(A, k)


def general_iteration(A, B, T0, k):
    return GeneralIteration.apply(A, B, T0, k)
