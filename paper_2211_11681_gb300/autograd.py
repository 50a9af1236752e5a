"""torch.autograd.Functions over the S-format library (argument marshalling only; every
forward and backward step runs in libsformat.so).

    MaskedMul.apply(A, B, plan)            C = P_{S_C}(A B); backward by s_mul_masked_adjoint
    SqrtmNS.apply(A, pattern, steps, c, prec, refine)
                                           A^{1/2} by coupled Newton-Schulz with per-step
                                           checkpoints (Y_k, Z_k); backward by
                                           s_funm_sqrt_backward_prec with c frozen.
                                           prec "fp64": double iteration and reverse mode;
                                           "fp32": float iteration with `refine` double
                                           residual corrections, float checkpoints, float
                                           reverse mode
    QuadForm.apply(X, pattern, z)          z^T X z over the pattern's blocks
"""
import torch

from . import sformat as sf


class MaskedMul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, plan):
        C = torch.empty(plan.pats[2].nnz, dtype=A.dtype, device=A.device)
        plan.mul(A.contiguous(), B.contiguous(), C)
        ctx.save_for_backward(A, B)
        ctx.plan = plan
        return C

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dA = torch.empty_like(A) if ctx.needs_input_grad[0] else None
        dB = torch.empty_like(B) if ctx.needs_input_grad[1] else None
        ctx.plan.adjoint(dC.contiguous(), A, B, dA, dB)
        return dA, dB, None


class SqrtmNS(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, pattern, steps, c, prec="fp64", refine=0):
        if c is None or c <= 0:
            # resolve the automatic scale here, so that backward differentiates the same
            # iteration with the same frozen c
            c = 1.01 * sf.norm_est(pattern, A.contiguous(), 50)
        nnz = pattern.nnz
        ck = torch.empty(2 * steps * nnz + 4, dtype=torch.float32 if prec == "fp32" else torch.float64,
                         device=A.device)
        F = torch.empty_like(A)
        sf.funm(pattern, "sqrt", A.contiguous(), F, steps=steps, scale=c, checkpoints=ck, prec=prec, refine=refine)
        ctx.save_for_backward(ck)
        ctx.pattern, ctx.steps, ctx.c, ctx.prec = pattern, steps, c, prec
        return F

    @staticmethod
    def backward(ctx, dF):
        (ck,) = ctx.saved_tensors
        dA = torch.empty_like(dF)
        sf.sqrt_backward(ctx.pattern, ctx.steps, ctx.c, ck, dF.contiguous(), dA, prec=ctx.prec)
        return dA, None, None, None, None, None


class QuadForm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, pattern, z):
        ctx.pattern = pattern
        ctx.save_for_backward(z)
        return torch.tensor(sf.quad_form(pattern, X.contiguous(), z), dtype=torch.float64)

    @staticmethod
    def backward(ctx, dL):
        (z,) = ctx.saved_tensors
        dX = torch.empty(ctx.pattern.nnz, dtype=torch.float64, device=z.device)
        sf.quad_form_grad(ctx.pattern, z, dX)
        return dX * float(dL), None, None
