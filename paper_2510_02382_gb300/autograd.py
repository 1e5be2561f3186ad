"""torch.autograd.Function wrappers of the differentiable form (argument marshalling only:
the forward and backward passes and the loss run in libctfmnmf's kernels).

    solver = Grad(M, N, L, B, F, J, batch=S, n_iter=20, ckpt_every=5)
    C = separate(X, T0, V0, solver)          # [S][N][M][F][J] images after n_iter iterations
    loss = mse(C, C_true, solver)            # mean |C - C_true|^2, float64 scalar
    loss.backward()                          # X.grad, T0.grad, V0.grad

Complex gradients follow PyTorch's convention (dL/da + i dL/db for z = a + ib), which is
also the library's. Each forward pass of a solver allows one backward pass.
"""
import torch

from .api import Grad


class _Separate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, T0, V0, solver):
        ctx.solver = solver
        return solver.forward(X.contiguous(), T0.contiguous(), V0.contiguous())

    @staticmethod
    def backward(ctx, gC):
        gX, gT0, gV0 = ctx.solver.backward(gC.contiguous())
        return gX, gT0, gV0, None


class _MSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C, Cref, solver):
        loss = torch.zeros((), dtype=torch.float64, device=C.device)
        solver.mse(C, Cref, loss=loss)
        ctx.solver = solver
        ctx.save_for_backward(C, Cref)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        C, Cref = ctx.saved_tensors
        gC = torch.empty_like(C)
        ctx.solver.mse(C, Cref, dloss=gloss.to(torch.float64).contiguous(), gC=gC)
        return gC, None, None


def separate(X, T0, V0, solver: Grad):
    """Separated images of a batch after the solver's n_iter iterations (differentiable)."""
    return _Separate.apply(X, T0, V0, solver)


def mse(C, Cref, solver: Grad):
    """Mean over all elements of |C - Cref|^2 (differentiable in C)."""
    return _MSE.apply(C, Cref.contiguous(), solver)
