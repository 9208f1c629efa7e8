"""torch.autograd.Function around the library's Cholesky routines.

Forward:  L = cd_chol_fwd(Sigma)  (Sec. 4.2 chol_blocked).
Backward: tril(Sigma_bar) = cd_chol_rev(L, tril(L_bar))  (Sec. 4.2
chol_blocked_rev), returned to torch as the symmetric gradient
(tril(Sigma_bar) + tril(Sigma_bar)^T) / 2, the convention of
torch.linalg.cholesky (f depends on Sigma only through its symmetric part).

The only torch operations here are argument marshalling (a tril copy, the
symmetrisation); the factorisation and its derivative run in the library.
``gp_nlml`` is the Gaussian-process negative log marginal likelihood used to
exercise the backward pass end to end.
"""
import torch

from . import native


class CholeskyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma, nb=0, prec="fp64", check=True):
        A = torch.tril(sigma).contiguous()
        info = native.chol_fwd(A, nb=nb, prec=prec)
        if check:
            bad = int(info.item())
            if bad:
                raise torch.linalg.LinAlgError(
                    f"cd_chol_fwd: leading minor of order {bad} is not positive definite")
        ctx.save_for_backward(A)
        ctx.nb, ctx.prec = nb, prec
        return A

    @staticmethod
    def backward(ctx, L_bar):
        (L,) = ctx.saved_tensors
        Abar = torch.tril(L_bar).contiguous()
        native.chol_rev(L, Abar, nb=ctx.nb, prec=ctx.prec)
        return 0.5 * (Abar + Abar.transpose(0, 1)), None, None, None


def cholesky(sigma, nb=0, prec="fp64", check=True):
    """Differentiable lower Cholesky factor of a CUDA float64 SPD matrix."""
    return CholeskyFn.apply(sigma, nb, prec, check)


def sqdist(X):
    sq = (X * X).sum(1)
    return (sq[:, None] + sq[None, :] - 2.0 * (X @ X.transpose(0, 1))).clamp_min(0.0)


def gp_sigma(theta, X):
    """Sigma(theta) = s^2 exp(-r^2 / (2 l^2)) + sigma^2 I for theta = (s, l, sigma)."""
    s, ell, sig = theta[0], theta[1], theta[2]
    r2 = sqdist(X)
    n = X.shape[0]
    eye = torch.eye(n, dtype=X.dtype, device=X.device)
    return s * s * torch.exp(-r2 / (2.0 * ell * ell)) + sig * sig * eye


def gp_nlml(theta, X, y, nb=0, prec="fp64"):
    """0.5 y^T Sigma(theta)^{-1} y + sum_i log L_ii, differentiable in theta."""
    L = cholesky(gp_sigma(theta, X), nb=nb, prec=prec)
    v = torch.linalg.solve_triangular(L, y.reshape(-1, 1), upper=False)
    return 0.5 * (v * v).sum() + torch.log(torch.diagonal(L)).sum()
