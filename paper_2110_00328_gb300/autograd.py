"""Differentiable scalar-field solve: torch.autograd.Function over the C-ABI.

``ScalarSolve.apply(rho, log_fR0, prm, a, tol)`` returns the converged field u*
(mgglam_solve_scalar).  Its backward runs mgglam_solve_adjoint: the adjoint
field lambda of J^T lambda = dl/du*, from which the library forms the gradients
with respect to the caller's density (through the solver's mean-1
normalisation) and ln|f_R0|.  Only u* (and the density) is kept between forward
and backward; the adjoint rebuilds its coarse levels from u*.

``fifth_force_power_loss`` is a loss of the kind used for emulators: the log of
the binned power spectrum of the f(R) fifth force F = (c~^2/2) grad f_R on the
mesh (three-point differences, Eq. F5_fR_codeunit), summed over logarithmic
wavenumber bins.  It uses torch's FFT (a library transform, not the solver path).
"""
from __future__ import annotations

import math
from dataclasses import replace

import torch

from . import binding

C_OVER_H0 = 299792.458 / 100.0  # Mpc/h


class ScalarSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, log_fR0, prm: binding.Params, a: float, tol: float):
        p = replace(prm, fR0_abs=float(math.exp(float(log_fR0))))
        N = rho.shape[0]
        field = torch.full((N, N, N), float("nan"), dtype=torch.float64, device=rho.device)
        binding.solve_scalar(p, a, rho.contiguous(), field, tol)
        ctx.save_for_backward(rho, field)
        ctx.p, ctx.a, ctx.tol = p, a, tol
        return field

    @staticmethod
    def backward(ctx, grad_field):
        rho, field = ctx.saved_tensors
        g_rho, g_theta, _ = binding.solve_adjoint(ctx.p, ctx.a, field, rho.contiguous(),
                                                  grad_field.contiguous().to(torch.float64), tol=ctx.tol * 0.1,
                                                  raw=True)
        return g_rho.to(rho.dtype), torch.tensor(g_theta, dtype=torch.float64, device=rho.device), None, None, None


def solve(rho, log_fR0, prm: binding.Params, a: float = 1.0, tol: float = 1e-10):
    return ScalarSolve.apply(rho, log_fR0, prm, a, tol)


def fifth_force_power_loss(u, prm: binding.Params, nbins: int = 32):
    """sum_b log P_F(k_b), P_F the shell-averaged |FFT(F)|^2 of F = (c~^2/2) grad f_R, f_R = -u^{n+1}.

    Bins: nbins logarithmic bins in k between 2 pi/L and pi N/L (h/Mpc)."""
    N = u.shape[0]
    ct = N / prm.box * C_OVER_H0
    fR = -u ** (prm.n + 1)
    F = [0.5 * ct * ct * 0.5 * (torch.roll(fR, -1, d) - torch.roll(fR, 1, d)) for d in range(3)]
    pk = sum(torch.fft.rfftn(Fd).abs() ** 2 for Fd in F)
    kf = 2 * math.pi / prm.box
    kx = torch.fft.fftfreq(N, d=1.0 / N, device=u.device, dtype=torch.float64) * kf
    kz = torch.fft.rfftfreq(N, d=1.0 / N, device=u.device, dtype=torch.float64) * kf
    k = torch.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    edges = torch.logspace(math.log10(kf), math.log10(math.pi * N / prm.box), nbins + 1,
                           device=u.device, dtype=torch.float64)
    idx = torch.bucketize(k.reshape(-1), edges) - 1
    valid = (idx >= 0) & (idx < nbins)
    sums = torch.zeros(nbins, dtype=torch.float64, device=u.device).index_add(0, idx[valid], pk.reshape(-1)[valid])
    counts = torch.zeros(nbins, dtype=torch.float64, device=u.device).index_add(
        0, idx[valid], torch.ones_like(pk.reshape(-1)[valid]))
    ok = counts > 0
    return torch.log(sums[ok] / counts[ok]).sum()
