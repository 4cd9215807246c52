"""Manufactured discrete solutions (the method of the paper's code tests, Sec. 4.2.2).

Pick the field, compute from the model equation the density that makes it an
exact solution of the discrete problem (7-point Laplacian, periodic), and hand
that density to a solver: it must give the field back.  The paper does this
for its sine tests (Eq. fR_eom_codeunit2_CodeTestForm and the densities printed
after Eqs. sine_field_sym, sine_field_cs); the cases here extend it to the two
branches of the equations that those tests leave out:

- coupled quintessence with the factor exp(beta phi~/c~^2) kept in front of
  (1 + delta) (Eq. csf_eom_code as written, before the simplification of
  Sec. 3.2.3);
- the symmetron with a field that changes sign across high-density walls
  (domain walls, Sec. 2.2: the field sits at +-phi_* in the low-density regions
  and near 0 where the density restores the symmetry).

Test helper only: numpy, no oracle and no CUDA code.  Each case returns plain
parameter values (keys shared by ``oracle.Params`` and the binding's
``Params``), the density with mean 1, and the exact field.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

C_OVER_H0 = 2997.92458  # c / (100 km/s/Mpc) in Mpc/h


def laplacian(f):
    """Sum of the six face neighbours minus 6 f (Eq. Lijk), periodic, h = 1."""
    return sum(np.roll(f, s, ax) for ax in range(3) for s in (1, -1)) - 6.0 * f


def _centres(N):
    x = 2.0 * np.pi * (np.arange(N) + 0.5) / N
    return np.meshgrid(x, x, x, indexing="ij")


def cq_exp_kept(N: int, alpha: float = 0.1, beta: float = -0.2, lam: float = 1.0, phibar: float = 0.5,
                omega_m: float = 0.3, a: float = 1.0, keep_exp: bool = True):
    """CQ manufactured case.  The box is N c/H0 so that c~ = 1 and the
    exponential and potential terms of Eq. csf_eom_code are of order 1e-2 of
    the field (at c~ ~ 1e3 they would be invisible).

    phi~ = phi0 + smooth 3D pattern; Eq. csf_eom_code solved for the density:
        1 + delta = [ (Lap phi~ + P(phi~)) / s + 1 ] / E(phi~),
        s = 3 beta Om e^{beta phibar} / a,   E = exp(beta phi~ / c~^2) (1 if not kept),
        P = alpha lambda^2 a^2 [ (phibar + phi~/c~^2)^{-1-alpha} - phibar^{-1-alpha} ].
    The solvers rescale the density to mean 1 (reading C12), so the constant
    phi0 is chosen (root of a 1D function) to make mean(1 + delta) = 1 exactly."""
    box = N * C_OVER_H0
    c2 = (N / box * C_OVER_H0) ** 2
    s = 3.0 * beta * omega_m * np.exp(beta * phibar) / a
    X, Y, Z = _centres(N)
    shape = 0.05 * np.sin(X) * np.cos(2 * Y) + 0.03 * np.cos(Z + 0.4) + 0.02 * np.sin(X + Y + Z)

    def rho_of(phi0):
        phi = phi0 + shape
        E = np.exp(beta * phi / c2) if keep_exp else 1.0
        P = alpha * lam ** 2 * a ** 2 * ((phibar + phi / c2) ** (-1.0 - alpha) - phibar ** (-1.0 - alpha))
        return ((laplacian(phi) + P) / s + 1.0) / E, phi

    phi0 = brentq(lambda t: rho_of(t)[0].mean() - 1.0, -0.3, 0.3, xtol=1e-16, rtol=1e-15)
    rho, phi = rho_of(phi0)
    params = dict(alpha=alpha, beta=beta, lam=lam, phibar=phibar, omega_m=omega_m, box=box, keep_exp=keep_exp)
    return params, rho, phi


def symmetron_domain_walls(N: int, B: float = 0.8, range_cells: float = 0.5, power: float = 1.5, a: float = 1.0):
    """Symmetron manufactured case whose field changes sign.

    u(x, y, z) = B sign(sin kx) |sin kx|^power (1 + 0.1 cos(ky) sin(kz + 0.2)),
    k = 2 pi / N: two planar walls (u = 0 on the planes x = 0 and x = N/2, cell
    faces), with u near +-B between them.  Eq. sym_eom_code_unit solved for the
    density (box = N Mpc/h, xi from the range in cells, m = a^2/(2 xi^2)):
        rho r = 1 - u^2 + c~^2 Lap(u) / (m u),   r = (a_*/a)^3.
    With power > 1 the field is convex away from zero near a wall, so the
    density there exceeds the symmetry-restoring value (rho r > 1) and pins the
    wall; r is set to mean(rho r), which gives the density mean 1.

    The solution is a strict local minimum of the field energy when
    m_eff = 2 m u^2 + c~^2 Lap(u)/u (the diagonal of the Jacobian, minus the
    Laplacian) is positive everywhere; this is returned for the tests to
    assert.  The same density has other exact solutions (the everywhere
    positive one among them)."""
    box = float(N)
    ct = N / box * C_OVER_H0
    xi = range_cells / ct
    m = a * a / (2.0 * xi * xi)
    X, Y, Z = _centres(N)
    sx = np.sin(X)
    u = B * np.sign(sx) * np.abs(sx) ** power * (1.0 + 0.1 * np.cos(Y) * np.sin(Z + 0.2))
    L = laplacian(u)
    rr = 1.0 - u ** 2 + ct * ct * L / (m * u)
    r = rr.mean()
    rho = rr / r
    m_eff = 2.0 * m * u ** 2 + ct * ct * L / u
    params = dict(a_star=a * r ** (1.0 / 3.0), xi=xi, beta_star=1.0, omega_m=0.3, box=box)
    return params, rho, u, m_eff / m
