"""Spherically symmetric reference solutions for the tophat test.

Sec. 4.2 (spherical tophat overdensity): for a density that depends on the
distance r from the box centre only, the scalar-field equations reduce to
radial ODEs, solved on [0, R] with u'(0) = 0 and u(R) = the far-field value
(the paper puts this boundary at R = N/2 as a stand-in for infinity):

- symmetron (Eq. sym_eom_code_unit_spherical):
    c^2 (1/r^2) (r^2 u')' = (a^2 / 2 xi^2) [ (rho (a*/a)^3 - 1) u + u^3 ]
- f(R), the radial form of Eq. fR_eom_codeunit2 with w = u^{n+1} = -f_R:
    c^2 (1/r^2) (r^2 w')' = Om delta / a + (Rbar a^2 / 3) (1 - ubar / u)

Both are solved here as boundary-value problems by Newton's method on a fine
vertex-centred grid (conservative second-order differences; at r = 0 the
limit 3 w'' of the spherical Laplacian), with a tridiagonal Jacobian.  The
coefficients come from the paper's definitions (c~ = N c / (100 L),
Rbar(a) = 3 (Om a^-3 + 4 OL), fbar_R(a) = -|fR0| (Rbar(1)/Rbar(a))^{n+1}),
computed here: this module shares nothing with the oracle or the CUDA path.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded

C_OVER_H0 = 2997.92458  # c / (100 km/s/Mpc) in Mpc/h


def c_tilde(N: int, box: float) -> float:
    return N * C_OVER_H0 / box


def fr_background(fR0_abs: float, n: int, omega_m: float, omega_l: float, a: float):
    """(Rbar(a), ubar) of Hu-Sawicki f(R): Rbar = 3 (Om a^-3 + 4 OL), ubar = (-fbar_R)^{1/(n+1)}."""
    Rbar = 3.0 * (omega_m / a ** 3 + 4.0 * omega_l)
    R1 = 3.0 * (omega_m + 4.0 * omega_l)
    fbar = -fR0_abs * (R1 / Rbar) ** (n + 1)
    return Rbar, (-fbar) ** (1.0 / (n + 1))


def _laplacian_coeffs(r: np.ndarray):
    """Coefficients (lo, di, up) of the radial Laplacian at nodes 0..M-1:
    Lap_i = lo_i w_{i-1} + di_i w_i + up_i w_{i+1}."""
    M = len(r) - 1
    dr = r[1] - r[0]
    lo = np.zeros(M)
    di = np.zeros(M)
    up = np.zeros(M)
    # r = 0: (1/r^2)(r^2 w')' -> 3 w'', with w'(0) = 0: 6 (w_1 - w_0) / dr^2
    di[0] = -6.0 / dr ** 2
    up[0] = 6.0 / dr ** 2
    ri = r[1:M]
    rp = ri + 0.5 * dr
    rm = ri - 0.5 * dr
    lo[1:] = rm ** 2 / (ri ** 2 * dr ** 2)
    up[1:] = rp ** 2 / (ri ** 2 * dr ** 2)
    di[1:] = -(rm ** 2 + rp ** 2) / (ri ** 2 * dr ** 2)
    return lo, di, up


def _newton(r, c2, w, dw, F, dF, u0, uR, positive: bool, tol=1e-13, max_iter=200):
    """Solve c2 Lap(w(u)) = F(u, r) for u at nodes 0..M-1, u(r_M) = uR."""
    lo, di, up = _laplacian_coeffs(r)
    M = len(r) - 1
    u = np.array(u0[:M], dtype=np.float64)

    def G(u):
        W = w(u)
        Wr = np.append(W, w(np.array([uR]))[0])
        lap = di * W + up * Wr[1:M + 1]
        lap[1:] += lo[1:] * W[:-1]
        return c2 * lap - F(u)

    g = G(u)
    scale = np.abs(F(np.full(M, uR))).max() + np.abs(c2 * di * w(u)).max()
    for _ in range(max_iter):
        if np.abs(g).max() <= tol * scale:
            return np.append(u, uR)
        d = dw(u)
        ab = np.zeros((3, M))
        ab[0, 1:] = c2 * up[:-1] * d[1:]     # superdiagonal J[i, i+1]
        ab[1, :] = c2 * di * d - dF(u)
        ab[2, :-1] = c2 * lo[1:] * d[:-1]    # subdiagonal J[i+1, i]
        s = solve_banded((1, 1), ab, -g)
        t = 1.0
        while True:
            un = u + t * s
            if (not positive or np.all(un > 0.05 * u)):
                gn = G(un)
                if np.abs(gn).max() < np.abs(g).max() or t < 1e-4:
                    break
            t *= 0.5
        u, g = un, gn
    raise RuntimeError("radial Newton did not converge")


def symmetron_profile(rho_in: float, rho_out: float, R_th: float, R: float, *, N: int, box: float,
                      a: float, a_star: float, xi: float, M: int = 4000):
    """(r, u) of the symmetron tophat: density rho_in for r <= R_th, rho_out beyond
    (both already normalised), u(R) = the homogeneous root for rho_out."""
    r = np.linspace(0.0, R, M + 1)
    c2 = c_tilde(N, box) ** 2
    k = a * a / (2.0 * xi * xi)
    s3 = (a_star / a) ** 3
    rho = np.where(r <= R_th, rho_in, rho_out)[:M]
    uR = np.sqrt(max(0.0, 1.0 - rho_out * s3))
    F = lambda u: k * ((rho * s3 - 1.0) * u + u ** 3)
    dF = lambda u: k * ((rho * s3 - 1.0) + 3.0 * u * u)
    u = _newton(r, c2, lambda u: u, lambda u: np.ones_like(u), F, dF, np.full(M + 1, uR), uR,
                positive=False)
    return r, u


def fr_profile(rho_in: float, rho_out: float, R_th: float, R: float, *, N: int, box: float, n: int,
               fR0_abs: float, omega_m: float, omega_l: float, a: float, M: int = 4000):
    """(r, u) of the f(R) tophat, u = (-f_R)^{1/(n+1)}; u(R) = the homogeneous root
    for rho_out: Om (rho_out - 1)/a + (Rbar a^2/3)(1 - ubar/u) = 0."""
    r = np.linspace(0.0, R, M + 1)
    c2 = c_tilde(N, box) ** 2
    Rbar, ubar = fr_background(fR0_abs, n, omega_m, omega_l, a)
    K = Rbar * a * a / 3.0
    delta = np.where(r <= R_th, rho_in, rho_out)[:M] - 1.0
    uR = ubar / (1.0 + omega_m * (rho_out - 1.0) / (a * K))
    F = lambda u: omega_m * delta / a + K * (1.0 - ubar / u)
    dF = lambda u: K * ubar / (u * u)
    u = _newton(r, c2, lambda u: u ** (n + 1), lambda u: (n + 1) * u ** n, F, dF,
                np.full(M + 1, uR), uR, positive=True)
    return r, u


def tophat_density(N: int, delta_in: float, R_frac: float = 0.1):
    """The test density of Sec. 4.2 on the mesh: 1 + delta_in inside the sphere of radius
    R_frac N about the box centre (N/2, N/2, N/2), 1 outside, with cell centres at index + 1/2.
    Returns (rho, r) with r each cell's distance from the centre."""
    x = np.arange(N) + 0.5 - N / 2.0
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    rho = np.where(r <= R_frac * N, 1.0 + delta_in, 1.0)
    return rho, r
