"""FP64 reference of one particle-mesh time step (test infrastructure).

Only the tests, the package's smoke check and the benchmark's CPU baseline use
this module: the library never calls it.  It restates the step in the paper's
order with numpy, for small meshes:

- Sec. 3.1: CIC density, the periodic Poisson equation
  grad_h^2 Phi_N = (3/2) Om/a delta (Eq. GR_poisson_codeunit) solved with the
  discrete Green's function of the 7-point Laplacian, Phi_0 = 0;
- the scalar field from the oracle's multigrid solve (Secs. 3.2.3-3.2.5);
- forces from three-point central differences at cell centres, CIC-
  interpolated to the particles: dp/da = -(H0/adot) [sN grad Phi_N] + the fifth
  force (Eqs. F_N_codeunit, F5_fR_codeunit, F_5_codeunit,
  csf_particle_geodesic_code2; sN = e^{beta phibar} for CQ) minus the drag
  gamma p (CQ: beta dphibar/da; symmetron: Eq. F_x_codeunit);
- leapfrog: p from a - da/2 to a + da/2 with the force at a (drag at the
  midpoint), then x from a to a + da with dx/da = H0 p / (a^2 adot) at a + da/2
  (the positive sign of Eq. csf_particle_geodesic_code1).
H0/adot = 1 / (a E(a)), E = H/H0.
"""
from __future__ import annotations

import numpy as np

from . import Params, FR, SYMMETRON, CQ, KIND_NEWTON, KIND_NONLINEAR, background, deposit_cic, solve


def discrete_k2(N: int) -> np.ndarray:
    """Eigenvalues of minus the 7-point periodic Laplacian: sum_d 4 sin^2(pi k_d / N)."""
    s = 4.0 * np.sin(np.pi * np.arange(N) / N) ** 2
    return s[:, None, None] + s[None, :, None] + s[None, None, :]


def poisson_fft(rho: np.ndarray, coef: float) -> np.ndarray:
    """Phi with grad_h^2 Phi = coef (rho/mean - 1), mean(Phi) = 0."""
    N = rho.shape[0]
    delta = rho / rho.mean() - 1.0
    k2 = discrete_k2(N)
    k2[0, 0, 0] = 1.0
    phik = -coef * np.fft.fftn(delta) / k2
    phik[0, 0, 0] = 0.0
    return np.fft.ifftn(phik).real


def grad_at(T: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """CIC interpolation to the particles of the central differences (T_{c+1} - T_{c-1})/2
    at cell centres (centre of cell c at c + 1/2), periodic."""
    N = T.shape[0]
    x = np.mod(np.asarray(pos, dtype=np.float64), N) - 0.5
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    g = [0.5 * (np.roll(T, -1, d) - np.roll(T, 1, d)) for d in range(3)]
    out = np.zeros((x.shape[0], 3))
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                w = ((f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) *
                     (f[:, 2] if dk else 1 - f[:, 2]))
                i, j, k = (i0[:, 0] + di) % N, (i0[:, 1] + dj) % N, (i0[:, 2] + dk) % N
                for d in range(3):
                    out[:, d] += w * g[d][i, j, k]
    return out


def interp_at(U: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """CIC interpolation of the mesh U to the particles."""
    N = U.shape[0]
    x = np.mod(np.asarray(pos, dtype=np.float64), N) - 0.5
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    out = np.zeros(x.shape[0])
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                w = ((f[:, 0] if di else 1 - f[:, 0]) * (f[:, 1] if dj else 1 - f[:, 1]) *
                     (f[:, 2] if dk else 1 - f[:, 2]))
                out += w * U[(i0[:, 0] + di) % N, (i0[:, 1] + dj) % N, (i0[:, 2] + dk) % N]
    return out


def fifth_force_potential(p: Params, u: np.ndarray) -> np.ndarray:
    """The potential whose gradient is the fifth force per unit H0/adot:
    f(R) (c~^2/2)(f_R - fbar_R); symmetron -3 xi^2 Om beta*^2 c~^2 a*^-3 (u^2 - ubar^2);
    CQ -beta phi~."""
    N = u.shape[0]
    b = background(p, N)
    if p.model == FR:
        ub = b["ubar"]
        return 0.5 * b["c2"] * (-(u ** (p.n + 1)) + ub ** (p.n + 1))
    if p.model == SYMMETRON:
        ub = b["ubar"]
        s = -3.0 * p.xi ** 2 * p.omega_m * p.beta_star ** 2 * b["c2"] / p.a_star ** 3
        return s * (u * u - ub * ub)
    return -p.beta * u


def pm_step(p: Params, pos, mom, da: float, E_a: float, E_half: float, field=None, tol: float = 1e-10,
            dphibar_da: float = 0.0, scalar: bool = True):
    """One step from p.a to p.a + da.  Returns (pos, mom, field, rho, psi); field is
    the scalar solution at p.a (None for a LCDM step)."""
    a = p.a
    N = None if field is None else field.shape[0]
    pos = np.asarray(pos, dtype=np.float64)
    mom = np.asarray(mom, dtype=np.float64)
    if N is None:
        raise ValueError("pass field (a mesh of the right size; its values are the initial guess)")
    rho = deposit_cic(pos.astype(np.float32), N)
    psi = -poisson_fft(rho, 1.5 * p.omega_m / a)
    u = None
    if scalar:
        # CQ by Newton-Gauss-Seidel (Sec. 3.2.3), the others by nonlinear Gauss-Seidel
        u = solve(p, rho, u0=field, tol=tol, max_cycles=80, kind=KIND_NEWTON if p.model == CQ else KIND_NONLINEAR).u
        if p.model == CQ:
            psi = psi * np.exp(p.beta * p.phibar)
        psi = psi + fifth_force_potential(p, u)
    gamma = np.zeros(pos.shape[0])
    if scalar and p.model == CQ:
        gamma[:] = p.beta * dphibar_da
    if scalar and p.model == SYMMETRON and p.a_star < a:
        k = 9.0 * p.omega_m * p.beta_star ** 2 * p.xi ** 2 * np.sqrt(1.0 - (p.a_star / a) ** 3) / a ** 4
        gamma = k * interp_at(u, pos)
    F = grad_at(psi, pos) / (a * E_a)
    g = (gamma * da)[:, None]
    mom = (mom * (1.0 - 0.5 * g) + da * F) / (1.0 + 0.5 * g)
    ah = a + 0.5 * da
    pos = np.mod(pos + da * mom / (ah ** 3 * E_half), N)
    return pos, mom, u, rho, psi
