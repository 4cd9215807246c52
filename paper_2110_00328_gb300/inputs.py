"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random fields and particle positions; it contains none
of the solver's arithmetic (no deposit, no multigrid, no force).  The paper's
workloads are CAMB-based N-body density fields (Sec. 5), which are not
available here; these generators stand in for them with the same mesh/box
shapes and comparable density statistics:

* ``lognormal_density``: a Gaussian random field g with power spectrum
  P(k) ~ k^slope exp(-(k/k_c)^2), rescaled to pixel standard deviation sigma_g,
  mapped to delta = exp(g - sigma_g^2/2) - 1 and returned as rho = 1 + delta
  renormalised to mean 1 (float64, [x][y][z] with z fastest).
* ``zeldovich_positions``: particles on the lattice q = (i + 1/2) displaced by
  the Zel'dovich displacement psi_k = i k delta_k / k^2 of a Gaussian field with
  P(k) ~ k^-2 (k <= k_Nyquist), pixel sigma fixed; positions in cell units in
  [0, N), float32, shape [np, 3].

Random numbers come from numpy's PCG64 ``default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np


def _kgrid(N: int):
    """Wavenumbers in radians per cell for an rfftn layout."""
    kx = 2.0 * np.pi * np.fft.fftfreq(N)
    kz = 2.0 * np.pi * np.fft.rfftfreq(N)
    return kx[:, None, None], kx[None, :, None], kz[None, None, :]


def gaussian_field(N: int, seed: int, slope: float = -1.5, kc_frac: float = 0.5,
                   sigma: float = 1.0, cutoff: bool = True) -> np.ndarray:
    """Zero-mean Gaussian field with P(k) ~ k^slope [exp(-(k/k_c)^2)], pixel std = sigma."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((N, N, N))
    wk = np.fft.rfftn(white)
    kx, ky, kz = _kgrid(N)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    k[0, 0, 0] = 1.0
    pk = k ** slope
    if cutoff:
        kc = kc_frac * np.pi
        pk = pk * np.exp(-((k / kc) ** 2))
    else:
        pk = np.where(k <= np.pi, pk, 0.0)
    pk[0, 0, 0] = 0.0
    g = np.fft.irfftn(wk * np.sqrt(pk), s=(N, N, N), axes=(0, 1, 2))
    g -= g.mean()
    std = g.std()
    return g * (sigma / std) if std > 0 else g


def lognormal_density(N: int, sigma_g: float, seed: int, slope: float = -1.5,
                      kc_frac: float = 0.5) -> np.ndarray:
    """rho = 1 + delta, delta = exp(g - sigma_g^2/2) - 1, renormalised to mean exactly 1 (FP64)."""
    g = gaussian_field(N, seed, slope=slope, kc_frac=kc_frac, sigma=sigma_g)
    rho = np.exp(g - 0.5 * sigma_g * sigma_g)
    return rho / rho.mean()


def zeldovich_positions(N: int, seed: int, sigma: float = 1.5, npart_side: int | None = None,
                        slope: float = -2.0) -> np.ndarray:
    """Particle positions [np,3] float32 in cell units of an N^3 mesh (np = npart_side^3).

    The displacement field is computed on an npart_side^3 lattice (default N)
    and scaled to mesh cell units.
    """
    M = N if npart_side is None else npart_side
    delta = gaussian_field(M, seed, slope=slope, sigma=sigma, cutoff=False)
    dk = np.fft.rfftn(delta)
    kx, ky, kz = _kgrid(M)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    scale = N / M
    q = (np.arange(M, dtype=np.float64) + 0.5)
    pos = np.empty((M, M, M, 3), dtype=np.float64)
    for d, kd in enumerate((kx, ky, kz)):
        psi = np.fft.irfftn(1j * kd * dk / k2, s=(M, M, M), axes=(0, 1, 2))
        base = q[:, None, None] if d == 0 else (q[None, :, None] if d == 1 else q[None, None, :])
        pos[..., d] = (base + psi) * scale
    pos = np.mod(pos, float(N))
    pos = pos.reshape(-1, 3).astype(np.float32)
    # float32 rounding of values just below N can produce exactly N; keep [0, N)
    pos[pos >= np.float32(N)] = 0.0
    return pos


def point_mass_density(N: int, amp: float = 1e-4) -> np.ndarray:
    """The point-mass configuration of Sec. 4.2.3: rho = 1 + delta with
    delta = amp (N^3 - 1) in cell (0,0,0) and -amp elsewhere."""
    rho = np.full((N, N, N), 1.0 - amp)
    rho[0, 0, 0] = 1.0 + amp * (N ** 3 - 1)
    return rho


def uniform_random_field(N: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Uniform random initial guesses in [lo, hi] (the homogeneous-density test, Sec. 4.2.1)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=(N, N, N))
