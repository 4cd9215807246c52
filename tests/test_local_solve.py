"""Properties of the f(R) local equation (Sec. 3.2.5) that the single-precision
smoother relies on when it starts Newton's method from a cell's current
correction instead of the closed form.

With U = u + x the total field, the correction equation of one cell is
  G(x) = U^{n+1} - u^{n+1} + al K (1/u - 1/U) - B = 0,
  G'(x) = (n+1) U^n + al K / U^2 > 0,   G''(x) = n(n+1) U^{n-1} - 2 al K / U^3.
For n <= 2, |G''| / (2 G') <= 1/U on the whole positive branch, so a Newton step
from a start eps U away from the root leaves at most ~eps^2 U.  These are checks
of that mathematics in FP64, independent of the library and of the oracle.
"""
import numpy as np
import pytest


def dw(n, u, x):
    """U^{n+1} - u^{n+1}, factored so that a small x loses nothing."""
    return x * (2.0 * u + x) if n == 1 else x * (3.0 * u * u + 3.0 * u * x + x * x)


def G(n, u, alK, B, x):
    return dw(n, u, x) + alK * x / (u * (u + x)) - B


def dG(n, alK, U):
    return (n + 1) * U ** n + alK / U ** 2


def d2G(n, alK, U):
    return n * (n + 1) * U ** (n - 1) - 2.0 * alK / U ** 3


@pytest.mark.parametrize("n", [1, 2])
def test_curvature_bound_holds_for_n_up_to_2(n):
    rng = np.random.default_rng(11 + n)
    U = 10.0 ** rng.uniform(-4, 1, 200000)
    alK = 10.0 ** rng.uniform(-14, 2, 200000)
    ratio = np.abs(d2G(n, alK, U)) / (2.0 * dG(n, alK, U)) * U
    assert ratio.max() <= 1.0 + 1e-12


def test_curvature_bound_fails_for_n_3():
    """The bound is tight in n: for n = 3 (not a model here) the U^{n-1} term
    exceeds it, so the test above would catch an exponent slip."""
    U, alK = np.array([1.0]), np.array([1e-12])
    assert (np.abs(d2G(3, alK, U)) / (2.0 * dG(3, alK, U)) * U).max() > 1.4


@pytest.mark.parametrize("n", [1, 2])
def test_two_newton_steps_from_within_one_percent(n):
    """From any start within 1% of U of the root, two Newton steps leave an
    error below eps^4 U (eps = start offset / U), i.e. below eps^3 of the step."""
    rng = np.random.default_rng(20 + n)
    m = 20000
    u = 10.0 ** rng.uniform(-4, 0, m)
    alK = u ** (n + 2) * 10.0 ** rng.uniform(-6, 4, m)     # screened to unscreened
    U_root = u * 10.0 ** rng.uniform(-1.5, 1.5, m)          # the solution's total field
    x_root = U_root - u
    B = G(n, u, alK, 0.0, x_root)                            # the right-hand side this root solves
    eps = 10.0 ** rng.uniform(-8, -2, m) * rng.choice([-1.0, 1.0], m)
    x = x_root + eps * U_root
    for _ in range(2):
        x = x - G(n, u, alK, B, x) / dG(n, alK, u + x)
    err = np.abs(x - x_root) / U_root
    # the bound holds at the root; between start and root the ratio grows by
    # O(eps), hence the 10% margin.  FP64 rounding of G's terms adds ~1e-16 of
    # them, divided by G'.
    terms = np.abs(dw(n, u, x_root)) + np.abs(alK * x_root / (u * U_root)) + np.abs(B)
    rounding = 64 * np.finfo(float).eps * terms / dG(n, alK, U_root) / U_root
    assert np.all(err <= 1.1 * np.abs(eps) ** 4 + rounding)
