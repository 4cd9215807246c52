"""Coupled-quintessence background (mgglam_cq_background, host code in the
library) against the oracle's independent RK4 shooting.  Runs without a GPU:
the entry point touches no device state.

The library integrates the cosmic-time form with an adaptive Dormand-Prince
5(4) pair and shoots lambda by safeguarded secant steps; the oracle integrates
the paper's conformal code-unit form with fixed-step RK4 and bisects.  Both
start at z = 1e5 from phi = 1e-4, x = 0.  Agreement: lambda and H(a)/H0 to
1e-9 relative, phibar and dphibar/dln a to 1e-7 (the fixed-step oracle's
truncation error dominates).
"""
import pytest

from paper_2110_00328_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_radiation_density_matches_oracle(lib, orc):
    assert binding.radiation_density(0.6774) == pytest.approx(orc.radiation_density(0.6774), rel=1e-12)


@pytest.mark.parametrize("alpha,beta", [(0.1, -0.05), (0.5, -0.2), (0.1, 0.0)])
@pytest.mark.parametrize("a", [1.0, 0.5])
def test_cq_background_matches_oracle(lib, orc, alpha, beta, a):
    Or = orc.radiation_density(0.6774)
    lam, phi, dphi, E = orc.cq_background(alpha, beta, 0.3, Or, a=a)
    got = binding.cq_background(alpha, beta, 0.3, 0.6774, a)
    assert got["lambda"] == pytest.approx(lam, rel=1e-9)
    assert got["E"] == pytest.approx(E, rel=1e-9)
    assert got["phibar"] == pytest.approx(phi, rel=1e-7)
    assert got["dphibar_dlna"] == pytest.approx(dphi, rel=1e-7)


def test_cq_background_argument_errors(lib):
    with pytest.raises(binding.MgglamError):
        binding.cq_background(-0.1, -0.05)
    with pytest.raises(binding.MgglamError):
        binding.cq_background(0.1, -0.05, a=1.5)
