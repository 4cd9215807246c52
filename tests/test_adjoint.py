"""Adjoint of the scalar-field solve: oracle pins (CPU) and GPU parity.

Oracle pins: the assembled Jacobian against central differences of the
oracle's residual, and the adjoint gradients against central differences of a
loss through the oracle's own FAS solve (in the density along a mean-zero
direction, and in ln|f_R0|).

GPU: mgglam_solve_adjoint against the oracle's sparse-LU adjoint on the same
u* (tolerance 1e-8 relative: FP64 outer refinement to 1e-12), and the
torch.autograd.Function on a fifth-force power-spectrum loss against central
finite differences of GPU solves (step 1e-3; agreement 1e-4 relative, the
gradient target stated for this path).
"""
import math

import numpy as np
import pytest

from paper_2110_00328_gb300 import inputs

CASES = {
    "fr0": dict(model=0, n=0, fR0_abs=1e-5, box=16.0),
    "fr1": dict(model=0, n=1, fR0_abs=1e-5, box=16.0),
    "fr2": dict(model=0, n=2, fR0_abs=1e-5, box=16.0),
    "sym": dict(model=1, a_star=0.5, xi=1e-3, beta_star=1.0, box=8.0),
}


def solved(orc, key, N=8, seed=70):
    p = orc.Params(**CASES[key])
    rho = inputs.lognormal_density(N, 0.8, seed=seed)
    r = orc.solve(p, rho, tol=1e-14, max_cycles=80)
    return p, rho, r.u


@pytest.mark.parametrize("key", list(CASES))
def test_oracle_jacobian_matches_residual_differences(orc, key):
    p, rho, u = solved(orc, key)
    J = orc.jacobian(p, u, rho)
    v = np.random.default_rng(1).normal(size=u.shape)
    eps = 1e-6 * np.abs(u).mean()
    fd = (orc.residual(p, u + eps * v, rho) - orc.residual(p, u - eps * v, rho)) / (2 * eps)
    assert np.linalg.norm(J @ v.ravel() - fd.ravel()) <= 1e-7 * np.linalg.norm(fd)


@pytest.mark.parametrize("key", list(CASES))
def test_oracle_adjoint_gradient_matches_solve_differences(orc, key):
    """l(u*) = sum c_i u*_i: the adjoint gradient against central differences of FAS solves."""
    N = 8
    p, rho, u = solved(orc, key, N)
    rng = np.random.default_rng(2)
    c = rng.normal(size=u.shape)
    _, gd, gt = orc.adjoint(p, u, rho, c)
    loss = lambda pp, rr: float(np.sum(c * orc.solve(pp, rr, tol=1e-14, max_cycles=80).u))
    v = rng.normal(size=u.shape)
    v -= v.mean()                      # keeps the mean density at 1 (the solver's normalisation)
    h = 1e-4
    fd = (loss(p, rho + h * v) - loss(p, rho - h * v)) / (2 * h)
    assert fd == pytest.approx(float(np.sum(gd * v)), rel=1e-5)
    if key.startswith("fr"):
        th = math.log(p.fR0_abs)
        pp = lambda t: orc.Params(**{**CASES[key], "fR0_abs": math.exp(t)})
        fdt = (loss(pp(th + h), rho) - loss(pp(th - h), rho)) / (2 * h)
        assert fdt == pytest.approx(gt, rel=1e-5)


def test_normalisation_jacobian_matches_differences_in_the_raw_density(orc):
    """The solver rescales any positive density to mean 1 (reading C12), so the
    gradient with respect to the density as passed in is dl/d delta composed with
    the Jacobian of rho -> rho/mean(rho): (g_j - sum_i g_i rho_i / sum rho)/mean.
    Central differences of oracle solves along a direction that changes the mean
    check that composition (the GPU's grad_rho_raw is compared with it)."""
    N = 8
    p, rho, u = solved(orc, "fr1", N)
    rho = 1.7 * rho                     # a mean other than 1
    rng = np.random.default_rng(4)
    c = rng.normal(size=u.shape)
    _, gd, _ = orc.adjoint(p, u, rho / rho.mean(), c)
    mu = rho.mean()
    g_raw = (gd - np.mean(gd * rho / mu)) / mu
    loss = lambda rr: float(np.sum(c * orc.solve(p, rr, tol=1e-14, max_cycles=80).u))
    v = rng.normal(size=u.shape) + 0.5  # mean 0.5: the mean density changes too
    h = 1e-4
    fd = (loss(rho + h * v) - loss(rho - h * v)) / (2 * h)
    assert fd == pytest.approx(float(np.sum(g_raw * v)), rel=1e-5)
    # a uniform rescaling of the density changes nothing
    assert abs(float(np.sum(g_raw * rho))) <= 1e-10 * np.abs(g_raw).sum() * rho.max()


# ---------------------------------------------------------------- GPU

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_00328_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.gpu
@pytest.mark.parametrize("key", list(CASES))
@pytest.mark.parametrize("N", [16, 24])
def test_gpu_adjoint_matches_oracle(orc, mg, key, N):
    """FP64 fine residual (meshes the float-float residual's 8 x 32 tiles do not divide)."""
    _adjoint_case(orc, mg, key, N)


@pytest.mark.gpu
def test_gpu_adjoint_float_float_residual_matches_oracle(orc, mg):
    """32^3: the float-float fine residual (one model: the oracle's sparse LU at
    32^3 takes most of a minute)."""
    _adjoint_case(orc, mg, "fr1", 32)


def _adjoint_case(orc, mg, key, N):
    kw = dict(CASES[key])
    kw["box"] = kw["box"] * N / 8
    p = orc.Params(**kw)
    rho = inputs.lognormal_density(N, 0.8, seed=71).astype(np.float32)
    rho_n = rho.astype(np.float64) / rho.astype(np.float64).mean()
    u = orc.solve(p, rho_n, tol=1e-14, max_cycles=80).u
    g = np.random.default_rng(3).normal(size=u.shape)
    lam, gd, gt = orc.adjoint(p, u, rho_n, g)
    pg = mg.Params(**kw, precision=1, max_cycles=80)
    grad_rho, gth, st = mg.solve_adjoint(pg, 1.0, torch.from_numpy(u).cuda(), torch.from_numpy(rho).cuda(),
                                         torch.from_numpy(g).cuda(), tol=1e-12)
    assert st.converged
    got = grad_rho.cpu().numpy()
    assert np.linalg.norm(got - gd) <= 1e-8 * np.linalg.norm(gd)
    if key.startswith("fr"):
        assert gth == pytest.approx(gt, rel=1e-8)
    # the gradient with respect to the caller's (unnormalised) density: the oracle's
    # dl/d delta composed with the Jacobian of rho -> rho / mean(rho)
    raw, _, _ = mg.solve_adjoint(pg, 1.0, torch.from_numpy(u).cuda(), torch.from_numpy(rho).cuda(),
                                 torch.from_numpy(g).cuda(), tol=1e-12, raw=True)
    r64 = rho.astype(np.float64)
    mu = r64.mean()
    ref_raw = (gd - np.mean(gd * r64 / mu)) / mu
    assert np.linalg.norm(raw.cpu().numpy() - ref_raw) <= 1e-8 * np.linalg.norm(ref_raw)


@pytest.mark.gpu
def test_autograd_fifth_force_loss_matches_finite_differences(mg):
    """Gradient of sum_b log P_F(k_b) w.r.t. the density and ln|f_R0| against
    central differences (step 1e-3) of GPU solves, 64^3 f(R) n=1."""
    from paper_2110_00328_gb300 import autograd as ag
    N = 64
    prm = mg.Params(model=0, n=1, fR0_abs=1e-5, box=64.0, precision=1, max_cycles=80)
    rho0 = torch.from_numpy(inputs.lognormal_density(N, 1.5, seed=72).astype(np.float32)).cuda()
    rho = rho0.clone().requires_grad_(True)
    th = torch.tensor(math.log(1e-5), dtype=torch.float64, requires_grad=True)
    loss = ag.fifth_force_power_loss(ag.solve(rho, th, prm, 1.0, 1e-11), prm)
    loss.backward()
    g_rho, g_th = rho.grad.double(), float(th.grad)

    def L(r, t):
        with torch.no_grad():
            return float(ag.fifth_force_power_loss(ag.solve(r, torch.tensor(t, dtype=torch.float64), prm, 1.0,
                                                             1e-11), prm))

    h = 1e-3
    t0 = math.log(1e-5)
    fdt = (L(rho0, t0 + h) - L(rho0, t0 - h)) / (2 * h)
    assert fdt == pytest.approx(g_th, rel=1e-4)
    for seed in range(2):
        v = torch.from_numpy(np.random.default_rng(80 + seed).normal(size=(N, N, N))).cuda() * rho0.double()
        # relative density perturbation of 1e-3; the densities are float32, so the
        # direction is the perturbation actually realised after rounding
        rp = (rho0.double() + h * v).float()
        rm = (rho0.double() - h * v).float()
        v_eff = (rp.double() - rm.double()) / (2 * h)
        fd = (L(rp, t0) - L(rm, t0)) / (2 * h)
        assert fd == pytest.approx(float((g_rho * v_eff).sum()), rel=1e-4)
