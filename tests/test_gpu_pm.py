"""CUDA particle-mesh step vs the FP64 oracle (oracle/pm.py), through the C-ABI.

Tolerances:
* FFT Poisson: single-precision FFTs of length N carry ~log2(N) x 6e-8 relative
  rounding per transform; 2e-5 of max|phi| covers the five passes up to N = 1024.
* One PM step: positions and momenta are float32 (rounding 6e-8 relative, i.e.
  ~2e-6 cells at x ~ 32); the mixed scalar solve agrees with the FP64 oracle to
  ~1e-6 of the field, the FP32 potential and gradient to ~1e-5 of the force.
  Bounds: |dx| <= 1e-4 cells, |dp| <= 1e-4 of max|p| + 2e-4 of the kick.
"""
import numpy as np
import pytest

from paper_2110_00328_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_00328_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def pm(orc):
    from oracle import pm as pm_mod
    return pm_mod


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256])
def test_poisson_fft_matches_oracle(mg, pm, N):
    rho = inputs.lognormal_density(N, 1.0, seed=60 + N).astype(np.float32) * 2.5
    coef = 1.5 * 0.3 / 0.7
    phi = mg.poisson_fft(torch.from_numpy(rho).cuda(), coef).cpu().numpy().astype(np.float64)
    ref = pm.poisson_fft(rho.astype(np.float64), coef)
    assert np.abs(phi - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("N", [512, 1024])
def test_poisson_fft_single_mode_closed_form(mg, N):
    """The largest transforms (32 x 16 and 32 x 32 splits): rho = 1 + A cos(2 pi m x / N)
    along each axis in turn gives phi = -coef A cos(...) / (4 sin^2(pi m / N))."""
    coef, A, m = 0.9, 0.4, 3
    x = (torch.arange(N, device="cuda", dtype=torch.float64) + 0.5) * (2 * np.pi * m / N)
    expect_line = (-coef * A * torch.cos(x) / (4 * np.sin(np.pi * m / N) ** 2)).cpu().numpy()
    for axis in range(3):
        shape = [1, 1, 1]
        shape[axis] = N
        rho = (1 + A * torch.cos(x)).to(torch.float32).reshape(shape).expand(N, N, N).contiguous()
        phi = mg.poisson_fft(rho, coef)
        idx = [slice(0, 1)] * 3
        idx[axis] = slice(None)
        got = phi[tuple(idx)].reshape(-1).double().cpu().numpy()
        assert np.abs(got - expect_line).max() <= 2e-5 * np.abs(expect_line).max()
        # every line along the other axes is the same
        assert float((phi - phi[tuple(idx)]).abs().max()) <= 2e-5 * np.abs(expect_line).max()
        del rho, phi
    torch.cuda.empty_cache()


def test_poisson_fft_rejects_unsupported_meshes(mg):
    x = torch.ones((12, 12, 12), dtype=torch.float32, device="cuda")
    with pytest.raises(mg.MgglamError):
        mg.poisson_fft(x, 1.0)


PM_MODELS = {
    "lcdm": None,
    "fr1": dict(model=0, n=1, fR0_abs=1e-5),
    "fr2": dict(model=0, n=2, fR0_abs=1e-5),
    "sym": dict(model=1, a_star=0.5, xi=1e-3, beta_star=1.0),
    "cq": dict(model=2, alpha=0.1, beta=-0.2, lam=1.0, phibar=0.5),
}


@pytest.mark.parametrize("key", list(PM_MODELS))
def test_pm_step_matches_oracle(orc, mg, pm, key):
    """One step of a 32^3-particle Zel'dovich realisation on a 32^3 mesh (box 64 Mpc/h)
    at a = 0.7: deposit, FFT Poisson, the scalar solve (mixed precision, warm-started
    from the background), forces, drag and leapfrog, against the oracle's step."""
    N, a, da = 32, 0.7, 0.02
    box = 64.0
    pos = inputs.zeldovich_positions(N, seed=61, sigma=0.8)
    rng = np.random.default_rng(62)
    mom = (0.05 * rng.standard_normal(pos.shape)).astype(np.float32)
    Om, OL = 0.3, 0.7
    E = lambda x: np.sqrt(Om / x ** 3 + OL)
    dphi = 0.8 if key == "cq" else 0.0
    kw = dict(PM_MODELS[key] or dict(model=0, n=1, fR0_abs=1e-5))
    po = orc.Params(box=box, a=a, **{k: v for k, v in kw.items() if k in orc.Params.__dataclass_fields__})
    pg = mg.Params(box=box, precision=1, max_cycles=60, **kw)
    scalar = PM_MODELS[key] is not None
    b = orc.background(po, N)
    field0 = np.full((N, N, N), b["ubar"] if key != "cq" else 0.0)
    rpos, rmom, _, _, _ = pm.pm_step(po, pos.astype(np.float64), mom.astype(np.float64), da, E(a), E(a + da / 2),
                                     field=field0, tol=1e-11, dphibar_da=dphi, scalar=scalar)
    gpos, gmom = torch.from_numpy(pos).cuda(), torch.from_numpy(mom).cuda()
    rho_w = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    psi_w = torch.empty_like(rho_w)
    field = torch.full((N, N, N), float("nan"), dtype=torch.float64, device="cuda") if scalar else None
    st = mg.pm_step(pg, a, da, gpos, gmom, rho_w, psi_w, field=field, tol=1e-10, E_a=E(a), E_half=E(a + da / 2),
                    dphibar_da=dphi)
    if scalar:
        assert st.converged
    gp, gm = gpos.cpu().numpy().astype(np.float64), gmom.cpu().numpy().astype(np.float64)
    dx = (gp - rpos + N / 2) % N - N / 2
    kick = np.abs(rmom - mom).max()
    assert kick > 1e-4  # the step moved the momenta
    assert np.abs(dx).max() <= 1e-4
    assert np.abs(gm - rmom).max() <= 1e-4 * np.abs(rmom).max() + 2e-4 * kick


def test_pm_plane_wave_grows_like_the_discrete_linear_mode(mg):
    """The oracle's plane-wave pin (test_pm.py) on the GPU: EdS, lattice at cell corners,
    final amplitude 0.025 cells after 40 steps from a = 0.2 to 0.6."""
    from test_pm import growth_exponent
    N, A_final, a0, a1, nsteps = 32, 0.025, 0.2, 0.6, 40
    k = 2 * np.pi / N
    alpha = growth_exponent(N)
    q = np.stack(np.meshgrid(*(np.arange(N),) * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    psi = np.sin(k * q[:, 0])
    A0 = A_final * (a0 / a1) ** alpha
    da = (a1 - a0) / nsteps
    pos = q.copy()
    pos[:, 0] += A0 * psi
    ah = a0 - 0.5 * da
    mom = np.zeros_like(q)
    mom[:, 0] = alpha * A0 * (ah / a0) ** alpha * ah ** 0.5 * psi
    gpos = torch.from_numpy(pos.astype(np.float32)).cuda()
    gmom = torch.from_numpy(mom.astype(np.float32)).cuda()
    rho_w = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    psi_w = torch.empty_like(rho_w)
    prm = mg.Params(model=0, n=1, fR0_abs=1e-5, omega_m=1.0, omega_l=0.0, box=64.0)
    a = a0
    for _ in range(nsteps):
        mg.pm_step(prm, a, da, gpos, gmom, rho_w, psi_w, E_a=a ** -1.5, E_half=(a + 0.5 * da) ** -1.5)
        a += da
    disp = (gpos.cpu().numpy().astype(np.float64) - q + N / 2) % N - N / 2
    # float32 positions near 32 resolve ~2e-6 cells: 1e-4 of the 0.025-cell amplitude
    assert np.abs(disp[:, 0] - A_final * psi).max() / A_final < 2e-3
    assert np.abs(disp[:, 1:]).max() < 1e-5


@pytest.mark.parametrize("N,steps", [(32, 5), (256, 1)])
def test_pm_step_conserves_momentum(mg, N, steps):
    """CIC deposit and interpolation with a symmetric Green's function and an
    antisymmetric difference exert no net force (test_pm.py pins this for the
    oracle); it holds at any size, so it checks the GPU step at the headline size
    (256^3 mesh, 256^3 Zel'dovich particles): a LCDM step changes the total momentum
    by float32 rounding only, far below the sum of the kicks."""
    pos = torch.from_numpy(inputs.zeldovich_positions(N, seed=1, sigma=1.5)).cuda()
    mom = torch.zeros_like(pos)
    rho_w = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    psi_w = torch.empty_like(rho_w)
    prm = mg.Params(model=0, n=1, fR0_abs=1e-6, box=float(N))
    a, da = 0.5, 0.01
    for s in range(steps):
        before = mom.double().sum(0)
        prev = mom.clone()
        mg.pm_step(prm, a + s * da, da, pos, mom, rho_w, psi_w)
        kick = (mom - prev).double()
        total = float(kick.abs().sum())
        assert total > 0
        assert float((mom.double().sum(0) - before).abs().max()) <= 1e-5 * total
