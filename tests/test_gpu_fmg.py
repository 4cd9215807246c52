"""The full-multigrid start (mgglam_params.fmg) on the GPU against the oracle's.

* FP64: the GPU's FMG stages (the coarsest level relaxed from the background,
  each finer level from the prolonged coarser solution with one V-cycle) are the
  oracle's fmg_start, so the residual history agrees cycle by cycle (rtol 1e-7,
  the FP64 rounding floor of the relative residual) and the solutions to 1e-10.
* Mixed: from the background the correction-form FMG of the first outer step is
  the total-field FMG; after that one cycle the iterate follows the oracle's to
  single precision (2e-5 of the deviation from the background, as for the
  V-cycles), and the solves reach the oracle's solution (rel-L2 1e-6; CQ: the
  mean-subtracted fields, the mean being fixed only by the potential's tiny
  mass, as in test_gpu_parity).
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


def relL2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


MODELS = {
    "fr1": dict(model=0, n=1, fR0_abs=1e-6),
    "fr2": dict(model=0, n=2, fR0_abs=1e-6),
    "sym": dict(model=1, a_star=0.5, xi=1e-3, beta_star=1.0),
    "cq": dict(model=2, alpha=0.1, beta=-0.2, lam=1.0, phibar=0.5),
}


def pair(orc, mg, key, box, **extra):
    kw = dict(MODELS[key])
    okw = {k: v for k, v in kw.items() if k in orc.Params.__dataclass_fields__}
    return orc.Params(box=box, **okw), mg.Params(box=box, **kw, **extra)


def gpu_solve(mg, pg, rho32, tol):
    N = rho32.shape[0]
    f = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device="cuda")
    st = mg.solve_scalar(pg, 1.0, torch.from_numpy(rho32).cuda(), f, tol, allow_unconverged=True)
    return f.cpu().numpy(), st


def test_fp64_fmg_matches_oracle_cycle_by_cycle(orc, mg):
    """The 32^3 workload (f(R) n = 1, |fR0| = 1e-5, box 64, 5 levels, tol 1e-10)."""
    N = 32
    rho32 = inputs.lognormal_density(N, 1.0, seed=0).astype(np.float32)
    po = orc.Params(model=0, n=1, fR0_abs=1e-5, box=64.0)
    ref = orc.solve(po, rho32.astype(np.float64), tol=1e-10, max_cycles=30, levels=5, fmg=True)
    pg = mg.Params(model=0, n=1, fR0_abs=1e-5, box=64.0, precision=0, max_cycles=30, levels=5, fmg=1)
    got, st = gpu_solve(mg, pg, rho32, 1e-10)
    assert st.converged and st.cycles == ref.cycles
    np.testing.assert_allclose(st.hist, ref.hist, rtol=1e-7, atol=1e-13)
    assert relL2(got, ref.u) <= 1e-10


@pytest.mark.parametrize("key", ["fr1", "sym"])
@pytest.mark.parametrize("N", [64, 96])
def test_mixed_fmg_start_follows_oracle(orc, mg, key, N):
    """One cycle (the FMG start) from the background: split finest level with
    stored Delta w (f(R)) at 64^3 and 96^3 (levels 96-48-24-12-6)."""
    rho32 = inputs.lognormal_density(N, 1.0, seed=50 + N).astype(np.float32)
    box = float(N) if key == "sym" else 2.0 * N
    po, pg = pair(orc, mg, key, box, precision=1, max_cycles=1, fmg=1)
    ref = orc.solve(po, rho32.astype(np.float64), tol=0.0, max_cycles=1, fmg=True)
    got, st = gpu_solve(mg, pg, rho32, 0.0)
    assert st.cycles == 1
    ub = orc.background(po, N)["ubar"]
    assert relL2(got - ub, ref.u - ub) <= 2e-5


@pytest.mark.parametrize("key", list(MODELS))
def test_mixed_fmg_solve_matches_oracle(orc, mg, key):
    """f(R) n = 1, 2 and the symmetron with the FMG start; CQ, which ignores the
    flag (its mean is fixed only by a mass far below the mesh scales), solves as
    without it."""
    N = 64 if key != "cq" else 32
    rho32 = inputs.lognormal_density(N, 1.5, seed=90).astype(np.float32)
    box = {"sym": float(N), "cq": 64.0}.get(key, float(N))
    po, pg = pair(orc, mg, key, box, precision=1, max_cycles=40, fmg=1)
    kind = orc.KIND_NEWTON if key == "cq" else orc.KIND_NONLINEAR
    ref = orc.solve(po, rho32.astype(np.float64), tol=1e-11, max_cycles=60, kind=kind)
    got, st = gpu_solve(mg, pg, rho32, 1e-10)
    assert st.converged, st
    if key != "cq":
        assert relL2(got, ref.u) <= 1e-6
    else:
        assert relL2(got - got.mean(), ref.u - ref.u.mean()) <= 1e-6
