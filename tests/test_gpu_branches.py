"""CUDA path vs the FP64 oracle on the two branches the paper's own tests leave out:

* coupled quintessence with exp(beta phi~/c~^2) kept in front of (1 + delta)
  (Eq. csf_eom_code as written; Sec. 3.2.3 drops the factor);
* the symmetron with a sign-changing field (two domain walls pinned by
  high-density planes).

Both use the manufactured densities of tests/manufactured.py, whose exact
solutions the oracle recovers to 1e-10 (test_oracle_pins.py).  Each GPU solve is
compared with the oracle's solve of the same float32 density from the same
start: FP64 rel-L2 <= 1e-9 (the same fixed point to rounding), mixed rel-L2
<= 1e-6 (the mixed-precision target); and with the exact field within the
float32 rounding of the density (5e-6).  Meshes: 32 (the split finest level for
the symmetron), 48 (ragged levels 48-24-12-6), 64 (several rows per warp).
"""
import numpy as np
import pytest

import manufactured as mf

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


def gpu_solve(mg, pg, rho32, u0, tol):
    N = rho32.shape[0]
    if u0 is None:
        field = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device="cuda")
    else:
        field = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float64)).cuda()
    st = mg.solve_scalar(pg, 1.0, torch.from_numpy(rho32).cuda(), field, tol, allow_unconverged=True)
    return field.cpu().numpy(), st


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [16, 32, 48])
def test_cq_exp_factor_kept_matches_oracle(orc, mg, N, precision):
    kw, rho, phi = mf.cq_exp_kept(N)
    rho32 = rho.astype(np.float32)
    po = orc.Params(model=orc.CQ, a=1.0, **kw)
    ref = orc.solve(po, rho32.astype(np.float64), u0=np.zeros((N,) * 3), tol=1e-12, max_cycles=60,
                    kind=orc.KIND_NEWTON)
    assert ref.eps <= 1e-12
    pg = mg.Params(model=mg.CQ, precision=precision, max_cycles=60, **kw)
    got, st = gpu_solve(mg, pg, rho32, np.zeros((N,) * 3), 1e-10)
    assert st.converged, st
    assert relL2(got, ref.u) <= (1e-9 if precision == 0 else 1e-6)
    assert relL2(got, phi) <= 5e-6
    # the kept factor is exercised: the dropped-factor solution is ~1e-2 away
    pg0 = mg.Params(model=mg.CQ, precision=precision, max_cycles=60, **{**kw, "keep_exp": False})
    got0, _ = gpu_solve(mg, pg0, rho32, np.zeros((N,) * 3), 1e-10)
    assert relL2(got0, phi) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [32, 48, 64])
def test_symmetron_domain_walls_match_oracle(orc, mg, N, precision):
    """From the walls' sign pattern (+-ubar) both the GPU and the oracle recover
    the sign-changing solution; from the background both relax to the
    everywhere-positive solution of the same density."""
    kw, rho, u, m_eff = mf.symmetron_domain_walls(N)
    assert m_eff.min() > 0 and rho.min() > 0
    rho32 = rho.astype(np.float32)
    po = orc.Params(model=orc.SYMMETRON, a=1.0, **kw)
    ub = orc.background(po, N)["ubar"]
    pg = mg.Params(model=mg.SYMMETRON, precision=precision, max_cycles=60, **kw)
    bound = 1e-9 if precision == 0 else 1e-6
    for sgn in (1.0, -1.0):
        start = sgn * np.sign(u) * ub
        ref = orc.solve(po, rho32.astype(np.float64), u0=start, tol=1e-12, max_cycles=60)
        assert ref.eps <= 1e-12
        got, st = gpu_solve(mg, pg, rho32, start, 1e-10)
        assert st.converged, st
        assert np.array_equal(np.sign(got), sgn * np.sign(u))
        assert relL2(got, ref.u) <= bound
        assert relL2(got, sgn * u) <= 5e-6
    ref = orc.solve(po, rho32.astype(np.float64), tol=1e-12, max_cycles=60)
    got, st = gpu_solve(mg, pg, rho32, None, 1e-10)
    assert st.converged and got.min() > 0 and ref.u.min() > 0
    assert relL2(got, ref.u) <= bound
