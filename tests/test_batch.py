"""Batched solves (mgglam_solve_batch): argument checks on CPU, and on the GPU each
batched solution against the same solve run alone and against the oracle.

Tolerance: every solve is carried to relative residual 1e-10; the batched and
individual runs may take different cycle counts (the adaptive inner-cycle count
follows the worst solve in the batch), so they agree to the solution accuracy,
field rel-L2 <= 1e-6 (the stated target for the mixed path), as does the oracle.
"""
import ctypes

import numpy as np
import pytest

from paper_2110_00328_gb300 import binding, build, inputs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_batch_argument_checks(lib):
    p = (binding.CParams * 2)(binding.Params().c(), binding.Params().c())
    a = (ctypes.c_double * 2)(1.0, 1.0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the checks return first
    ptrs = (ctypes.c_void_p * 2)(fake, fake)
    st = (binding.CStats * 2)()
    lib.mgglam_solve_batch.argtypes = None
    n_bad = (ctypes.c_int * 2)(64, 48)
    assert lib.mgglam_solve_batch(2, p, a, ptrs, n_bad, ptrs, ctypes.c_double(1e-8), st, None) == -2
    n_ok = (ctypes.c_int * 2)(64, 96)
    p2 = (binding.CParams * 2)(binding.Params().c(), binding.Params(nu1=3).c())
    assert lib.mgglam_solve_batch(2, p2, a, ptrs, n_ok, ptrs, ctypes.c_double(1e-8), st, None) == -1
    assert lib.mgglam_solve_batch(0, p, a, ptrs, n_ok, ptrs, ctypes.c_double(1e-8), st, None) == -1
    nulls = (ctypes.c_void_p * 2)(fake, None)
    assert lib.mgglam_solve_batch(2, p, a, nulls, n_ok, ptrs, ctypes.c_double(1e-8), st, None) == -1
    lib.mgglam_solve_batch.argtypes = None
    binding._lib = None  # re-bind argtypes on the next load()


torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_batch_matches_individual_solves_and_oracle(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    binding.load()
    cases = [
        (32, dict(model=0, n=1, fR0_abs=1e-5, box=32.0)),
        (64, dict(model=0, n=1, fR0_abs=1e-6, box=64.0)),
        (96, dict(model=0, n=1, fR0_abs=3e-5, box=96.0)),
        (64, dict(model=1, a_star=0.5, xi=100 / 299792.458, beta_star=1.0, box=64.0)),
        (32, dict(model=1, a_star=0.5, xi=2 * 100 / 299792.458, beta_star=1.0, box=32.0)),
        (64, dict(model=0, n=1, fR0_abs=1e-4, box=64.0)),
    ]
    prms, rhos, fields, singles = [], [], [], []
    for idx, (N, kw) in enumerate(cases):
        rho = inputs.lognormal_density(N, 1.0 + 0.2 * idx, seed=90 + idx).astype(np.float32)
        prms.append(binding.Params(**kw, max_cycles=60))
        rhos.append(torch.from_numpy(rho).cuda())
        fields.append(torch.full((N, N, N), float("nan"), dtype=torch.float64, device="cuda"))
    stats = binding.solve_batch(prms, [1.0] * len(cases), rhos, fields, 1e-10)
    for k, ((N, kw), st) in enumerate(zip(cases, stats)):
        assert st.converged, (k, st)
        f1 = torch.full((N, N, N), float("nan"), dtype=torch.float64, device="cuda")
        binding.solve_scalar(prms[k], 1.0, rhos[k], f1, 1e-10)
        got, one = fields[k].cpu().numpy(), f1.cpu().numpy()
        assert np.linalg.norm(got - one) <= 1e-6 * np.linalg.norm(one), k
        okw = {key: v for key, v in kw.items() if key in orc.Params.__dataclass_fields__}
        ref = orc.solve(orc.Params(**okw), rhos[k].cpu().numpy().astype(np.float64), tol=1e-11, max_cycles=60)
        assert np.linalg.norm(got - ref.u) <= 1e-6 * np.linalg.norm(ref.u), k
    # a second call with the same shapes reuses the cached batch and its graph
    for f in fields:
        f.fill_(float("nan"))
    stats2 = binding.solve_batch(prms, [1.0] * len(cases), rhos, fields, 1e-10)
    assert all(s.converged for s in stats2)
