"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

CPU only: no call here reaches a CUDA kernel.  Argument checks that return
before any device work are exercised.
"""
import ctypes
import glob
import os
import re

import pytest

from paper_2110_00328_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(mgglam_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("mgglam_deposit_cic", "mgglam_solve_scalar", "mgglam_gather_force"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.mgglam_version()
    assert lib.mgglam_status_string(0) == b"ok"
    assert lib.mgglam_status_string(-4) == b"not converged"


def test_default_params_match_binding_defaults(lib):
    p = binding.default_params()
    q = binding.Params().c()
    for name, _ in binding.CParams._fields_:
        if name == "reserved":
            continue
        assert getattr(p, name) == pytest.approx(getattr(q, name)), name
    assert lib.mgglam_default_params(None) == -1


def test_argument_errors_are_reported_before_any_device_work(lib):
    p = binding.Params().c()
    st = binding.CStats()
    nullp = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the checks return first
    assert lib.mgglam_solve_scalar(ctypes.byref(p), 1.0, nullp, 32, fake, 1e-8, ctypes.byref(st), None) == -1
    assert lib.mgglam_solve_scalar(ctypes.byref(p), 1.0, fake, 33, fake, 1e-8, ctypes.byref(st), None) == -2
    assert lib.mgglam_solve_scalar(ctypes.byref(p), 1.0, fake, 2, fake, 1e-8, ctypes.byref(st), None) == -2
    assert lib.mgglam_solve_scalar(ctypes.byref(p), 1.0, fake, 32, fake, -1.0, ctypes.byref(st), None) == -1
    bad = binding.Params(precision=7).c()
    assert lib.mgglam_solve_scalar(ctypes.byref(bad), 1.0, fake, 32, fake, 1e-8, ctypes.byref(st), None) == -1
    bad = binding.Params(fmg=2).c()
    assert lib.mgglam_solve_scalar(ctypes.byref(bad), 1.0, fake, 32, fake, 1e-8, ctypes.byref(st), None) == -1
    assert lib.mgglam_deposit_cic(nullp, 10, 32, fake, None) == -1
    assert lib.mgglam_deposit_cic(fake, 0, 32, fake, None) == -1
    assert lib.mgglam_deposit_cic(fake, 10, 4096, fake, None) == -2
    assert lib.mgglam_gather_force(ctypes.byref(p), 1.0, fake, 31, fake, 10, fake, 1.0, None) == -2
    assert lib.mgglam_gather_force(None, 1.0, fake, 32, fake, 10, fake, 1.0, None) == -1
    assert lib.mgglam_smooth(ctypes.byref(p), 1.0, 7, 1.0, fake, fake, None, 1, None) == -2
    assert lib.mgglam_restrict(5, fake, fake, None) == -2
    assert lib.mgglam_prolong_correct(ctypes.byref(p), 8, nullp, fake, fake, None) == -1


def test_binding_refuses_cpu_tensors(lib):
    import torch
    rho = torch.ones((8, 8, 8), dtype=torch.float32)
    field = torch.full((8, 8, 8), float("nan"), dtype=torch.float64)
    with pytest.raises(TypeError):
        binding.solve_scalar(binding.Params(), 1.0, rho, field, 1e-8)


def test_pm_entry_points_reject_bad_arguments_before_device_work(lib):
    """mgglam_poisson_fft and mgglam_pm_step check their arguments (NULL or aliased
    buffers, mesh sides that are not powers of two in 8..1024, non-positive steps
    or Hubble rates) and return before any device call."""
    fake, fake2 = ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000)
    lib.mgglam_poisson_fft.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p]
    assert lib.mgglam_poisson_fft(None, 32, 1.0, fake2, None) == -1
    assert lib.mgglam_poisson_fft(fake, 32, 1.0, fake, None) == -1       # rho aliases phi
    assert lib.mgglam_poisson_fft(fake, 32, float("nan"), fake2, None) == -1
    for N in (4, 12, 96, 2048):
        assert lib.mgglam_poisson_fft(fake, N, 1.0, fake2, None) == -2
    lib.mgglam_pm_step.argtypes = [ctypes.POINTER(binding.CParams), ctypes.POINTER(binding.CPmStepDesc),
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                   ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(binding.CStats), ctypes.c_void_p]
    p = binding.Params().c()
    st = binding.CStats()
    ok = binding.CPmStepDesc(0.5, 0.01, 1.0, 1.0, 0.0, 1)

    def call(desc=ok, N=32, pos=fake, mom=fake, np_=10, field=fake, tol=1e-8, rw=fake, pw=fake2, prm=p):
        return lib.mgglam_pm_step(ctypes.byref(prm), ctypes.byref(desc) if desc is not None else None, N, pos, mom,
                                  np_, field, tol, rw, pw, ctypes.byref(st), None)

    assert call(desc=None) == -1
    assert call(pos=None) == -1
    assert call(np_=0) == -1
    assert call(rw=fake2) == -1                    # rho_work aliases psi_work
    assert call(field=None) == -1                  # a scalar step needs the field
    assert call(tol=-1.0) == -1
    assert call(desc=binding.CPmStepDesc(0.5, 0.0, 1.0, 1.0, 0.0, 1)) == -1     # da <= 0
    assert call(desc=binding.CPmStepDesc(0.5, 0.01, -1.0, 1.0, 0.0, 1)) == -1   # E <= 0
    assert call(desc=binding.CPmStepDesc(0.0, 0.01, 1.0, 1.0, 0.0, 1)) == -1    # a <= 0
    for N in (4, 48, 2048):
        assert call(N=N) == -2
    assert call(prm=binding.Params(precision=9).c()) == -1
