"""mgglam_deposit_cic_static: the CIC deposit that allocates no device memory.

Some callers cannot let the library call cudaMalloc: applications whose
device memory is owned by their own pool allocator under a fixed budget, and
time-stepping loops that cannot take cudaMalloc's implicit device-wide
synchronisation.  For them the library offers a deposit whose accumulator is a
fixed device array compiled into the library (meshes up to 128^3).  These tests call it through
the C-ABI and compare it with the regular mgglam_deposit_cic on two calls in a
row: the second call must not see the first call's sums, since every call
shares the one array.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2110_00328_gb300 import inputs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg():
    from paper_2110_00328_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def test_static_deposit_rejects_meshes_above_its_array_before_any_work(mg):
    lib = mg.load()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the size check returns first
    assert lib.mgglam_deposit_cic_static(fake, 10, 130, fake, None) == -2
    assert lib.mgglam_deposit_cic_static(fake, 10, 1, fake, None) == -2
    assert lib.mgglam_deposit_cic_static(None, 10, 64, fake, None) == -1


@pytest.mark.gpu
def test_static_deposit_matches_regular_deposit_on_two_calls(mg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    N = 64
    pos1 = torch.from_numpy(inputs.zeldovich_positions(N, seed=60, sigma=1.5)).cuda()
    pos2 = torch.from_numpy(inputs.zeldovich_positions(N, seed=61, sigma=1.0, npart_side=48)).cuda()
    ref1 = mg.deposit_cic(pos1, N)
    ref2 = mg.deposit_cic(pos2, N)
    out = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    got1 = mg.deposit_cic_static(pos1, N, out).clone()
    got2 = mg.deposit_cic_static(pos2, N, out).clone()
    torch.cuda.synchronize()
    # same fixed-point arithmetic on both paths: the results agree bit for bit
    # (the parity tests hold the deposit to rtol 2e-7 against the oracle)
    assert torch.equal(got1, ref1)
    assert torch.equal(got2, ref2)
    assert not torch.equal(got1, got2)
    assert float(got2.double().sum()) == pytest.approx(N ** 3, rel=1e-6)
    # a smaller mesh after a larger one uses (and clears) only the front of the array
    N3 = 32
    pos3 = torch.from_numpy(inputs.zeldovich_positions(N3, seed=62, sigma=1.0)).cuda()
    assert torch.equal(mg.deposit_cic_static(pos3, N3), mg.deposit_cic(pos3, N3))
