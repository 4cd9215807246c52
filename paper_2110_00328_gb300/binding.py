"""ctypes binding of libmgglam.so (declared in include/mgglam.h).

Argument marshalling only: torch CUDA tensors are passed as raw device pointers
together with the current CUDA stream; every step of the computation runs in
the library's kernels.  There is no CPU fallback: if the library is missing or
the tensors are not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field, fields

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgglam.so")

FR, SYMMETRON, CQ = 0, 1, 2
FP64, MIXED = 0, 1

STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported mesh size", -3: "CUDA error",
          -4: "not converged", -5: "non-finite residual", -6: "device wait timed out",
          -7: "out of device memory"}


class MgglamError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class CParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("n", ctypes.c_int), ("keep_exp", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("fR0_abs", ctypes.c_double), ("omega_m", ctypes.c_double), ("omega_l", ctypes.c_double),
                ("box", ctypes.c_double), ("a_star", ctypes.c_double), ("xi", ctypes.c_double),
                ("beta_star", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("lam", ctypes.c_double), ("phibar", ctypes.c_double),
                ("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("coarse_sweeps", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("check_every", ctypes.c_int),
                ("sweep_chunk", ctypes.c_int), ("sweep_slab", ctypes.c_int), ("tail_cells", ctypes.c_int),
                ("cycle", ctypes.c_int), ("fmg", ctypes.c_int)]


class CStats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer", ctypes.c_int), ("converged", ctypes.c_int),
                ("pad", ctypes.c_int), ("guarded", ctypes.c_longlong), ("resid0", ctypes.c_double),
                ("resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("resid_hist", ctypes.c_double * 64)]


@dataclass
class Params:
    """Mirror of mgglam_params (defaults = mgglam_default_params)."""
    model: int = FR
    n: int = 1
    keep_exp: bool = False
    precision: int = MIXED
    fR0_abs: float = 1e-5
    omega_m: float = 0.3
    omega_l: float = 0.7
    box: float = 256.0
    a_star: float = 0.5
    xi: float = 100.0 / 299792.458
    beta_star: float = 1.0
    alpha: float = 0.1
    beta: float = -0.05
    lam: float = 1.0
    phibar: float = 1.0
    levels: int = 0
    nu1: int = 2
    nu2: int = 2
    coarse_sweeps: int = 16
    max_cycles: int = 50
    inner_cycles: int = 0
    check_every: int = 1
    sweep_chunk: int = 0
    sweep_slab: int = 0
    tail_cells: int = 0
    cycle: int = 0
    fmg: int = 0

    def c(self) -> CParams:
        p = CParams()
        for f in fields(self):
            setattr(p, f.name, int(getattr(self, f.name)) if f.name == "keep_exp" else getattr(self, f.name))
        return p


@dataclass
class Stats:
    cycles: int
    outer: int
    converged: bool
    resid0: float
    resid: float
    seconds: float
    hist: list = field(default_factory=list)
    guarded: int = 0  # f(R) positivity-guard replacements


_lib = None
EXPORTS = ["mgglam_version", "mgglam_status_string", "mgglam_default_params", "mgglam_deposit_cic",
           "mgglam_solve_scalar", "mgglam_gather_force", "mgglam_smooth", "mgglam_residual",
           "mgglam_restrict", "mgglam_prolong_correct", "mgglam_release", "mgglam_profile_start",
           "mgglam_profile_stop", "mgglam_launch_count", "mgglam_deposit_cic_static",
           "mgglam_solve_adjoint", "mgglam_solve_batch", "mgglam_cq_background", "mgglam_radiation_density",
           "mgglam_deposit_cic_host", "mgglam_gather_force_host", "mgglam_poisson_fft", "mgglam_pm_step"]


class CKernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


def load(path: str = LIB_PATH):
    """Load the library (no CUDA context is created by loading)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, i, d, ll, vp = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_void_p
    lib.mgglam_version.restype = ctypes.c_char_p
    lib.mgglam_status_string.restype = ctypes.c_char_p
    lib.mgglam_status_string.argtypes = [i]
    lib.mgglam_default_params.argtypes = [P(CParams)]
    lib.mgglam_deposit_cic.argtypes = [vp, ll, i, vp, vp]
    lib.mgglam_deposit_cic_static.argtypes = [vp, ll, i, vp, vp]
    lib.mgglam_solve_scalar.argtypes = [P(CParams), d, vp, i, vp, d, P(CStats), vp]
    lib.mgglam_gather_force.argtypes = [P(CParams), d, vp, i, vp, ll, vp, d, vp]
    lib.mgglam_smooth.argtypes = [P(CParams), d, i, d, vp, vp, vp, i, vp]
    lib.mgglam_residual.argtypes = [P(CParams), d, i, d, vp, vp, vp, vp, P(ctypes.c_double), vp]
    lib.mgglam_restrict.argtypes = [i, vp, vp, vp]
    lib.mgglam_prolong_correct.argtypes = [P(CParams), i, vp, vp, vp, vp]
    lib.mgglam_release.argtypes = []
    lib.mgglam_profile_start.argtypes = []
    lib.mgglam_profile_stop.argtypes = [P(CKernelProfile), i, P(ctypes.c_int)]
    lib.mgglam_launch_count.restype = ll
    lib.mgglam_launch_count.argtypes = []
    lib.mgglam_solve_adjoint.argtypes = [P(CParams), d, vp, vp, i, vp, vp, vp, P(ctypes.c_double), d, P(CStats), vp]
    lib.mgglam_solve_batch.argtypes = [i, P(CParams), P(d), P(vp), P(i), P(vp), d, P(CStats), vp]
    lib.mgglam_deposit_cic_host.argtypes = [vp, vp, ll, i, vp, i, vp]
    lib.mgglam_gather_force_host.argtypes = [P(CParams), d, vp, i, vp, ll, vp, vp, d, i, vp]
    lib.mgglam_poisson_fft.argtypes = [vp, i, d, vp, vp]
    lib.mgglam_pm_step.argtypes = [P(CParams), P(CPmStepDesc), i, vp, vp, ll, vp, d, vp, vp, P(CStats), vp]
    lib.mgglam_cq_background.argtypes = [d, d, d, d, d, P(d), P(d), P(d), P(d)]
    lib.mgglam_radiation_density.argtypes = [d]
    lib.mgglam_radiation_density.restype = d
    for name in EXPORTS:
        getattr(lib, name).restype = getattr(lib, name).restype or i
    lib.mgglam_version.restype = ctypes.c_char_p
    lib.mgglam_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(fn: str, rc: int, allow=(0,)):
    if rc not in allow:
        raise MgglamError(fn, rc)
    return rc


def _ptr(t, dtype=None, host_ok=False):
    """Device address of a contiguous tensor.  host_ok: page-locked host tensors
    are accepted as well (the kernels read or write them directly over the
    host link); pageable host memory never is (there is no CPU path)."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise TypeError("expected a CUDA tensor" + (" or a pinned host tensor" if host_ok else "") +
                        " (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_params() -> CParams:
    p = CParams()
    _check("mgglam_default_params", load().mgglam_default_params(ctypes.byref(p)))
    return p


def deposit_cic(pos, N: int, rho=None, stream=None):
    """CIC density (mean 1) of particles pos [np,3] float32 (cell units) on an N^3 float32 mesh.
    pos may be a CUDA tensor or a pinned host tensor (read in place by the kernel)."""
    import torch
    if rho is None:
        rho = torch.empty((N, N, N), dtype=torch.float32, device="cuda" if not pos.is_cuda else pos.device)
    _check("mgglam_deposit_cic", load().mgglam_deposit_cic(_ptr(pos, torch.float32, host_ok=True), pos.shape[0], N,
                                                          _ptr(rho, torch.float32), _stream(stream)))
    return rho


def deposit_cic_host(pos_host, pos_dev, N: int, rho=None, chunks: int = 8, stream=None):
    """Deposit from pinned host positions, the copy into pos_dev (device staging)
    overlapped with the deposit (mgglam_deposit_cic_host)."""
    import torch
    if not (isinstance(pos_host, torch.Tensor) and pos_host.is_pinned()):
        raise TypeError("pos_host must be a pinned host tensor")
    if rho is None:
        rho = torch.empty((N, N, N), dtype=torch.float32, device=pos_dev.device)
    lib = load()
    _check("mgglam_deposit_cic_host",
           lib.mgglam_deposit_cic_host(ctypes.c_void_p(pos_host.data_ptr()), _ptr(pos_dev, torch.float32),
                                       pos_host.shape[0], N, _ptr(rho, torch.float32), chunks, _stream(stream)))
    return rho


def gather_force_host(prm: Params, a: float, field, pos_dev, force_dev, force_host, prefactor: float = 1.0,
                      chunks: int = 8, stream=None):
    """Gather with the forces delivered to a pinned host tensor, the copy
    overlapped with the gather (mgglam_gather_force_host)."""
    import torch
    if not (isinstance(force_host, torch.Tensor) and force_host.is_pinned()):
        raise TypeError("force_host must be a pinned host tensor")
    lib = load()
    _check("mgglam_gather_force_host",
           lib.mgglam_gather_force_host(ctypes.byref(prm.c()), a, _ptr(field, torch.float64), field.shape[0],
                                        _ptr(pos_dev, torch.float32), pos_dev.shape[0], _ptr(force_dev, torch.float32),
                                        ctypes.c_void_p(force_host.data_ptr()), prefactor, chunks, _stream(stream)))
    return force_host


def solve_scalar(prm: Params, a: float, rho, field, tol: float, stream=None, allow_unconverged=False) -> Stats:
    """Solve in place into field (N^3 float64; NaN first element = start from the background)."""
    import torch
    N = rho.shape[0]
    st = CStats()
    rc = load().mgglam_solve_scalar(ctypes.byref(prm.c()), a, _ptr(rho, torch.float32), N,
                                    _ptr(field, torch.float64), tol, ctypes.byref(st), _stream(stream))
    _check("mgglam_solve_scalar", rc, (0, -4) if allow_unconverged else (0,))
    nh = min(64, (st.outer if prm.precision == MIXED else st.cycles) + 1)
    return Stats(st.cycles, st.outer, bool(st.converged), st.resid0, st.resid, st.seconds,
                 list(st.resid_hist[:nh]), st.guarded)


def gather_force(prm: Params, a: float, field, pos, prefactor: float = 1.0, force=None, stream=None):
    """Fifth force on the particles.  pos and force may be CUDA tensors or pinned
    host tensors (read and written in place by the kernel)."""
    import torch
    N = field.shape[0]
    if force is None:
        force = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=field.device)
    _check("mgglam_gather_force", load().mgglam_gather_force(ctypes.byref(prm.c()), a, _ptr(field, torch.float64), N,
                                                            _ptr(pos, torch.float32, host_ok=True), pos.shape[0],
                                                            _ptr(force, torch.float32, host_ok=True), prefactor,
                                                            _stream(stream)))
    return force


def smooth(prm: Params, a: float, u, rho, S=None, sweeps: int = 1, h: float = 1.0, stream=None):
    import torch
    _check("mgglam_smooth", load().mgglam_smooth(ctypes.byref(prm.c()), a, u.shape[0], h, _ptr(u, torch.float64),
                                                _ptr(rho, torch.float64), _ptr(S, torch.float64), sweeps,
                                                _stream(stream)))
    return u


def residual(prm: Params, a: float, u, rho, S=None, h: float = 1.0, stream=None):
    import torch
    d = torch.empty_like(u)
    ss = ctypes.c_double()
    _check("mgglam_residual", load().mgglam_residual(ctypes.byref(prm.c()), a, u.shape[0], h, _ptr(u, torch.float64),
                                                    _ptr(rho, torch.float64), _ptr(S, torch.float64),
                                                    _ptr(d, torch.float64), ctypes.byref(ss), _stream(stream)))
    return d, ss.value


def restrict(fine, stream=None):
    import torch
    n = fine.shape[0]
    out = torch.empty((n // 2,) * 3, dtype=torch.float64, device=fine.device)
    _check("mgglam_restrict", load().mgglam_restrict(n, _ptr(fine, torch.float64), _ptr(out, torch.float64),
                                                    _stream(stream)))
    return out


def prolong_correct(prm: Params, uH, RuH, u_fine, stream=None):
    import torch
    _check("mgglam_prolong_correct", load().mgglam_prolong_correct(ctypes.byref(prm.c()), u_fine.shape[0],
                                                                  _ptr(uH, torch.float64), _ptr(RuH, torch.float64),
                                                                  _ptr(u_fine, torch.float64), _stream(stream)))
    return u_fine


def release():
    _check("mgglam_release", load().mgglam_release())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().mgglam_launch_count())


def profile_start():
    _check("mgglam_profile_start", load().mgglam_profile_start())


def profile_stop() -> dict:
    """Per-class {launches, ms, bytes} of the event-timed launches since profile_start()."""
    arr = (CKernelProfile * 32)()
    n = ctypes.c_int()
    _check("mgglam_profile_stop", load().mgglam_profile_stop(arr, 32, ctypes.byref(n)))
    return {arr[k].name.decode(): {"launches": arr[k].launches, "ms": arr[k].ms, "bytes": arr[k].bytes}
            for k in range(min(n.value, 32))}


def deposit_cic_static(pos, N: int, rho=None, stream=None):
    """CIC density through mgglam_deposit_cic_static (no device allocation; N <= 128).

    rho must be supplied by a caller that cannot allocate; it is created here
    only for convenience when omitted.
    """
    import torch
    lib = load()
    if rho is None:
        rho = torch.empty((N, N, N), dtype=torch.float32, device=pos.device)
    _check("mgglam_deposit_cic_static", lib.mgglam_deposit_cic_static(_ptr(pos, torch.float32), pos.shape[0], N,
                                                                    _ptr(rho, torch.float32), _stream(stream)))
    return rho


def solve_adjoint(prm: Params, a: float, field, rho, grad_field, tol: float = 1e-10, stream=None,
                  allow_unconverged=False, raw: bool = False):
    """Adjoint solve: returns (grad_rho [N^3 float64], dl/d ln|fR0|, Stats).

    grad_rho is dl/d delta; with raw=True it is dl/d rho for the rho passed in
    (the library composes the mean-1 normalisation's Jacobian)."""
    import torch
    lib = load()
    N = field.shape[0]
    grad_delta = torch.empty_like(field)
    grad_raw = torch.empty_like(field) if raw else None
    gth = ctypes.c_double()
    st = CStats()
    rc = lib.mgglam_solve_adjoint(ctypes.byref(prm.c()), a, _ptr(field, torch.float64), _ptr(rho, torch.float32), N,
                                  _ptr(grad_field, torch.float64), _ptr(grad_delta, torch.float64),
                                  _ptr(grad_raw, torch.float64) if raw else None, ctypes.byref(gth),
                                  tol, ctypes.byref(st), _stream(stream))
    _check("mgglam_solve_adjoint", rc, (0, -4) if allow_unconverged else (0,))
    nh = min(64, st.outer + 1)
    return (grad_raw if raw else grad_delta), gth.value, Stats(st.cycles, st.outer, bool(st.converged), st.resid0,
                                                               st.resid, st.seconds, list(st.resid_hist[:nh]))


def cq_background(alpha: float, beta: float, omega_m: float = 0.3, h: float = 0.6774, a: float = 1.0):
    """Coupled-quintessence background (mgglam_cq_background): dict with lambda,
    phibar(a), dphibar_dlna(a) and E = H(a)/H0."""
    lib = load()
    lam, ph, dph, E = (ctypes.c_double() for _ in range(4))
    _check("mgglam_cq_background",
           lib.mgglam_cq_background(ctypes.c_double(alpha), ctypes.c_double(beta), ctypes.c_double(omega_m),
                                    ctypes.c_double(h), ctypes.c_double(a), ctypes.byref(lam), ctypes.byref(ph),
                                    ctypes.byref(dph), ctypes.byref(E)))
    return {"lambda": lam.value, "phibar": ph.value, "dphibar_dlna": dph.value, "E": E.value}


def radiation_density(h: float = 0.6774) -> float:
    lib = load()
    lib.mgglam_radiation_density.restype = ctypes.c_double
    return lib.mgglam_radiation_density(ctypes.c_double(h))


def poisson_fft(rho, coef: float, phi=None, stream=None):
    """phi with grad_h^2 phi = coef (rho/mean - 1), mean(phi) = 0 (mgglam_poisson_fft)."""
    import torch
    N = rho.shape[0]
    if phi is None:
        phi = torch.empty_like(rho)
    lib = load()
    _check("mgglam_poisson_fft", lib.mgglam_poisson_fft(_ptr(rho, torch.float32), N, coef,
                                                        _ptr(phi, torch.float32), _stream(stream)))
    return phi


class CPmStepDesc(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("da", ctypes.c_double), ("E_a", ctypes.c_double),
                ("E_half", ctypes.c_double), ("dphibar_da", ctypes.c_double), ("scalar", ctypes.c_int)]


def lcdm_E(a: float, omega_m: float = 0.3, omega_l: float = 0.7) -> float:
    """H(a)/H0 of the flat LCDM background (matter and Lambda)."""
    return (omega_m / a ** 3 + omega_l) ** 0.5


def pm_step(prm: Params, a: float, da: float, pos, mom, rho_work, psi_work, field=None, tol: float = 1e-8,
            E_a: float | None = None, E_half: float | None = None, dphibar_da: float = 0.0, stream=None,
            allow_unconverged=False) -> Stats | None:
    """One PM leapfrog step in place on pos/mom (mgglam_pm_step); field=None is a
    LCDM step.  E_a, E_half default to the LCDM H/H0 of prm's Om, OL."""
    import torch
    N = rho_work.shape[0]
    if E_a is None:
        E_a = lcdm_E(a, prm.omega_m, prm.omega_l)
    if E_half is None:
        E_half = lcdm_E(a + 0.5 * da, prm.omega_m, prm.omega_l)
    d = CPmStepDesc(a, da, E_a, E_half, dphibar_da, 1 if field is not None else 0)
    st = CStats()
    lib = load()
    rc = lib.mgglam_pm_step(ctypes.byref(prm.c()), ctypes.byref(d), N, _ptr(pos, torch.float32),
                            _ptr(mom, torch.float32), pos.shape[0],
                            _ptr(field, torch.float64) if field is not None else None, tol,
                            _ptr(rho_work, torch.float32), _ptr(psi_work, torch.float32), ctypes.byref(st),
                            _stream(stream))
    _check("mgglam_pm_step", rc, (0, -4) if allow_unconverged else (0,))
    if field is None:
        return None
    nh = min(64, (st.outer if prm.precision == MIXED else st.cycles) + 1)
    return Stats(st.cycles, st.outer, bool(st.converged), st.resid0, st.resid, st.seconds, list(st.resid_hist[:nh]),
                 st.guarded)


def solve_batch(prms, a_list, rhos, fields, tol: float, stream=None, allow_unconverged=False):
    """Batched solve: prms, a_list, rhos (float32 N^3 CUDA), fields (float64 N^3 CUDA) per solve.

    Returns a list of Stats (one per solve)."""
    import torch
    lib = load()
    n = len(prms)
    cp = (CParams * n)(*[p.c() for p in prms])
    ca = (ctypes.c_double * n)(*a_list)
    cr = (ctypes.c_void_p * n)(*[_ptr(r, torch.float32).value for r in rhos])
    cn = (ctypes.c_int * n)(*[r.shape[0] for r in rhos])
    cf = (ctypes.c_void_p * n)(*[_ptr(f, torch.float64).value for f in fields])
    st = (CStats * n)()
    rc = lib.mgglam_solve_batch(n, cp, ca, cr, cn, cf, tol, st, _stream(stream))
    _check("mgglam_solve_batch", rc, (0, -4) if allow_unconverged else (0,))
    return [Stats(s.cycles, s.outer, bool(s.converged), s.resid0, s.resid, s.seconds,
                  list(s.resid_hist[:min(64, s.outer + 1)]), s.guarded) for s in st]
