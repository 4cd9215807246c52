"""Plain FP64 CPU oracle for the MG-GLAM scalar-field solve (arXiv:2110.00328).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing here is imported by
the CUDA path and nothing here imports it.

The arithmetic lives in ``mgoracle.c`` (loops written out from the paper, see its
header); this module loads it with ctypes and adds the numpy-level references
used to pin it: FFT solutions of the linearised and zero-coupling problems and a
dense Newton solve of the full discrete system on tiny meshes.

Parity status: every function is pinned by a ``-m "not gpu"`` test, including
the symmetron in sign-changing (domain-wall) regimes and CQ with the exp factor
kept, which are pinned by manufactured exact discrete solutions (the field is
chosen, the density derived from the equation with the 7-point Laplacian, and
the solve must return the field).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmgoracle.so")
_SRC = os.path.join(_HERE, "mgoracle.c")

FR, SYMMETRON, CQ = 0, 1, 2
KIND_NONLINEAR, KIND_NEWTON = 0, 1


def build(force: bool = False) -> str:
    """Compile mgoracle.c with gcc (OpenMP) into libmgoracle.so next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class CParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("n", ctypes.c_int), ("keep_exp", ctypes.c_int),
                ("pad0", ctypes.c_int),
                ("fR0_abs", ctypes.c_double), ("omega_m", ctypes.c_double),
                ("omega_l", ctypes.c_double), ("box", ctypes.c_double),
                ("a_star", ctypes.c_double), ("xi", ctypes.c_double), ("beta_star", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("lam", ctypes.c_double),
                ("phibar", ctypes.c_double), ("a", ctypes.c_double)]


class CBackground(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("ctilde", "c2", "Rbar", "fRbar", "ubar", "K0", "K", "msym", "cq_src", "cq_pot")]


@dataclass
class Params:
    """Model parameters in GLAM code units (box in Mpc/h)."""
    model: int = FR
    n: int = 1
    fR0_abs: float = 1e-5
    omega_m: float = 0.3
    omega_l: float = 0.7
    box: float = 64.0
    a_star: float = 0.5
    xi: float = 1e-3
    beta_star: float = 1.0
    alpha: float = 0.1
    beta: float = -0.05
    lam: float = 1.0
    phibar: float = 1.0
    a: float = 1.0
    keep_exp: bool = False

    def c(self) -> CParams:
        return CParams(self.model, self.n, int(self.keep_exp), 0, self.fR0_abs, self.omega_m,
                       self.omega_l, self.box, self.a_star, self.xi, self.beta_star, self.alpha,
                       self.beta, self.lam, self.phibar, self.a)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        dp = P(ctypes.c_double)
        fp = P(ctypes.c_float)
        _lib.or_compute_background.argtypes = [P(CParams), i, P(CBackground)]
        _lib.or_residual.argtypes = [P(CParams), P(CBackground), i, d, dp, dp, dp, dp]
        _lib.or_residual.restype = d
        _lib.or_smooth.argtypes = [P(CParams), P(CBackground), i, d, dp, dp, dp, i, i]
        _lib.or_restrict.argtypes = [i, dp, dp]
        _lib.or_prolong.argtypes = [i, dp, dp]
        _lib.or_prolong_correct.argtypes = [P(CParams), i, dp, dp, dp]
        _lib.or_prolong_correct.restype = ctypes.c_long
        _lib.or_solve.argtypes = [P(CParams), i, dp, dp, d, i, i, i, i, i, i, dp, dp,
                                  P(ctypes.c_long)]
        _lib.or_solve_cycle.argtypes = [P(CParams), i, dp, dp, d, i, i, i, i, i, i, i, i, dp, dp,
                                        ctypes.POINTER(ctypes.c_long)]
        _lib.or_solve_cycle.restype = i
        _lib.or_solve.restype = i
        _lib.or_source_rms.argtypes = [P(CParams), i, dp]
        _lib.or_source_rms.restype = d
        _lib.or_deposit_cic.argtypes = [fp, ll, i, dp]
        _lib.or_gather_force.argtypes = [P(CParams), i, dp, dp, fp, ll, d, dp]
        _lib.or_num_threads.restype = i
        _lib.or_set_num_threads.argtypes = [i]
        _lib.or_set_num_threads.restype = None
        _lib.or_local_root.argtypes = [i, i, d, d, d]
        _lib.or_local_root.restype = d
        _lib.or_cq_background.argtypes = [d, d, d, d, d, d, d, d, i, dp, dp, dp, dp]
        _lib.or_cq_background.restype = i
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def background(p: Params, N: int) -> dict:
    """Code-unit background scalars (c~, Rbar, fbar_R, ubar, ...) at p.a."""
    b = CBackground()
    lib().or_compute_background(ctypes.byref(p.c()), N, ctypes.byref(b))
    return {k: getattr(b, k) for k, _ in CBackground._fields_}


def residual(p: Params, u, rho, S=None, h: float = 1.0):
    """Local residual d = N_h(u) - S on one periodic level (rho must have mean 1 on the fine level)."""
    u, rho = _f64(u), _f64(rho)
    n = u.shape[0]
    b = CBackground()
    cp = p.c()
    lib().or_compute_background(ctypes.byref(cp), _fine_N(p, n, h), ctypes.byref(b))
    d = np.empty_like(u)
    S = _f64(S) if S is not None else None
    lib().or_residual(ctypes.byref(cp), ctypes.byref(b), n, h, _dp(u), _dp(rho), _dp(S), _dp(d))
    return d


def _fine_N(p: Params, n: int, h: float) -> int:
    # c~ is fixed by the finest mesh: N_fine = n * h
    return int(round(n * h))


def smooth(p: Params, u, rho, S=None, sweeps: int = 1, kind: int = KIND_NONLINEAR, h: float = 1.0):
    """Red-black sweeps (black first) on one level; returns the relaxed field."""
    u = _f64(u).copy()
    rho = _f64(rho)
    n = u.shape[0]
    b = CBackground()
    cp = p.c()
    lib().or_compute_background(ctypes.byref(cp), _fine_N(p, n, h), ctypes.byref(b))
    S = _f64(S) if S is not None else None
    lib().or_smooth(ctypes.byref(cp), ctypes.byref(b), n, h, _dp(u), _dp(rho), _dp(S), sweeps, kind)
    return u


def restrict(f):
    f = _f64(f)
    n = f.shape[0]
    out = np.empty((n // 2,) * 3)
    lib().or_restrict(n, _dp(f), _dp(out))
    return out


def prolong(c):
    c = _f64(c)
    n = c.shape[0]
    out = np.empty((2 * n,) * 3)
    lib().or_prolong(n, _dp(c), _dp(out))
    return out


def prolong_correct(p: Params, uH, RuH, uh):
    uh = _f64(uh).copy()
    g = lib().or_prolong_correct(ctypes.byref(p.c()), _f64(uH).shape[0], _dp(_f64(uH)), _dp(_f64(RuH)), _dp(uh))
    return uh, int(g)


@dataclass
class SolveResult:
    u: np.ndarray
    cycles: int
    eps: float
    hist: np.ndarray
    guarded: int = 0


def solve(p: Params, rho, u0=None, tol: float = 1e-10, max_cycles: int = 50, nu1: int = 2,
          nu2: int = 2, coarse_sweeps: int = 16, kind: int = KIND_NONLINEAR, levels: int = 0,
          cycle: int = 0, fmg: bool = False) -> SolveResult:
    """FAS cycles (cycle 0 V, 1 F, 2 W) to relative residual tol (or max_cycles).  u0=None starts
    from the background.  fmg: the first cycle is the full-multigrid start (the coarse problems
    first; it replaces the initial guess)."""
    rho = _f64(rho)
    N = rho.shape[0]
    u = np.full(rho.shape, np.nan) if u0 is None else _f64(u0).copy()
    hist = np.zeros(max_cycles + 1)
    eps = ctypes.c_double()
    g = ctypes.c_long()
    cyc = lib().or_solve_cycle(ctypes.byref(p.c()), N, _dp(rho), _dp(u), tol, max_cycles, nu1, nu2,
                               coarse_sweeps, kind, levels, cycle, int(fmg), _dp(hist), ctypes.byref(eps),
                               ctypes.byref(g))
    return SolveResult(u, cyc, eps.value, hist[: cyc + 1], g.value)


def source_rms(p: Params, rho) -> float:
    rho = _f64(rho)
    return lib().or_source_rms(ctypes.byref(p.c()), rho.shape[0], _dp(rho))


def deposit_cic(pos, N: int):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    rho = np.empty((N, N, N))
    lib().or_deposit_cic(pos.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), pos.shape[0], N, _dp(rho))
    return rho


def gather_force(p: Params, u, pos, prefactor: float = 1.0, phiN=None):
    u = _f64(u)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    out = np.empty((pos.shape[0], 3))
    phiN = _f64(phiN) if phiN is not None else None
    lib().or_gather_force(ctypes.byref(p.c()), u.shape[0], _dp(u), _dp(phiN),
                          pos.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), pos.shape[0],
                          prefactor, _dp(out))
    return out


def local_root(model: int, n: int, p: float, q: float, u_old: float = 1.0) -> float:
    """The admissible root of the local polynomial (u^{n+2} or u^3) + p u + q = 0."""
    return lib().or_local_root(model, n, p, q, u_old)


def radiation_density(h: float, T_cmb: float = 2.7255, N_eff: float = 3.046) -> float:
    """Omega_r today: CMB photons at T_cmb plus N_eff massless neutrino species (Sec. 3.2.3).

    rho_gamma = (4 sigma_SB / c) T^4 (radiation constant), rho_crit = 3 H0^2 / (8 pi G),
    neutrinos add N_eff (7/8) (4/11)^(4/3) of the photon density."""
    import math
    sigma_sb, c, G = 5.670374419e-8, 299792458.0, 6.67430e-11
    mpc = 3.0856775814913673e22
    H0 = 100.0 * h * 1e3 / mpc
    rho_gamma = 4.0 * sigma_sb / c ** 3 * T_cmb ** 4        # kg m^-3
    rho_crit = 3.0 * H0 * H0 / (8.0 * math.pi * G)
    return rho_gamma / rho_crit * (1.0 + N_eff * 7.0 / 8.0 * (4.0 / 11.0) ** (4.0 / 3.0))


def cq_background(alpha: float, beta: float, omega_m: float, omega_r: float, a: float = 1.0,
                  z_init: float = 1e5, phi_init: float = 1e-4, dphi_init: float = 0.0, steps: int = 50000):
    """Coupled-quintessence background by RK4 shooting: (lambda, phibar(a), dphibar/dlna(a), H(a)/H0)."""
    lam, ph, dph, E = (ctypes.c_double() for _ in range(4))
    it = lib().or_cq_background(alpha, beta, omega_m, omega_r, a, z_init, phi_init, dphi_init, steps,
                                ctypes.byref(lam), ctypes.byref(ph), ctypes.byref(dph), ctypes.byref(E))
    if it < 0:
        raise RuntimeError("no bracket for lambda")
    return lam.value, ph.value, dph.value, E.value


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (OpenMP)."""
    lib().or_set_num_threads(int(n))


# ---------------------------------------------------------------------------
# Adjoint (plain definition: the Jacobian assembled from the operator's
# derivatives, J^T lambda = g solved by sparse LU)
# ---------------------------------------------------------------------------

def _neighbour_index(N):
    idx = np.arange(N ** 3).reshape(N, N, N)
    return [np.roll(idx, s, ax).ravel() for ax in range(3) for s in (1, -1)]


def jacobian(p: Params, u, rho_n):
    """J = dN/du of the fine-level operator at u (scipy CSR), rho_n the mean-1 density.

    f(R) (Eq. fR_eom_codeunit2, w = u^{n+1}): dN_i/du_j = -c^2 (n+1) u_j^n for a
    face neighbour j, dN_i/du_i = 6 c^2 (n+1) u_i^n + K/u_i^2.
    symmetron (Eq. sym_eom_code_unit): dN_i/du_j = c^2, dN_i/du_i = -6 c^2 -
    msym (rho a*^3/a^3 - 1 + 3 u_i^2).
    """
    import scipy.sparse as sp
    u = _f64(u)
    N = u.shape[0]
    b = background(p, N)
    n3 = N ** 3
    rows = np.arange(n3)
    nbrs = _neighbour_index(N)
    uf = u.ravel()
    if p.model == FR:
        dwdu = (p.n + 1) * uf ** p.n
        diag = 6 * b["c2"] * dwdu + b["K"] / uf ** 2
        offv = [-b["c2"] * dwdu[nb] for nb in nbrs]   # column j = neighbour, value uses u_j
    elif p.model == SYMMETRON:
        r3 = (p.a_star / p.a) ** 3
        diag = -6 * b["c2"] - b["msym"] * (_f64(rho_n).ravel() * r3 - 1 + 3 * uf ** 2)
        offv = [np.full(n3, b["c2"]) for _ in nbrs]
    else:
        raise ValueError("adjoint: f(R) and symmetron only")
    r = [rows] + [rows] * 6
    c = [rows] + nbrs
    v = [diag] + offv
    return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))), shape=(n3, n3))


def adjoint(p: Params, u, rho_n, g):
    """lambda = J^{-T} g; returns (lambda, dl/d delta, dl/d ln|fR0|).

    dl/d delta_i = -(dN_i/d delta_i) lambda_i: f(R) dN/d delta = Om/a; symmetron
    dN/d delta = -msym (a*/a)^3 u.  dl/d ln|fR0| = -lambda . dN/d ln|fR0| with
    dN_i/d ln|fR0| = -K/((n+1) u_i) (ubar scales as |fR0|^{1/(n+1)}).
    """
    import scipy.sparse.linalg as spla
    u = _f64(u)
    N = u.shape[0]
    b = background(p, N)
    J = jacobian(p, u, rho_n)
    lam = spla.spsolve(J.T.tocsc(), _f64(g).ravel()).reshape(u.shape)
    if p.model == FR:
        gd = -(p.omega_m / p.a) * lam
        gt = float(np.sum(lam * b["K"] / ((p.n + 1) * u)))
    else:
        gd = b["msym"] * (p.a_star / p.a) ** 3 * u * lam
        gt = 0.0
    return lam, gd, gt
