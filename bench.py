#!/usr/bin/env python
"""Benchmark of the MG-GLAM scalar-field hot path on GB300.

One step = the whole per-time-step path on the 256^3 f(R) workload
(Hu-Sawicki n=1, |f_R0| = 1e-6, box 256 Mpc/h, a = 1): CIC deposit of 256^3
Zel'dovich particles (pixel sigma 1.5, seed 1 + rank), the mixed-precision FAS
solve from the background field to relative residual 1e-8, and the fifth-force
gather back to every particle.  Inputs are resident in HBM before timing
starts; every step recomputes everything from the particle positions.

Metric: cell updates per second (one nonlinear Gauss-Seidel relaxation of one
cell on any multigrid level is one update), with time-to-tolerance and the
fraction of the HBM roofline reported beside it.  With torchrun (N > 1) each
rank solves its own independent realisation (weak scaling, no collective on
the data path); the timings are reduced with a max over ranks.

--impl reference times the FP64 CPU oracle (the test-suite reference) on the
host cores over a bounded sample of the same workload (deposit, one V-cycle,
gather per step).
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_MESH = 256
BOX = 256.0
FR0 = 1e-6
TOL = 1e-8
SIGMA = 1.5
WORKLOAD = "fR_HS_n1_fR0_1e-6_256cube_box256_zeldovich_sigma1.5_cic_tol1e-8"


def workload_config() -> dict:
    """The workload keys both arms' lines share."""
    return {"workload": WORKLOAD, "N": N_MESH, "box_mpch": BOX, "fR0": FR0, "n": 1, "tol": TOL,
            "particles": N_MESH ** 3}
METRIC = "f(R) solve time-to-1e-8 residual at 256^3; Mcell-updates/s and % HBM peak"
UNIT = "Mcell-updates/s"


# The solver schedule the bench times: V(2,1) cycles with 4 sweeps on the 4^3
# level (the fastest time to 1e-8 on this workload; the library's defaults are
# V(2,2) with 16), every other knob at the library default (split finest level,
# dependent-launch colour passes, warm-started local solve, adaptive inner cycles).
SCHEDULE = dict(nu1=2, nu2=1, coarse_sweeps=4, inner_cycles=0, sweep_chunk=0, tail_cells=0, cycle=0)


def headline_params(mg, precision=None, **override):
    """mgglam_params of the timed 256^3 f(R) solve (the tests import this too)."""
    kw = {**SCHEDULE, **override}
    return mg.Params(model=mg.FR, n=1, fR0_abs=FR0, box=BOX, precision=mg.MIXED if precision is None else precision,
                     max_cycles=60, **kw)


def models_params(mg, name: str, precision=None, lam=None, phibar=None):
    """mgglam_params of the 256^3 symmetron (a* = 0.5, beta* = 1, range 1 Mpc/h) and
    coupled-quintessence (alpha = 0.1, beta = -0.05; lambda and phibar(1) from the
    background solver) solves, with the headline schedule."""
    prec = mg.MIXED if precision is None else precision
    if name == "symmetron":
        kw = dict(model=mg.SYMMETRON, a_star=0.5, beta_star=1.0, xi=100.0 / 299792.458, box=256.0)
    else:
        kw = dict(model=mg.CQ, alpha=0.1, beta=-0.05, lam=lam, phibar=phibar, box=256.0)
    return mg.Params(**kw, precision=prec, max_cycles=80, nu1=2, nu2=1, coarse_sweeps=4)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes per fine-level sweep of the smoother at 256^3: dram__bytes_read.sum +
# dram__bytes_write.sum of both colour launches of a warm sweep (cycle 6, the
# path every pass after an inner solve's first sweep takes), from one ncu
# capture; valid while the kernel's sources hash to the value recorded with it.
SMOOTHER_TRAFFIC = {"bytes_per_sweep": (134.520576 + 43.065344 + 134.503680 + 38.631680) * 1e6,
                    "source_sha256_16": "255035e13679efa1"}


def smoother_traffic_per_sweep():
    import hashlib
    h = hashlib.sha256()
    for f in ("sweep32.cuh", "mg_common.cuh", "mg_model.cuh"):
        with open(os.path.join(ROOT, "paper_2110_00328_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != SMOOTHER_TRAFFIC["source_sha256_16"]:
        return None  # the kernel changed since the counters were taken
    return SMOOTHER_TRAFFIC["bytes_per_sweep"]


def level_sizes(N: int):
    """Mesh sides of the multigrid levels (halve while even and the half is >= 4 and even)."""
    ns = [N]
    n = N
    while n % 2 == 0 and n // 2 >= 4 and (n // 2) % 2 == 0:
        n //= 2
        ns.append(n)
    return ns


def level_visits(l: int, cycle: int) -> int:
    """Visits of level l in one cycle: V once; W 2^l; F l + 1 (F then V below the finest)."""
    if cycle == 2:
        return 2 ** l
    if cycle == 1:
        return l + 1
    return 1


def updates_per_cycle(N: int, nu1=2, nu2=2, coarse=16, cycle=0) -> int:
    ns = level_sizes(N)
    L = len(ns)
    return (sum(level_visits(l, cycle) * (nu1 + nu2) * ns[l] ** 3 for l in range(L - 1)) +
            level_visits(L - 1, cycle) * coarse * ns[-1] ** 3)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.p = None
        self.gpu = gpu_index
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x: float, world: int, device) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput in millions per second: every rank processes
    units_per_rank; the job takes the slowest rank's time (max over ranks)."""
    return units_per_rank * world / (max_ms * 1e-3) / 1e6


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_step(pos, cycles: int | None):
    """Deposit, FAS solve (cycles=None: to tolerance; else that many V-cycles), gather."""
    import oracle
    rho = oracle.deposit_cic(pos, N_MESH)
    p = oracle.Params(model=oracle.FR, n=1, fR0_abs=FR0, box=BOX)
    r = oracle.solve(p, rho, tol=TOL if cycles is None else 0.0, max_cycles=cycles or 50)
    oracle.gather_force(p, r.u, pos)
    return r


def run_oracle_baseline(pos) -> dict:
    """The oracle as it stands on the host cores: one full step with every core,
    and a bounded sample (deposit, one V-cycle, gather) on one thread."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    r = oracle_step(pos, None)
    dt = time.perf_counter() - t0
    ups = r.cycles * updates_per_cycle(N_MESH)
    oracle.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        oracle_step(pos, 1)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    return {"value": ups / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one full step at 256^3 (deposit, {r.cycles} V-cycles to {r.eps:.1e}, gather) in {dt:.1f} s",
            "seconds": dt, "time_to_tol_ms": dt * 1e3,
            "single_thread": {"value": updates_per_cycle(N_MESH) / dt1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"deposit, one V-cycle, gather at 256^3 on one thread in {dt1:.1f} s",
                              "seconds": dt1}}


def run_reference(args) -> None:
    world, rank, _ = dist_init()
    if rank != 0:
        return
    from paper_2110_00328_gb300 import inputs
    import oracle
    oracle.build()
    pos = inputs.zeldovich_positions(N_MESH, seed=1, sigma=SIGMA)
    for _ in range(args.warmup):
        oracle_step(pos, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(pos, 1)
    dt = time.perf_counter() - t0
    ups = args.steps * updates_per_cycle(N_MESH)
    value = ups / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {**workload_config(), "sample": "deposit + 1 V-cycle + gather"},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(),
                             "sample": "per step: CIC deposit, one FAS V-cycle, gather at 256^3", "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Extra measurements: adjoint at 512^3, batch of 48 uneven solves
# ---------------------------------------------------------------------------

def batch_workload(seed: int = 4, count: int = 48):
    """48 solves: N from {64, 96, 128, 192} (L = N Mpc/h), f(R) n=1 with |fR0|
    log-uniform in [1e-7, 1e-4] or symmetron (a* = 0.5, beta* = 1, range log-uniform
    in [0.5, 3] Mpc/h), 50/50; lognormal densities with sigma_g ~ U[0.8, 2.0], seed 100 + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice([64, 96, 128, 192]))
        sg = float(rng.uniform(0.8, 2.0))
        if rng.random() < 0.5:
            kw = dict(model=0, n=1, fR0_abs=float(10 ** rng.uniform(-7, -4)), box=float(N))
        else:
            rng_mpch = float(10 ** rng.uniform(np.log10(0.5), np.log10(3.0)))
            kw = dict(model=1, a_star=0.5, beta_star=1.0, xi=rng_mpch * 100.0 / 299792.458, box=float(N))
        out.append((N, sg, 100 + i, kw))
    return out


def run_batch_extra(mg, torch, dev, tol=TOL) -> dict:
    from paper_2110_00328_gb300 import inputs
    work = batch_workload()
    prms = [mg.Params(**kw, max_cycles=60) for (_, _, _, kw) in work]
    rhos = [torch.from_numpy(inputs.lognormal_density(N, sg, seed).astype(np.float32)).to(dev)
            for (N, sg, seed, _) in work]
    fields = [torch.empty((N,) * 3, dtype=torch.float64, device=dev) for (N, _, _, _) in work]
    cells = sum(N ** 3 for (N, _, _, _) in work)

    def reset():
        for f in fields:
            f.fill_(float("nan"))
        torch.cuda.synchronize()

    def timed(fn, reps):
        best = []
        for _ in range(reps):
            reset()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            best.append((time.perf_counter() - t0) * 1e3)
        return min(best), out

    reset()
    mg.solve_batch(prms, [1.0] * len(work), rhos, fields, tol)  # allocation, autotune, graph capture
    t_batch, stats = timed(lambda: mg.solve_batch(prms, [1.0] * len(work), rhos, fields, tol), 2)

    def seq(precision):
        out = []
        for p, r, f in zip(prms, rhos, fields):
            q = mg.Params(**{**p.__dict__, "precision": precision})
            out.append(mg.solve_scalar(q, 1.0, r, f, tol, allow_unconverged=True))
        return out

    seq(mg.MIXED)  # workspaces for every mesh size
    t_seq_mixed, st_mixed = timed(lambda: seq(mg.MIXED), 1)
    t_seq_fp64, st_fp64 = timed(lambda: seq(mg.FP64), 1)
    return {"workload": "48 solves, N in {64,96,128,192}, f(R) n=1 |fR0| log-U[1e-7,1e-4] / symmetron range "
                        "log-U[0.5,3] Mpc/h, lognormal sigma_g U[0.8,2], seeds 4 and 100+i, tol 1e-8",
            "cells": int(cells), "batched_ms": round(t_batch, 2),
            "sequential_mixed_ms": round(t_seq_mixed, 2), "sequential_fp64_ms": round(t_seq_fp64, 2),
            "speedup_vs_sequential_mixed": round(t_seq_mixed / t_batch, 2),
            "speedup_vs_sequential_fp64": round(t_seq_fp64 / t_batch, 2),
            "all_converged": bool(all(s.converged for s in stats)),
            "max_resid": float(max(s.resid for s in stats)),
            "max_cycles": int(max(s.cycles for s in stats)),
            "fp64_all_converged": bool(all(s.converged for s in st_fp64))}


def run_models_extra(mg, torch, dev, tol=TOL) -> dict:
    """256^3, box 256 Mpc/h, lognormal density (sigma_g = 2.0, P ~ k^-1.5 with a
    Gaussian cut at half the Nyquist wavenumber, seed 2): symmetron (a* = 0.5,
    beta* = 1, range 1 Mpc/h) and coupled quintessence (alpha = 0.1, beta = -0.05,
    phibar(1) and lambda from the background solver), mixed precision vs plain
    FP64, from the background field to relative residual 1e-8."""
    from paper_2110_00328_gb300 import inputs
    N = 256
    rho = torch.from_numpy(inputs.lognormal_density(N, 2.0, seed=2).astype(np.float32)).to(dev)
    bg = mg.cq_background(0.1, -0.05, 0.3, 0.6774, 1.0)
    out = {"workload": "256^3 lognormal sigma_g 2.0 seed 2, tol 1e-8; CQ background: lambda %.6f phibar(1) %.6f"
                       % (bg["lambda"], bg["phibar"])}
    field = torch.empty((N,) * 3, dtype=torch.float64, device=dev)
    for name in ("symmetron", "cq"):
        res = {}
        for prec, pname in ((mg.MIXED, "mixed"), (mg.FP64, "fp64")):
            p = models_params(mg, name, prec, lam=bg["lambda"], phibar=bg["phibar"])
            times = []
            for rep in range(3):
                field.fill_(float("nan"))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = mg.solve_scalar(p, 1.0, rho, field, tol, allow_unconverged=True)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            res[pname] = {"time_to_tol_ms": round(min(times[1:]), 3), "cycles": st.cycles, "converged": bool(st.converged),
                          "resid": st.resid}
        res["speedup_mixed_vs_fp64"] = round(res["fp64"]["time_to_tol_ms"] / res["mixed"]["time_to_tol_ms"], 2)
        out[name] = res
    return out


def run_fmg_extra(mg, torch, rho, field, stream) -> dict:
    """Time to 1e-8 on the headline density with the full-multigrid start against
    the V-cycle start (the background), mixed and plain FP64, same schedule."""
    out = {"workload": "the headline density (deposited 256^3 Zel'dovich particles), tol 1e-8"}
    for prec, pname in ((mg.MIXED, "mixed"), (mg.FP64, "fp64")):
        for fmg in (0, 1):
            p = headline_params(mg, precision=prec, fmg=fmg)
            times = []
            for _ in range(3 if prec == mg.MIXED else 2):
                field.fill_(float("nan"))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = mg.solve_scalar(p, 1.0, rho, field, TOL)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            out[f"{pname}_{'fmg' if fmg else 'v'}"] = {"time_to_tol_ms": round(min(times[1:] or times), 3),
                                                      "cycles": st.cycles, "outer_steps": st.outer,
                                                      "resid": st.resid, "hist": st.hist}
    for pname in ("mixed", "fp64"):
        out[f"{pname}_fmg_speedup"] = round(out[f"{pname}_v"]["time_to_tol_ms"] / out[f"{pname}_fmg"]["time_to_tol_ms"], 3)
    return out


def run_pm_extra(mg, torch, dev) -> dict:
    """One particle-mesh time step at 256^3 (the headline workload's 256^3 Zel'dovich
    particles and mesh, box 256 Mpc/h, a = 0.9, da = 0.01, momenta from rest):
    LCDM (deposit, FFT Poisson, gather-kick-drift) against f(R) n=1, |fR0| = 1e-6
    (the same plus the mixed scalar solve to 1e-8, warm-started from the previous
    step's field as in a simulation, or from the background), and the FFT Poisson
    solve alone (algorithmic 72 B/cell: density in, five complex passes, potential out).
    The paper reports an MG-GLAM run at 3-5x the time of the LCDM GLAM run (Sec. 1)."""
    from paper_2110_00328_gb300 import inputs
    N = N_MESH
    pos0 = torch.from_numpy(inputs.zeldovich_positions(N, seed=1, sigma=SIGMA)).to(dev)
    rho_w = torch.empty((N,) * 3, dtype=torch.float32, device=dev)
    psi_w = torch.empty_like(rho_w)
    prm = mg.Params(model=0, n=1, fR0_abs=FR0, box=BOX, precision=mg.MIXED, max_cycles=80, nu2=1, coarse_sweeps=4)
    a0, da, steps = 0.9, 0.01, 6

    def run(scalar: bool, warm: bool):
        pos, mom = pos0.clone(), torch.zeros_like(pos0)
        field = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device=dev) if scalar else None
        times, cycles = [], []
        for s in range(steps):
            if scalar and not warm:
                field.fill_(float("nan"))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = mg.pm_step(prm, a0 + s * da, da, pos, mom, rho_w, psi_w, field=field, tol=TOL)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            if st is not None:
                cycles.append(st.cycles)
        return times, cycles

    t_l, _ = run(False, True)
    t_w, c_w = run(True, True)
    t_c, c_c = run(True, False)
    ms = lambda t: round(float(np.median(t[1:])), 3)
    fft = []
    for _ in range(8):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mg.poisson_fft(rho_w, 1.5 * 0.3 / a0, psi_w)
        e1.record()
        torch.cuda.synchronize()
        fft.append(e0.elapsed_time(e1))
    fft_ms = float(np.median(fft[2:]))
    peak, _ = measured_peaks()
    gbs = 72.0 * N ** 3 / (fft_ms * 1e-3) / 1e9
    return {"workload": "256^3 mesh, 256^3 Zel'dovich particles (pixel sigma 1.5, seed 1), box 256, a = 0.9, "
                        "da = 0.01, 6 steps (median of steps 2-6)",
            "lcdm_step_ms": ms(t_l), "fr_step_warm_ms": ms(t_w), "fr_cycles_warm": c_w,
            "fr_step_cold_ms": ms(t_c), "fr_cycles_cold": c_c,
            "mg_over_lcdm_warm": round(ms(t_w) / ms(t_l), 2), "mg_over_lcdm_cold": round(ms(t_c) / ms(t_l), 2),
            "paper_mg_over_lcdm": "3-5 (whole runs, Sec. 1)",
            "poisson_fft_ms": round(fft_ms, 4), "poisson_fft_GBps": round(gbs, 1),
            "poisson_fft_frac_hbm": round(gbs / peak, 4)}


def run_adjoint_extra(mg, torch, dev) -> dict:
    """Gradient of sum_b log P_F(k_b) (fifth-force power, 32 log bins) w.r.t. the
    density and ln|fR0| at 512^3 (f(R) n=1, |fR0| = 1e-5, box 512 Mpc/h, lognormal
    sigma_g = 1.5, seed 3), timed, and checked against central differences (step 1e-3)."""
    import math
    from paper_2110_00328_gb300 import autograd as ag
    from paper_2110_00328_gb300 import inputs
    N = 512
    prm = mg.Params(model=0, n=1, fR0_abs=1e-5, box=512.0, precision=mg.MIXED, max_cycles=80)
    rho0 = torch.from_numpy(inputs.lognormal_density(N, 1.5, seed=3).astype(np.float32)).to(dev)
    t0v = math.log(1e-5)
    tol = 1e-10

    def fwd_bwd():
        rho = rho0.clone().requires_grad_(True)
        th = torch.tensor(t0v, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        a = time.perf_counter()
        u = ag.solve(rho, th, prm, 1.0, tol)
        loss = ag.fifth_force_power_loss(u, prm)
        torch.cuda.synchronize()
        b = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        c = time.perf_counter()
        return rho.grad.double(), float(th.grad), (b - a) * 1e3, (c - b) * 1e3

    fwd_bwd()
    g_rho, g_th, f_ms, b_ms = fwd_bwd()

    def L(r, t):
        with torch.no_grad():
            return float(ag.fifth_force_power_loss(ag.solve(r, torch.tensor(t, dtype=torch.float64), prm, 1.0, tol),
                                                   prm))

    h = 1e-3
    fdt = (L(rho0, t0v + h) - L(rho0, t0v - h)) / (2 * h)
    v = torch.from_numpy(np.random.default_rng(5).normal(size=(N, N, N))).to(dev) * rho0.double()
    rp, rm = (rho0.double() + h * v).float(), (rho0.double() - h * v).float()
    v_eff = (rp.double() - rm.double()) / (2 * h)
    fdd = (L(rp, t0v) - L(rm, t0v)) / (2 * h)
    adj = float((g_rho * v_eff).sum())
    # the plain FP64 forward solve on the same input, for comparison
    p64 = mg.Params(**{**prm.__dict__, "precision": mg.FP64})
    f64 = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    a = time.perf_counter()
    mg.solve_scalar(p64, 1.0, rho0, f64, tol, allow_unconverged=True)
    torch.cuda.synchronize()
    fp64_ms = (time.perf_counter() - a) * 1e3
    # the library calls alone (no loss, no torch glue): forward solve and adjoint solve
    pf = mg.Params(**{**prm.__dict__, "fR0_abs": 1e-5})
    fld = torch.full((N,) * 3, float("nan"), dtype=torch.float64, device=dev)
    g = torch.from_numpy(np.random.default_rng(6).normal(size=(N, N, N))).to(dev)
    raw = {}
    for rep in range(2):
        fld.fill_(float("nan"))
        torch.cuda.synchronize()
        a = time.perf_counter()
        st_f = mg.solve_scalar(pf, 1.0, rho0, fld, tol)
        torch.cuda.synchronize()
        b = time.perf_counter()
        mg.solve_adjoint(pf, 1.0, fld, rho0, g, tol=tol * 0.1)
        torch.cuda.synchronize()
        c = time.perf_counter()
        raw = {"solve_ms": round((b - a) * 1e3, 2), "adjoint_solve_ms": round((c - b) * 1e3, 2),
               "solve_cycles": st_f.cycles}
    return {"workload": "fR n=1 |fR0|=1e-5 512^3 box 512 lognormal sigma_g 1.5 seed 3; loss sum_b log P_F(k_b), "
                        "32 log bins; tol 1e-10",
            "forward_ms": round(f_ms, 2), "backward_ms": round(b_ms, 2), "plain_fp64_forward_ms": round(fp64_ms, 2),
            "library_calls": raw,
            "grad_logfR0": g_th, "fd_logfR0": fdt, "rel_err_logfR0": abs(g_th - fdt) / abs(fdt),
            "grad_dir": adj, "fd_dir": fdd, "rel_err_density_dir": abs(adj - fdd) / abs(fdd)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args) -> None:
    import torch
    from paper_2110_00328_gb300 import binding as mg
    from paper_2110_00328_gb300 import build, inputs

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    mg.load()

    prec = mg.FP64 if args.precision == "fp64" else mg.MIXED
    prm = headline_params(mg, precision=prec, inner_cycles=args.inner_cycles, sweep_chunk=args.chunk, nu1=args.nu1,
                          nu2=args.nu2, coarse_sweeps=args.coarse_sweeps, tail_cells=args.tail_cells,
                          cycle="VFW".index(args.cycle))
    pos_h = inputs.zeldovich_positions(N_MESH, seed=1 + rank, sigma=SIGMA)
    npart = pos_h.shape[0]
    pos = torch.from_numpy(pos_h).to(dev)
    rho = torch.empty((N_MESH,) * 3, dtype=torch.float32, device=dev)
    field = torch.empty((N_MESH,) * 3, dtype=torch.float64, device=dev)
    force = torch.empty((npart, 3), dtype=torch.float32, device=dev)
    nan1 = torch.tensor([float("nan")], dtype=torch.float64).pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2
    stream = torch.cuda.current_stream()

    def step(stats_out):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        mg.deposit_cic(pos, N_MESH, rho)
        ev[1].record(stream)
        field.view(-1)[:1].copy_(nan1, non_blocking=True)  # start from the background field
        st = mg.solve_scalar(prm, 1.0, rho, field, TOL)
        ev[2].record(stream)
        mg.gather_force(prm, 1.0, field, pos, 1.0, force)
        ev[3].record(stream)
        stats_out.append((st, ev))

    warm = []
    for _ in range(args.warmup):
        step(warm)
        flush.zero_()
    torch.cuda.synchronize()
    barrier(world)

    clocks = ClockSampler(local) if rank == 0 else None
    time.sleep(0.4 if rank == 0 else 0.0)
    mg.profile_start()
    n0 = mg.launch_count()
    recs = []
    torch.cuda.synchronize()
    barrier(world)
    for _ in range(args.steps):
        step(recs)
        torch.cuda.synchronize()
        flush.zero_()  # L2 flush between steps, outside the step's events
    torch.cuda.synchronize()
    launches = mg.launch_count() - n0
    prof = mg.profile_stop()
    clk = clocks.stop() if clocks else None

    dep = sum(e[0].elapsed_time(e[1]) for _, e in recs)
    sol = sum(e[1].elapsed_time(e[2]) for _, e in recs)
    gat = sum(e[2].elapsed_time(e[3]) for _, e in recs)
    total_ms = dep + sol + gat
    total_ms = reduce_max(total_ms, world, dev)
    cycles = [st.cycles for st, _ in recs]
    ups_rank = sum(c * updates_per_cycle(N_MESH, prm.nu1, prm.nu2, prm.coarse_sweeps, prm.cycle) for c in cycles)
    value = job_rate(ups_rank, world, total_ms)

    # End to end through the public API with the particles in pinned host memory:
    # (a) the host-I/O entry points (copies in chunks overlapped with the deposit
    #     and the gather); (b) one explicit copy each way around the device calls.
    pos_host = torch.from_numpy(pos_h).pin_memory()
    force_host = torch.empty((npart, 3), dtype=torch.float32).pin_memory()

    def e2e_run(zero_copy):
        times = []
        for it in range(1 + max(1, args.steps)):  # one untimed warm-up step (host-side state, page mappings)
            torch.cuda.synchronize()
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if zero_copy:
                mg.deposit_cic_host(pos_host, pos, N_MESH, rho)
            else:
                pos.copy_(pos_host, non_blocking=True)
                mg.deposit_cic(pos, N_MESH, rho)
            field.view(-1)[:1].copy_(nan1, non_blocking=True)
            st_ = mg.solve_scalar(prm, 1.0, rho, field, TOL)
            if zero_copy:
                mg.gather_force_host(prm, 1.0, field, pos, force, force_host, 1.0)
            else:
                mg.gather_force(prm, 1.0, field, pos, 1.0, force)
                force_host.copy_(force, non_blocking=True)
            torch.cuda.synchronize()
            if it > 0:
                times.append((time.perf_counter() - t0) * 1e3)
        return times, st_

    e2e_ms, st = e2e_run(True)
    e2e_total = reduce_max(sum(e2e_ms), world, dev)
    e2e_value = job_rate(st.cycles * updates_per_cycle(N_MESH, prm.nu1, prm.nu2, prm.coarse_sweeps, prm.cycle) *
                         len(e2e_ms), world, e2e_total)
    copy_ms, st_c = e2e_run(False)
    copy_total = reduce_max(sum(copy_ms), world, dev)
    copy_value = job_rate(st_c.cycles * updates_per_cycle(N_MESH, prm.nu1, prm.nu2, prm.coarse_sweeps, prm.cycle) *
                          len(copy_ms), world, copy_total)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    # Roofline of the dominant kernel, the fine-level smoother k_smooth32s, per
    # red-black sweep (its two colour launches): algorithmic 12 B/cell (read u
    # and rho, write u: the FP32 field and density once each), time per sweep
    # from the library's event profile.  The correction form also reads the
    # fixed base field (16 B/cell); that figure is reported beside it.
    roof = None
    d = prof.get("smooth32_fine")
    sweeps = sum(cycles) * (prm.nu1 + prm.nu2)
    if d and d["ms"] > 0 and sweeps > 0:
        per_sweep_s = d["ms"] / sweeps * 1e-3
        alg = 12.0 * N_MESH ** 3
        achieved = alg / per_sweep_s / 1e9
        impl = 16.0 * N_MESH ** 3
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": smoother_traffic_per_sweep(),
                "kernel": "k_smooth32s (split fine level, one red-black sweep = 2 launches)",
                "peak_source": peak_kind, "algorithmic_bytes_per_sweep": alg,
                "ms_per_sweep": round(per_sweep_s * 1e3, 4),
                "correction_form_bytes_per_sweep": impl,
                "correction_form_frac": round(impl / per_sweep_s / 1e9 / peak, 4)}
    # Whole-solve roofline: per V(nu1,nu2) cycle b (3 nu + 4.5) 8/7 bytes per fine
    # cell with b = 4 (nu sweeps at 3b, residual-restriction and prolongation at
    # 2.25b each, levels adding 1/7), plus 36 B/cell per outer FP64 defect step
    # (residual: field 8 + density 4 + correction source 4; update: field 16 + e 4).
    nu = prm.nu1 + prm.nu2
    outer = recs[-1][0].outer
    solve_bytes = (cycles[-1] * 4.0 * (3 * nu + 4.5) * 8.0 / 7.0 + outer * 36.0) * N_MESH ** 3
    t_solve = sol / args.steps
    solve_roof = {"algorithmic_bytes": solve_bytes, "cycles": cycles[-1], "outer_steps": outer,
                  "bound_ms": round(solve_bytes / (peak * 1e9) * 1e3, 4), "time_to_tol_ms": round(t_solve, 4),
                  "frac": round(solve_bytes / (peak * 1e9) * 1e3 / t_solve, 4), "peak": peak,
                  "formula": "cycles x 4 (3 nu + 4.5) 8/7 + outer x 36 bytes per fine cell"}
    # the plain FP64 GPU multigrid on the same density, same schedule, same tolerance
    p64 = headline_params(mg, precision=mg.FP64, nu1=prm.nu1, nu2=prm.nu2, coarse_sweeps=prm.coarse_sweeps)
    f64 = torch.empty_like(field)
    t64 = []
    for _ in range(2):
        f64.fill_(float("nan"))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = mg.solve_scalar(p64, 1.0, rho, f64, TOL)
        e1.record(stream)
        torch.cuda.synchronize()
        t64.append(e0.elapsed_time(e1))
    fp64_gpu = {"time_to_tol_ms": round(min(t64), 3), "cycles": st64.cycles, "resid": st64.resid,
                "mixed_speedup": round(min(t64) / t_solve, 2),
                "field_relL2_mixed_vs_fp64": float(torch.linalg.vector_norm(field - f64) /
                                                   torch.linalg.vector_norm(f64))}
    timed_total = sum(v["ms"] for v in prof.values())
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "share_of_step": round(v["ms"] / max(total_ms, 1e-9), 4),
                   "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["bytes"] else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == mg.MIXED else "f64",
        "data": "synthetic",
        "config": {**workload_config(), "particles": npart, "precision": args.precision, "inner_cycles": args.inner_cycles, "sweep_chunk": args.chunk,
                   "nu1": prm.nu1, "nu2": prm.nu2, "coarse_sweeps": prm.coarse_sweeps, "tail_cells": prm.tail_cells, "cycle": args.cycle,
                   "levels": level_sizes(N_MESH),
                   "l2": "512 MB written between timed steps; positions (201 MB) exceed L2",
                   "parallelism": f"independent realisation per GPU x{world}"},
        "time_to_tol_ms": round(sol / args.steps, 3), "deposit_ms": round(dep / args.steps, 3),
        "gather_ms": round(gat / args.steps, 3), "cycles": cycles, "outer_steps": recs[-1][0].outer,
        "final_resid": recs[-1][0].resid, "resid_per_outer_step": recs[-1][0].hist, "solved_Mcells_per_s": round(N_MESH ** 3 * args.steps * world / (sol * 1e-3) / 1e6, 1),
        "roofline": roof, "solve_roofline": solve_roof, "fp64_gpu": fp64_gpu, "kernels": kernels, "timed_kernel_ms": round(timed_total, 3),
        "gpu_launches": int(launches),
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT, "h2d_bytes_per_step": int(pos_host.numel() * 4),
                "d2h_bytes_per_step": int(force_host.numel() * 4), "ms_per_step": round(e2e_total / len(e2e_ms), 3),
                "host_io": "mgglam_deposit_cic_host / mgglam_gather_force_host: copies overlapped with the kernels",
                "explicit_copies": {"value": round(copy_value, 1), "ms_per_step": round(copy_total / len(copy_ms), 3),
                                    "h2d_bytes_per_step": int(pos_host.numel() * 4),
                                    "d2h_bytes_per_step": int(force_host.numel() * 4)}},
        "clocks": clk,
    }
    extras = {"all": ("fmg", "batch", "adjoint", "models", "pm"), "none": ()}.get(args.extras, (args.extras,))
    if args.no_extras:
        extras = ()
    if "fmg" in extras:
        line["fmg"] = run_fmg_extra(mg, torch, rho, field, stream)
    if "batch" in extras:
        line["batch"] = run_batch_extra(mg, torch, dev)
    if "adjoint" in extras:
        line["adjoint"] = run_adjoint_extra(mg, torch, dev)
    if "models" in extras:
        line["models"] = run_models_extra(mg, torch, dev)
    if "pm" in extras:
        line["pm"] = run_pm_extra(mg, torch, dev)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_oracle_baseline(pos_h)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--inner-cycles", type=int, default=0, help="0 = adaptive")
    ap.add_argument("--chunk", type=int, default=0, help="planes per CTA of the fused sweep (0 = library default)")
    ap.add_argument("--nu1", type=int, default=2, help="pre-smoothing sweeps")
    ap.add_argument("--nu2", type=int, default=1, help="post-smoothing sweeps (2+1 gives the shortest time to 1e-8 here)")
    ap.add_argument("--coarse-sweeps", type=int, default=4,
                    help="red-black sweeps on the coarsest level (4 reach the same cycle count and residual as 16 here)")
    ap.add_argument("--tail-cells", type=int, default=0, help="largest level run by the one-block tail (0 = default)")
    ap.add_argument("--cycle", choices=["V", "F", "W"], default="V", help="multigrid cycle")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", choices=["all", "none", "fmg", "batch", "adjoint", "models", "pm"], default="all",
                    help="extra measurements after the main step: the 48-solve batch, the 512^3 adjoint, "
                         "the symmetron and CQ solves at 256^3")
    ap.add_argument("--no-extras", action="store_true", help="same as --extras none")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
