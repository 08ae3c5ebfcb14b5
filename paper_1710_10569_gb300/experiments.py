"""The paper's Rayleigh-Benard experiments (Sec. 3.3) run on the GPU path, many instances per batch.

* table1: Nusselt numbers of Table 1 (60 x 30, Pr = 0.71, Ma = 0.3).
* critical_rayleigh: growth rate of the disturbance for Ra near onset and the least-squares zero of
  the growth rate (the paper measures V_max over time at Ra = 1702..1710 and finds 1706.82 against
  1707.76 from linear stability theory).
* ma_sweep: steps to convergence and Nu over a range of Mach numbers (Nu changes by ~0.1% over the
  range; steps scale with 1/Ma).
* stability: a long run at high Ra (the paper reports stability at Ra = 1e9 with 220 vertical nodes).
"""
from __future__ import annotations

import math

import numpy as np

from . import clb
from . import workloads as W

TABLE1_RA = (2000, 2500, 3000, 5000, 10000, 20000, 30000, 50000)


def table1(storage=W.STORAGE_F64, steps: int = 200000, ras=TABLE1_RA, seed_T: float = 0.0, seed: int = 0):
    """Nu after `steps` steps for each Ra of Table 1, all instances in one batch. seed_T > 0 adds a
    seeded uniform temperature disturbance of that amplitude to the paper's initial state (reduced
    precision storage cannot grow the instability from disturbances below its resolution)."""
    probs = [W.rayleigh_benard_table1(float(ra), storage=storage) for ra in ras]
    if seed_T > 0:
        rng = np.random.default_rng(seed)
        for p in probs:
            p.T = p.T + rng.uniform(-seed_T, seed_T, p.T.shape)
    b = clb.Batch(probs)
    b.step(steps)
    nu, er = b.diagnostics()
    b.close()
    return {int(ra): float(n) for ra, n in zip(ras, nu)}


def roll_amplitude(uy):
    """Amplitude of the convection roll: the x-Fourier component of u_y at wavenumber 2 pi / nx
    (mean over rows). The x-uniform odd-even mode of u_y that the D2Q5 step can carry has no x
    structure and does not enter it."""
    ny, nx = uy.shape
    ph = np.exp(-2j * math.pi * np.arange(nx) / nx)
    return float(abs(np.mean(uy @ ph)) * 2 / nx)


def roll_series(ras, storage=W.STORAGE_F64, steps: int = 40000, every: int = 1000, Ma: float = 0.3,
                nx: int = 60, ny: int = 30):
    """Roll amplitude every `every` steps for each Ra (one batch)."""
    probs = [W.rayleigh_benard_table1(float(ra), Ma=Ma, nx=nx, ny=ny, storage=storage) for ra in ras]
    b = clb.Batch(probs)
    t, series = [], [[] for _ in ras]
    done = 0
    while done < steps:
        b.step(every)
        done += every
        t.append(done)
        for k in range(len(ras)):
            series[k].append(roll_amplitude(b.fields(k)[2]))
    b.close()
    return np.array(t), np.array(series)


def critical_rayleigh(ras=(1702, 1704, 1706, 1708, 1710), storage=W.STORAGE_F64, steps: int = 40000,
                      every: int = 1000, fit_from: int = 10000):
    """Growth rate sigma(Ra) of ln(roll amplitude) over [fit_from, steps] (least squares), and the Ra
    where the least-squares line through (Ra, sigma) crosses zero (Sec. 3.3)."""
    t, s = roll_series(ras, storage, steps, every)
    sel = t >= fit_from
    rates = []
    for k in range(len(ras)):
        y = np.log(s[k][sel])
        rates.append(float(np.polyfit(t[sel], y, 1)[0]))
    slope, icpt = np.polyfit(np.array(ras, dtype=float), np.array(rates), 1)
    return {"ra": list(ras), "growth_rate": rates, "ra_c": float(-icpt / slope)}


def ma_sweep(Ra: float, mas=(0.1, 0.15, 0.2, 0.25, 0.3), storage=W.STORAGE_F64, tol: float = 1e-7,
             check: int = 1000, max_steps: int = 600000):
    """For each Ma: the step count at which Nu changes by less than `tol` (relative) between checks
    `check` steps apart, and that Nu (batched; instances stop counting when they converge)."""
    probs = [W.rayleigh_benard_table1(Ra, Ma=m, storage=storage) for m in mas]
    b = clb.Batch(probs)
    prev = np.full(len(mas), np.nan)
    steps = np.zeros(len(mas), dtype=np.int64)
    nus = np.zeros(len(mas))
    done = 0
    active = np.ones(len(mas), dtype=bool)
    while active.any() and done < max_steps:
        b.step(check)
        done += check
        nu, _ = b.diagnostics()
        for k in range(len(mas)):
            if active[k]:
                if nu[k] > 1.01 and abs(nu[k] - prev[k]) < tol * nu[k]:
                    active[k] = False
                    steps[k] = done
                    nus[k] = nu[k]
                prev[k] = nu[k]
    for k in range(len(mas)):
        if active[k]:
            steps[k] = done
            nus[k] = prev[k]
    b.close()
    return {"ma": list(mas), "steps": steps.tolist(), "nu": nus.tolist(),
            "nu_rel_change": float((nus.max() - nus.min()) / nus.min())}


def stability(Ra: float = 1e9, ny: int = 220, aspect: int = 2, Pr: float = 0.71, Ma: float = 0.3,
              steps: int = 200000, storage=W.STORAGE_F32, seed: int = 0):
    """A long Rayleigh-Benard run at high Ra: returns whether the fields stayed finite, the final Nu
    and the maximum speed over the run's checkpoints (relative to u_c)."""
    u_c = Ma * W.CS
    prob = W.rayleigh_benard(aspect * ny, ny, Ra=Ra, Pr=Pr, u_c=u_c, perturb=1e-3, seed=seed,
                             storage=storage)
    lat = clb.Lattice.from_problem(prob)
    finite = True
    umax = 0.0
    nu = float("nan")
    done = 0
    chunk = 10000
    try:
        while done < steps:
            lat.step(chunk)
            done += chunk
            nu = lat.nusselt(1)
            _, ux, uy, _ = lat.fields()
            umax = max(umax, float(np.max(np.hypot(ux, uy))) / u_c)
    except clb.CLBError as e:
        if e.status != clb.CLB_ENAN:
            raise
        finite = False
    lat.close()
    return {"Ra": Ra, "ny": ny, "nx": aspect * ny, "steps": done, "finite": finite, "nu": nu,
            "max_speed_over_uc": umax, "nu_visc": prob.params["nu"]}


def normal_plate_convergence(Ls=(30, 60, 90, 120, 150), Re=(10.0, 20.0, 30.0), Pr: float = 0.71,
                             storage=W.STORAGE_F64, tol: float = 1e-11, max_steps: int = 1500000,
                             wet: bool = False):
    """Sec. 3.2: steady profiles of the normal-plate channel for every (Re, L) in one batch, their
    relative errors E_u and E_T against the analytic profiles, and the least-squares slopes of
    log E against log(1/L) per Re (the paper finds slopes of about 2)."""
    probs = [W.normal_plate_channel(L=L, Re=re, Pr=Pr, storage=storage, wet=wet) for re in Re for L in Ls]
    b = clb.Batch(probs)
    steps, er, status = b.run(tol, max_steps, 1000)
    out = {"Re": list(Re), "L": list(Ls), "E_u": {}, "E_T": {}, "slope_u": {}, "slope_T": {},
           "steps": steps.tolist()}
    k = 0
    for re in Re:
        eu, et = [], []
        for L in Ls:
            prob = probs[k]
            _, ux, uy, T = b.fields(k)
            ua, Ta = W.normal_plate_analytic(prob)
            eu.append(float(np.sqrt(np.sum((ux[:, 0] - ua) ** 2) / np.sum(ua ** 2))))
            et.append(float(np.sqrt(np.sum((T[:, 0] - Ta) ** 2) / np.sum(Ta ** 2))))
            k += 1
        out["E_u"][str(re)] = eu
        out["E_T"][str(re)] = et
        x = np.log(1.0 / np.array(Ls, dtype=float))
        out["slope_u"][str(re)] = float(np.polyfit(x, np.log(eu), 1)[0])
        out["slope_T"][str(re)] = float(np.polyfit(x, np.log(et), 1)[0])
    b.close()
    return out
