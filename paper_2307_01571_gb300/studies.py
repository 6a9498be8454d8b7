"""The paper's parameter studies of Sec. IV as batched runs of this library.

``e3``: spin-flip scaling (Sec. IV, sec:scaling_effects): the showcase setup of Sec. II.D
(2048 x 128 grid over 80 x 40 wavelengths, co-moving box, A0 = 0.1 m c / q, packet at
(-hbar k_L, m c) with spin +x, run time 280 lambda sqrt 2 / c) for
epsilon in {0.01, 0.02, 0.05, 0.1} and hbar k_L in {0.05, 0.07, 0.1} m c.  The paper reports
that the flipped-spin population of the diffracted peak grows as (k_L / epsilon)^2.
``e4``: the longitudinal field component on and off (Sec. IV, sec:longitudinal_component)
at hbar k_L = 0.1 m c for the same four epsilon: the paper reports that the difference of
the spin populations with and without the longitudinal component grows as epsilon^2.

Read-outs are window sums (half width hbar k_L / 2) of |c^+|^2 and |c^-|^2 around the
diffracted peak p0 + 2 hbar k_L e_x, the populations the library's observation records
carry (cp_diff, cm_diff).  ``fit_slope`` fits the power law in log-log.  Everything runs on
the GPU through kd_batch_step; nothing here computes the method.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import showcase
from . import workloads as W

EPSILONS = (0.01, 0.02, 0.05, 0.1)
K_NAT = (0.05, 0.07, 0.1)


def run(units: W.Units = W.NATURAL, eps: float = 0.02, k_nat: float = 0.1, longitudinal: int = 1,
        nx: int = 2048, ny: int = 128, nsteps: int | None = None,
        precision: int = W.FP32) -> W.Workload:
    """The showcase setup with laser wave number k_nat m c / hbar, waist 1/(k_L epsilon) and
    the longitudinal component switched on or off."""
    k, lam = W.laser(units, k_nat)
    dt = W.dt_of(units)
    y0 = -140.0
    g = W.Grid(nx, ny, -40 * lam, 40 * lam, (y0 - 20) * lam, (y0 + 20) * lam)
    f = W.Field(kind=W.GAUSS, longitudinal=longitudinal, a0=0.1, k_L=k, epsilon=eps, env_T=0.0,
                p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
    lam_c = 2.0 * math.pi * units.hbar / units.mc
    p = W.Packet(-units.hbar * k, units.mc, 140.0 * lam_c, y0 * lam, units.hbar * k / 200.0, 1, 0)
    T = 280.0 * lam * math.sqrt(2.0) / units.c
    n = int(round(T / dt)) if nsteps is None else nsteps
    return W.Workload(f"study eps {eps:g} hbar k_L {k_nat:g} mc long {longitudinal}", units, g, f,
                      p, dt, n, obs_every=0, precision=precision,
                      extra={"eps": eps, "k_nat": k_nat, "longitudinal": longitudinal})


def e3(**kw) -> list:
    return [run(eps=e, k_nat=k, **kw) for e in EPSILONS for k in K_NAT]


def e4(**kw) -> list:
    return [run(eps=e, k_nat=0.1, longitudinal=lo, **kw) for e in EPSILONS for lo in (1, 0)]


def fit_slope(x, y) -> float:
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(x, float)), np.log(np.asarray(y, float))
    return float(np.polyfit(lx, ly, 1)[0])


def execute(kd, workloads: list, stream: int | None = None) -> list:
    """Runs the workloads to their end as one batch (members of equal step counts together)
    and returns per workload the diffracted-peak read-outs {cp_diff, cm_diff, norm}."""
    groups: dict = {}
    for i, wl in enumerate(workloads):
        groups.setdefault(wl.nsteps, []).append(i)
    out = [None] * len(workloads)
    for n, idx in groups.items():
        sims = [kd.Sim.from_workload(workloads[i], stream=stream) for i in idx]
        for s, i in zip(sims, idx):
            wl = workloads[i]
            s.init_packet(wl.packet)
            s.set_obs_spec(showcase.readout_spec(wl, 1.0))
        with kd.Batch(sims, stream=stream) as b:
            b.step([workloads[i].dt for i in idx], n)
        for s, i in zip(sims, idx):
            o = s.observe()
            out[i] = {"cp_diff": o["cp_diff"], "cm_diff": o["cm_diff"], "norm": o["norm"]}
            s.close()
    return out


def studies(kd, stream: int | None = None) -> dict:
    """E3 and E4 in full; returns the read-outs, the fitted slopes and the GPU time."""
    t0 = time.perf_counter()
    w3 = e3()
    r3 = execute(kd, w3, stream)
    w4 = [w for w in e4() if w.field.longitudinal == 0]
    r4 = execute(kd, w4, stream)
    secs = time.perf_counter() - t0
    x3 = [w.extra["k_nat"] / w.extra["eps"] for w in w3]
    e3_rows = [{"eps": w.extra["eps"], "k_nat": w.extra["k_nat"], "steps": w.nsteps, **r}
               for w, r in zip(w3, r3)]
    on = {w.extra["eps"]: r for w, r in zip(w3, r3) if w.extra["k_nat"] == 0.1}
    e4_rows = []
    for w, r in zip(w4, r4):
        e = w.extra["eps"]
        e4_rows.append({"eps": e, "cp_on": on[e]["cp_diff"], "cp_off": r["cp_diff"],
                        "cm_on": on[e]["cm_diff"], "cm_off": r["cm_diff"],
                        "d_cp": abs(on[e]["cp_diff"] - r["cp_diff"]),
                        "d_cm": abs(on[e]["cm_diff"] - r["cm_diff"])})
    return {
        "e3": e3_rows,
        "e3_slope_cm_vs_kL_over_eps": fit_slope(x3, [r["cm_diff"] for r in r3]),
        "e4": e4_rows,
        "e4_slope_dcm_vs_eps": fit_slope([r["eps"] for r in e4_rows], [r["d_cm"] for r in e4_rows]),
        "e4_slope_dcp_vs_eps": fit_slope([r["eps"] for r in e4_rows], [r["d_cp"] for r in e4_rows]),
        "paper": {"e3_slope": 2.0, "e4_slope": 2.0},
        "gpu_seconds": secs,
    }
