"""The paper's parameter studies of Sec. IV as batched runs of this library.

``e3``: spin-flip scaling (Sec. IV, sec:scaling_effects): the showcase setup of Sec. II.D
(2048 x 128 grid over 80 x 40 wavelengths, co-moving box, A0 = 0.1 m c / q, packet at
(-hbar k_L, m c) with spin +x, run time 280 lambda sqrt 2 / c) for
epsilon in {0.01, 0.02, 0.05, 0.1} and hbar k_L in {0.05, 0.07, 0.1} m c.  The paper reports
that the flipped-spin population of the diffracted peak grows as (k_L / epsilon)^2.
``e4``: the longitudinal field component on and off (Sec. IV, sec:longitudinal_component)
at hbar k_L = 0.1 m c for the same four epsilon: the paper reports that the difference of
the spin populations with and without the longitudinal component grows as epsilon^2.

Read-outs are the three forms the library's observation records carry around the
diffracted peak p0 + 2 hbar k_L e_x: window sums (half width hbar k_L / 2) of |c^+|^2 and
|c^-|^2 (populations: cp_diff, cm_diff), window maxima, and the value at the cell
(hbar k_L, m c) that the paper plots (cp_target, cm_target).  ``fit_slope`` fits the power law in log-log.  Everything runs on
the GPU through kd_batch_step; nothing here computes the method.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import showcase
from . import workloads as W

EPSILONS = (0.01, 0.02, 0.05, 0.1)
# read-outs per run: window sums (a population), window maxima and the value at the cell
# (hbar k_L, m c) of the diffracted peak (the paper's |c^-(hbar k_L, m c, T)|^2)
READOUTS = ("cp_diff", "cm_diff", "cp_max_diff", "cm_max_diff", "cp_target", "cm_target", "norm")
K_NAT = (0.05, 0.07, 0.1)


def run(units: W.Units = W.NATURAL, eps: float = 0.02, k_nat: float = 0.1, longitudinal: int = 1,
        nx: int = 2048, ny: int = 128, nsteps: int | None = None,
        precision: int = W.FP32, y0: float = -140.0) -> W.Workload:
    """The showcase setup with laser wave number k_nat m c / hbar, waist 1/(k_L epsilon) and
    the longitudinal component switched on or off; ``y0`` is the box's (and the packet's)
    initial centre in wavelengths (the setup's -140; 0 puts both at the focus)."""
    k, lam = W.laser(units, k_nat)
    dt = W.dt_of(units)
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
            out[i] = {k: o[k] for k in READOUTS}
            s.close()
    return out


def _slopes(rows, form):
    """Power-law exponents of one read-out form over the E3 grid: against k_L / eps over
    every run, against eps at each k_L and against k_L at each eps."""
    return {
        "vs_kL_over_eps": fit_slope([r["k_nat"] / r["eps"] for r in rows], [r[form] for r in rows]),
        "vs_eps": {k: fit_slope([r["eps"] for r in rows if r["k_nat"] == k],
                                [r[form] for r in rows if r["k_nat"] == k]) for k in K_NAT},
        "vs_kL": {e: fit_slope([r["k_nat"] for r in rows if r["eps"] == e],
                               [r[form] for r in rows if r["eps"] == e]) for e in EPSILONS},
    }


FORMS = ("cp_diff", "cm_diff", "cp_max_diff", "cm_max_diff", "cp_target", "cm_target")


def studies(kd, stream: int | None = None, e4_precision: int | None = W.DW) -> dict:
    """E3 and E4 in full; returns the read-outs, the fitted slopes and the GPU time.

    E4's differences (1e-6 ... 1e-5 of populations ~1e-2) are near the accumulated FP32
    rounding of a 5e5-step run, so E4 also runs on and off in ``e4_precision`` (default the
    double-word FP64-accurate form; None skips it) and its slopes are fitted on both."""
    t0 = time.perf_counter()
    w3 = e3()
    r3 = execute(kd, w3, stream)
    w4 = [w for w in e4() if w.field.longitudinal == 0]
    r4 = execute(kd, w4, stream)
    hp = {}
    if e4_precision is not None:
        wh = e4(precision=e4_precision)
        for w, r in zip(wh, execute(kd, wh, stream)):
            hp[(w.extra["eps"], w.extra["longitudinal"])] = r
    secs = time.perf_counter() - t0
    e3_rows = [{"eps": w.extra["eps"], "k_nat": w.extra["k_nat"], "steps": w.nsteps, **r}
               for w, r in zip(w3, r3)]
    on = {w.extra["eps"]: r for w, r in zip(w3, r3) if w.extra["k_nat"] == 0.1}
    off = {w.extra["eps"]: r for w, r in zip(w4, r4)}
    e4_rows = []
    for e in EPSILONS:
        row = {"eps": e}
        for f in FORMS:
            row[f"fp32_{f}_on"], row[f"fp32_{f}_off"] = on[e][f], off[e][f]
            row[f"fp32_d_{f}"] = abs(on[e][f] - off[e][f])
            if hp:
                a, b = hp[(e, 1)], hp[(e, 0)]
                row[f"hp_{f}_on"], row[f"hp_{f}_off"] = a[f], b[f]
                row[f"hp_d_{f}"] = abs(a[f] - b[f])
                row[f"fp32_err_{f}_on"] = abs(on[e][f] - a[f])
        e4_rows.append(row)
    e4_slopes = {}
    for f in FORMS:
        for tag in ("fp32", "hp") if hp else ("fp32",):
            e4_slopes[f"{tag}_d_{f}"] = fit_slope(EPSILONS, [r[f"{tag}_d_{f}"] for r in e4_rows])
    return {
        "e3": e3_rows,
        "e3_slopes": {f: _slopes(e3_rows, f) for f in FORMS},
        "e4": e4_rows,
        "e4_precision": e4_precision,
        "e4_slopes_vs_eps": e4_slopes,
        "paper": {"e3_slope_vs_eps": -2.0, "e3_slope_vs_kL": 2.0, "e4_slope_vs_eps": 2.0},
        "gpu_seconds": secs,
    }
