"""The paper's own simulations, as workloads of this library.

``e1``: the showcase run of Sec. II.D and Sec. III (2048 x 128 grid over 80 x 40 wavelengths,
epsilon = 0.02, hbar k_L = 0.1 m c, A0 = 0.1 m c / q, dt = 0.05 hbar/(m c^2), co-moving box
starting at y in [-160, -120] lambda, packet at (140 lambda_C, -140 lambda) with kinetic
momentum (-hbar k_L, m c) and sigma_p = hbar k_L / 200, spin +x, run time
280 lambda sqrt 2 / c), whose diffracted peak the paper reads out at (0.1, 1) m c.
``e5`` / ``e6``: the diffraction-regime runs of Tables I and II (2048 x 256, epsilon = 0.1,
A0 = 0.4 m c / q, p_x = -hbar k_L and p_x = 0).

The paper's printed populations depend on normalisation conventions it leaves open
(bispinor and momentum-space normalisation), so they are an order-of-magnitude reference
for these runs, not a parity target.
"""
from __future__ import annotations

import math

from . import workloads as W

PAPER_E1 = {"cp_at_0.1_1": 4.6e-5, "cm_at_0.1_1": 3.9e-3}   # Sec. III.B


def _run(units, nx, ny, eps, a0, px0_hk, y0_lambda=-140.0, x0=None, nsteps=None, precision=W.FP32,
         name="showcase"):
    k, lam = W.laser(units)
    dt = W.dt_of(units)
    g = W.Grid(nx, ny, -40 * lam, 40 * lam, (y0_lambda - 20) * lam, (y0_lambda + 20) * lam)
    f = W.Field(kind=W.GAUSS, longitudinal=1, a0=a0, k_L=k, epsilon=eps, env_T=0.0,
                p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
    lam_c = 2.0 * math.pi * units.hbar / units.mc
    p = W.Packet(px0_hk * units.hbar * k, units.mc, 140.0 * lam_c if x0 is None else x0,
                 y0_lambda * lam, units.hbar * k / 200.0, 1, 0)
    T = 280.0 * lam * math.sqrt(2.0) / units.c
    n = int(round(T / dt)) if nsteps is None else nsteps
    return W.Workload(name, units, g, f, p, dt, n, obs_every=0, precision=precision)


def e1(units: W.Units = W.NATURAL, nsteps=None, precision=W.FP32) -> W.Workload:
    return _run(units, 2048, 128, 0.02, 0.1, -1.0, nsteps=nsteps, precision=precision,
                name="paper showcase E1: 2048x128, eps 0.02, A0 0.1")


def e5(units: W.Units = W.NATURAL, nsteps=None, precision=W.FP32) -> W.Workload:
    return _run(units, 2048, 256, 0.1, 0.4, -1.0, nsteps=nsteps, precision=precision,
                name="paper Table I: 2048x256, eps 0.1, A0 0.4, p_x = -hbar k_L")


def e6(units: W.Units = W.NATURAL, nsteps=None, precision=W.FP32) -> W.Workload:
    return _run(units, 2048, 256, 0.1, 0.4, 0.0, x0=0.0, nsteps=nsteps, precision=precision,
                name="paper Table II: 2048x256, eps 0.1, A0 0.4, p_x = 0")


def readout_spec(wl: W.Workload, px_hk: float) -> W.ObsSpec:
    """Windows around p0 and p0 + 2 hbar k_L e_x; target cell at (px_hk hbar k_L, m c)."""
    u, f, pk = wl.units, wl.field, wl.packet
    hk = u.hbar * f.k_L
    return W.ObsSpec(pk.p0x, pk.p0y, pk.p0x + 2 * hk, pk.p0y, px_hk * hk, u.mc, 0.5 * hk, 0)
