"""Parameter sets and seeded synthetic inputs for the Kapitza-Dirac split-operator step.

This module holds no arithmetic of the method: only unit systems, named parameter
sets shaped like the paper's simulations (Sec. II.D and Sec. IV of arXiv 2307.01571)
and seeded random generators.  It is the one module that both the CUDA path's
callers and the CPU oracle's callers use, so that both sides see identical inputs.

Field kinds: ``NONE`` (free particle), ``PLANE`` (plane-wave standing wave, the
epsilon -> 0 limit of the beams) and ``GAUSS`` (Gaussian-beam standing wave of
Eqs. Equation_of_Gaussian_beam / Phase_of_Gaussian_beam / Equation_of_vector_potential).
The amplitude is the dimensionless a0 = q A0 / (m c^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

NONE, PLANE, GAUSS = 0, 1, 2
FP64, FP32, FP32_TC, DW = 0, 1, 2, 3


@dataclass(frozen=True)
class Units:
    m: float = 1.0
    c: float = 137.035999
    hbar: float = 1.0
    q: float = -1.0

    @property
    def mc(self) -> float:
        return self.m * self.c

    @property
    def mc2(self) -> float:
        return self.m * self.c * self.c


ATOMIC = Units()
NATURAL = Units(1.0, 1.0, 1.0, -1.0)


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    x_min: float
    x_max: float
    y_min: float
    y_max: float


@dataclass(frozen=True)
class Field:
    kind: int = NONE
    longitudinal: int = 0
    a0: float = 0.0
    k_L: float = 1.0
    epsilon: float = 0.0
    env_T: float = 0.0
    phase0: float = 0.0
    p_shift_x: float = 0.0
    p_shift_y: float = 0.0
    box_vy: float = 0.0


@dataclass(frozen=True)
class Packet:
    p0x: float
    p0y: float
    r0x: float
    r0y: float
    sigma_p: float
    spin: int = 1
    basis: int = 0


@dataclass(frozen=True)
class ObsSpec:
    p_in_x: float
    p_in_y: float
    p_diff_x: float
    p_diff_y: float
    target_x: float
    target_y: float
    half_width: float
    basis: int = 0


@dataclass(frozen=True)
class Workload:
    name: str
    units: Units
    grid: Grid
    field: Field
    packet: Packet
    dt: float
    nsteps: int
    obs_every: int = 0
    precision: int = FP64
    extra: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.grid.nx * self.grid.ny

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def default_obs_spec(units: Units, field_: Field, packet: Packet) -> ObsSpec:
    """Windows around the incoming peak p0 and the two-photon Bragg peak p0 + 2 hbar k_L e_x
    (the diffracted beam appears two photon momenta to the right, Sec. III.B), half width
    hbar k_L / 2; single-cell read-out at the diffracted peak."""
    hk = units.hbar * field_.k_L
    return ObsSpec(packet.p0x, packet.p0y, packet.p0x + 2.0 * hk, packet.p0y,
                   packet.p0x + 2.0 * hk, packet.p0y, 0.5 * hk, packet.basis)


def laser(units: Units, k_nat: float = 0.1):
    """Laser wave number k_L = k_nat m c / hbar and wavelength."""
    k = k_nat * units.m * units.c / units.hbar
    return k, 2.0 * math.pi / k


def dt_of(units: Units, dt_nat: float = 0.05) -> float:
    """Time step in units of hbar / (m c^2) (the paper's 0.05, Sec. II.D)."""
    return dt_nat * units.hbar / units.mc2


def c1(units: Units = ATOMIC) -> Workload:
    """Plain FP64 plane-wave run: 128x128 periodic grid, 16 lambda square box, Bragg packet
    p0 = (-hbar k_L, m c), spin +x, a0 = 0.1, sin^2 envelope over 200 steps, 200 steps."""
    k, lam = laser(units)
    dt = dt_of(units)
    g = Grid(128, 128, -8 * lam, 8 * lam, -8 * lam, 8 * lam)
    f = Field(kind=PLANE, longitudinal=0, a0=0.1, k_L=k, epsilon=0.0, env_T=200 * dt,
              p_shift_x=0.0, p_shift_y=units.mc, box_vy=0.0)
    p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k / 8.0, 1, 0)
    return Workload("plane-wave standing wave 128x128 c128, 200 steps", units, g, f, p, dt, 200,
                    obs_every=100, precision=FP64)


def c2(units: Units = ATOMIC, w0_lambda: float = 10.0, longitudinal: int = 1,
       precision: int = FP64, nsteps: int = 2000) -> Workload:
    """Gaussian-beam standing wave with its longitudinal component on a 1024x512 grid,
    40 lambda x 40 lambda co-moving box (v = c/sqrt 2) centred on the beam, waist w0 in
    lambda, a0 = 0.1, packet p0 = (-hbar k_L, m c), sigma_p = hbar k_L / 20, 2000 steps,
    observables every 100 steps."""
    k, lam = laser(units)
    dt = dt_of(units)
    eps = 1.0 / (k * w0_lambda * lam)
    g = Grid(1024, 512, -20 * lam, 20 * lam, -20 * lam, 20 * lam)
    f = Field(kind=GAUSS, longitudinal=longitudinal, a0=0.1, k_L=k, epsilon=eps, env_T=0.0,
              p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
    p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k / 20.0, 1, 0)
    tag = {FP64: "c128", DW: "c128 as double-word FP32 pairs"}.get(precision, "c64")
    return Workload(f"Gaussian-beam standing wave 1024x512 {tag}, w0={w0_lambda:g} lambda, "
                    f"{nsteps} steps", units, g, f, p, dt, nsteps, obs_every=100,
                    precision=precision)


def c3(units: Units = ATOMIC, precision: int = FP32, nsteps: int = 2000) -> Workload:
    """2048x1024 grid over the paper's 80 lambda x-box and a 40 lambda co-moving y-box,
    epsilon = 0.02, otherwise as the 1024x512 case."""
    k, lam = laser(units)
    dt = dt_of(units)
    g = Grid(2048, 1024, -40 * lam, 40 * lam, -20 * lam, 20 * lam)
    f = Field(kind=GAUSS, longitudinal=1, a0=0.1, k_L=k, epsilon=0.02, env_T=0.0,
              p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
    p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k / 20.0, 1, 0)
    return Workload(f"Gaussian-beam standing wave 2048x1024, {nsteps} steps", units, g, f, p,
                    dt, nsteps, obs_every=100, precision=precision)


def hbm(units: Units = ATOMIC, precision: int = FP32, nsteps: int = 200) -> Workload:
    """A grid whose state does not fit in L2 (4096x2048: 256 MiB spinor in FP32), over a
    160 lambda x 80 lambda co-moving box, epsilon = 0.02, otherwise as the 1024x512 case."""
    k, lam = laser(units)
    dt = dt_of(units)
    g = Grid(4096, 2048, -80 * lam, 80 * lam, -40 * lam, 40 * lam)
    f = Field(kind=GAUSS, longitudinal=1, a0=0.1, k_L=k, epsilon=0.02, env_T=0.0,
              p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
    p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k / 20.0, 1, 0)
    return Workload(f"Gaussian-beam standing wave 4096x2048, {nsteps} steps", units, g, f, p,
                    dt, nsteps, obs_every=100, precision=precision)


def small(nx: int, ny: int, kind: int = GAUSS, units: Units = NATURAL, nsteps: int = 20,
          longitudinal: int = 1, a0: float = 0.1, box_vy: float | None = None,
          precision: int = FP64, env: bool = False) -> Workload:
    """A small grid with the same physics as the large cases, for oracle-sized parity runs.
    The box is nx/16 by ny/16 wavelengths (momentum cell hbar k_L / (n/16))."""
    k, lam = laser(units)
    dt = dt_of(units)
    Lx, Ly = nx / 16 * lam, ny / 16 * lam
    g = Grid(nx, ny, -Lx / 2, Lx / 2, -Ly / 2, Ly / 2)
    w0 = max(2.0 * lam, Ly / 4)
    eps = 1.0 / (k * w0) if kind == GAUSS else 0.0
    vy = units.c / math.sqrt(2.0) if box_vy is None else box_vy
    f = Field(kind=kind, longitudinal=longitudinal if kind == GAUSS else 0, a0=a0, k_L=k,
              epsilon=eps, env_T=(nsteps * dt if env else 0.0), phase0=0.3,
              p_shift_x=0.0, p_shift_y=units.mc, box_vy=vy)
    p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k * 16 / min(nx, ny) * 2, 1, 0)
    return Workload(f"small {nx}x{ny}", units, g, f, p, dt, nsteps, obs_every=0,
                    precision=precision)


def c4(units: Units = ATOMIC, n: int = 64, seed: int = 0, nsteps: int = 2000,
       precision: int = FP32) -> list:
    """Batched form: n independent Gaussian-beam runs with seeded parameters.  Grid per run
    uniform from {128x128, 256x128, 256x256, 512x256} over (nx/16) x (ny/16) wavelengths,
    waist U[5, 20] wavelengths, a0 log-uniform in [1e-2, 0.4], sin^2 envelope
    U[100, 2000] steps, spin +-1 along x, p0 = (-hbar k_L, m c), box moving at c/sqrt 2."""
    rng = np.random.default_rng(seed)
    k, lam = laser(units)
    dt = dt_of(units)
    shapes = [(128, 128), (256, 128), (256, 256), (512, 256)]
    out = []
    for i in range(n):
        nx, ny = shapes[int(rng.integers(0, len(shapes)))]
        w0 = float(rng.uniform(5.0, 20.0)) * lam
        a0 = float(np.exp(rng.uniform(np.log(1e-2), np.log(0.4))))
        env = float(rng.uniform(100.0, 2000.0)) * dt
        spin = int(rng.choice([1, -1]))
        Lx, Ly = nx / 16 * lam, ny / 16 * lam
        g = Grid(nx, ny, -Lx / 2, Lx / 2, -Ly / 2, Ly / 2)
        f = Field(kind=GAUSS, longitudinal=1, a0=a0, k_L=k, epsilon=1.0 / (k * w0), env_T=env,
                  p_shift_x=0.0, p_shift_y=units.mc, box_vy=units.c / math.sqrt(2.0))
        p = Packet(-units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k * 16 / min(nx, ny), spin, 0)
        out.append(Workload(f"batch member {i}: {nx}x{ny}", units, g, f, p, dt, nsteps,
                            obs_every=100, precision=precision,
                            extra={"w0_lambda": w0 / lam, "a0": a0, "env_steps": env / dt}))
    return out


def random_spinor(nx: int, ny: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian spinor, shape (ny, nx, 4), unit sum of |psi|^2."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((ny, nx, 4)) + 1j * rng.standard_normal((ny, nx, 4))
    return (a / np.sqrt(np.sum(np.abs(a) ** 2))).astype(np.complex128)
