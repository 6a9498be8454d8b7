"""Learned surrogate of the Kapitza-Dirac solver (the batched-form runs of Sec. II.D).

Maps the run parameters (beam waist, peak field a0, envelope length, incident transverse
momentum p_x0, initial x-spin) to the run's final momentum-space read-outs: the
population of the incoming peak, of the two-photon Bragg peak, and the spin-resolved
Bragg populations (same spin and flipped spin, Sec. III.B).  Training data come from the
batched solver (``kd.Batch``), training and inference run in the library's own MLP
kernels (``kd.MLP``); the solver stays the fallback outside the trained parameter box and
the reference for the surrogate's error.

Targets are log10 of the four populations (they span many decades); inputs and targets
are standardised with the training set's mean and spread.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import kd
from . import workloads as W

WIDTHS = [5, 256, 256, 256, 4]
FLOOR = 1e-14          # added before log10 of a population
RANGES = {             # parameter box of the draws (also the surrogate's domain)
    "w0_lambda": (5.0, 20.0),
    "log10_a0": (math.log10(1e-2), math.log10(0.4)),
    "env_steps": (100.0, 2000.0),
    "px0_hk": (-1.2, -0.8),
}


def draw_params(n: int, seed: int = 1) -> np.ndarray:
    """n seeded parameter rows (w0 [lambda], log10 a0, envelope [steps], p_x0 [hbar k_L], spin)."""
    rng = np.random.default_rng(seed)
    cols = [rng.uniform(*RANGES[k], n) for k in ("w0_lambda", "log10_a0", "env_steps", "px0_hk")]
    cols.append(rng.choice([-1.0, 1.0], n))
    return np.stack(cols, 1)


def workload(row, units: W.Units = W.ATOMIC, grid=(256, 128), nsteps: int = 2000,
             env_scale: float = 1.0) -> W.Workload:
    """The solver run of one parameter row (FP32, Gaussian beam with its longitudinal part,
    co-moving box, box (nx/16) x (ny/16) wavelengths)."""
    w0_l, la0, env_steps, px0, spin = [float(v) for v in row]
    k, lam = W.laser(units)
    dt = W.dt_of(units)
    nx, ny = grid
    Lx, Ly = nx / 16 * lam, ny / 16 * lam
    g = W.Grid(nx, ny, -Lx / 2, Lx / 2, -Ly / 2, Ly / 2)
    f = W.Field(kind=W.GAUSS, longitudinal=1, a0=10.0 ** la0, k_L=k, epsilon=1.0 / (k * w0_l * lam),
                env_T=env_steps * env_scale * dt, p_shift_x=0.0, p_shift_y=units.mc,
                box_vy=units.c / math.sqrt(2.0))
    p = W.Packet(px0 * units.hbar * k, units.mc, 0.0, 0.0, units.hbar * k * 16 / min(nx, ny),
                 int(spin), 0)
    return W.Workload("surrogate run", units, g, f, p, dt, nsteps, obs_every=0, precision=W.FP32)


def targets_from_obs(o: dict, spin: float) -> list:
    same, flip = (o["cp_diff"], o["cm_diff"]) if spin > 0 else (o["cm_diff"], o["cp_diff"])
    return [math.log10(max(o["pop_in"], 0.0) + FLOOR), math.log10(max(o["pop_diff"], 0.0) + FLOOR),
            math.log10(max(same, 0.0) + FLOOR), math.log10(max(flip, 0.0) + FLOOR)]


def solve(rows, batch: int = 256, stream=None, **wkw):
    """Runs the solver for every parameter row (batched), returns (targets [n, 4], seconds)."""
    rows = np.asarray(rows, np.float64)
    out = np.zeros((len(rows), 4))
    t0 = time.perf_counter()
    for s0 in range(0, len(rows), batch):
        chunk = rows[s0:s0 + batch]
        wls = [workload(r, **wkw) for r in chunk]
        sims = [kd.Sim.from_workload(w, stream=stream) for w in wls]
        for s, w in zip(sims, wls):
            s.init_packet(w.packet)
            s.autotune(w.dt)      # launch variants of this grid (timed once per process)
        with kd.Batch(sims, stream=stream) as b:
            b.step([w.dt for w in wls], wls[0].nsteps)
        for i, (s, r) in enumerate(zip(sims, chunk)):
            out[s0 + i] = targets_from_obs(s.observe(), r[4])
            s.close()
    return out, time.perf_counter() - t0


@dataclass
class Scaler:
    mean: np.ndarray
    std: np.ndarray

    @classmethod
    def fit(cls, a):
        return cls(a.mean(0), np.maximum(a.std(0), 1e-6))

    def fwd(self, a):
        return ((a - self.mean) / self.std).astype(np.float32)

    def inv(self, a):
        return a * self.std + self.mean


def he_init(widths, seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, from a seeded numpy generator."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(widths) - 1):
        fi, fo = widths[l], widths[l + 1]
        lim = math.sqrt(6.0 / fi)
        parts += [rng.uniform(-lim, lim, fo * fi), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    """MLP surrogate with the solver as fallback outside the trained parameter box."""

    def __init__(self, seed: int = 0, widths=WIDTHS, precision: int = kd.KD_MLP_FP32):
        """precision: kd.KD_MLP_FP32 (CUDA-core GEMMs) or kd.KD_MLP_BF16 (tensor cores)."""
        self.widths = list(widths)
        self.net = kd.MLP(self.widths)
        self.net.set_precision(precision)
        self.net.set_params(he_init(self.widths, seed))
        self.xs = self.ys = None

    def fit(self, X, Y, steps: int = 3000, batch: int = 256, lr: float = 1e-3, seed: int = 0):
        """Adam on minibatches drawn with a seeded generator; cosine-decayed step size.
        Returns the wall time in seconds."""
        import torch
        self.xs, self.ys = Scaler.fit(X), Scaler.fit(Y)
        xn = torch.from_numpy(self.xs.fwd(X)).cuda()
        yn = torch.from_numpy(self.ys.fwd(Y)).cuda()
        n = len(X)
        rng = np.random.default_rng(seed)
        # every step's minibatch indices, drawn up front and copied once; the library's
        # gather kernel selects the rows on the device
        idx = torch.from_numpy(rng.integers(0, n, (steps, batch)).astype(np.int32)).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(steps):
            lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / steps))
            self.net.train_step_gather(xn.data_ptr(), yn.data_ptr(), n, idx[it].data_ptr(), batch, lr_t,
                                       stream=stream)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def predict(self, X) -> np.ndarray:
        return self.ys.inv(self.net.forward(self.xs.fwd(np.asarray(X, np.float64))))

    @staticmethod
    def in_domain(X) -> np.ndarray:
        X = np.asarray(X, np.float64)
        ok = np.ones(len(X), bool)
        for j, k in enumerate(("w0_lambda", "log10_a0", "env_steps", "px0_hk")):
            lo, hi = RANGES[k]
            ok &= (X[:, j] >= lo) & (X[:, j] <= hi)
        return ok & np.isin(X[:, 4], [-1.0, 1.0])

    def predict_or_solve(self, X, **wkw):
        """Surrogate inside the trained box, the solver outside it; returns (targets, used_solver)."""
        X = np.asarray(X, np.float64)
        ok = self.in_domain(X)
        out = np.zeros((len(X), 4))
        if ok.any():
            out[ok] = self.predict(X[ok])
        if (~ok).any():
            out[~ok] = solve(X[~ok], **wkw)[0]
        return out, ~ok


TARGET_NAMES = ["log10_P_in", "log10_P_bragg", "log10_P_bragg_same_spin", "log10_P_bragg_flip"]
PARAM_NAMES = ["w0_lambda", "log10_a0", "env_steps", "px0_hk", "spin"]


def heldout_error(pred, truth) -> dict:
    """Errors in log10 space per target (RMS and max |error|, decades)."""
    d = np.asarray(pred) - np.asarray(truth)
    return {n: {"rms": float(np.sqrt(np.mean(d[:, j] ** 2))), "max": float(np.max(np.abs(d[:, j])))}
            for j, n in enumerate(TARGET_NAMES)}


def worst_cases(pred, truth, params, k: int = 3) -> dict:
    """Per target, the k held-out rows of largest |error|: parameters, truth and prediction
    (log10), and the row's other targets (to see where in the physics the error sits)."""
    pred, truth, params = np.asarray(pred), np.asarray(truth), np.asarray(params)
    out = {}
    for j, n in enumerate(TARGET_NAMES):
        idx = np.argsort(-np.abs(pred[:, j] - truth[:, j]))[:k]
        out[n] = [{"params": dict(zip(PARAM_NAMES, map(float, params[i]))),
                   "truth": [float(v) for v in truth[i]], "pred": [float(v) for v in pred[i]]}
                  for i in idx]
    return out
