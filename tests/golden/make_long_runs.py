"""Writes the oracle's full-length records of the benchmark workloads (calls only oracle/):

    python tests/golden/make_long_runs.py c2    # 1024x512 Gaussian beam, 200 and 2000 steps
    python tests/golden/make_long_runs.py c3    # 2048x1024 grid, 200 and 2000 steps

For each step count the record holds the oracle's read-outs (default observation spec)
and the spinor at 256 points: the 128 of largest |psi| (where the packet is) and 128
drawn with a seeded generator, with max |psi| over the whole grid for relative errors.
Single-threaded FP64; about 1 s (c2) and 5 s (c3) per Strang step.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2307_01571_gb300 import workloads as W  # noqa: E402

CHECKPOINTS = (200, 2000)


def sample(psi, seed=0, top=128, rand=128):
    mag = np.sum(np.abs(psi) ** 2, axis=2).ravel()
    big = np.argsort(mag)[::-1][:top]
    rng = np.random.default_rng(seed)
    others = rng.choice(np.setdiff1d(np.arange(mag.size), big), rand, replace=False)
    idx = np.concatenate([big, np.sort(others)])
    ny, nx = psi.shape[:2]
    pts = [(int(i // nx), int(i % nx)) for i in idx]
    vals = [[[float(psi[y, x, c].real), float(psi[y, x, c].imag)] for c in range(4)] for y, x in pts]
    return pts, vals


def main(name):
    wl = W.c2(precision=W.FP64) if name == "c2" else W.c3(precision=W.FP64)
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    spec = W.default_obs_spec(u, f, pk)
    psi = oracle.init_packet(u, g, f, pk)
    done, out = 0, {"workload": wl.name, "grid": [g.nx, g.ny], "dt": wl.dt, "records": []}
    path = os.path.join(HERE, f"{name}_long_oracle.json")
    for n in CHECKPOINTS:
        t0 = time.perf_counter()
        psi = oracle.step(u, g, f, psi, done * wl.dt, wl.dt, n - done)
        done = n
        pts, vals = sample(psi)
        out["records"].append({
            "steps": n, "max_abs_psi": float(np.max(np.abs(psi))),
            "obs": oracle.observe(u, g, f, spec, psi, n * wl.dt),
            "points_yx": pts, "psi": vals, "oracle_seconds": time.perf_counter() - t0})
        with open(path, "w") as fh:
            json.dump(out, fh)
        print(name, n, "steps written", flush=True)


if __name__ == "__main__":
    main(sys.argv[1])
