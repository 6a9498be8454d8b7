"""Writes the oracle regression fixtures in this folder.  Calls only ``oracle`` (and the
parameter sets of ``workloads``); run it from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2307_01571_gb300 import workloads as W  # noqa: E402


def c1_obs():
    wl = W.c1()
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    spec = W.default_obs_spec(u, f, pk)
    psi = oracle.init_packet(u, g, f, pk)
    rec = {"workload": wl.name, "dt": wl.dt, "obs": []}
    t = 0.0
    for chunk in (100, 100):
        psi = oracle.step(u, g, f, psi, t, wl.dt, chunk)
        t += chunk * wl.dt
        o = oracle.observe(u, g, f, spec, psi, t)
        rec["obs"].append(o)
    return rec


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "c1_oracle_obs.json"), "w") as fh:
        json.dump(c1_obs(), fh, indent=1)
    print("wrote c1_oracle_obs.json")
