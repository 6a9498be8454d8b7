"""Full-length parity: the benchmark workloads (1024x512 for 2000 Strang steps, 2048x1024
for 200 and 2000) run through kd_step in the bench's launch configuration (graph-captured
chunks, observations every 100 steps) and compared with the oracle's stored records
(tests/golden/*_long_oracle.json, written by tests/golden/make_long_runs.py, which calls
only the oracle) at 256 points: the 128 of largest |psi| and 128 seeded ones, errors
relative to the oracle's max |psi| over the grid.  Tolerances per form are the bars of
the short parity tests, except where a long run is stated to need more (below)."""
import json
import os

import numpy as np
import pytest

from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

# relative error bound over the runs per precision: the FP64 and FP32 bars (measured at 2000
# steps: 6e-13 and 3.3e-6); the double-word form (3) has FP64's bar; the precision form (2)
# is held to the FP32 bar and misses it: its tensor cores truncate in their FP32
# accumulation, so its norm decays by ~7e-7 per step and its error grows with it (measured
# 1.3e-4 after 200 steps, 1.4e-3 after 2000) -- an expected failure
TOL = {0: 1e-10, 1: 1e-4, 2: 1e-4, 3: 1e-10}
PRECS = [0, 1, pytest.param(2, marks=pytest.mark.xfail(
    strict=True, reason="tensor-core FP32 accumulation truncates: error 1.4e-3 after 2000 steps")), 3]


def records(name):
    path = os.path.join(HERE, "golden", f"{name}_long_oracle.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    with open(path) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def kd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


def run_and_compare(kd, wl, rec_set, prec):
    out = {}
    with kd.Sim.from_workload(wl.with_(precision=prec)) as sim:
        sim.init_packet(wl.packet)
        done = 0
        for rec in rec_set["records"]:
            n = rec["steps"]
            obs = sim.step(wl.dt, n - done, obs_every=100)
            done = n
            psi = sim.get_spinor()
            pts = np.array(rec["points_yx"])
            ref = np.array(rec["psi"])
            ref = ref[..., 0] + 1j * ref[..., 1]
            got = psi[pts[:, 0], pts[:, 1], :].astype(np.complex128)
            err = float(np.max(np.abs(got - ref)) / rec["max_abs_psi"])
            oerr = {k: abs(obs[-1][k] - v) / max(1.0, abs(v)) for k, v in rec["obs"].items() if k != "t"}
            out[n] = (err, max(oerr.values()))
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_1024x512_full_run(kd, prec):
    rs = records("c2")
    res = run_and_compare(kd, W.c2(), rs, prec)
    for n, (err, oerr) in res.items():
        assert err <= TOL[prec], (n, err)
        assert oerr <= TOL[prec], (n, oerr)


@pytest.mark.parametrize("prec", PRECS)
def test_2048x1024_full_run(kd, prec):
    rs = records("c3")
    res = run_and_compare(kd, W.c3(), rs, prec)
    for n, (err, oerr) in res.items():
        assert err <= TOL[prec], (n, err)
        assert oerr <= TOL[prec], (n, oerr)
