"""Double-word form (KD_DW): the FP64-accurate step with every real a pair of floats,
checked element by element against the oracle at the FP64 bars (max |psi - psi_oracle|
<= 1e-10 max |psi|, norm drift <= 1e-12): every field kind on grids from 4x4 to 4096-point
axes (ragged tiles, the radix-8 schedule of 4096-point axes), rotation angles up to ~1
(the closed-form branch of the potential factor), the packet, read-outs and densities,
checkpoints, a batch member, and the 1024x512 benchmark workload's norm over 2000 steps."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DW = 3
TOL = 1e-10


@pytest.fixture(scope="module")
def kd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - b)) / np.max(np.abs(b)))


FIELDS = {
    "none": dict(kind=W.NONE),
    "plane": dict(kind=W.PLANE),
    "plane_env": dict(kind=W.PLANE, env=True),
    "gauss": dict(kind=W.GAUSS, longitudinal=1),
    "gauss_transverse_static": dict(kind=W.GAUSS, longitudinal=0, box_vy=0.0),
}


@pytest.mark.parametrize("fname", list(FIELDS))
@pytest.mark.parametrize("nx,ny", [(4, 4), (32, 16), (64, 128), (256, 32), (4096, 4), (8, 4096)])
def test_dw_step_random_spinor(kd, fname, nx, ny):
    wl = W.small(nx, ny, units=W.ATOMIC, a0=0.4, nsteps=6, **FIELDS[fname])
    psi = W.random_spinor(nx, ny, 7 * nx + ny)
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, wl.dt, wl.nsteps)
    with kd.Sim(wl.units, wl.grid, wl.field, DW) as sim:
        sim.set_spinor(psi)
        sim.step(wl.dt, wl.nsteps)
        got = sim.get_spinor()
        t, n = sim.get_time()
    assert got.dtype == np.complex128
    assert rel(got, ref) <= TOL
    assert n == wl.nsteps


@pytest.mark.parametrize("fname", ["plane", "gauss", "gauss_transverse_static"])
def test_dw_large_rotation_angle(kd, fname):
    wl = W.small(64, 32, units=W.NATURAL, a0=2.0, nsteps=5, **FIELDS[fname])
    dt = 10 * wl.dt
    psi = W.random_spinor(64, 32, 5)
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, dt, wl.nsteps)
    with kd.Sim(wl.units, wl.grid, wl.field, DW) as sim:
        sim.set_spinor(psi)
        sim.step(dt, wl.nsteps)
        got = sim.get_spinor()
    assert rel(got, ref) <= TOL


@pytest.mark.parametrize("units", ["atomic", "natural"])
def test_dw_packet_run_with_observables(kd, units):
    u = W.ATOMIC if units == "atomic" else W.NATURAL
    wl = W.small(128, 64, W.GAUSS, units=u, a0=0.2, nsteps=60)
    g, f, pk = wl.grid, wl.field, wl.packet
    spec = W.default_obs_spec(u, f, pk)
    psi = oracle.init_packet(u, g, f, pk)
    with kd.Sim(u, g, f, DW) as sim:
        sim.init_packet(pk)
        assert rel(sim.get_spinor(), psi) <= TOL
        refs = []
        t = 0.0
        for _ in range(3):
            psi = oracle.step(u, g, f, psi, t, wl.dt, 20)
            t += 20 * wl.dt
            refs.append(oracle.observe(u, g, f, spec, psi, t))
        obs = sim.step(wl.dt, 60, obs_every=20)
        got = sim.get_spinor()
        md = sim.momentum_density(0)
        dens = sim.density_x()
    assert rel(got, psi) <= TOL
    for o, r in zip(obs, refs):
        for k, v in r.items():
            if k != "t":
                assert abs(o[k] - v) <= TOL * max(1.0, abs(v)), (k, o[k], v)
    ref_md = oracle.momentum_density(u, g, f, psi, basis=0)
    assert np.max(np.abs(md - ref_md)) <= TOL * np.max(ref_md)
    ref_d = oracle.density_x(g, psi)
    assert np.max(np.abs(dens - ref_d)) <= TOL * np.max(ref_d)


def test_dw_checkpoint_resume_and_batch_member(kd):
    wl = W.small(128, 64, W.GAUSS, units=W.ATOMIC, a0=0.3)
    with kd.Sim.from_workload(wl.with_(precision=DW)) as a:
        a.init_packet(wl.packet)
        a.step(wl.dt, 30)
        want = a.get_spinor()
    with kd.Sim.from_workload(wl.with_(precision=DW)) as b:
        b.init_packet(wl.packet)
        b.step(wl.dt, 11)
        blob = b.get_state()
    with kd.Sim.from_workload(wl.with_(precision=DW)) as c:
        c.set_state(blob)
        c.step(wl.dt, 19)
        # two calls close and reopen the half steps at step 11: equal to rounding
        assert rel(c.get_spinor(), want) <= 1e-13
    # an FP64 simulation does not accept the double-word checkpoint
    with kd.Sim.from_workload(wl.with_(precision=0)) as d:
        with pytest.raises(kd.KdError):
            d.set_state(blob)
    sims = [kd.Sim.from_workload(wl.with_(precision=DW)), kd.Sim.from_workload(wl.with_(precision=1))]
    for s_ in sims:
        s_.init_packet(wl.packet)
    with kd.Batch(sims) as bt:
        bt.step([wl.dt, wl.dt], 30)
    assert np.array_equal(sims[0].get_spinor(), want)
    for s_ in sims:
        s_.close()


def test_dw_norm_drift_over_the_benchmark_run(kd):
    wl = W.c2(precision=DW)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        n0 = sim.observe()["norm"]
        obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
    drift = max(abs(o["norm"] - n0) for o in obs)
    assert drift <= 1e-12, drift
    assert all(math.isfinite(o["pop_diff"]) for o in obs)
