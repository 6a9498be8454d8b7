"""Precision form (KD_FP32_TC): the full sweeps of 1024-point axes evaluate their FFTs as
32-point DFT matrix products on the tensor cores.  Parity with the oracle element by
element on both axes and every field kind (several tiles: 4 lines per work item, many
items per CTA), at the 1024x512 and 2048x1024 grids, observables through the mixed path
(tensor-core full sweeps, CUDA-core half sweeps), checkpoints interchangeable with KD_FP32,
the FP32 norm-drift bar as an expected failure (the truncating tensor-core accumulation
misses it) beside a regression guard, and the bounded-wait timeout path."""
import math

import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TC = 2


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


FIELDS = {"none": dict(kind=W.NONE), "plane": dict(kind=W.PLANE),
          "gauss": dict(kind=W.GAUSS, longitudinal=1), "gauss_static": dict(kind=W.GAUSS, box_vy=0.0)}


@pytest.mark.parametrize("fname", list(FIELDS))
@pytest.mark.parametrize("nx,ny", [(1024, 8), (8, 1024), (1024, 64), (64, 1024), (1024, 1024)])
def test_tc_step_against_oracle(kd, fname, nx, ny):
    wl = W.small(nx, ny, units=W.ATOMIC, a0=0.4, nsteps=4, **FIELDS[fname])
    psi = W.random_spinor(nx, ny, 5 * nx + ny)
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, wl.dt, wl.nsteps)
    with kd.Sim(wl.units, wl.grid, wl.field, TC) as sim:
        sim.set_spinor(psi)
        sim.step(wl.dt, wl.nsteps)
        got = sim.get_spinor()
    assert rel(got, ref) <= 1e-4


@pytest.mark.parametrize("fname", ["plane", "gauss"])
@pytest.mark.parametrize("nx,ny", [(1024, 16), (16, 1024)])
def test_tc_step_large_rotation_angle(kd, fname, nx, ny):
    """The tensor-core sweeps' potential step at rotation angles up to ~1 (natural units,
    dt = 0.5 hbar/mc^2, a0 = 2): the closed-form branch for theta >= 1/4."""
    wl = W.small(nx, ny, units=W.NATURAL, a0=2.0, nsteps=4, **FIELDS[fname])
    dt = 10 * wl.dt
    psi = W.random_spinor(nx, ny, 3 * nx + ny)
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, dt, wl.nsteps)
    with kd.Sim(wl.units, wl.grid, wl.field, TC) as sim:
        sim.set_spinor(psi)
        sim.step(dt, wl.nsteps)
        got = sim.get_spinor()
    assert rel(got, ref) <= 1e-4


@pytest.mark.parametrize("wlf", [lambda: W.c2(precision=TC, nsteps=3), lambda: W.c3(precision=TC, nsteps=3)])
def test_tc_full_size_with_observables(kd, wlf):
    wl = wlf()
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    ref = oracle.step(u, g, f, oracle.init_packet(u, g, f, pk), 0.0, wl.dt, 3)
    spec = W.default_obs_spec(u, f, pk)
    oref = oracle.observe(u, g, f, spec, ref, 3 * wl.dt)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(pk)
        obs = sim.step(wl.dt, 3, obs_every=3)
        got = sim.get_spinor()
    assert rel(got, ref) <= 1e-4
    for k, v in oref.items():
        assert abs(obs[-1][k] - v) <= 1e-4 * max(1.0, abs(v)), k


def _tc_drift(kd):
    wl = W.c2(precision=TC)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        n0 = sim.observe()["norm"]
        obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
    assert all(math.isfinite(o["pop_diff"]) for o in obs)
    return max(abs(o["norm"] - n0) for o in obs)


@pytest.mark.xfail(strict=True, reason="the tensor cores' FP32 accumulation truncates (bias toward "
                   "zero); the norm of the 1024x512 run decays by ~1.5e-3 over 2000 steps")
def test_tc_norm_drift_meets_fp32_bar(kd):
    """The FP32 bar of norm drift <= 1e-6 over the 2000-step run: the precision form does not
    meet it (an expected failure; the FP32 CUDA-core form does, test_gpu_long)."""
    assert _tc_drift(kd) <= 1e-6


def test_tc_norm_drift_regression_guard(kd):
    """Not the bar: guards the measured behaviour of the form (drift 1.5e-3, monotone decay
    from the truncating accumulation) against getting worse."""
    assert _tc_drift(kd) <= 3e-3


def test_tc_checkpoint_interchangeable_with_fp32(kd):
    wl = W.small(1024, 32, W.GAUSS, units=W.ATOMIC, a0=0.3)
    with kd.Sim.from_workload(wl.with_(precision=TC)) as sim:
        sim.init_packet(wl.packet)
        sim.step(wl.dt, 5)
        blob = sim.get_state()
        a = sim.get_spinor()
    with kd.Sim.from_workload(wl.with_(precision=1)) as s32:
        s32.set_state(blob)
        assert np.array_equal(s32.get_spinor(), a)
        assert s32.get_time()[1] == 5


def test_tc_bounded_wait_gives_up_and_context_survives(kd):
    wl = W.small(1024, 16, W.GAUSS, units=W.ATOMIC, a0=0.3, nsteps=2)
    psi = W.random_spinor(1024, 16, 9)
    with kd.Sim.from_workload(wl.with_(precision=TC)) as sim:
        sim.set_spinor(psi)
        sim.inject_fault()
        with pytest.raises(kd.KdError) as e:
            sim.step(wl.dt, 2)
        assert e.value.code == kd.KD_ERR_TIMEOUT
        # the hook lasted one call; the same simulation runs correctly afterwards
        sim.set_spinor(psi)
        sim.set_time(0.0)
        sim.step(wl.dt, 2)
        got = sim.get_spinor()
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, wl.dt, 2)
    assert rel(got, ref) <= 1e-4
    with kd.Sim.from_workload(wl.with_(precision=1)) as s32:
        with pytest.raises(kd.KdError):
            s32.inject_fault()


def test_tc_member_in_a_batch_matches_it_alone(kd):
    """A KD_FP32_TC simulation advanced as one branch of a batch (its operand scales set by
    the batch's per-member prologue) equals the same simulation run alone, bit for bit."""
    wls = [W.small(1024, 32, W.GAUSS, units=W.ATOMIC, a0=0.3), W.small(128, 256, W.GAUSS, units=W.ATOMIC)]
    precs = [TC, 1]
    alone = []
    for wl, p in zip(wls, precs):
        with kd.Sim.from_workload(wl.with_(precision=p)) as sim:
            sim.init_packet(wl.packet)
            sim.step(wl.dt, 25, obs_every=5)
            alone.append(sim.get_spinor())
    sims = [kd.Sim.from_workload(wl.with_(precision=p)) for wl, p in zip(wls, precs)]
    for s, wl in zip(sims, wls):
        s.init_packet(wl.packet)
    with kd.Batch(sims) as b:
        b.step([wl.dt for wl in wls], 25, obs_every=5)
    for s, a in zip(sims, alone):
        assert np.array_equal(s.get_spinor(), a)
        s.close()


def test_tc_injected_wait_fault_lasts_one_batch_step(kd):
    """The bounded-wait test hook on a batch member: the next kd_batch_step returns
    KD_ERR_TIMEOUT (the member's waits give up), the one after it runs normally and
    matches the member run alone."""
    wl = W.small(1024, 16, W.GAUSS, units=W.ATOMIC, a0=0.3, nsteps=2)
    psi = W.random_spinor(1024, 16, 21)
    with kd.Sim.from_workload(wl.with_(precision=TC)) as alone:
        alone.set_spinor(psi)
        alone.step(wl.dt, 2)
        ref = alone.get_spinor()
    sim = kd.Sim.from_workload(wl.with_(precision=TC))
    sim.set_spinor(psi)
    with kd.Batch([sim]) as b:
        sim.inject_fault()
        with pytest.raises(kd.KdError) as e:
            b.step([wl.dt], 2)
        assert e.value.code == kd.KD_ERR_TIMEOUT
        sim.set_spinor(psi)
        sim.set_time(0.0)
        b.step([wl.dt], 2)
    assert np.array_equal(sim.get_spinor(), ref)
    sim.close()


def test_tensor_core_fp32_accumulation_rounds_toward_zero(kd):
    """Why the precision form misses the FP32 bars: the FP32 accumulation of a
    tcgen05.mma (kind::f16) rounds toward zero.  Sums whose exact value lies between two
    floats, formed through the library's BF16 tensor-core GEMM (a one-layer network
    y = W x, W = 1, bias 0, so y is the MMA's sum): 1 + 0.75 ulp comes back as 1 (round to
    nearest: 1 + 1 ulp), -(1 + 0.75 ulp) as -1, 1 + 1.5 ulp as 1 + 1 ulp (nearest: + 2 ulp),
    also when the small part arrives in a later 64-deep slab (accumulation in tensor
    memory).  Every operand is exact in BF16."""
    u = 2.0 ** -23
    rows = [[1.0, 0.75 * u], [-1.0, -0.75 * u], [1.0, 1.5 * u], [1.0, 0.25 * u, 0.25 * u, 0.25 * u]]
    want_rz = [1.0, -1.0, 1.0 + u, 1.0]
    net = kd.MLP([16, 1])
    net.set_precision(kd.KD_MLP_BF16)
    p = np.zeros(17, np.float32)
    p[:16] = 1.0
    net.set_params(p)
    x = np.zeros((len(rows), 16), np.float32)
    for i, r in enumerate(rows):
        x[i, :len(r)] = r
    y = net.forward(x)[:, 0].astype(np.float64)
    assert list(y) == want_rz
    # round to nearest would differ in every row
    assert all(float(np.float32(sum(r))) != w for r, w in zip(rows, want_rz))
    net.close()
    # across k slabs: the 1 in slab 0, the small part in slab 1
    net2 = kd.MLP([80, 1])
    net2.set_precision(kd.KD_MLP_BF16)
    p2 = np.zeros(81, np.float32)
    p2[:80] = 1.0
    net2.set_params(p2)
    x2 = np.zeros((2, 80), np.float32)
    x2[0, 0], x2[0, 70] = 1.0, 0.75 * u
    x2[1, 0], x2[1, 70] = -1.0, -0.75 * u
    assert list(net2.forward(x2)[:, 0].astype(np.float64)) == [1.0, -1.0]
    net2.close()
