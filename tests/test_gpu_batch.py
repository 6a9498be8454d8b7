"""Batched form: independent simulations of different grids, precisions and fields
advanced by kd_batch_step (one graph launch per chunk, the simulations as concurrent
branches) give exactly the states and observations of the same simulations advanced one
by one with kd_step, which the parity tests check against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


def _members():
    m = W.c4(n=6, seed=3, nsteps=60)
    m[1] = m[1].with_(precision=W.FP64)
    m.append(W.small(64, 32, W.PLANE, units=W.ATOMIC, nsteps=60, precision=W.FP64))
    return m


@pytest.mark.parametrize("obs_every", [0, 20])
def test_batch_equals_individual_runs(kd, obs_every):
    members = _members()
    ref_psi, ref_obs = [], []
    for wl in members:
        # the same call split as the batch below: a call boundary closes and reopens the
        # potential half step, which rounds differently from the merged step
        with kd.Sim.from_workload(wl) as s:
            s.init_packet(wl.packet)
            ref_obs.append(s.step(wl.dt, 40, obs_every=obs_every) + s.step(wl.dt, 20, obs_every=obs_every))
            ref_psi.append(s.get_spinor())
    sims = [kd.Sim.from_workload(wl) for wl in members]
    for s, wl in zip(sims, members):
        s.init_packet(wl.packet)
    with kd.Batch(sims) as b:
        obs = b.step([wl.dt for wl in members], 40, obs_every=obs_every)
        obs2 = b.step([wl.dt for wl in members], 20, obs_every=obs_every)
    for i, s in enumerate(sims):
        assert np.array_equal(s.get_spinor(), ref_psi[i]), i
        assert s.get_time()[1] == 60
        if obs_every:
            got = obs[i] + obs2[i]
            assert len(got) == 3
            for a, r in zip(got, ref_obs[i]):
                assert a == r
        s.close()


def test_batch_rejects_duplicates_and_bad_dt(kd):
    wl = W.small(32, 32, W.GAUSS, units=W.ATOMIC)
    with kd.Sim.from_workload(wl) as s:
        with pytest.raises(kd.KdError):
            kd.Batch([s, s])
        s.init_packet(wl.packet)
        with kd.Batch([s]) as b:
            with pytest.raises(kd.KdError):
                b.step([-1.0], 3)


def test_batch_autotune_keeps_states_and_steps_like_members_alone(kd):
    """kd_batch_autotune times launch variants on the whole batch and restores every
    member's state and clock; afterwards the batch still equals its members run alone
    with the chosen variants, bit for bit."""
    wls = [W.small(128, 128, W.GAUSS, units=W.ATOMIC, a0=0.2), W.small(256, 128, W.GAUSS, units=W.ATOMIC),
           W.small(128, 128, W.PLANE, units=W.ATOMIC, a0=0.3), W.small(64, 256, W.GAUSS, units=W.ATOMIC)]
    sims = [kd.Sim.from_workload(wl.with_(precision=1)) for wl in wls]
    before = []
    for s, wl in zip(sims, wls):
        s.init_packet(wl.packet)
        s.step(wl.dt, 3)
        before.append((s.get_spinor(), s.get_time(), s.get_state()))
    dts = [wl.dt for wl in wls]
    with kd.Batch(sims) as b:
        chosen = b.autotune(dts, steps=10)
        for s, (psi, tm, _), v in zip(sims, before, chosen):
            assert np.array_equal(s.get_spinor(), psi)
            assert s.get_time() == tm
            assert s.sweep_variants == v and all(0 <= x < kd.KD_SWEEP_VARIANTS for x in v)
        # members of the same grid and form share their variants
        assert chosen[0] == chosen[2]
        b.step(dts, 20)
    batched = [s.get_spinor() for s in sims]
    for s in sims:
        s.close()
    for wl, (psi, tm, blob), v, got in zip(wls, before, chosen, batched):
        with kd.Sim.from_workload(wl.with_(precision=1)) as alone:
            alone.sweep_variants = v
            alone.set_state(blob)         # the member's state and clock before the batch
            alone.step(wl.dt, 20)
            assert np.array_equal(alone.get_spinor(), got)


# ------------------------------------------------------------ persistent form
PERSIST_VARIANTS = (0, 3)


def _mixed_members():
    return [W.small(128, 64, W.GAUSS, units=W.ATOMIC, a0=0.3),
            W.small(64, 256, W.GAUSS, units=W.ATOMIC, a0=0.2),
            W.small(32, 32, W.PLANE, units=W.ATOMIC, a0=0.4),
            W.small(512, 128, W.GAUSS, units=W.ATOMIC, a0=0.1),
            W.small(16, 512, W.NONE, units=W.ATOMIC)]


def _persist_ran(var, ny):
    """The launch variants a member with sweep variants `var` runs in the persistent
    kernel: x 0 or 2; y 3, or 2 on y axes up to 256 points."""
    vx = 2 if var[0] == 2 else 0
    vy = 2 if var[1] == 2 and ny <= 256 else 3
    return (vx, vy)


@pytest.mark.parametrize("variants", [None, (2, 2)])
def test_persistent_batch_equals_members_alone(kd, variants):
    """One persistent kernel per chunk (device work queue, per-member completion counters)
    advances every member exactly as its own sweeps would: bitwise equal to the members
    run alone on the same launch variants, over chunks with observations and two calls;
    with the default variants and with the radix-4 alternates of both axes."""
    wls = _mixed_members()
    alone, alone_obs = [], []
    for wl in wls:
        with kd.Sim.from_workload(wl.with_(precision=1)) as sim:
            # the packet is built on the variants the member has when it is initialised
            # (its own), the steps on those the persistent kernel runs for it
            if variants is not None:
                sim.sweep_variants = variants
            sim.init_packet(wl.packet)
            sim.sweep_variants = PERSIST_VARIANTS if variants is None else _persist_ran(variants, wl.grid.ny)
            o1 = sim.step(wl.dt, 45, obs_every=15)
            o2 = sim.step(wl.dt, 30, obs_every=15)
            alone.append(sim.get_spinor())
            alone_obs.append(o1 + o2)
    sims = [kd.Sim.from_workload(wl.with_(precision=1)) for wl in wls]
    for s, wl in zip(sims, wls):
        if variants is not None:
            s.sweep_variants = variants
        s.init_packet(wl.packet)
    with kd.Batch(sims) as b:
        b.set_mode(kd.KD_BATCH_PERSISTENT)
        # the members now report the variants the kernel runs for them
        for s, wl in zip(sims, wls):
            assert s.sweep_variants == (PERSIST_VARIANTS if variants is None
                                        else _persist_ran(variants, wl.grid.ny))
        o1 = b.step([wl.dt for wl in wls], 45, obs_every=15)
        o2 = b.step([wl.dt for wl in wls], 30, obs_every=15)
    for i, s in enumerate(sims):
        assert np.array_equal(s.get_spinor(), alone[i]), i
        assert o1[i] + o2[i] == alone_obs[i], i
        assert s.get_time()[1] == 75
        s.close()


def test_persistent_batch_against_oracle(kd):
    wl = W.small(64, 32, W.GAUSS, units=W.ATOMIC, a0=0.4, nsteps=6)
    psi = W.random_spinor(64, 32, 77)
    ref = oracle.step(wl.units, wl.grid, wl.field, psi, 0.0, wl.dt, 6)
    sims = [kd.Sim.from_workload(wl.with_(precision=1)), kd.Sim.from_workload(wl.with_(precision=1))]
    for s in sims:
        s.set_spinor(psi)
    with kd.Batch(sims) as b:
        b.set_mode(kd.KD_BATCH_PERSISTENT)
        b.step([wl.dt, wl.dt], 6)
    for s in sims:
        got = s.get_spinor().astype(np.complex128)
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
        s.close()


def test_persistent_batch_many_members_equals_graph_form(kd):
    """150 small members (three grid shapes, seeded fields): far more members than the
    kernel keeps in registers or shared memory, so every item's member lookup runs over the
    prefix sums; the persistent form equals the graph-branch form bit for bit (both on the
    variants the kernel holds), over two calls with observations."""
    rng = np.random.default_rng(11)
    shapes = [(16, 16), (32, 16), (16, 64)]
    wls = [W.small(*shapes[i % 3], W.GAUSS, units=W.ATOMIC, a0=float(rng.uniform(0.05, 0.4)))
           for i in range(150)]
    finals = {}
    for mode in (kd.KD_BATCH_GRAPH, kd.KD_BATCH_PERSISTENT):
        sims = [kd.Sim.from_workload(wl.with_(precision=1)) for wl in wls]
        for s, wl in zip(sims, wls):
            s.sweep_variants = PERSIST_VARIANTS
            s.init_packet(wl.packet)
        with kd.Batch(sims) as b:
            b.set_mode(mode)
            o1 = b.step([wl.dt for wl in wls], 12, obs_every=6)
            o2 = b.step([wl.dt for wl in wls], 7, obs_every=6)
        finals[mode] = ([s.get_spinor() for s in sims], [a + c for a, c in zip(o1, o2)])
        for s in sims:
            s.close()
    (pg, og), (pp, op) = finals[kd.KD_BATCH_GRAPH], finals[kd.KD_BATCH_PERSISTENT]
    for i in range(len(wls)):
        assert np.array_equal(pg[i], pp[i]), i
        assert og[i] == op[i], i


def test_persistent_batch_withheld_producer_times_out(kd):
    """A member's first work item never signals completion (test hook): the items waiting
    for it give up after their bounded waits, the call returns KD_ERR_TIMEOUT, and the
    context stays usable."""
    wls = [W.small(64, 64, W.GAUSS, units=W.ATOMIC), W.small(128, 32, W.GAUSS, units=W.ATOMIC)]
    sims = [kd.Sim.from_workload(wl.with_(precision=1)) for wl in wls]
    for s, wl in zip(sims, wls):
        s.init_packet(wl.packet)
    with kd.Batch(sims) as b:
        b.set_mode(kd.KD_BATCH_PERSISTENT)
        sims[1].inject_fault(kd.KD_FAULT_PERSIST_HOLD)
        with pytest.raises(kd.KdError) as e:
            b.step([wl.dt for wl in wls], 10)
        assert e.value.code == kd.KD_ERR_TIMEOUT
        # the hook lasted one call: fresh states step correctly afterwards
        for s, wl in zip(sims, wls):
            s.init_packet(wl.packet)
        b.step([wl.dt for wl in wls], 10)
    for s, wl in zip(sims, wls):
        with kd.Sim.from_workload(wl.with_(precision=1)) as alone:
            alone.sweep_variants = PERSIST_VARIANTS
            alone.init_packet(wl.packet)
            alone.step(wl.dt, 10)
            assert np.array_equal(alone.get_spinor(), s.get_spinor())
        s.close()


def test_persistent_batch_rejects_unsupported_members(kd):
    for wl, prec in [(W.small(64, 64, W.GAUSS), 0), (W.small(1024, 64, W.GAUSS), 1),
                     (W.small(64, 64, W.GAUSS), 2)]:
        sims = [kd.Sim.from_workload(wl.with_(precision=prec))]
        with kd.Batch(sims) as b:
            with pytest.raises(kd.KdError) as e:
                b.set_mode(kd.KD_BATCH_PERSISTENT)
            assert e.value.code == kd.KD_ERR_UNSUPPORTED_SIZE
        sims[0].close()
