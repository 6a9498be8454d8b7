"""Failure handling on the host side of the C ABI, with no GPU fault: cancellation of a
running kd_step at a chunk boundary (the state stays a valid evolution of the steps that
ran), and out-of-memory handling through the allocation-failure test hook (every failing
allocation in kd_create and kd_step returns KD_ERR_NOMEM, releases what the call had
allocated, and leaves the simulation usable)."""
import threading
import time

import numpy as np
import pytest

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


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("obs_every", [0, 20])
def test_cancel_before_step_runs_one_closed_chunk(kd, prec, obs_every):
    wl = W.small(64, 32, W.GAUSS, units=W.ATOMIC, a0=0.3, precision=prec)
    chunk = obs_every if obs_every else 64
    with kd.Sim.from_workload(wl) as ref:
        ref.init_packet(wl.packet)
        ref_obs = ref.step(wl.dt, chunk, obs_every=obs_every)
        want = ref.get_spinor()
        t_want = ref.get_time()
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        sim.cancel()
        with pytest.raises(kd.KdCancelled) as e:
            sim.step(wl.dt, 1000, obs_every=obs_every)
        assert e.value.code == kd.KD_ERR_CANCELLED
        assert sim.get_time() == t_want
        assert np.array_equal(sim.get_spinor(), want)
        assert e.value.obs == ref_obs
        # the request was consumed: the next call runs to the end
        sim.step(wl.dt, 3)
        assert sim.get_time()[1] == chunk + 3


def test_cancel_from_another_thread(kd):
    wl = W.small(128, 128, W.GAUSS, units=W.ATOMIC, a0=0.3, precision=1)
    n = 400_000
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        th = threading.Thread(target=lambda: (time.sleep(0.2), sim.cancel()))
        th.start()
        with pytest.raises(kd.KdCancelled):
            sim.step(wl.dt, n)
        th.join()
        _, done = sim.get_time()
        assert 0 < done < n and done % 64 == 0
        got = sim.get_spinor()
    with kd.Sim.from_workload(wl) as ref:
        ref.init_packet(wl.packet)
        ref.step(wl.dt, done)                  # the same chunks, the last one closing
        assert np.array_equal(ref.get_spinor(), got)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_alloc_failure_in_create_releases_everything(kd, prec):
    wl = W.small(1024, 64, W.GAUSS, units=W.ATOMIC, precision=prec)
    kd.Sim.from_workload(wl).close()          # kernels and runtime state loaded once
    free0 = _free_bytes()
    failures = 0
    try:
        for k in range(64):
            kd.inject_alloc_failure(k)
            try:
                sim = kd.Sim.from_workload(wl)
            except kd.KdError as e:
                assert e.code == kd.KD_ERR_NOMEM, e
                failures += 1
                assert _free_bytes() == free0, k
                continue
            kd.inject_alloc_failure(-1)
            sim.init_packet(wl.packet)
            sim.step(wl.dt, 4)
            sim.close()
            break
    finally:
        kd.inject_alloc_failure(-1)
    assert failures >= 12                      # every buffer of kd_create was reached
    assert _free_bytes() == free0


def test_alloc_failure_in_step_leaves_simulation_usable(kd):
    wl = W.small(128, 64, W.GAUSS, units=W.ATOMIC, a0=0.3, precision=1)
    with kd.Sim.from_workload(wl) as ref:
        ref.init_packet(wl.packet)
        ref.step(wl.dt, 100, obs_every=10)
        ref.step(wl.dt, 3000)
        ref_obs = ref.step(wl.dt, 100, obs_every=1)
        want = ref.get_spinor()
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        sim.step(wl.dt, 100, obs_every=10)
        state = sim.get_time()
        try:
            kd.inject_alloc_failure(0)         # the per-step table grows for 3000 steps
            with pytest.raises(kd.KdError) as e:
                sim.step(wl.dt, 3000)
            assert e.value.code == kd.KD_ERR_NOMEM
            assert sim.get_time() == state
            sim.step(wl.dt, 3000)
            kd.inject_alloc_failure(0)         # the observation buffer grows for 100 records
            with pytest.raises(kd.KdError) as e:
                sim.step(wl.dt, 100, obs_every=1)
            assert e.value.code == kd.KD_ERR_NOMEM
        finally:
            kd.inject_alloc_failure(-1)
        obs = sim.step(wl.dt, 100, obs_every=1)
        assert np.array_equal(sim.get_spinor(), want)
        assert obs == ref_obs
