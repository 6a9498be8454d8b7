"""The parameter studies of Sec. IV (spin-flip scaling and longitudinal on/off) as batched
runs: every study configuration's first steps on a reduced grid, advanced together through
kd_batch_step, against the oracle element by element (FP32 bar)."""
import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import studies
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


def test_study_configurations_first_steps_against_oracle(kd):
    cfgs = [(e, k, 1) for e in studies.EPSILONS for k in studies.K_NAT] + \
           [(e, 0.1, 0) for e in studies.EPSILONS]
    wls = [studies.run(eps=e, k_nat=k, longitudinal=lo, nx=256, ny=32, nsteps=3) for e, k, lo in cfgs]
    sims = [kd.Sim.from_workload(w) for w in wls]
    for s, w in zip(sims, wls):
        s.init_packet(w.packet)
    with kd.Batch(sims) as b:
        b.step([w.dt for w in wls], 3)
    for s, w in zip(sims, wls):
        u, g, f, pk = w.units, w.grid, w.field, w.packet
        ref = oracle.step(u, g, f, oracle.init_packet(u, g, f, pk), 0.0, w.dt, 3)
        got = s.get_spinor().astype(np.complex128)
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), w.name
        s.close()
