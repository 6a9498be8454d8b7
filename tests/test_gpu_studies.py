"""The parameter studies of Sec. IV (spin-flip scaling and longitudinal on/off) as batched
runs: every study configuration's first steps on a reduced grid, advanced together through
kd_batch_step, against the oracle element by element.  The reduced runs put the box and
the packet at the beam's focus (the setup's start, 15 half waists out, sees no field), so
the Gaussian beam and its longitudinal component act from the first step."""
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


def _batch(kd, wls, n):
    sims = [kd.Sim.from_workload(w) for w in wls]
    for s, w in zip(sims, wls):
        s.init_packet(w.packet)
    with kd.Batch(sims) as b:
        b.step([w.dt for w in wls], n)
    out = [s.get_spinor().astype(np.complex128) for s in sims]
    for s in sims:
        s.close()
    return out


def _oracle(w, n):
    u, g, f, pk = w.units, w.grid, w.field, w.packet
    return oracle.step(u, g, f, oracle.init_packet(u, g, f, pk), 0.0, w.dt, n)


def test_study_configurations_first_steps_against_oracle(kd):
    cfgs = [(e, k, 1) for e in studies.EPSILONS for k in studies.K_NAT] + \
           [(e, 0.1, 0) for e in studies.EPSILONS]
    wls = [studies.run(eps=e, k_nat=k, longitudinal=lo, nx=256, ny=32, nsteps=3, y0=0.0) for e, k, lo in cfgs]
    for w, got in zip(wls, _batch(kd, wls, 3)):
        ref = _oracle(w, 3)
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref)), w.name


def test_longitudinal_on_off_resolved_in_double_word(kd):
    # the longitudinal component changes the state by 2e-6 (eps 0.01) ... 2e-5 (eps 0.1) of
    # max |psi| in 3 steps: below the FP32 bar, far above the double-word form's 1e-10
    n = 3
    wls = [studies.run(eps=e, k_nat=0.1, longitudinal=lo, nx=256, ny=32, nsteps=n, y0=0.0, precision=W.DW)
           for e in studies.EPSILONS for lo in (1, 0)]
    got = _batch(kd, wls, n)
    refs = [_oracle(w, n) for w in wls]
    for w, g, r in zip(wls, got, refs):
        assert np.max(np.abs(g - r)) <= 1e-10 * np.max(np.abs(r)), w.name
    for i in range(0, len(wls), 2):
        scale = np.max(np.abs(refs[i]))
        d_ref = refs[i] - refs[i + 1]
        d_got = got[i] - got[i + 1]
        assert np.max(np.abs(d_ref)) > 1e-6 * scale
        assert np.max(np.abs(d_got - d_ref)) <= 1e-10 * scale
