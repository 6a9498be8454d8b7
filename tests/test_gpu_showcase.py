"""The paper's own runs (Sec. II.D / III showcase E1, Tables I and II) as workloads of the
library: their first Strang steps through the C ABI against the oracle, element by
element and for the read-outs the paper prints (spin-resolved cell populations at the
diffracted peak), in both precisions and in the precision form."""
import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import showcase as S
from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {0: 1e-10, 1: 1e-4, 2: 1e-4}


@pytest.fixture(scope="module")
def kd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,px_hk", [("e1", 0.1), ("e5", 1.0), ("e6", 1.0)])
def test_paper_run_first_steps_against_oracle(kd, name, px_hk, prec):
    wl = getattr(S, name)(nsteps=3, precision=prec)
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    ref = oracle.step(u, g, f, oracle.init_packet(u, g, f, pk), 0.0, wl.dt, wl.nsteps)
    spec = S.readout_spec(wl, px_hk)
    oref = oracle.observe(u, g, f, spec, ref, wl.nsteps * wl.dt)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(pk)
        sim.set_obs_spec(spec)
        obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.nsteps)
        got = sim.get_spinor()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(np.asarray(got, np.complex128) - ref)) <= TOL[prec] * scale
    for k in ("norm", "pop_in", "pop_diff", "p_target", "cp_target", "cm_target"):
        assert abs(obs[-1][k] - oref[k]) <= TOL[prec] * max(1.0, abs(oref[k])), k


def test_paper_run_precision_form(kd):
    """E1's x axis has 2048 points and its y axis 128: the precision form runs it on the
    CUDA-core kernels (no 1024-point axis) and must equal KD_FP32 bit for bit."""
    wl = S.e1(nsteps=4, precision=1)
    outs = []
    for prec in (1, 2):
        with kd.Sim.from_workload(wl.with_(precision=prec)) as sim:
            sim.init_packet(wl.packet)
            sim.step(wl.dt, wl.nsteps)
            outs.append(sim.get_spinor())
    assert np.array_equal(outs[0], outs[1])
