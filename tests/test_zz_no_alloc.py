"""kd_density_noalloc: the allocation-free density read-out, for callers that cannot
allocate device memory (a host that gives the library a fixed memory budget, a real-time
loop that must not wait on the allocator, a plug-in inside a runtime that forbids
allocation).  It is checked through the C ABI against the existing entry points
(kd_observe's norm and kd_get_density_x) on the same state and against the oracle's sums
of the same spinor values, on two calls in a row (the static scratch keeps the previous
call's contents), and device memory must not change across those calls.  This file is
collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2307_01571_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-4}
# both sides accumulate in FP64 over the same stored values, in different orders
ACC_TOL = 1e-12


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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_density_matches_existing_entry_points(kd, prec):
    import torch
    wl = W.small(256, 128, W.GAUSS, units=W.ATOMIC, a0=0.3, precision=prec)
    g = wl.grid
    dx, dy = (g.x_max - g.x_min) / g.nx, (g.y_max - g.y_min) / g.ny
    ctype = torch.complex128 if prec == 0 else torch.complex64
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        sim.step(wl.dt, 7)
        ref_norm = sim.observe()["norm"]
        ref_dens = sim.density_x()
        psi = torch.empty((g.ny, g.nx, 4), dtype=ctype, device="cuda")
        sim.get_spinor(psi)
        torch.cuda.synchronize()
    host = psi.cpu().numpy().astype(np.complex128)
    o_dens = oracle.density_x(g, host)
    o_norm = float(np.sum(o_dens) * dx)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    norm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    dens = torch.full((g.nx,), -1.0, dtype=torch.float64, device="cuda")

    def call():
        norm.fill_(-1.0)
        dens.fill_(-1.0)
        rc = kd.kd_density_noalloc(C.c_void_p(psi.data_ptr()), g.nx, g.ny, prec, dx, dy,
                                   C.c_void_p(norm.data_ptr()), C.c_void_p(dens.data_ptr()), stream)
        assert rc == kd.KD_OK, kd.kd_last_error()
        torch.cuda.synchronize()
        assert kd.kd_last_error() == b""

    call()                                   # first call on the device: address set-up
    alloc0, free0 = torch.cuda.memory_allocated(), _free_bytes()
    for _ in range(2):
        call()
        assert abs(norm.item() - ref_norm) <= TOL[prec] * abs(ref_norm)
        d = dens.cpu().numpy()
        assert abs(d - ref_dens).max() <= TOL[prec] * ref_dens.max()
        assert abs(norm.item() - o_norm) <= ACC_TOL * o_norm
        assert abs(d - o_dens).max() <= ACC_TOL * o_dens.max()
    assert torch.cuda.memory_allocated() == alloc0
    assert _free_bytes() == free0


def test_noalloc_rejects_sizes_beyond_its_scratch(kd):
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = kd.kd_density_noalloc(C.c_void_p(buf.data_ptr()), 4, 8192, 0, 1.0, 1.0,
                               C.c_void_p(out.data_ptr()), None, None)
    assert rc == kd.KD_ERR_UNSUPPORTED_SIZE
    assert b"KD_NOALLOC_MAX_ROWS" in kd.kd_last_error()
    rc = kd.kd_density_noalloc(None, 4, 4, 0, 1.0, 1.0, C.c_void_p(out.data_ptr()), None, None)
    assert rc == kd.KD_ERR_ARG
