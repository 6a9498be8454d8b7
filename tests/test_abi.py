"""Host-side checks of the C ABI that need no GPU: the library builds and loads, exports
every function declared in include/kd.h, rejects bad arguments before touching the
device, and fails (no CPU fallback) when no CUDA device is present."""
import ctypes as C
import os
import re

import pytest
import torch

from paper_2307_01571_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kd():
    _build.build()
    from paper_2307_01571_gb300 import kd as mod
    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "kd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(kd):
    names = _declared()
    assert len(names) >= 17
    lib = C.CDLL(kd.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(kd.EXPORTS)


def test_version_and_no_error(kd):
    assert kd.kd_version() >= 100


def test_bad_sizes_rejected_before_device(kd):
    from paper_2307_01571_gb300 import workloads as W
    u = kd.kd_units(1, 1, 1, -1)
    f = kd.kd_field()
    h = C.c_void_p()
    for nx, ny in [(6, 8), (2, 8), (8192, 8), (8, 0)]:
        g = kd.kd_grid(nx, ny, -1.0, 1.0, -1.0, 1.0)
        assert kd.kd_create(C.byref(u), C.byref(g), C.byref(f), 0, None, C.byref(h)) == kd.KD_ERR_UNSUPPORTED_SIZE
        assert b"power" in kd.kd_last_error()
    g = kd.kd_grid(8, 8, 1.0, -1.0, -1.0, 1.0)
    assert kd.kd_create(C.byref(u), C.byref(g), C.byref(f), 0, None, C.byref(h)) == kd.KD_ERR_ARG
    g = kd.kd_grid(8, 8, -1.0, 1.0, -1.0, 1.0)
    assert kd.kd_create(C.byref(u), C.byref(g), C.byref(f), 7, None, C.byref(h)) == kd.KD_ERR_ARG
    fb = kd.kd_field(kind=2, k_L=1.0, epsilon=0.0)
    assert kd.kd_create(C.byref(u), C.byref(g), C.byref(fb), 0, None, C.byref(h)) == kd.KD_ERR_ARG
    assert kd.kd_create(None, C.byref(g), C.byref(f), 0, None, C.byref(h)) == kd.KD_ERR_ARG
    # null simulation handles are rejected, destroy(NULL) is a no-op
    assert kd.kd_step(None, 0.1, 1, 0, None, 0, None) == kd.KD_ERR_ARG
    kd.kd_destroy(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_cpu_fallback_without_device(kd):
    from paper_2307_01571_gb300 import workloads as W
    wl = W.small(8, 8)
    with pytest.raises(kd.KdError) as e:
        kd.Sim.from_workload(wl)
    assert e.value.code == kd.KD_ERR_CUDA


def test_launch_variant_count_agrees_everywhere(kd):
    """The FP32 sweep launch variants are compiled one object file per variant (build
    script), enumerated by the internal variant table, exported as KD_SWEEP_VARIANTS in the
    public header and mirrored by the Python binding: all four must agree."""
    hdr = open(os.path.join(ROOT, "include", "kd.h")).read()
    m = re.search(r"#define\s+KD_SWEEP_VARIANTS\s+(\d+)", hdr)
    assert m
    n = int(m.group(1))
    internal = open(os.path.join(ROOT, "paper_2307_01571_gb300", "csrc", "kd_internal.h")).read()
    assert re.search(rf"constexpr int kNumSweepVariants = {n};", internal)
    # one table entry per variant and axis (the default closes each axis's chain)
    table = internal[internal.index("sweep_variant(int axis, int v)"):internal.index("sweep_nc(")]
    assert table.count("SweepVariant{") == 2 * n
    assert _build.SWEEP_VARIANTS == n
    assert kd.KD_SWEEP_VARIANTS == n
    assert sum(1 for u in _build.UNITS if u[0] == "kd_sweep_f32.cu") == n


def test_cancel_and_alloc_hook_argument_checks(kd):
    assert kd.kd_cancel(None) == kd.KD_ERR_ARG
    assert kd.kd_inject_alloc_failure(-2) == kd.KD_ERR_ARG
    assert kd.kd_inject_alloc_failure(-1) == kd.KD_OK
