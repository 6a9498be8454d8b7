"""ctypes binding of ``libkd.so`` (C ABI in ``include/kd.h``).

Argument marshalling only: every step of the split-operator path runs in the library's
CUDA kernels.  The raw entry points are exported under their C names (``kd_create``,
``kd_step``, ...); :class:`Sim` wraps them for numpy arrays and torch tensors.  There is
no CPU fallback: importing this module raises if the library is missing, and
``kd_create`` fails without a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkd.so")

KD_OK = 0
KD_ERR_ARG, KD_ERR_UNSUPPORTED_SIZE, KD_ERR_CUDA = -1, -2, -3
KD_ERR_NONFINITE, KD_ERR_NORM_DRIFT, KD_ERR_TIMEOUT = -4, -5, -6
KD_ERR_STATE_MISMATCH, KD_ERR_NOMEM, KD_ERR_CANCELLED = -7, -8, -9
KD_FP64, KD_FP32, KD_FP32_TC, KD_DW = 0, 1, 2, 3
KD_HOST, KD_DEVICE = 0, 1
KD_SWEEP_VARIANTS, KD_TUNE_FORCE = 4, 1
KD_FAULT_TC_WAIT, KD_FAULT_PERSIST_HOLD = 1, 2
KD_BATCH_GRAPH, KD_BATCH_PERSISTENT = 0, 1
KD_MLP_FP32, KD_MLP_BF16 = 0, 1


class KdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kd error {code}: {msg}")
        self.code = code


class KdCancelled(KdError):
    """kd_step stopped early at a kd_cancel request; ``obs`` holds the records of the
    steps that ran."""

    def __init__(self, code: int, msg: str, obs: list):
        super().__init__(code, msg)
        self.obs = obs


class kd_units(C.Structure):
    _fields_ = [("m", C.c_double), ("c", C.c_double), ("hbar", C.c_double), ("q", C.c_double)]


class kd_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x_min", C.c_double),
                ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double)]


class kd_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("longitudinal", C.c_int32), ("a0", C.c_double),
                ("k_L", C.c_double), ("epsilon", C.c_double), ("env_T", C.c_double),
                ("phase0", C.c_double), ("p_shift_x", C.c_double), ("p_shift_y", C.c_double),
                ("box_vy", C.c_double)]


class kd_packet(C.Structure):
    _fields_ = [("p0x", C.c_double), ("p0y", C.c_double), ("r0x", C.c_double),
                ("r0y", C.c_double), ("sigma_p", C.c_double), ("spin", C.c_int32),
                ("basis", C.c_int32)]


class kd_obs_spec(C.Structure):
    _fields_ = [("p_in_x", C.c_double), ("p_in_y", C.c_double), ("p_diff_x", C.c_double),
                ("p_diff_y", C.c_double), ("target_x", C.c_double), ("target_y", C.c_double),
                ("half_width", C.c_double), ("basis", C.c_int32), ("pad_", C.c_int32)]


OBS_FIELDS = ["t", "norm", "pop_in", "pop_diff", "cp_in", "cm_in", "cp_diff", "cm_diff",
              "max_diff", "cp_max_diff", "cm_max_diff", "p_target", "cp_target", "cm_target"]


class kd_obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in OBS_FIELDS]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(the CUDA library is the only compute path)")
_lib = C.CDLL(LIB_PATH)

_vp, _P = C.c_void_p, C.POINTER
_SIGS = {
    "kd_create": (C.c_int, [_P(kd_units), _P(kd_grid), _P(kd_field), C.c_int32, _vp, _P(_vp)]),
    "kd_init_packet": (C.c_int, [_vp, _P(kd_packet)]),
    "kd_set_obs_spec": (C.c_int, [_vp, _P(kd_obs_spec)]),
    "kd_set_spinor": (C.c_int, [_vp, _vp, C.c_int32]),
    "kd_get_spinor": (C.c_int, [_vp, _vp, C.c_int32]),
    "kd_set_time": (C.c_int, [_vp, C.c_double]),
    "kd_get_time": (C.c_int, [_vp, _P(C.c_double), _P(C.c_int64)]),
    "kd_step": (C.c_int, [_vp, C.c_double, C.c_int64, C.c_int64, _P(kd_obs), C.c_int64,
                          _P(C.c_int64)]),
    "kd_observe": (C.c_int, [_vp, _P(kd_obs_spec), _P(kd_obs)]),
    "kd_get_momentum_density": (C.c_int, [_vp, C.c_int32, _vp, C.c_int32]),
    "kd_get_density_x": (C.c_int, [_vp, _vp, C.c_int32]),
    "kd_set_watchdog": (C.c_int, [_vp, C.c_double]),
    "kd_get_state": (C.c_int, [_vp, _vp, _P(C.c_size_t)]),
    "kd_set_state": (C.c_int, [_vp, _vp, C.c_size_t]),
    "kd_bench_sweep": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "kd_get_launch_count": (C.c_int, [_vp, _P(C.c_int64)]),
    "kd_autotune": (C.c_int, [_vp, C.c_double, C.c_int32, C.c_int32, _P(C.c_int32), _P(C.c_int32),
                              _P(C.c_float)]),
    "kd_set_sweep_variants": (C.c_int, [_vp, C.c_int32, C.c_int32]),
    "kd_inject_fault": (C.c_int, [_vp, C.c_int32]),
    "kd_cancel": (C.c_int, [_vp]),
    "kd_inject_alloc_failure": (C.c_int, [C.c_int32]),
    "kd_get_sweep_variants": (C.c_int, [_vp, _P(C.c_int32), _P(C.c_int32)]),
    "kd_density_noalloc": (C.c_int, [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                     C.c_double, _vp, _vp, _vp]),
    "kd_batch_create": (C.c_int, [_P(_vp), C.c_int32, _vp, _P(_vp)]),
    "kd_batch_step": (C.c_int, [_vp, _P(C.c_double), C.c_int64, C.c_int64, _P(kd_obs), C.c_int64,
                                _P(C.c_int64)]),
    "kd_batch_destroy": (None, [_vp]),
    "kd_batch_autotune": (C.c_int, [_vp, _P(C.c_double), C.c_int32, _P(C.c_int32)]),
    "kd_batch_set_mode": (C.c_int, [_vp, C.c_int32]),
    "kd_mlp_create": (C.c_int, [_P(C.c_int32), C.c_int32, _P(_vp)]),
    "kd_mlp_num_params": (C.c_int, [_vp, _P(C.c_int64)]),
    "kd_mlp_set_params": (C.c_int, [_vp, _vp, C.c_int32]),
    "kd_mlp_get_params": (C.c_int, [_vp, _vp, C.c_int32]),
    "kd_mlp_forward": (C.c_int, [_vp, _vp, C.c_int32, _vp, C.c_int32, _vp]),
    "kd_mlp_gradients": (C.c_int, [_vp, _vp, _vp, C.c_int32, _vp, _vp, C.c_int32, _vp]),
    "kd_mlp_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_float, _vp, _vp]),
    "kd_mlp_train_step_gather": (C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, C.c_int32, C.c_float, _vp, _vp]),
    "kd_mlp_set_precision": (C.c_int, [_vp, C.c_int32]),
    "kd_mlp_destroy": (None, [_vp]),
    "kd_destroy": (None, [_vp]),
    "kd_last_error": (C.c_char_p, []),
    "kd_version": (C.c_int, []),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn

EXPORTS = list(_SIGS)


def _check(rc: int):
    if rc != KD_OK:
        raise KdError(rc, kd_last_error().decode())


def inject_alloc_failure(after: int):
    """Test hook (``kd_inject_alloc_failure``): the device allocation after ``after``
    further successful ones fails as if the device were out of memory; -1 turns it off."""
    _check(kd_inject_alloc_failure(after))


def _fill(cls, obj):
    s = cls()
    for name, _ in cls._fields_:
        if name != "pad_":
            setattr(s, name, getattr(obj, name))
    return s


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


class Sim:
    """One simulation on the current CUDA device (see ``kd_create``)."""

    def __init__(self, units: W.Units, grid: W.Grid, field: W.Field, precision: int = KD_FP64,
                 stream: int | None = None):
        self.units, self.grid, self.field, self.precision = units, grid, field, precision
        self.cdtype = np.complex128 if precision in (KD_FP64, KD_DW) else np.complex64
        h = _vp()
        _check(kd_create(C.byref(_fill(kd_units, units)), C.byref(_fill(kd_grid, grid)),
                         C.byref(_fill(kd_field, field)), precision,
                         _vp(stream) if stream else None, C.byref(h)))
        self._h = h

    @classmethod
    def from_workload(cls, wl: W.Workload, stream: int | None = None) -> "Sim":
        return cls(wl.units, wl.grid, wl.field, wl.precision, stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            kd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        return (self.grid.ny, self.grid.nx, 4)

    def init_packet(self, packet: W.Packet):
        _check(kd_init_packet(self._h, C.byref(_fill(kd_packet, packet))))

    def set_obs_spec(self, spec: W.ObsSpec):
        _check(kd_set_obs_spec(self._h, C.byref(_fill(kd_obs_spec, spec))))

    def set_spinor(self, psi):
        if _is_torch(psi):
            assert psi.is_contiguous() and tuple(psi.shape) == self.shape
            where = KD_DEVICE if psi.is_cuda else KD_HOST
            _check(kd_set_spinor(self._h, _vp(psi.data_ptr()), where))
        else:
            a = np.ascontiguousarray(psi, dtype=self.cdtype)
            assert a.shape == self.shape
            _check(kd_set_spinor(self._h, a.ctypes.data_as(_vp), KD_HOST))

    def get_spinor(self, out=None):
        if out is not None and _is_torch(out):
            assert out.is_contiguous() and tuple(out.shape) == self.shape
            _check(kd_get_spinor(self._h, _vp(out.data_ptr()), KD_DEVICE if out.is_cuda else KD_HOST))
            return out
        a = np.empty(self.shape, self.cdtype) if out is None else out
        _check(kd_get_spinor(self._h, a.ctypes.data_as(_vp), KD_HOST))
        return a

    def set_time(self, t: float):
        _check(kd_set_time(self._h, t))

    def get_time(self):
        t, n = C.c_double(), C.c_int64()
        _check(kd_get_time(self._h, C.byref(t), C.byref(n)))
        return t.value, n.value

    def step(self, dt: float, nsteps: int, obs_every: int = 0, obs_cap: int | None = None):
        nobs = nsteps // obs_every if obs_every > 0 else 0
        cap = nobs if obs_cap is None else obs_cap
        buf = (kd_obs * max(cap, 1))()
        n = C.c_int64()
        rc = kd_step(self._h, dt, nsteps, obs_every, buf if cap > 0 else None, cap, C.byref(n))
        obs = [{k: getattr(buf[i], k) for k in OBS_FIELDS} for i in range(min(n.value, cap))]
        if rc == KD_ERR_CANCELLED:
            raise KdCancelled(rc, kd_last_error().decode(errors="replace"), obs)
        _check(rc)
        return obs

    def cancel(self):
        """Asks the running (or next) ``step`` to stop at its next chunk boundary
        (``kd_cancel``; callable from another thread)."""
        _check(kd_cancel(self._h))

    def observe(self, spec: W.ObsSpec | None = None) -> dict:
        o = kd_obs()
        _check(kd_observe(self._h, C.byref(_fill(kd_obs_spec, spec)) if spec else None,
                          C.byref(o)))
        return {k: getattr(o, k) for k in OBS_FIELDS}

    def momentum_density(self, basis: int = 0) -> np.ndarray:
        out = np.empty((self.grid.ny, self.grid.nx, 3), np.float64)
        _check(kd_get_momentum_density(self._h, basis, out.ctypes.data_as(_vp), KD_HOST))
        return out

    def density_x(self) -> np.ndarray:
        out = np.empty(self.grid.nx, np.float64)
        _check(kd_get_density_x(self._h, out.ctypes.data_as(_vp), KD_HOST))
        return out

    def set_watchdog(self, tol: float):
        _check(kd_set_watchdog(self._h, tol))

    def bench_sweep(self, kind: int, reps: int):
        _check(kd_bench_sweep(self._h, kind, reps))

    def autotune(self, dt: float, reps: int = 20, force: bool = False) -> dict:
        """Times the launch variants of both sweeps (``kd_autotune``) and applies the
        fastest; returns {"variants": (x, y), "ms": {"x": [...], "y": [...]}} (the recorded
        times when the choice came from the process-wide record; -1 for FP64)."""
        vx, vy = C.c_int32(), C.c_int32()
        ms = (C.c_float * (2 * KD_SWEEP_VARIANTS))()
        _check(kd_autotune(self._h, dt, reps, KD_TUNE_FORCE if force else 0, C.byref(vx),
                           C.byref(vy), ms))
        return {"variants": (vx.value, vy.value),
                "ms": {"x": list(ms[:KD_SWEEP_VARIANTS]), "y": list(ms[KD_SWEEP_VARIANTS:])}}

    @property
    def sweep_variants(self) -> tuple:
        vx, vy = C.c_int32(), C.c_int32()
        _check(kd_get_sweep_variants(self._h, C.byref(vx), C.byref(vy)))
        return vx.value, vy.value

    @sweep_variants.setter
    def sweep_variants(self, v):
        _check(kd_set_sweep_variants(self._h, int(v[0]), int(v[1])))

    def inject_fault(self, kind: int = KD_FAULT_TC_WAIT):
        """Test hooks (``kd_inject_fault``): KD_FAULT_TC_WAIT -- the next ``step`` call's
        tensor-core sweeps issue no matrix products, so their bounded waits run out and
        ``step`` raises KD_ERR_TIMEOUT; KD_FAULT_PERSIST_HOLD -- in the next persistent
        batch step the completion of this member's first work item is never signalled."""
        _check(kd_inject_fault(self._h, kind))

    def launch_count(self) -> int:
        n = C.c_int64()
        _check(kd_get_launch_count(self._h, C.byref(n)))
        return n.value

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _check(kd_get_state(self._h, None, C.byref(n)))
        buf = (C.c_char * n.value)()
        _check(kd_get_state(self._h, buf, C.byref(n)))
        return bytes(buf)

    def set_state(self, blob: bytes):
        buf = (C.c_char * len(blob)).from_buffer_copy(blob)
        _check(kd_set_state(self._h, buf, len(blob)))


class Batch:
    """Several simulations advanced together by one graph launch per chunk of steps
    (``kd_batch_*``)."""

    def __init__(self, sims, stream: int | None = None):
        self.sims = list(sims)
        arr = (_vp * len(self.sims))(*[s.handle for s in self.sims])
        h = _vp()
        _check(kd_batch_create(arr, len(self.sims), _vp(stream) if stream else None, C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            kd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_mode(self, mode: int):
        """KD_BATCH_GRAPH (graph branches) or KD_BATCH_PERSISTENT (one persistent kernel per
        chunk with a device work queue) -- ``kd_batch_set_mode``."""
        _check(kd_batch_set_mode(self._h, mode))

    def autotune(self, dts, steps: int = 20) -> list:
        """Launch variants timed on the whole batch (``kd_batch_autotune``); the members'
        states are unchanged.  Returns [(vx, vy)] per member."""
        n = len(self.sims)
        dt_arr = (C.c_double * n)(*[float(d) for d in dts])
        out = (C.c_int32 * (2 * n))()
        _check(kd_batch_autotune(self._h, dt_arr, steps, out))
        return [(out[2 * i], out[2 * i + 1]) for i in range(n)]

    def step(self, dts, nsteps: int, obs_every: int = 0):
        n = len(self.sims)
        nobs = nsteps // obs_every if obs_every > 0 else 0
        dt_arr = (C.c_double * n)(*[float(d) for d in dts])
        buf = (kd_obs * max(n * nobs, 1))()
        got = C.c_int64()
        _check(kd_batch_step(self._h, dt_arr, nsteps, obs_every, buf if nobs > 0 else None, nobs,
                             C.byref(got)))
        return [[{k: getattr(buf[i * nobs + j], k) for k in OBS_FIELDS} for j in range(nobs)]
                for i in range(n)]


class MLP:
    """The surrogate network (``kd_mlp_*``): widths[0] -> ... -> widths[-1], GELU hidden."""

    def __init__(self, widths):
        self.widths = [int(w) for w in widths]
        arr = (C.c_int32 * len(self.widths))(*self.widths)
        h = _vp()
        _check(kd_mlp_create(arr, len(self.widths) - 1, C.byref(h)))
        self._h = h
        n = C.c_int64()
        _check(kd_mlp_num_params(h, C.byref(n)))
        self.nparam = n.value

    def close(self):
        if getattr(self, "_h", None):
            kd_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: int):
        """KD_MLP_FP32 or KD_MLP_BF16 (tensor-core products) -- ``kd_mlp_set_precision``."""
        _check(kd_mlp_set_precision(self._h, precision))

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        assert a.size == self.nparam
        _check(kd_mlp_set_params(self._h, a.ctypes.data_as(_vp), KD_HOST))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.nparam, np.float32)
        _check(kd_mlp_get_params(self._h, a.ctypes.data_as(_vp), KD_HOST))
        return a

    def forward(self, x) -> np.ndarray:
        xa = np.ascontiguousarray(x, np.float32)
        y = np.empty((xa.shape[0], self.widths[-1]), np.float32)
        _check(kd_mlp_forward(self._h, xa.ctypes.data_as(_vp), xa.shape[0], y.ctypes.data_as(_vp),
                              KD_HOST, None))
        return y

    def gradients(self, x, t):
        xa = np.ascontiguousarray(x, np.float32)
        ta = np.ascontiguousarray(t, np.float32)
        g = np.empty(self.nparam, np.float32)
        loss = np.empty(1, np.float32)
        _check(kd_mlp_gradients(self._h, xa.ctypes.data_as(_vp), ta.ctypes.data_as(_vp), xa.shape[0],
                                loss.ctypes.data_as(_vp), g.ctypes.data_as(_vp), KD_HOST, None))
        return float(loss[0]), g

    def train_step(self, x_dev, t_dev, batch: int, lr: float, loss_dev=None, stream=None):
        """Device pointers (ints, e.g. torch data_ptr())."""
        _check(kd_mlp_train_step(self._h, _vp(x_dev), _vp(t_dev), batch, lr,
                                 _vp(loss_dev) if loss_dev else None, _vp(stream) if stream else None))

    def train_step_gather(self, x_all_dev, t_all_dev, n_all: int, idx_dev, batch: int, lr: float,
                          loss_dev=None, stream=None):
        """Training step on rows idx of the device arrays (gathered by the library)."""
        _check(kd_mlp_train_step_gather(self._h, _vp(x_all_dev), _vp(t_all_dev), n_all, _vp(idx_dev),
                                        batch, lr, _vp(loss_dev) if loss_dev else None,
                                        _vp(stream) if stream else None))
