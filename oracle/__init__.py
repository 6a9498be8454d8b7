"""Plain FP64 CPU oracle for the 2D Dirac FFT split-operator step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The product path (the CUDA
library and its binding) never imports it, and it imports nothing from the product.

The arithmetic lives in ``kd_oracle.c`` (see its header for the paper passages and
the readings it implements).  This module only compiles it with gcc and marshals
numpy arrays.  Parameter objects are duck-typed: anything with the attribute names
of the C structs works.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kd_oracle.c")
_HDR = os.path.join(_HERE, "kd_oracle.h")
_LIB = os.path.join(_HERE, "libkd_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libkd_oracle_omp.so")   # timing variant: rows/columns on threads
_lock = threading.Lock()
_lib = None
_use_omp = False


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile ``libkd_oracle.so`` beside the source (FP64, no fast-math, no FMA contraction);
    with openmp=True the OpenMP timing variant ``libkd_oracle_omp.so`` (same source, the
    independent rows, columns and grid points on several threads, identical results)."""
    out = _LIB_OMP if openmp else _LIB
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def use_openmp(on: bool) -> None:
    """Route the calls below to the OpenMP timing variant (on) or the plain build (off)."""
    global _lib, _use_omp
    with _lock:
        if on != _use_omp:
            _use_omp = on
            _lib = None


class Units(C.Structure):
    _fields_ = [("m", C.c_double), ("c", C.c_double), ("hbar", C.c_double), ("q", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x_min", C.c_double),
                ("x_max", C.c_double), ("y_min", C.c_double), ("y_max", C.c_double)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("longitudinal", C.c_int32), ("a0", C.c_double),
                ("k_L", C.c_double), ("epsilon", C.c_double), ("env_T", C.c_double),
                ("phase0", C.c_double), ("p_shift_x", C.c_double), ("p_shift_y", C.c_double),
                ("box_vy", C.c_double)]


class Packet(C.Structure):
    _fields_ = [("p0x", C.c_double), ("p0y", C.c_double), ("r0x", C.c_double),
                ("r0y", C.c_double), ("sigma_p", C.c_double), ("spin", C.c_int32),
                ("basis", C.c_int32)]


class ObsSpec(C.Structure):
    _fields_ = [("p_in_x", C.c_double), ("p_in_y", C.c_double), ("p_diff_x", C.c_double),
                ("p_diff_y", C.c_double), ("target_x", C.c_double), ("target_y", C.c_double),
                ("half_width", C.c_double), ("basis", C.c_int32), ("pad_", C.c_int32)]


OBS_FIELDS = ["t", "norm", "pop_in", "pop_diff", "cp_in", "cm_in", "cp_diff", "cm_diff",
              "max_diff", "cp_max_diff", "cm_max_diff", "p_target", "cp_target", "cm_target"]


class Obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in OBS_FIELDS]


_P = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build(openmp=_use_omp))
            sig = {
                "or_fft1d": [_P, C.c_int32, C.c_int32],
                "or_fft2d": [_P, C.c_int32, C.c_int32, C.c_int32],
                "or_field_a": [C.POINTER(Units), C.POINTER(Field), C.c_double, C.c_double,
                               C.c_double, _P, _P],
                "or_init_packet": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field),
                                   C.POINTER(Packet), _P],
                "or_potential_step": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field), _P,
                                      C.c_double, C.c_double],
                "or_kinetic_step": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field), _P,
                                    C.c_double],
                "or_step": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field), _P, C.c_double,
                            C.c_double, C.c_int64],
                "or_observe": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field),
                               C.POINTER(ObsSpec), _P, C.c_double, C.POINTER(Obs)],
                "or_momentum_density": [C.POINTER(Units), C.POINTER(Grid), C.POINTER(Field),
                                        C.c_int32, _P, _P],
                "or_density_x": [C.POINTER(Grid), _P, _P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            for name, args in {
                "or_dirac_matrices": [_P, _P, _P],
                "or_potential_factor": [C.POINTER(Units), C.c_double, C.c_double, C.c_double, _P],
                "or_kinetic_factor": [C.POINTER(Units), C.c_double, C.c_double, C.c_double, _P],
                "or_spinor_u": [C.POINTER(Units), C.c_double, C.c_double, C.c_int32, C.c_int32,
                                _P],
                "or_momentum": [C.POINTER(Grid), C.POINTER(Units), C.POINTER(Field), C.c_int32,
                                C.c_int32, _P, _P],
            }.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = None
            _lib = L
    return _lib


def _fill(cls, obj):
    s = cls()
    for name, _ in cls._fields_:
        if name == "pad_":
            continue
        setattr(s, name, getattr(obj, name))
    return s


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _cplx(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def fft1d(a, sign: int) -> np.ndarray:
    out = _cplx(a).copy()
    _check(lib().or_fft1d(_ptr(out), out.size, sign), "fft1d")
    return out


def fft2d(psi, sign: int) -> np.ndarray:
    out = _cplx(psi).copy()
    ny, nx, nc = out.shape
    assert nc == 4
    _check(lib().or_fft2d(_ptr(out), nx, ny, sign), "fft2d")
    return out


def dirac_matrices():
    ax = np.zeros((4, 4), np.complex128)
    ay = np.zeros((4, 4), np.complex128)
    b = np.zeros((4, 4), np.complex128)
    lib().or_dirac_matrices(_ptr(ax), _ptr(ay), _ptr(b))
    return ax, ay, b


def field_a(units, field, x: float, y: float, t: float):
    ax, ay = C.c_double(), C.c_double()
    _check(lib().or_field_a(C.byref(_fill(Units, units)), C.byref(_fill(Field, field)),
                            x, y, t, C.byref(ax), C.byref(ay)), "field_a")
    return ax.value, ay.value


def potential_factor(units, ax: float, ay: float, tau: float) -> np.ndarray:
    M = np.zeros((4, 4), np.complex128)
    lib().or_potential_factor(C.byref(_fill(Units, units)), ax, ay, tau, _ptr(M))
    return M


def kinetic_factor(units, pix: float, piy: float, dt: float) -> np.ndarray:
    M = np.zeros((4, 4), np.complex128)
    lib().or_kinetic_factor(C.byref(_fill(Units, units)), pix, piy, dt, _ptr(M))
    return M


def spinor_u(units, pix: float, piy: float, spin: int, basis: int = 0) -> np.ndarray:
    v = np.zeros(4, np.complex128)
    lib().or_spinor_u(C.byref(_fill(Units, units)), pix, piy, spin, basis, _ptr(v))
    return v


def momentum(grid, units, field, kx: int, ky: int):
    a, b = C.c_double(), C.c_double()
    lib().or_momentum(C.byref(_fill(Grid, grid)), C.byref(_fill(Units, units)),
                      C.byref(_fill(Field, field)), kx, ky, C.byref(a), C.byref(b))
    return a.value, b.value


def init_packet(units, grid, field, packet) -> np.ndarray:
    psi = np.zeros((grid.ny, grid.nx, 4), np.complex128)
    _check(lib().or_init_packet(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                                C.byref(_fill(Field, field)), C.byref(_fill(Packet, packet)),
                                _ptr(psi)), "init_packet")
    return psi


def potential_step(units, grid, field, psi, t: float, tau: float) -> np.ndarray:
    out = _cplx(psi).copy()
    _check(lib().or_potential_step(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                                   C.byref(_fill(Field, field)), _ptr(out), t, tau),
           "potential_step")
    return out


def kinetic_step(units, grid, field, phi, dt: float) -> np.ndarray:
    out = _cplx(phi).copy()
    _check(lib().or_kinetic_step(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                                 C.byref(_fill(Field, field)), _ptr(out), dt), "kinetic_step")
    return out


def step(units, grid, field, psi, t0: float, dt: float, nsteps: int) -> np.ndarray:
    out = _cplx(psi).copy()
    _check(lib().or_step(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                         C.byref(_fill(Field, field)), _ptr(out), t0, dt, nsteps), "step")
    return out


def observe(units, grid, field, spec, psi, t: float) -> dict:
    o = Obs()
    a = _cplx(psi)
    _check(lib().or_observe(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                            C.byref(_fill(Field, field)), C.byref(_fill(ObsSpec, spec)),
                            _ptr(a), t, C.byref(o)), "observe")
    return {n: getattr(o, n) for n in OBS_FIELDS}


def momentum_density(units, grid, field, psi, basis: int = 0) -> np.ndarray:
    a = _cplx(psi)
    out = np.zeros((grid.ny, grid.nx, 3), np.float64)
    _check(lib().or_momentum_density(C.byref(_fill(Units, units)), C.byref(_fill(Grid, grid)),
                                     C.byref(_fill(Field, field)), basis, _ptr(a), _ptr(out)),
           "momentum_density")
    return out


def density_x(grid, psi) -> np.ndarray:
    a = _cplx(psi)
    out = np.zeros(grid.nx, np.float64)
    _check(lib().or_density_x(C.byref(_fill(Grid, grid)), _ptr(a), _ptr(out)), "density_x")
    return out
