"""GB300-native FFT split-operator step for the 2D Dirac equation in a standing light wave.

Ge, Ahrens & Shen, "Two-dimensional simulation of the spin-flip in the Kapitza-Dirac
effect" (arXiv 2307.01571), Sec. II.D: the Strang-split FFT split-operator time step of
the four-component Dirac spinor, with the Gaussian-beam potential of Sec. II.A and the
observables of Sec. III.

The compute path is the CUDA library ``libkd.so`` (C ABI declared in ``include/kd.h``);
``paper_2307_01571_gb300.kd`` is its thin ctypes binding.  ``workloads`` holds parameter
sets and seeded inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "kd"]


def __getattr__(name):
    if name == "kd":
        import importlib
        return importlib.import_module(__name__ + ".kd")
    raise AttributeError(name)
