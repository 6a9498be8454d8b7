"""Runs a few fused sweeps on the 1024x512 benchmark grid so that a profiler can capture
them in isolation:

    python -m paper_2307_01571_gb300.prof_sweeps PRECISION KIND REPS

PRECISION 0 = FP64, 1 = FP32, 2 = FP32 with the tensor-core sweeps (x axis of this grid);
KIND 0 = x sweep, 1 = y sweep.  The simulation is created (one warm-up launch of every
sweep shape), initialised with the benchmark packet, advanced 2 Strang steps, and then
``kd_bench_sweep(KIND, REPS)`` runs REPS back-to-back full sweeps on the default launch
variants.  For the FP32/FP64 sweep kernels (ncu ``-k regex:sweep_kernel``) the benchmarked
launches are numbers 14 .. 13 + REPS; for the tensor-core kernel (``-k regex:tc_sweep``)
numbers 3 .. 2 + REPS.
"""
import sys

from . import kd
from . import workloads as W


def main(argv):
    prec = int(argv[0]) if argv else 1
    kind = int(argv[1]) if len(argv) > 1 else 0
    reps = int(argv[2]) if len(argv) > 2 else 4
    wl = W.c2(precision=prec, nsteps=2)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        sim.step(wl.dt, 2)
        sim.bench_sweep(kind, reps)
        sim.get_time()
    print("ok", prec, kind, reps)


if __name__ == "__main__":
    main(sys.argv[1:])
