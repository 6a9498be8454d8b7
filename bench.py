#!/usr/bin/env python
"""Benchmark of the FFT split-operator step (arXiv 2307.01571, Sec. II.D) on GB300.

Workload (one bench step): the Gaussian-beam standing wave with its longitudinal
component on a 1024 x 512 grid (40 x 40 wavelengths, co-moving box, waist 10
wavelengths), 2000 Strang steps with observables every 100 steps, through the public C
ABI (kd_step).  Metric: spinor grid-point-steps/s; the FP32 form is the headline
``value`` and the FP64 form is reported beside it.  Inputs are synthetic (the paper's
packet and field parameters) and resident in HBM when the timed region starts; L2 is
flushed (a 256 MiB write) between timed bench steps.

``--impl reference`` times the CPU oracle (the plain FP64 C implementation) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_01571_gb300 import workloads as W  # noqa: E402

METRIC = "spinor grid-point-steps/s"
UNIT = "grid-point-steps/s"
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes per grid point per Strang step: two read+write sweeps of the
# four-component spinor (x sweep and y sweep)
BYTES_PER_PT_STEP = {"fp32": 2 * 2 * 4 * 8, "fp64": 2 * 2 * 4 * 16, "dw": 2 * 2 * 4 * 16}
BYTES_PER_PT_SWEEP = {"fp32": 2 * 4 * 8, "fp64": 2 * 4 * 16, "dw": 2 * 4 * 16}
# FP64 FMA peak of one GB300 (the recipe's nominal 1.25 TFLOP/s; an FMA-chain probe
# measured 1.256): the FP64 sweeps are bound by this pipe, not by HBM
FP64_PEAK_TFLOPS = 1.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--strang", type=int, default=2000, help="Strang steps per bench step")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-surrogate", action="store_true")
    p.add_argument("--no-tc", action="store_true", help="skip the tensor-core precision form")
    p.add_argument("--no-hbm", action="store_true", help="skip the HBM-resident 4096x2048 grid")
    p.add_argument("--no-dw", action="store_true", help="skip the double-word (FP64-accurate) form")
    p.add_argument("--profile-persist", default=None, metavar="N,CHUNK",
                   help="run the persistent batch kernel on N runs for a profiler")
    p.add_argument("--profile-mlp", default=None, metavar="BATCH,STEPS",
                   help="run the BF16 tensor-core surrogate training for a profiler")
    p.add_argument("--profile-sweep", default=None, metavar="PREC,KIND,REPS[,GRID]",
                   help="profiling mode: build the GRID workload (1024x512 default, or 4096x2048), "
                        "step it twice, then run REPS back-to-back sweeps of KIND (0 x, 1 y) at "
                        "precision PREC (0 FP64, 1 FP32, 2 tensor-core form) on the default "
                        "launch variants, and exit")
    p.add_argument("--sweep-variants", default=None,
                   help="X,Y: launch variants of the FP32 sweeps instead of the autotuner's choice "
                        "(a profiler distorts the tuner's timings)")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_01571_gb300", "csrc")
    for f in ("kd_sweep.cuh", "kd_sweep_f32.cu", "kd_sweep_f64.cu", "kd_internal.h", "kd_dw.cuh",
              "kd_sweep_dw.cu"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, form: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d[f"{kernel}_{form}"]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


def ncu_instructions(kernel: str, form: str):
    """Warp instructions per launch from the committed ncu summary (smsp__inst_executed.sum),
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            e = json.load(fh)[f"{kernel}_{form}"]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return e.get("warp_instructions_per_launch")
    except Exception:
        return None


def roofline_issue(form: str, sweep_ms: dict, sm_mhz, sms: int, profiled_variants: bool = True) -> dict:
    """The sweeps against their instruction-issue bound: warp instructions per launch (ncu)
    over the launch time, against one warp instruction per clock per scheduler (four per
    SM) at the SM clock sampled during the timed region.  The bound says how close a
    kernel is to what its instruction count allows, whatever memory it moves."""
    peak = 4.0 * sms * (sm_mhz or 0.0) * 1e6
    out = {"bound": "issue", "unit": "warp instructions/s", "peak": peak,
           "peak_source": f"4 schedulers x {sms} SMs x {sm_mhz} MHz (sampled)", "kernels": {}}
    for kern, ms in sweep_ms.items():
        # the counts were taken on the default launch variants (bench.py --profile-sweep)
        inst = ncu_instructions(kern, form) if profiled_variants else None
        if inst is None or not peak:
            out["kernels"][kern] = {"warp_instructions_per_launch": None, "frac": None}
            continue
        ach = inst / (ms * 1e-3)
        out["kernels"][kern] = {"warp_instructions_per_launch": inst, "achieved": ach,
                                "frac": ach / peak, "launch_ms": round(ms, 5),
                                "time_at_full_issue_us": inst / peak * 1e6}
    return out


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid: str | None):
        self.proc = None
        import tempfile
        fd, self.out = tempfile.mkstemp(prefix="kd_clocks_", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if dev_uuid:
            cmd += ["-i", dev_uuid]
        try:
            self.fh = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.out) as fh:
            lines = fh.readlines()
        os.remove(self.out)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms_local: float, points_per_rank: float, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    points_per_rank grid-point-steps; the job time is the slowest rank's (max over ranks).
    Returns (grid-point-steps/s, job ms)."""
    import torch
    ms = float(ms_local)
    world = 1
    if dist is not None and dist.is_initialized():
        t = torch.tensor([ms], dtype=torch.float64, device=device or "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        world = dist.get_world_size()
    return points_per_rank * world / (ms * 1e-3), ms


def host_info() -> dict:
    """Core count and CPU model of the host the oracle ran on."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                key = ln.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.machine()
    return {"nproc": os.cpu_count(), "cpu": model}


def oracle_rate(wl, nsteps: int):
    """The CPU oracle as it stands, single-threaded, on nsteps Strang steps of wl's grid."""
    import oracle
    u, g, f, pk = wl.units, wl.grid, wl.field, wl.packet
    psi = oracle.init_packet(u, g, f, pk)
    t0 = time.perf_counter()
    psi = oracle.step(u, g, f, psi, 0.0, wl.dt, nsteps)
    dt = time.perf_counter() - t0
    return wl.points * nsteps / dt, dt, psi


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = W.c2(precision=W.FP64)
    per = 2  # Strang steps of the 1024x512 grid per bench step (about 1 s of CPU work)
    for _ in range(args.warmup):
        oracle_rate(wl, 1)
    total_t, total_pts = 0.0, 0
    for _ in range(args.steps):
        r, dt, _ = oracle_rate(wl, per)
        total_t += dt
        total_pts += wl.points * per
    v = total_pts / total_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.ny],
                   "strang_steps_per_step": per, "parallelism": "cpu oracle, 1 thread"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_info(),
                         "sample": f"{per} Strang steps of the 1024x512 FP64 run per bench step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def batched_form(kd, stream, K, barrier, dist):
    """Config 4: 64 independent seeded Gaussian-beam runs on mixed grids (128x128 to
    512x256, FP32) advanced by kd_batch_step (one graph launch per 100-step chunk, the
    runs as concurrent branches), against the same runs one after the other."""
    import torch
    members = W.c4()
    pts = sum(w.points for w in members) * members[0].nsteps
    sims = [kd.Sim.from_workload(w, stream=stream.cuda_stream) for w in members]
    chosen = {}
    for s_, w in zip(sims, members):
        s_.init_packet(w.packet)
        # launch variants per grid shape (timed once per shape, then looked up)
        chosen[f"{w.grid.nx}x{w.grid.ny}"] = s_.autotune(w.dt, reps=50)["variants"]
    dts = [w.dt for w in members]
    res = {"sweep_variants": chosen}
    with kd.Batch(sims, stream=stream.cuda_stream) as b:
        # launch variants timed on the batch as a whole (members' states are kept)
        bv = b.autotune(dts, steps=20)
        res["sweep_variants_batch"] = {f"{w.grid.nx}x{w.grid.ny}": v for w, v in zip(members, bv)}
        b.step(dts, members[0].nsteps, obs_every=100)           # warm-up: graphs captured
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            b.step(dts, members[0].nsteps, obs_every=100)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / K
    # every member after warm-up + K runs in the graph form, to check the persistent form
    psi_graph = [s_.get_spinor() for s_ in sims]
    # the persistent form: one kernel per chunk with a device work queue (fixed variants)
    for s_, w in zip(sims, members):
        s_.init_packet(w.packet)
    with kd.Batch(sims, stream=stream.cuda_stream) as b:
        b.set_mode(kd.KD_BATCH_PERSISTENT)
        pv = b.autotune(dts, steps=20)                           # x variants, work item size
        res["persistent_variants"] = {f"{w.grid.nx}x{w.grid.ny}": v for w, v in zip(members, pv)}
        b.step(dts, members[0].nsteps, obs_every=100)           # warm-up: graphs captured
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            b.step(dts, members[0].nsteps, obs_every=100)
        e1.record(stream)
        e1.synchronize()
        ms_p = e0.elapsed_time(e1) / K
    # same runs, same step count: the two forms differ only in launch variants (rounding)
    diff_p = max(float(np.max(np.abs(s_.get_spinor() - g)) / np.max(np.abs(g)))
                 for s_, g in zip(sims, psi_graph))
    del psi_graph
    for s_, w in zip(sims, members):                           # the same runs one by one,
        s_.autotune(w.dt)                                      # on the variants tuned alone
        s_.step(w.dt, w.nsteps, obs_every=100)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_, w in zip(sims, members):
        s_.step(w.dt, w.nsteps, obs_every=100)
    e1.record(stream)
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for s_ in sims:
        s_.close()
    value, ms = aggregate(ms, pts, dist, "cuda")
    res.update({"value": value, "unit": UNIT, "ms_per_step": ms, "steps": K, "sims": len(members),
                "workload": "64 seeded Gaussian-beam runs, grids 128x128..512x256, c64, "
                            "2000 steps, observations every 100",
                "sequential_value": pts / (ms_seq * 1e-3),
                "speedup_vs_sequential": ms_seq / ms,
                "persistent": {"value": pts / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p,
                               "form": "one persistent kernel per 100-step chunk, device work queue of "
                                       "(step, sweep, member, block group) items, bounded waits",
                               "over_graph_branches": ms / ms_p,
                               "max_rel_diff_vs_graph_form": diff_p}})
    return res


def precision_form(kd, stream, with_oracle: bool):
    """Precision form on the 2048x1024 grid: the 1024-point (y) sweeps as tensor-core DFT
    products (KD_FP32_TC), the 2048-point (x) sweeps on the CUDA cores, against the FP32
    CUDA-core form on the same run; error of both against the oracle after 2 Strang steps."""
    import torch
    wl = W.c3(precision=W.FP32_TC)
    res = {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.ny]}
    for prec, name in ((W.FP32_TC, "tc"), (W.FP32, "fp32")):
        w = wl.with_(precision=prec)
        sim = kd.Sim.from_workload(w, stream=stream.cuda_stream)
        sim.init_packet(w.packet)
        sim.autotune(w.dt)
        n0 = sim.observe()["norm"]
        sim.step(w.dt, w.nsteps, obs_every=w.obs_every)      # warm-up (graphs captured)
        sim.init_packet(w.packet)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        obs = sim.step(w.dt, w.nsteps, obs_every=w.obs_every)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sweep = {}
        for kind, nm in ((0, "x_sweep"), (1, "y_sweep")):
            sim.bench_sweep(kind, 100)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.bench_sweep(kind, 100)
            b.record(stream)
            b.synchronize()
            sweep[nm] = round(a.elapsed_time(b) / 100, 5)
        sim.close()
        res[name] = {"value": w.points * w.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms,
                     "norm_drift": max(abs(o["norm"] - n0) for o in obs), "launch_ms": sweep}
    res["tc_over_fp32"] = res["tc"]["value"] / res["fp32"]["value"]
    if with_oracle:
        wlo = wl.with_(precision=W.FP64, nsteps=2)
        _, _, ref = oracle_rate(wlo, 2)
        errs = {}
        for prec, name in ((W.FP32_TC, "tc"), (W.FP32, "fp32")):
            sim = kd.Sim.from_workload(wlo.with_(precision=prec), stream=stream.cuda_stream)
            sim.init_packet(wlo.packet)
            sim.step(wlo.dt, 2)
            got = sim.get_spinor().astype(np.complex128)
            sim.close()
            errs[name] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        errs.update({"strang_steps": 2, "measure": "max|psi-psi_oracle|/max|psi_oracle|"})
        res["error_vs_oracle"] = errs
    return res


def full_run_errors(kd, stream, precisions):
    """Error of the benchmark run itself (1024x512, 2000 Strang steps, observations every
    100) against the oracle's stored record of the same run (tests/golden/c2_long_oracle.json,
    written by tests/golden/make_long_runs.py from the oracle alone), at its 256 sampled
    points, relative to the oracle's max |psi|."""
    path = os.path.join(ROOT, "tests", "golden", "c2_long_oracle.json")
    try:
        with open(path) as fh:
            rec = [r for r in json.load(fh)["records"] if r["steps"] == 2000][0]
    except Exception:
        return None
    pts = np.array(rec["points_yx"])
    ref = np.array(rec["psi"])
    ref = ref[..., 0] + 1j * ref[..., 1]
    out = {}
    for prec, name in precisions:
        wl = W.c2(precision=prec)
        sim = kd.Sim.from_workload(wl, stream=stream.cuda_stream)
        sim.init_packet(wl.packet)
        obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
        got = sim.get_spinor()[pts[:, 0], pts[:, 1], :].astype(np.complex128)
        sim.close()
        out[name] = {"psi": float(np.max(np.abs(got - ref)) / rec["max_abs_psi"]),
                     "pop_diff": abs(obs[-1]["pop_diff"] - rec["obs"]["pop_diff"]) / rec["obs"]["pop_diff"],
                     "cm_target": abs(obs[-1]["cm_target"] - rec["obs"]["cm_target"]) / max(rec["obs"]["cm_target"], 1e-300)}
    out.update({"strang_steps": 2000, "points": len(pts),
                "measure": "max|psi-psi_oracle|/max|psi_oracle| at the record's points; relative read-out errors"})
    return out


def surrogate_form(n_runs: int = 4096):
    """Config 5: the MLP surrogate (5 -> 3 x 256 GELU -> 4) trained by the library's own
    kernels on n_runs batched-solver runs (seeded uniform draws, 256x128, 2000 steps),
    90/10 split; held-out error in log10 decades and time per prediction vs per run."""
    from paper_2307_01571_gb300 import surrogate as S
    X = S.draw_params(n_runs, seed=1)
    Y, secs = S.solve(X, batch=512)
    n_tr = int(0.9 * n_runs)
    sur = S.Surrogate(seed=0)
    t_fit = sur.fit(X[:n_tr], Y[:n_tr], steps=4000, batch=256, lr=2e-3)
    pred = sur.predict(X[n_tr:])
    t0 = time.perf_counter()
    for _ in range(20):
        sur.predict(X[n_tr:])
    t_pred = (time.perf_counter() - t0) / (20 * (n_runs - n_tr))
    err = S.heldout_error(pred, Y[n_tr:])
    base = S.heldout_error(np.tile(Y[:n_tr].mean(0), (n_runs - n_tr, 1)), Y[n_tr:])
    # the same network trained with BF16 tensor-core products
    from paper_2307_01571_gb300 import kd
    s16 = S.Surrogate(seed=0, precision=kd.KD_MLP_BF16)
    t_fit16 = s16.fit(X[:n_tr], Y[:n_tr], steps=4000, batch=256, lr=2e-3)
    err16 = S.heldout_error(s16.predict(X[n_tr:]), Y[n_tr:])
    return {"runs": n_runs, "train": n_tr, "heldout": n_runs - n_tr,
            "solver_s_per_run_batched": secs / n_runs, "train_s": t_fit,
            "predict_s_per_sample": t_pred, "speedup_vs_solver": secs / n_runs / t_pred,
            "heldout_rms_log10": {k: v["rms"] for k, v in err.items()},
            "bf16_tensor_core": {"train_s": t_fit16,
                                 "heldout_rms_log10": {k: v["rms"] for k, v in err16.items()},
                                 "heldout_max_log10": {k: v["max"] for k, v in err16.items()}},
            "heldout_max_log10": {k: v["max"] for k, v in err.items()},
            "heldout_worst": S.worst_cases(pred, Y[n_tr:], X[n_tr:], k=3),
            "constant_predictor_rms_log10": {k: v["rms"] for k, v in base.items()}}


def profile_sweep(spec: str):
    """Runs a few fused sweeps in isolation for a profiler.  The simulation is created (one
    warm-up launch of every sweep shape), initialised with the workload's packet and
    advanced 2 Strang steps; then kd_bench_sweep(KIND, REPS) runs REPS back-to-back full
    sweeps (for the FP32/FP64 sweep kernels, ncu -k regex:sweep_kernel, the benchmarked
    launches are numbers 14 .. 13 + REPS; for the tensor-core kernel, -k regex:tc_sweep,
    numbers 3 .. 2 + REPS)."""
    from paper_2307_01571_gb300 import kd
    f = spec.split(",")
    prec, kind, reps = int(f[0]), int(f[1]), int(f[2])
    grid = f[3] if len(f) > 3 else "1024x512"
    wl = {"1024x512": W.c2, "2048x1024": W.c3, "4096x2048": W.hbm}[grid](precision=prec, nsteps=2)
    with kd.Sim.from_workload(wl) as sim:
        sim.init_packet(wl.packet)
        sim.step(wl.dt, 2)
        sim.bench_sweep(kind, reps)
        sim.get_time()
    print("ok", prec, kind, reps, grid)


def profile_persist(spec: str):
    """The persistent batch kernel for a profiler: the first N runs of the 64-run batch
    (FP32, launch variants fixed at the radix-4 pair (2, 2) that the tuner picks for these
    grids), advanced in the persistent form by two calls of CHUNK steps, one launch of
    k_persist each (ncu -k regex:k_persist -s 1 -c 1 captures the second)."""
    from paper_2307_01571_gb300 import kd
    n, chunk = (int(v) for v in spec.split(","))
    members = W.c4()[:n]
    sims = [kd.Sim.from_workload(w) for w in members]
    for s_, w in zip(sims, members):
        s_.sweep_variants = (2, 2)
        s_.init_packet(w.packet)
    with kd.Batch(sims) as b:
        b.set_mode(kd.KD_BATCH_PERSISTENT)
        for _ in range(2):
            b.step([w.dt for w in members], chunk, obs_every=chunk)
    for s_ in sims:
        s_.get_time()
        s_.close()
    print("ok persistent", n, chunk)


def profile_mlp(spec: str):
    """The surrogate network's BF16 tensor-core GEMMs for a profiler: STEPS training steps
    of the 5 -> 3 x 256 -> 4 network on BATCH seeded rows (each step: 4 forward, 7 backward
    GEMMs of k_gemm_bf16)."""
    import torch
    from paper_2307_01571_gb300 import kd, surrogate as S
    batch, steps = (int(v) for v in spec.split(","))
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal((batch, S.WIDTHS[0])).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((batch, S.WIDTHS[-1])).astype(np.float32)).cuda()
    net = kd.MLP(S.WIDTHS)
    net.set_precision(kd.KD_MLP_BF16)
    net.set_params(S.he_init(S.WIDTHS, 0))
    for _ in range(steps):
        net.train_step(x.data_ptr(), t.data_ptr(), batch, 1e-3)
    torch.cuda.synchronize()
    net.get_params()
    net.close()
    print("ok mlp", batch, steps)


def hbm_resident(kd, stream, hbm_peak, hbm_src, flush, tuned):
    """FP32 step on a grid whose state does not fit in L2 (4096x2048, 256 MiB spinor plus
    a 64 MiB kinetic table): 200 Strang steps with observations every 100, and each sweep
    timed alone (back-to-back launches), with the roofline of the slower sweep."""
    import torch
    wl = W.hbm(precision=W.FP32)
    sim = kd.Sim.from_workload(wl, stream=stream.cuda_stream)
    sim.init_packet(wl.packet)
    tune = tuned(sim, wl.dt)
    sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)          # warm-up (graphs captured)
    sim.init_packet(wl.packet)
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    sweep = {}
    for kind, nm in ((0, "x_sweep"), (1, "y_sweep")):
        sim.bench_sweep(kind, 20)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.bench_sweep(kind, 20)
        b.record(stream)
        b.synchronize()
        sweep[nm] = a.elapsed_time(b) / 20
    sim.close()
    kern = max(sweep, key=sweep.get)
    byts = BYTES_PER_PT_SWEEP["fp32"] * wl.points
    ach = byts / (sweep[kern] * 1e-3) / 1e9
    return {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.ny], "dtype": "f32",
            "value": wl.points * wl.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_run": ms,
            "sweep_variants": tune["variants"],
            "roofline": {"bound": "hbm", "kernel": kern, "achieved": ach, "peak": hbm_peak,
                         "peak_source": hbm_src, "unit": "GB/s", "frac": ach / hbm_peak,
                         "traffic": ncu_traffic(f"{kern}_4096x2048", "fp32"),
                         "algorithmic_bytes_per_launch": byts,
                         "launch_ms": {k: round(v, 5) for k, v in sweep.items()}},
            "l2": "state 320 MiB > 129 MiB L2: every sweep streams from HBM"}


def main():
    args = parse()
    if args.profile_sweep:
        return profile_sweep(args.profile_sweep)
    if args.profile_persist:
        return profile_persist(args.profile_persist)
    if args.profile_mlp:
        return profile_mlp(args.profile_mlp)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2307_01571_gb300 import kd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    dev_uuid = f"GPU-{uuid}" if uuid else None
    hbm, hbm_src = peaks()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def tuned(sim, dt):
        if args.sweep_variants and sim.precision in (W.FP32, W.FP32_TC):
            v = tuple(int(x) for x in args.sweep_variants.split(","))
            sim.sweep_variants = v
            return {"variants": v, "ms": {"x": [], "y": []}, "pinned": True}
        return sim.autotune(dt, reps=50)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_form(prec: int, K: int, Wm: int, clocks: bool):
        wl = W.c2(precision=prec, nsteps=args.strang)
        sim = kd.Sim.from_workload(wl, stream=stream.cuda_stream)
        sim.init_packet(wl.packet)
        tune = tuned(sim, wl.dt)               # launch variants of both sweeps (untimed)
        n0 = sim.observe()["norm"]
        start = n0
        for _ in range(Wm):
            ow = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
            start = ow[-1]["norm"] if ow else start
        barrier()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        stops = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ck = Clocks(dev_uuid) if clocks else None
        l0 = sim.launch_count()
        obs = []
        runs = []
        for i in range(K):
            flush.zero_()
            starts[i].record(stream)
            obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
            stops[i].record(stream)
            runs.append(obs)
        barrier()
        launches = sim.launch_count() - l0
        ck_res = ck.stop() if ck else None
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, stops))
        _, ms = aggregate(ms, 0.0, dist, "cuda")
        # norm drift within each timed run of wl.nsteps steps (the bar is per run), and over
        # everything this simulation ran since its packet was set
        drift = None
        if obs:
            per_run = []
            for r in runs:
                per_run.append(max(abs(o["norm"] - start) for o in r))
                start = r[-1]["norm"]
            drift = {"per_run_max": max(per_run), "since_start": max(abs(o["norm"] - n0) for o in obs),
                     "steps_per_run": wl.nsteps, "runs_since_start": Wm + K}
        # dominant-kernel timing: back-to-back launches of each fused sweep
        sweep_ms = {}
        for kind, name in ((0, "x_sweep"), (1, "y_sweep")):
            reps = 200
            sim.bench_sweep(kind, reps)      # captures the replay graph (untimed)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.bench_sweep(kind, reps)
            e1.record(stream)
            e1.synchronize()
            sweep_ms[name] = e0.elapsed_time(e1) / reps
        sim.close()
        return wl, ms, launches, ck_res, drift, sweep_ms, tune

    def e2e_form(prec: int, K: int):
        wl = W.c2(precision=prec, nsteps=args.strang)
        sim = kd.Sim.from_workload(wl, stream=stream.cuda_stream)
        sim.init_packet(wl.packet)
        tuned(sim, wl.dt)                                 # the recorded choice (no timing)
        host_in = torch.from_numpy(sim.get_spinor()).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)
        barrier()
        t0 = time.perf_counter()
        obs = []
        for _ in range(K):
            sim.set_spinor(host_in)                       # H2D from pinned host memory
            obs = sim.step(wl.dt, wl.nsteps, obs_every=wl.obs_every)   # D2H of observables
            sim.get_spinor(host_out)                      # D2H of the final spinor
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sim.close()
        nb = host_in.numel() * host_in.element_size()
        obs_b = len(obs) * 14 * 8
        return wl.points * wl.nsteps * K / dt, nb, nb + obs_b

    def roofline_alu(wl, sweep_ms):
        # algorithmic FP64 flops per launch: the two 1D FFTs of every line and component
        # in the 5 N log2 N convention (the potential and kinetic factors not counted)
        kern = max(sweep_ms, key=sweep_ms.get)
        n, lines = (wl.grid.nx, wl.grid.ny) if kern == "x_sweep" else (wl.grid.ny, wl.grid.nx)
        flops = 2 * 4 * lines * 5.0 * n * np.log2(n)
        ach = flops / (sweep_ms[kern] * 1e-3) / 1e12
        return {"bound": "alu", "kernel": kern, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "peak_source": "nominal FP64 (1.25 TFLOP/s; 1.256 measured by an FMA probe)",
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "algorithmic_flops_per_launch": flops,
                "launch_ms": {k: round(v, 5) for k, v in sweep_ms.items()}}

    def roofline(form, wl, sweep_ms, hbm_peak):
        kern = max(sweep_ms, key=sweep_ms.get)
        b = BYTES_PER_PT_SWEEP[form] * wl.points
        ach = b / (sweep_ms[kern] * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": kern, "achieved": ach, "peak": hbm_peak,
                "peak_source": hbm_src, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": ncu_traffic(kern, form),
                "algorithmic_bytes_per_launch": b,
                "launch_ms": {k: round(v, 5) for k, v in sweep_ms.items()}}

    K, Wm = args.steps, max(3, args.warmup)
    wl, ms, launches, clk, drift, sweep_ms, tune = timed_form(W.FP32, K, Wm, True)
    pts = wl.points * wl.nsteps * K * world
    value = pts / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "grid": [wl.grid.nx, wl.grid.ny],
                   "strang_steps_per_step": wl.nsteps, "obs_every": wl.obs_every,
                   "l2": "flushed between timed steps (256 MiB write); the 20 MiB spinor and "
                         "tables stay L2-resident inside a step",
                   "parallelism": f"replicas x{world}",
                   "sweep_variants": {"chosen": tune["variants"], "pinned": tune.get("pinned", False),
                                      "us_per_launch": {k: [round(1e3 * m, 2) for m in v]
                                                        for k, v in tune["ms"].items()}}},
        "roofline": roofline("fp32", wl, sweep_ms, hbm),
        "gpu_launches": launches,
        "clocks": clk,
        "norm_drift_fp32": drift,
    }
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    line["roofline_issue"] = roofline_issue("fp32", sweep_ms, (clk or {}).get("sm_mhz"), sms,
                                            tuple(tune["variants"]) == (0, 0))
    e2e_v, bi, bo = e2e_form(W.FP32, K)
    line["e2e"] = {"value": e2e_v * world, "unit": UNIT, "h2d_bytes_per_step": bi,
                   "d2h_bytes_per_step": bo}
    if not args.no_fp64:
        K64 = max(1, min(K, 3))
        wl64, ms64, l64, _, drift64, sw64, _ = timed_form(W.FP64, K64, 3, False)
        v64 = wl64.points * wl64.nsteps * K64 * world / (ms64 * 1e-3)
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / K64, "steps": K64,
                        "norm_drift": drift64, "speedup_fp32_over_fp64": value / v64,
                        "roofline": roofline_alu(wl64, sw64),
                        "roofline_hbm": roofline("fp64", wl64, sw64, hbm), "gpu_launches": l64}
    if not args.no_dw:
        Kd = max(1, min(K, 3))
        wld, msd, ld, _, driftd, swd, _ = timed_form(W.DW, Kd, 3, False)
        vd = wld.points * wld.nsteps * Kd * world / (msd * 1e-3)
        line["dw"] = {"value": vd, "unit": UNIT, "ms_per_step": msd / Kd, "steps": Kd,
                      "dtype": "f32 pairs (double-word, 48-bit significand)",
                      "norm_drift": driftd, "gpu_launches": ld,
                      "roofline_hbm": roofline("dw", wld, swd, hbm),
                      "roofline_issue": roofline_issue("dw", swd, (line.get("clocks") or {}).get("sm_mhz"), sms)}
        if "fp64" in line:
            line["dw"]["speedup_over_fp64"] = vd / line["fp64"]["value"]
    if rank == 0 and not args.no_tc:
        line["precision_form"] = precision_form(kd, stream, not args.no_cpu)
        if "fp64" in line:
            # rates per grid-point-step of different grids: the precision form on 2048x1024,
            # the FP64 step on 1024x512
            line["precision_form"]["speedup_tc_2048x1024_vs_fp64_1024x512"] = (
                line["precision_form"]["tc"]["value"] / line["fp64"]["value"])
    if rank == 0 and not args.no_hbm:
        line["hbm_resident"] = hbm_resident(kd, stream, hbm, hbm_src, flush, tuned)
    if not args.no_batch:
        line["batched"] = batched_form(kd, stream, max(1, min(K, 3)), barrier, dist)
        if "fp64" in line:
            line["batched"]["speedup_vs_fp64_single"] = line["batched"]["value"] / line["fp64"]["value"]
    if rank == 0 and not args.no_surrogate:
        line["surrogate"] = surrogate_form()
    if rank == 0 and not args.no_cpu:
        # error of both forms against the oracle on the same grid (4 Strang steps), and the
        # oracle's own rate on that sample
        wlc = W.c2(precision=W.FP64, nsteps=4)
        r, dt, ref = oracle_rate(wlc, 4)
        errs = {}
        for prec, name in ((W.FP32, "fp32"), (W.FP64, "fp64"), (W.DW, "dw")):
            if (prec == W.FP64 and args.no_fp64) or (prec == W.DW and args.no_dw):
                continue
            s = kd.Sim.from_workload(wlc.with_(precision=prec), stream=stream.cuda_stream)
            s.init_packet(wlc.packet)
            s.step(wlc.dt, 4)
            got = s.get_spinor().astype(np.complex128)
            s.close()
            errs[name] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        line["error_vs_oracle"] = {**errs, "strang_steps": 4, "measure": "max|psi-psi_oracle|/max|psi_oracle|"}
        forms = [(W.FP32, "fp32")] + ([] if args.no_fp64 else [(W.FP64, "fp64")]) + \
                ([] if args.no_dw else [(W.DW, "dw")]) + ([] if args.no_tc else [(W.FP32_TC, "fp32_tc")])
        fr = full_run_errors(kd, stream, forms)
        if fr:
            line["error_vs_oracle"]["full_run"] = fr
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"4 Strang steps of the 1024x512 FP64 run ({dt:.1f} s)",
                                "host": host_info()}
        # the same oracle source built with OpenMP (independent rows, columns and points on
        # every host core; identical results), on the same sample
        import oracle
        oracle.use_openmp(True)
        try:
            r_omp, dt_omp, _ = oracle_rate(wlc, 32)
        finally:
            oracle.use_openmp(False)
        line["cpu_baseline_openmp"] = {"value": r_omp, "unit": UNIT, "cores": os.cpu_count(),
                                       "kind": "oracle, OpenMP over rows, columns and grid points",
                                       "sample": f"32 Strang steps of the 1024x512 FP64 run ({dt_omp:.1f} s)",
                                       "speedup_over_one_core": r_omp / r}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
