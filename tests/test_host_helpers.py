"""Host-side helpers of the studies and the surrogate (no GPU): the power-law fit, the
read-out bookkeeping of the studies, and the surrogate's error report."""
import numpy as np

from paper_2307_01571_gb300 import studies, surrogate


def test_fit_slope_recovers_power_laws():
    x = np.array([0.01, 0.02, 0.05, 0.1])
    assert abs(studies.fit_slope(x, 3.0 * x ** -2) + 2.0) < 1e-12
    assert abs(studies.fit_slope(x, 0.5 * x ** 2) - 2.0) < 1e-12
    assert abs(studies.fit_slope(x, np.full(4, 7.0))) < 1e-12


def test_studies_bookkeeping_with_synthetic_readouts(monkeypatch):
    # read-outs ~ (k/eps)^2 for the longitudinal component off, times (1 + 1e-3 eps^2) on:
    # the fitted E3 exponents are 2 / -2 / 2 and the on-off difference goes as eps^2 k^2
    def fake(kd, wls, stream=None):
        out = []
        for w in wls:
            e, k, lo = w.extra["eps"], w.extra["k_nat"], w.extra["longitudinal"]
            v = (k / e) ** 2 * 1e-6 * (1.0 + 1e-3 * lo * e ** 2)
            out.append({**{f: v for f in studies.FORMS}, "norm": 1.0})
        return out
    monkeypatch.setattr(studies, "execute", fake)
    r = studies.studies(None)
    s = r["e3_slopes"]["cm_target"]
    assert abs(s["vs_kL_over_eps"] - 2.0) < 1e-3
    assert all(abs(v + 2.0) < 1e-3 for v in s["vs_eps"].values())
    assert all(abs(v - 2.0) < 1e-3 for v in s["vs_kL"].values())
    assert abs(r["e4_slopes_vs_eps"]["hp_d_cm_diff"]) < 1e-6     # (k/eps)^2 eps^2: flat in eps
    assert len(r["e4"]) == len(studies.EPSILONS)
    assert all(row["fp32_err_cm_diff_on"] == 0.0 for row in r["e4"])


def test_surrogate_error_report_and_worst_cases():
    truth = np.zeros((10, 4))
    pred = np.zeros((10, 4))
    pred[3, 0] = 1.5
    pred[7, 0] = -0.5
    pred[:, 2] = 0.1
    params = np.arange(50, dtype=float).reshape(10, 5)
    e = surrogate.heldout_error(pred, truth)
    assert abs(e["log10_P_in"]["max"] - 1.5) < 1e-15
    assert abs(e["log10_P_in"]["rms"] - np.sqrt((1.5 ** 2 + 0.5 ** 2) / 10)) < 1e-15
    assert abs(e["log10_P_bragg_same_spin"]["rms"] - 0.1) < 1e-15
    w = surrogate.worst_cases(pred, truth, params, k=2)
    assert [c["params"]["w0_lambda"] for c in w["log10_P_in"]] == [15.0, 35.0]
    assert w["log10_P_in"][0]["pred"][0] == 1.5 and w["log10_P_in"][0]["truth"][0] == 0.0


def test_issue_bound_reads_the_committed_counts_only_for_the_current_source():
    import bench
    counts = {k: bench.ncu_instructions(k, f) for k, f in (("x_sweep", "fp32"), ("y_sweep", "fp32"))}
    r = bench.roofline_issue("fp32", {"x_sweep": 0.0131, "y_sweep": 0.0131}, 2070.0, 152)
    assert abs(r["peak"] - 4 * 152 * 2070e6) < 1.0
    for k, inst in counts.items():
        got = r["kernels"][k]
        if inst is None:   # counts taken on another kernel source: not reported
            assert got["frac"] is None
        else:
            assert got["warp_instructions_per_launch"] == inst
            assert abs(got["frac"] - inst / (0.0131e-3 * r["peak"])) < 1e-12
            assert abs(got["time_at_full_issue_us"] - inst / r["peak"] * 1e6) < 1e-9
    # launch variants other than the profiled ones: no count
    r2 = bench.roofline_issue("fp32", {"x_sweep": 0.0131}, 2070.0, 152, profiled_variants=False)
    assert r2["kernels"]["x_sweep"]["frac"] is None
