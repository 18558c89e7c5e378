"""CPU tests of host-side analysis code: the cycle driver's slip/curvature
scaling fit (Sec. "Scaling of slip distribution versus fault geometry") and
the bench's reader of recorded ncu traffic."""
import os

import numpy as np

from paper_2107_03550_gb300.cycle import scaling_fit
from paper_2107_03550_gb300.workloads import element_x, sinusoidal_cycle


def _law_slip(w, f, scale=1.0):
    # (1/(f du)) d(du)/dx = -kappa with kappa = -A q^2 sin(qx):
    # ln du = -f A q cos(qx) + (crack-shaped profile over the fault)
    x = element_x(w.N, w.dx)
    Lf = w.extra["fault_length"]
    q = 2 * np.pi / w.extra["wavelength"]
    crack = np.sqrt(np.clip(1 - (2 * x / Lf) ** 2, 1e-12, None))
    return x, Lf, np.where(np.abs(x) < Lf / 2, scale * crack * np.exp(-f * w.extra["amp"] * q * np.cos(q * x)), 0.0)


def test_scaling_fit_recovers_the_law_under_a_rupture_profile():
    w = sinusoidal_cycle()
    x, Lf, du = _law_slip(w, 0.6)
    fit = scaling_fit(du, w.kappa, x, Lf, 0.6)
    assert abs(fit["slope"] - 1.0) < 0.02 and fit["corr"] > 0.999
    # the rupture-scale profile spoils the raw (un-detrended) fit
    assert fit["raw_corr"] < 0.6


def test_scaling_fit_is_scale_free_and_sees_the_sign():
    w = sinusoidal_cycle()
    x, Lf, du = _law_slip(w, 0.6, scale=3.7)
    assert abs(scaling_fit(du, w.kappa, x, Lf, 0.6)["slope"] - 1.0) < 0.02
    # slip modulated the wrong way round (ln du = +f A q cos qx) fits with slope -1
    _, _, du_flip = _law_slip(w, -0.6)
    assert abs(scaling_fit(du_flip, w.kappa, x, Lf, 0.6)["slope"] + 1.0) < 0.02


def test_bench_reads_recorded_traffic_only_for_the_current_sweep_source(tmp_path, monkeypatch):
    # a profile of a smaller fault of the same family is scaled by ring slots
    import bench
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_sweep_source_sha", lambda: "0123456789abcdef")
    path = os.path.join(str(tmp_path), "profiles", "k_sweep_fp32_large_N65536.md")
    body = ("# k_sweep\n\n- k_sweep source sha256[:16]: {}\n- workload family: large\n- ring slots: 1000\n"
            "- dram bytes per launch: 16000\n")
    with open(path, "w") as fh:
        fh.write(body.format("0123456789abcdef"))
    t = bench._traffic("fp32", "large", 4000)
    assert t["bytes"] == 64000.0 and t["scaled_by_slots"] == 4.0
    assert bench._traffic("fp32", "rough", 4000) is None
    assert bench._traffic("fp64", "large", 4000) is None
    with open(path, "w") as fh:
        fh.write(body.format("fedcba9876543210"))
    assert bench._traffic("fp32", "large", 4000) is None
