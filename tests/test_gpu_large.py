"""CUDA path vs the FP64 oracle at the large sizes: the FP32 four-step and
16-CTA cluster spectral passes (N = 16384 .. 65536, whole-step parity), the
history sweep at N = 65536 (every mode), and the N = 262144 fault of the
benchmark, where the oracle checks sampled modes and a closed form.

Tolerances as in the other parity tests: FP64 1e-10 relative (max-norm),
FP32 history sums 2e-6, FP32 tractions 1e-4 of the larger traction scale and
1e-4 relative in slip, slip rate and state.
"""
import os

import numpy as np
import pytest

from paper_2107_03550_gb300.workloads import element_x, large_fault, rough_cycle, rough_fault
from tests.gpu_helpers import compare, gpu_for, oracle_for, prefill, rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_03550_gb300 import sbiem
    sbiem.load_library()


def _workload(N):
    # N = 65536: the rough-fault cycle at dx = 2 m (wavelengths 20 m .. 40 km)
    if N == 65536:
        return rough_cycle(N=65536, dx=2.0, seed=3)
    return rough_fault(N, {16384: 10.0, 32768: 4.0}[N], 3e-3, seed=N)


@pytest.mark.parametrize("N,precision", [(16384, 1), (32768, 1), (32768, 0), (65536, 1)])
def test_large_N_steps_match_oracle(N, precision):
    # N = 16384: the FP32 pass on a 16-CTA cluster; N > 16384: the four-step
    # col/row kernels (FP32 and FP64).  Full random history, three steps one
    # call at a time and three in the overlapped graph form.
    w = _workload(N)
    o = oracle_for(w, workers=WORKERS)
    g1 = gpu_for(w, precision=precision)
    g2 = gpu_for(w, precision=precision)
    HT, HN = prefill(o, g1, seed=N + 1, scale=1e-5)
    g2.set_history(HT, HN)
    for _ in range(3):
        assert o.step() == 0
        g1.step()
    g2.enqueue(3)
    assert g2.status()[0] == 0
    scale = max(np.abs(o.last["tau_el"]).max(), np.abs(o.last["sig_el"]).max())
    for g in (g1, g2):
        if precision == 0:
            err = compare(o, g)
            for k in ("delta", "tau_el", "sigma_el", "theta"):
                assert err[k] < TOL64, (k, err)
            assert err["V"] < 1e-9, err
        else:
            s = g.get_state()
            for k, ref in (("tau_el", o.last["tau_el"]), ("sigma_el", o.last["sig_el"])):
                assert np.abs(s[k] - ref).max() < 1e-4 * scale, k
            err = compare(o, g, fields=("delta", "V", "theta"))
            for k in ("delta", "V", "theta"):
                assert err[k] < 1e-4, (k, err)
    g1.close()
    g2.close()


@pytest.mark.parametrize("precision,gen_ds_max,tol", [(0, 0.0, 1e-10), (1, 1.0 / 32, 2e-6), (1, 1.0 / 64, 2e-6),
                                                      (1, 1.0 / 256, 2e-6), (1, 0.0, 2e-6)])
def test_history_sums_every_mode_at_65536(precision, gen_ds_max, tol):
    # the sweep alone on the N = 65536 rings (66 M slots): every mode's sums,
    # FP32 with the weights of the modes up to ds = 1/32 evaluated on chip
    # (eight-lag blocks to 1/64, four-lag blocks above), up to 1/64 (the
    # default), up to 1/256, and of none
    w = _workload(65536)
    o = oracle_for(w, workers=WORKERS)
    g = gpu_for(w, precision=precision)
    sw = g.get_sweep()
    assert sw["gen_ds_max"] == (1.0 / 64 if precision == 1 else 0.0)
    if precision == 1:
        assert 0 < sw["table_err"] < 2e-7
    g.set_sweep(3, gen_ds_max, 0)
    prefill(o, g, seed=17, scale=1e-3)
    for m in (1, 4):
        AT, AN = g.history_sums(m)
        rT, rN = o.history_sums(m)
        assert rel(AT, rT) < tol, (m, rel(AT, rT))
        assert rel(AN, rN) < tol, (m, rel(AN, rN))
    g.close()


def test_autotuner_keeps_results():
    # the autotuner picks shape, weight form and CTAs per SM by timing; the
    # sums (and the step) are those of any form up to FP32 rounding
    w = _workload(16384)
    o = oracle_for(w, workers=WORKERS)
    g = gpu_for(w, precision=1)
    prefill(o, g, seed=19, scale=1e-3)
    before = g.history_sums(1)
    choice = g.tune(reps=3)
    assert choice["shape"] in (3, 4)
    assert choice["ctas_per_sm"] >= 1 and choice["ms"] > 0
    sw = g.get_sweep()
    assert (sw["shape"], sw["gen_ds_max"], sw["ctas_per_sm"]) == (choice["shape"], choice["gen_ds_max"],
                                                                choice["ctas_per_sm"])
    after = g.history_sums(1)
    rT, rN = o.history_sums(1)
    for x, y, r in zip(before, after, (rT, rN)):
        assert rel(y, x) < 1e-6 and rel(y, r) < 2e-6
    g.step()
    assert o.step() == 0
    s = g.get_state()
    scale = max(np.abs(o.last["tau_el"]).max(), np.abs(o.last["sig_el"]).max())
    assert np.abs(s["tau_el"] - o.last["tau_el"]).max() < 1e-4 * scale
    g.close()


SAMPLE_MODES = [1, 17, 31, 32, 33, 500, 4096, 65536, 131071]


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-6)])
def test_history_sums_sampled_at_262144(precision, tol):
    # the benchmark's fault (311 M slots per field, 1,048,575 in each of the
    # modes below the cutting plane): the rings hold seeded random history
    # drawn on the device; the oracle sums the sampled modes from the same
    # values
    import torch
    from oracle import Params
    from oracle.sbiem import history_sums_sampled
    from paper_2107_03550_gb300.workloads import random_history_device
    w = large_fault()
    g = gpu_for(w, precision=precision)
    R = np.maximum(g.windows() - 1, 0)
    hoff = np.concatenate([[0], np.cumsum(R)])
    dt = torch.float64 if precision == 0 else torch.float32
    HT, HN = random_history_device(R, 23, 1e-3, torch, dtype=dt)
    g.set_history_device(HT, HN)
    sT = [HT[hoff[n]:hoff[n + 1]].cpu().numpy().astype(np.complex128) for n in SAMPLE_MODES]
    sN = [HN[hoff[n]:hoff[n + 1]].cpu().numpy().astype(np.complex128) for n in SAMPLE_MODES]
    del HT, HN
    torch.cuda.empty_cache()
    p = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min)
    for m in (1, 2):
        AT, AN = g.history_sums(m)
        rT, rN = history_sums_sampled(p, SAMPLE_MODES, sT, sN, m, workers=WORKERS)
        assert rel(AT[SAMPLE_MODES], rT) < tol, (m, rel(AT[SAMPLE_MODES], rT))
        assert rel(AN[SAMPLE_MODES], rN) < tol, (m, rel(AN[SAMPLE_MODES], rN))
        # per mode as well: the low modes' long windows dominate the max-norm
        for i in range(len(SAMPLE_MODES)):
            assert abs(AT[SAMPLE_MODES[i]] - rT[i]) <= 10 * tol * max(abs(rT[i]), np.abs(rT).max() * 1e-3)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_form_steady_modes_at_262144(precision):
    # The N = 262144, dx = 1 m fault stepped in the benchmark's launch
    # configuration.  Every element slides at a prescribed
    # V = sum_q Va_q cos(q x + phi_q) over sampled modes q, on a fault of
    # constant curvature k0, and each sampled mode's history holds that
    # spectrum over its whole window (as if V had held for T_w).  Then, with
    # zero slip at the start of the step, the spectral formulas of Sec. 3.1
    # give in closed form (shear: -|k| on cos gives -q cos; normal:
    # -i sgn(k) on cos gives sin):
    #   tau_el = sum_q -q Va_q cos(q x + phi_q) [S dt + mu sum_{j<M_q} w^T_{q,j}]
    #   sig_el = sum_q  k0 Va_q sin(q x + phi_q) [S dt + mu sum_{j<M_q} w^N_{q,j}]
    # with the oracle's weights of the sampled modes.
    import torch
    from oracle import Params
    from oracle.sbiem import weights, windows
    from paper_2107_03550_gb300.sbiem import Fault
    w = large_fault()
    N, dx = w.N, w.dx
    p = Params(N=N, dx=dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min)
    x = element_x(N, dx)
    rng = np.random.default_rng(5)
    modes = [1, 31, 40, 4096, 131071]
    Va = rng.uniform(1e-4, 1e-3, len(modes))
    phi = rng.uniform(0, 2 * np.pi, len(modes))
    k0 = 2e-4
    V = np.zeros(N)
    for q, a, f in zip(modes, Va, phi):
        V += a * np.cos(2 * np.pi * q / (N * dx) * x + f)
    w.kappa = np.full(N, k0)
    w.prescribed = np.ones(N, dtype=bool)
    w.V_presc = V.copy()
    w.V_init = V.copy()
    w.tau_load = np.zeros(N)
    Vhat = np.fft.rfft(V)          # the index-based DFT the library uses
    M = windows(p)
    wT, wN, woff = weights(p, M, modes=modes, workers=WORKERS)
    R = np.maximum(M - 1, 0)
    hoff = np.concatenate([[0], np.cumsum(R)])
    S, mu, dt = p.S, p.mu, p.dt_min
    tau = np.zeros(N)
    sig = np.zeros(N)
    for i, q in enumerate(modes):
        WT = wT[woff[q]:woff[q + 1]].sum()
        WN = wN[woff[q]:woff[q + 1]].sum()
        arg = 2 * np.pi * q / (N * dx) * x + phi[i]
        tau += -(2 * np.pi * q / (N * dx)) * Va[i] * np.cos(arg) * (S * dt + mu * WT)
        sig += k0 * Va[i] * np.sin(arg) * (S * dt + mu * WN)
    scale = max(np.abs(tau).max(), np.abs(sig).max())
    tol = TOL64 if precision == 0 else 1e-4
    dtype = torch.float64 if precision == 0 else torch.float32
    for form in ("step", "graph"):
        g = Fault.from_workload(w, precision=precision)
        HT = torch.zeros(int(R.sum()), 2, dtype=dtype, device="cuda")
        HN = torch.zeros_like(HT)
        for q in modes:
            v = torch.tensor([Vhat[q].real, Vhat[q].imag], dtype=dtype, device="cuda")
            HT[hoff[q]:hoff[q + 1]] = v
            HN[hoff[q]:hoff[q + 1]] = k0 * v
        g.set_history_device(HT, HN)
        del HT, HN
        if form == "step":
            g.step()
        else:
            g.enqueue(1)
            assert g.status()[0] == 0
        s = g.get_state()
        assert np.abs(s["tau_el"] - tau).max() < tol * scale, (form, np.abs(s["tau_el"] - tau).max() / scale)
        assert np.abs(s["sigma_el"] - sig).max() < tol * scale, (form, np.abs(s["sigma_el"] - sig).max() / scale)
        assert np.abs(s["delta"] - V * dt).max() <= 1e-12 * np.abs(V * dt).max()
        g.close()
        torch.cuda.empty_cache()


def test_autotuner_undoes_its_timed_steps_at_32768():
    # With the four-kernel passes (N > 16384) the autotuner also times real
    # overlapped steps and undoes each (state snapshot, overwritten ring slot
    # put back): the committed state and the history after tuning are those
    # before, bitwise, and the tuned handle then steps bitwise like a fresh
    # handle given the same history and the tuner's setting.
    w = _workload(32768)
    g = gpu_for(w, precision=1)
    R = np.maximum(g.windows() - 1, 0)
    from paper_2107_03550_gb300.workloads import random_history
    HT, HN, _ = random_history(R, 29, 1e-5)
    g.set_history(HT, HN)
    s0 = g.get_state()
    h0 = g.get_history()
    choice = g.tune(reps=2)
    s1 = g.get_state()
    h1 = g.get_history()
    for k in ("delta", "V", "theta", "t"):
        assert np.array_equal(s0[k], s1[k]), k
    for a, b in zip(h0, h1):
        assert np.array_equal(a, b)
    g2 = gpu_for(w, precision=1)
    g2.set_history(HT, HN)
    g2.set_sweep(choice["shape"], choice["gen_ds_max"], choice["ctas_per_sm"])
    g.enqueue(3)
    g2.enqueue(3)
    assert g.status()[0] == 0 and g2.status()[0] == 0
    a, b = g.get_state(), g2.get_state()
    for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
        assert np.array_equal(a[k], b[k]), k
    g.close()
    g2.close()
