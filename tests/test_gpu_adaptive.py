"""Variable time steps (dt = m dt_min) and the step-doubling run (Sec. 3.2):
CUDA path vs the FP64 oracle through the C ABI."""
import numpy as np
import pytest

from oracle.sbiem import adaptive_run
from paper_2107_03550_gb300.workloads import rough_cycle, seamount_rupture
from tests.gpu_helpers import compare, gpu_for, oracle_for, prefill

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_step_lengths_match_oracle(precision):
    # steps of 1, 2, 4, 3, 16, 5 dt_min: multi-slot pushes, current-interval
    # weights from the power-of-two table and from the direct sum
    w = seamount_rupture(N=256)
    o = oracle_for(w)
    g = gpu_for(w, precision=precision)
    prefill(o, g, seed=3, scale=1e-6)
    for m in (1, 2, 4, 3, 16, 5, 64, 1):
        assert o.step(m) == 0
        g.step(m * g.dt_min)
        err = compare(o, g)
        if precision == 0:
            for k in ("delta", "tau_el", "sigma_el", "theta"):
                assert err[k] < 1e-10, (m, k, err)
        else:
            # FP32 form: FFT rounding is relative to the largest spectral
            # coefficient, shared by shear and normal traction, so both are
            # measured against the larger of the two traction scales
            s = g.get_state()
            scale = max(np.abs(o.last["tau_el"]).max(), np.abs(o.last["sig_el"]).max())
            for k, ref in (("tau_el", o.last["tau_el"]), ("sigma_el", o.last["sig_el"])):
                assert np.abs(s[k] - ref).max() < 1e-4 * scale, (m, k, err)
            for k in ("delta", "theta"):
                assert err[k] < 1e-4, (m, k, err)
    hT, hN = g.get_history()
    HT, HN = o.get_history()
    assert np.abs(hT - np.concatenate(HT)).max() <= (1e-12 if precision == 0 else 1e-6) * np.abs(hT).max()
    g.close()


def test_steps_longer_than_every_window():
    # m larger than every ring: all slots hold the step's spectra
    w = rough_cycle(N=128, dx=10.0, lam_max=1280.0)
    o = oracle_for(w)
    g = gpu_for(w)
    for m in (1, 4096, 8192, 1):
        assert o.step(m) == 0
        g.step(m * g.dt_min)
    err = compare(o, g)
    for k in ("delta", "V", "theta"):
        assert err[k] < 1e-10, (k, err)
    # near-uniform sliding: the traction change is a small remainder of the
    # static term S |k| F[delta]; bound the difference by its rounding scale
    st = g.get_state()
    scale = o.p.S * (2 * np.pi * (w.N // 2) / (w.N * w.dx)) * np.abs(o.delta).max()
    assert np.abs(st["tau_el"] - o.last["tau_el"]).max() < 1e-12 * scale
    assert np.abs(st["sigma_el"] - o.last["sig_el"]).max() < 1e-12 * scale
    g.close()


def test_adaptive_run_matches_oracle():
    w = rough_cycle(N=128, dx=10.0, lam_max=1280.0, alpha=3e-3)
    o = oracle_for(w)
    g = gpu_for(w)
    eps0 = 1e-3 * 1e-3
    st, acc_o = adaptive_run(o, t_end=1e9, eps0=eps0, m0=1, m_max=1 << 30, max_steps=40)
    acc_g, m_next, t_g, code = g.run(t_end=1e9, eps0=eps0, m0=1, m_max=1 << 30, max_steps=40)
    assert st == 0 and code == 0
    assert acc_g == acc_o
    assert abs(t_g - o.t) <= 1e-12 * o.t
    err = compare(o, g, fields=("delta", "V", "theta"))
    assert err["delta"] < 1e-9 and err["theta"] < 1e-9, err
    assert err["V"] < 1e-8, err
    g.close()


def test_adaptive_run_rejects_and_recovers():
    # a rupture from a strong nucleation patch forces rejections; the state
    # after each rejection is restored exactly, so the run matches the oracle
    w = seamount_rupture(N=256)
    o = oracle_for(w)
    g = gpu_for(w)
    eps0 = 1e-3 * 1e-3
    st, acc_o = adaptive_run(o, t_end=1e9, eps0=eps0, m0=64, max_steps=30)
    acc_g, m_next, t_g, code = g.run(t_end=1e9, eps0=eps0, m0=64, max_steps=30)
    assert st == 0 and code == 0
    assert acc_g == acc_o
    err = compare(o, g, fields=("delta", "V", "theta"))
    assert err["delta"] < 1e-9, err
    g.close()


def test_run_output_callback_samples_and_stops():
    # the output callback of sbiem_run: called after every 4th accepted step
    # and the last one, with the committed slip and slip rate of that step;
    # a True return stops the run after that step
    w = seamount_rupture(N=256)
    g = gpu_for(w)
    calls = []

    def out(step, t, m, delta, V):
        calls.append((step, t, m, delta, V))
        return False

    g.set_output(out, every=4)
    hist, m_next, t, rc = g.run(t_end=1e9, eps0=1e-6, m0=1, max_steps=18)
    assert rc == 0 and len(hist) == 18
    assert [c[0] for c in calls] == [4, 8, 12, 16, 18]
    assert [c[2] for c in calls] == [hist[k - 1] for k in (4, 8, 12, 16, 18)]
    s = g.get_state()
    assert np.array_equal(calls[-1][3], s["delta"]) and np.array_equal(calls[-1][4], s["V"])
    assert calls[-1][1] == pytest.approx(s["t"], rel=1e-14)
    g.close()
    # stopping: the run ends after the step whose callback returned True
    g = gpu_for(w)
    g.set_output(lambda step, t, m, d, V: step >= 7, every=1)
    hist, _, _, rc = g.run(t_end=1e9, eps0=1e-6, m0=1, max_steps=50)
    assert rc == 0 and len(hist) == 7
    g.set_output(None)
    hist, _, _, rc = g.run(t_end=1e9, eps0=1e-6, m0=1, max_steps=3)
    assert rc == 0 and len(hist) == 3
    g.close()
