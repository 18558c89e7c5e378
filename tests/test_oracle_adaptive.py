"""Pins for the oracle's variable time step and step-doubling controller (Sec. 3.2)."""
import numpy as np

from oracle.sbiem import _restore, _snapshot, adaptive_run
from paper_2107_03550_gb300.workloads import rough_cycle, seamount_rupture
from tests.gpu_helpers import oracle_for


def _eps(o, m):
    snap = _snapshot(o)
    assert o.step(m) == 0
    full = o.delta.copy()
    _restore(o, snap)
    assert o.step(m // 2) == 0 and o.step(m // 2) == 0
    e = np.abs(o.delta - full).max()
    _restore(o, snap)
    return e


def test_step_doubling_error_is_third_order():
    # Sec. 3.2: eps = u1 - u2 = (3/4) phi dt^3 for a second-order scheme, so
    # doubling dt multiplies the estimate by about 8 (smooth nucleation phase).
    w = seamount_rupture(N=128, dx=25.0)
    o = oracle_for(w)
    for _ in range(40):
        assert o.step(1) == 0
    e = [_eps(o, m) for m in (4, 8, 16)]
    r1, r2 = e[1] / e[0], e[2] / e[1]
    assert 6.0 < r1 < 10.0, e
    assert 6.0 < r2 < 10.0, e


def test_steady_sliding_doubles_the_step():
    # steady state at the plate rate: no error, the controller doubles dt at
    # every accepted step up to its cap
    w = rough_cycle(N=64, dx=10.0, lam_max=640.0, alpha=0.0)
    o = oracle_for(w)
    st, acc = adaptive_run(o, t_end=1e12, eps0=1e-6, m0=1, m_max=1 << 12, max_steps=16)
    assert st == 0
    assert acc[:13] == [1 << k for k in range(13)]
    assert acc[13:] == [1 << 12] * 3


def test_variable_step_equals_dt_min_steps_when_history_is_constant():
    # with a constant slip rate the history of a step of m dt_min equals m
    # steps of dt_min: the tractions and slip must agree
    w = rough_cycle(N=64, dx=10.0, lam_max=640.0, alpha=3e-3)
    w.prescribed[:] = True
    w.V_presc[:] = 1e-3 * (1 + 0.5 * np.sin(np.arange(64) / 5.0))
    o1 = oracle_for(w)
    o2 = oracle_for(w)
    for _ in range(8):
        assert o1.step(1) == 0
    assert o2.step(8) == 0
    assert np.allclose(o1.delta, o2.delta, rtol=1e-13, atol=0)
    assert np.allclose(o1.last["tau_el"], o2.last["tau_el"], rtol=1e-10,
                       atol=1e-10 * np.abs(o1.last["tau_el"]).max())
