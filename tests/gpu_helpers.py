"""Shared helpers of the GPU parity tests: build the oracle and the CUDA path
from the same seeded workload and compare their outputs."""
import numpy as np

from oracle import Oracle, Params
from paper_2107_03550_gb300.workloads import Workload, random_history


def oracle_for(w: Workload, **kw) -> Oracle:
    p = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min,
               state_law=kw.pop("state_law", "analytic"), kc_L=kw.pop("kc_L", 200.0),
               kc_units=kw.pop("kc_units", "rad"), eta_w=kw.pop("eta_w", 1.0), kcN_L=kw.pop("kcN_L", 0.0),
               quadrature=kw.pop("quadrature", "midpoint"))
    return Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, w.tau_load, w.V_init,
                  w.theta_init, tau_load_rate=w.tau_load_rate,
                  prescribed=w.prescribed if np.any(w.prescribed) else None,
                  V_presc=w.V_presc if np.any(w.prescribed) else None, workers=kw.pop("workers", 1))


def gpu_for(w: Workload, **kw):
    from paper_2107_03550_gb300.sbiem import Fault
    return Fault.from_workload(w, **kw)


def rel(a, b) -> float:
    """max |a - b| / max |b| (norm-wise relative difference)."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max()
    if scale == 0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / scale)


def prefill(o: Oracle, g, seed: int, scale: float = 1e-9):
    """Same seeded history in both: flat arrays for the GPU, per-mode lists for the oracle."""
    M = g.windows()
    assert np.array_equal(M, o.M)
    R = np.maximum(M - 1, 0)
    HT, HN, off = random_history(R, seed, scale)
    g.set_history(HT, HN)
    o.set_history([HT[off[n]:off[n + 1]] for n in range(R.size)],
                  [HN[off[n]:off[n + 1]] for n in range(R.size)])
    return HT, HN


def compare(o: Oracle, g, fields=("delta", "V", "theta", "tau_el", "sigma_el")) -> dict:
    s = g.get_state()
    ref = {"delta": o.delta, "V": o.V, "theta": o.theta, "tau_el": o.last.get("tau_el"),
           "sigma_el": o.last.get("sig_el")}
    return {k: rel(s[k], ref[k]) for k in fields if ref[k] is not None}
