"""Earthquake cycle on the sinusoidal fault (Sec. "Seismic cycles") with the
adaptive step-doubling solver (Sec. 3.2), and the slip-versus-geometry
scaling of Sec. "Scaling of slip distribution versus fault geometry" on its
final slip.

    python -m paper_2107_03550_gb300.cycle [--events 3] [--years 400] [--precision 1]
                                           [--workload sinusoidal|rough]

(rough: the rough-fault cycle, Hurst-1 roughness with the outer 30 % of the
fault creeping at the plate rate, N = 4096, dx = 10 m.)

Prints one JSON line: simulated time, accepted steps and their step lengths,
the events (peak slip rate above 1e-2 m/s), wall time and element-steps/s,
and the scaling fit.  The scaling (Romanet et al. 2020) relates the scaled
slip gradient to the curvature, (1 / (f du)) d(du)/dx = -kappa: the fit is
the least-squares slope and the correlation of the left side against -kappa
over the inner 60 % of the fault (the relation does not hold near the
fault's edges, as the paper notes), after a smooth trend is removed from
both sides.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .sbiem import Fault
from .workloads import element_x, rough_cycle, sinusoidal_cycle


def scaling_fit(delta: np.ndarray, kappa: np.ndarray, x: np.ndarray, fault_length: float, f: float,
                inner: float = 0.6, trend_degree: int = 3) -> dict:
    """Slope and correlation of (1/(f du)) d(du)/dx against -kappa over the inner part of the fault.

    Both sides first lose their least-squares polynomial trend in x (degree
    trend_degree): the rupture-scale shape of the slip (a crack profile, a
    nucleation-side bias) is smooth over the fault, the geometric term
    varies with the profile's wavelength.  The raw fit is reported too.
    """
    dx = x[1] - x[0]
    grad = np.gradient(delta, dx)
    sel = (np.abs(x) < 0.5 * inner * fault_length) & (delta > 0)
    lhs = grad[sel] / (f * delta[sel])
    rhs = -kappa[sel]
    xi = x[sel] / (0.5 * inner * fault_length)
    P = np.vander(xi, trend_degree + 1)
    detrend = lambda y: y - P @ np.linalg.lstsq(P, y, rcond=None)[0]
    rl, rr = detrend(lhs), detrend(rhs)
    return {"slope": float(np.dot(rl, rr) / np.dot(rr, rr)), "corr": float(np.corrcoef(rl, rr)[0, 1]),
            "raw_slope": float(np.dot(lhs, rhs) / np.dot(rhs, rhs)), "raw_corr": float(np.corrcoef(lhs, rhs)[0, 1]),
            "points": int(sel.sum()), "trend_degree": trend_degree}


def run_cycle(events: int = 3, years: float = 400.0, precision: int = 1, eps0: float = 1e-7,
              chunk: int = 200, max_steps: int = 400_000, w=None) -> dict:
    w = w or sinusoidal_cycle()
    g = Fault.from_workload(w, precision=precision)
    x = element_x(w.N, w.dx)
    fault = ~w.prescribed  # the frictional part of the fault
    fault_length = float(fault.sum() * w.dx)
    t_end = years * 365.25 * 86400.0
    m = 1
    steps = 0
    m_hist: list[int] = []
    found: list[dict] = []
    in_event = False
    vmax_trace = []
    stop = "events reached" if events else ""
    t0 = time.perf_counter()
    t = 0.0
    while t < t_end and steps < max_steps and (len(found) < events or in_event):
        hist, m, t, rc = g.run(t_end, eps0, m0=m, max_steps=chunk)
        steps += len(hist)
        m_hist += hist
        if rc != 0:
            # SBIEM_ERR_DTMIN: a step failed at dt_min (state kept at its start);
            # the library's message carries the failing step's status bits
            msg = g.lib.sbiem_last_error().decode()
            bits = int(msg.split("status bits ")[1].split(")")[0]) if "status bits " in msg else 0
            why = [n for b, n in ((1, "Newton cap"), (2, "opening"), (4, "state")) if bits & b]
            stop = f"code {rc} at t = {t:.6g} s ({', '.join(why) or msg})"
            break
        s = g.get_state()
        vmax = float(s["V"][fault].max())
        vmax_trace.append((t, vmax))
        if not in_event and vmax > 1e-2:
            in_event = True
            found.append({"t_years": t / (365.25 * 86400.0), "x_km": float(x[fault][np.argmax(s["V"][fault])] / 1e3)})
        if in_event:
            found[-1]["peak_V"] = max(found[-1].get("peak_V", 0.0), vmax)
            if vmax < 1e-6:
                in_event = False
                found[-1]["slip_m"] = float(s["delta"][fault].mean())
        if not hist:
            stop = "no step accepted"
            break
    else:
        stop = ("events reached" if len(found) >= events and not in_event
                else ("t_end" if t >= t_end else "max_steps"))
    wall = time.perf_counter() - t0
    s = g.get_state()
    fit = scaling_fit(s["delta"], w.kappa, x, fault_length, w.f0)
    mh = np.asarray(m_hist)
    out = {
        "workload": w.name, "precision": precision, "eps0_m": eps0,
        "t_years": s["t"] / (365.25 * 86400.0), "accepted_steps": int(steps),
        "steps_at_dt_min": int((mh == 1).sum()), "largest_m": int(mh.max()) if mh.size else 0,
        "events": found, "stopped": stop, "wall_s": wall, "element_steps_per_s": w.N * steps / wall,
        "mean_slip_m": float(s["delta"][fault].mean()),
        "scaling": fit,
    }
    g.close()
    return out


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--events", type=int, default=3)
    ap.add_argument("--years", type=float, default=400.0)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--eps0", type=float, default=1e-7, help="step-doubling slip tolerance (m)")
    ap.add_argument("--max-steps", type=int, default=400_000)
    ap.add_argument("--workload", choices=["sinusoidal", "rough"], default="sinusoidal")
    a = ap.parse_args()
    w = sinusoidal_cycle() if a.workload == "sinusoidal" else rough_cycle()
    print(json.dumps(run_cycle(a.events, a.years, a.precision, a.eps0, max_steps=a.max_steps, w=w)), flush=True)


if __name__ == "__main__":
    main()
