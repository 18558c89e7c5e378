"""Train the learned Newton initial guess and measure what it gains.

    python -m paper_2107_03550_gb300.train_guess train [--rows 10000000] [--out PATH]
    python -m paper_2107_03550_gb300.train_guess compare [--params PATH] [--years 0.3]

train: harvest (ln V_prev, ln theta, tau/sigma, a, b, ln V*) rows from the
method's own solves on two families of runs, then fit the 5-64-64-1 network
with the library's GPU training (sbiem_mlp_train: Adam on the mean squared
error of the normalized residual ln V* - ln V_prev):
  * the rough-fault cycle (N = 4096, dx = 10 m, Hurst-1 alpha = 0.005,
    central 70 % rate-and-state, outer 30 % at the plate rate), run by the
    adaptive step-doubling solver (Sec. 3.2) from steady state through its
    first rupture;
  * rough-fault ruptures of the ensemble's sizes (N = 1024 .. 8192,
    dx = 10 m, alpha ~ U[0.001, 0.01]) stepped at dt_min.
Solves that moved ln V by more than 0.01 are kept whole; the others (most
of every run, and easy for plain Newton) are subsampled one in twenty.
Writes the FP32 parameter vector (SBIEM_MLP_PARAMS + SBIEM_MLP_NORM values)
and a JSON summary beside it.

compare: the rough-fault cycle at N = 65536, dx = 2 m (alpha = 0.005) run by
the adaptive solver from steady state, once with plain Newton and once with
the learned guess, over the same simulated time: accepted steps, Newton
iterations per solve and wall time of each.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from .sbiem import Fault, mlp_train
from .workloads import rough_cycle, rough_fault

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "newton_guess_mlp.f32")
YEAR = 365.25 * 86400.0


def _keep(rows: np.ndarray, rng, small_keep: float = 0.05) -> np.ndarray:
    big = np.abs(rows[:, 5] - rows[:, 0]) > 0.01
    pick = big | (rng.random(rows.shape[0]) < small_keep)
    rows = rows[pick]
    return rows[np.all(np.isfinite(rows), axis=1)]


def harvest_cycle(target: int, rng, years: float = 2.0, chunk: int = 200, cap: int = 4_000_000) -> tuple:
    """Rows from the rough-fault cycle (N = 4096) through its first rupture."""
    w = rough_cycle()
    g = Fault.from_workload(w, precision=1)
    g.harvest_enable(cap)
    out, m, t, steps = [], 1, 0.0, 0
    total = 0
    while t < years * YEAR and total < target:
        hist, m, t, rc = g.run(years * YEAR, 1e-7, m0=m, max_steps=chunk)
        steps += len(hist)
        rows = _keep(g.harvest_read(reset=True), rng)
        out.append(rows)
        total += rows.shape[0]
        if rc != 0 or not hist:
            break             # the cycle's rupture opened the fault (or failed at dt_min): enough
    g.close()
    return (np.concatenate(out) if out else np.zeros((0, 6), np.float32)), {"accepted_steps": steps,
                                                                          "years": t / YEAR}


def harvest_ruptures(target: int, rng, steps: int = 4000, chunk: int = 250, cap: int = 4_000_000) -> tuple:
    """Rows from rough-fault ruptures of the ensemble's sizes, stepped at dt_min."""
    out, total, runs = [], 0, 0
    Ns = [1024, 2048, 4096, 8192]
    while total < target and runs < 64:
        N = Ns[runs % 4]
        w = rough_fault(N, 10.0, float(rng.uniform(1e-3, 1e-2)), seed=2000 + runs)
        g = Fault.from_workload(w, precision=1)
        g.harvest_enable(cap)
        for _ in range(steps // chunk):
            g.enqueue(chunk)
            if g.status()[0]:
                break
            rows = _keep(g.harvest_read(reset=True), rng)
            out.append(rows)
            total += rows.shape[0]
            if total >= target:
                break
        g.close()
        runs += 1
    return (np.concatenate(out) if out else np.zeros((0, 6), np.float32)), {"runs": runs}


def train(rows_target: int, out: str, epochs: int = 4, seed: int = 7) -> dict:
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    rc_rows, rc_info = harvest_cycle(rows_target // 2, rng)
    ru_rows, ru_info = harvest_ruptures(rows_target - rc_rows.shape[0], rng)
    rows = np.concatenate([rc_rows, ru_rows]).astype(np.float32)
    rows = rows[rng.permutation(rows.shape[0])][:rows_target]
    t_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, loss = mlp_train(rows, epochs=epochs, batch=8192, lr=2e-3, seed=seed)
    t_t = time.perf_counter() - t0
    os.makedirs(os.path.dirname(out), exist_ok=True)
    params.astype(np.float32).tofile(out)
    res = rows[:, 5] - rows[:, 0]
    summary = {"rows": int(rows.shape[0]), "rows_cycle": int(rc_rows.shape[0]), "rows_ruptures": int(ru_rows.shape[0]),
               "cycle": rc_info, "ruptures": ru_info, "epochs": epochs, "final_batch_loss": loss,
               "residual_std": float(res.std()), "harvest_s": t_h, "train_s": t_t,
               "params": os.path.basename(out)}
    with open(os.path.splitext(out)[0] + ".json", "w") as fh:
        json.dump(summary, fh, indent=1)
    return summary


def compare(params_path: str, years: float, chunk: int = 500, max_steps: int = 200_000) -> dict:
    params = np.fromfile(params_path, dtype=np.float32)
    w = rough_cycle(N=65536, dx=2.0, seed=3)
    res = {}
    for name in ("plain", "guided"):
        g = Fault.from_workload(w, precision=1)
        if name == "guided":
            g.set_mlp(params)
        g.newton_totals(reset=True)
        t_end = years * YEAR
        m, t, steps, rc = 1, 0.0, 0, 0
        mh = []
        t0 = time.perf_counter()
        while t < t_end * (1 - 1e-12) and steps < max_steps:
            hist, m, t, rc = g.run(t_end, 1e-7, m0=m, max_steps=chunk)
            steps += len(hist)
            mh += hist
            if rc != 0 or not hist:
                break
        wall = time.perf_counter() - t0
        it, so = g.newton_totals()
        vmax = float(g.get_state()["V"].max())
        res[name] = {"accepted_steps": steps, "years": t / YEAR, "wall_s": wall, "newton_iters": it,
                     "newton_solves": so, "iters_per_solve": it / max(so, 1), "stop_code": rc, "V_max": vmax,
                     "steps_at_dt_min": int(sum(1 for q in mh if q == 1))}
        g.close()
    res["iteration_ratio"] = res["guided"]["iters_per_solve"] / res["plain"]["iters_per_solve"]
    res["time_ratio"] = res["guided"]["wall_s"] / res["plain"]["wall_s"]
    res["workload"] = "rough-fault cycle N=65536, dx=2 m, Hurst-1 alpha=0.005, FP32 form, adaptive (eps0 = 1e-7 m)"
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "compare"])
    ap.add_argument("--rows", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--params", default=DEFAULT_OUT)
    ap.add_argument("--years", type=float, default=0.3)
    a = ap.parse_args()
    if a.cmd == "train":
        print(json.dumps(train(a.rows, a.out, a.epochs)), flush=True)
    else:
        print(json.dumps(compare(a.params, a.years)), flush=True)


if __name__ == "__main__":
    main()
