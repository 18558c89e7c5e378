#!/usr/bin/env python3
"""Throughput of the non-planar spectral BIEM time step on one GB300.

Metric: element-steps/s (N elements x accepted steps / device time) of the
whole step -- history convolution, two passes of predictor / FFTs / spectral
assembly / Newton, commit -- on the rough-fault cycle workload (N = 4096,
dx = 10 m, Hurst-1 roughness) with every history window full (steady state).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
    python bench.py --impl reference     # the FP64 CPU oracle on the same workload

The headline is the chosen form (FP32 history convolution and FFTs, FP64
state, slip, time and Newton); the plain FP64 path is timed the same way and
reported beside it.

Timing: each timed step runs as one CUDA-graph launch bracketed by CUDA events
on the launch stream (the step sweeps the next step's history on a side
branch while its passes run); after it, the history convolution alone is
launched and timed the same way, with an event between its sweep kernel and
its per-mode finish (the roofline is the sweep's).  L2 is flushed (256 MiB written, then
256 MiB read) before every timed launch, outside the events; the timed
launches run back to back without host synchronization.  Under torchrun every rank runs an independent replica (the path
has no exchange step), the maximum device time over ranks is taken and the
value sums all ranks' element-steps.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element-steps/s"
UNIT = "element-steps/s"
L2_FLUSH_BYTES = 256 << 20
HIST_AMP = 1e-3   # m/s: slip-rate amplitude of the seeded history (spectral scale amp*sqrt(N))


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp32")
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the other precision's measurement (profiling runs)")
    ap.add_argument("--workload", choices=["rough", "sinusoidal"], default="rough",
                    help="rough: the rough-fault cycle (headline); sinusoidal: the paper's own cycle setup")
    ap.add_argument("--kcN-L", type=float, default=0.0,
                    help="k_c * eta * L of the normal-traction kernel (the second cutting plane); 0: one plane")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


_KIND = "rough"  # --workload


def _workload(N):
    from paper_2107_03550_gb300.workloads import rough_cycle, sinusoidal_cycle
    if _KIND == "sinusoidal":
        return sinusoidal_cycle(N=N)
    return rough_cycle(N=N, lam_max=min(40e3, N * 10.0))


def _history(M, seed, N):
    from paper_2107_03550_gb300.workloads import random_history
    R = np.maximum(np.asarray(M) - 1, 0)
    return random_history(R, seed, HIST_AMP * np.sqrt(N))


def _workload_name(w, N):
    if _KIND == "sinusoidal":
        return (f"sinusoidal-fault cycle (Table 1), steady state: N={N}, dx={w.dx:g} m, fault "
                f"{w.extra['fault_length'] / 1e3:g} km of a 4L periodic domain, null slip rate on 1.5L each "
                f"side, h = {w.extra['amp']:g} m sin(2 pi x / {w.extra['wavelength'] / 1e3:g} km); "
                f"dt = dt_min = 0.25 dx/cs; every history window full")
    return (f"rough-fault cycle, steady state: N={N}, dx={w.dx:g} m, Hurst-1 roughness alpha=0.005, "
            f"lambda in [20 m, {min(40e3, N * 10.0) / 1e3:g} km], central 70% rate-and-state, "
            f"outer 30% at V_pl; dt = dt_min = 0.25 dx/cs; every history window full")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.idx = device_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
def _oracle_leg(N: int, seconds: float, max_steps: int | None = None) -> dict:
    """The FP64 oracle, as it stands, on the same workload (steady state)."""
    from oracle import Oracle, Params
    w = _workload(N)
    p = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min)
    o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init,
               prescribed=w.prescribed, V_presc=w.V_presc)
    HT, HN, off = _history(o.M, 11, N)
    o.set_history([HT[off[n]:off[n + 1]] for n in range(o.M.size)],
                  [HN[off[n]:off[n + 1]] for n in range(o.M.size)])
    steps = 0
    t0 = time.perf_counter()
    while True:
        if o.step() != 0:
            raise RuntimeError("oracle step failed")
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and steps >= max_steps):
            break
    return {"value": N * steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steady-state steps of the N={N} rough-fault workload "
                      f"(numpy FP64, single thread), {el:.1f} s"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _sweep_source_sha() -> str:
    """Hash of the history sweep's source section of kernels.cu (from its banner to the finish kernel)."""
    src = open(os.path.join(ROOT, "paper_2107_03550_gb300", "csrc", "kernels.cu")).read()
    a = src.index("// ---------------------------------------------- history sweep (bulk-async)")
    b = src.index("// Per-mode sums of the sweep's segment partials")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def _traffic(precision: str, N: int):
    """ncu DRAM bytes per sweep launch, if recorded for the current sweep source (else None)."""
    sha = _sweep_source_sha()
    path = os.path.join(ROOT, "profiles", f"k_sweep_{precision}_rough_cycle_N{N}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            fields[k.strip()] = v.strip()
    if fields.get("k_sweep source sha256[:16]") != sha:
        return None
    try:
        return float(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


# -------------------------------------------------------------- reference
def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    # bounded sample: at most K steps and at most about a minute of CPU time
    cpu = _oracle_leg(a.N, 60.0, max_steps=max(a.steps, 1))
    line = {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(_workload(a.N), a.N), "N": a.N, "precision": "fp64"},
            "cpu_baseline": {"value": cpu["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": cpu["sample"]},
            "e2e": {"value": cpu["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- ours
def _flusher(torch):
    w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    out = torch.empty((), dtype=torch.int32, device="cuda")

    def flush():
        # write 256 MiB (evicts the history), then read another 256 MiB so the
        # evicted dirty lines are written back before the timed step starts
        w.fill_(1)
        torch.amax(r, dim=0, out=out)

    return flush


def _measure(torch, a, precision: str, rank: int, world: int, flush, clock_index: int, extra=None):
    """Time K steps (and K history-only launches) back to back on one stream."""
    from paper_2107_03550_gb300.sbiem import Fault
    N = a.N
    w = _workload(N)
    g = Fault.from_workload(w, precision=1 if precision == "fp32" else 0, **(extra or {}))
    g.set_stream(torch.cuda.current_stream())
    HT, HN, _ = _history(g.windows(), 11 + rank, N)
    g.set_history(HT, HN)
    hist_bytes, dev_bytes = g.footprint()
    for _ in range(max(a.warmup, 3)):
        flush()
        g.enqueue(1)
        flush()
        g.history_enqueue(1)
    torch.cuda.synchronize()
    flags, _ = g.status(clear=True)
    if flags:
        raise RuntimeError(f"warm-up step failed, status {flags}")
    K = a.steps
    ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    ev_h = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    ev_m = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e in ev_m:
        e.record()  # creates the event; the library records it again after the sweep
    clocks = ClockSampler(clock_index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(K):
        flush()
        ev_s[k][0].record()
        g.enqueue(1)
        ev_s[k][1].record()
        flush()
        ev_h[k][0].record()
        g.history_enqueue(1, sweep_done=ev_m[k])
        ev_h[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    flags, done = g.status(clear=True)
    if flags:
        raise RuntimeError(f"timed step failed, status {flags}")
    ms_step = [x.elapsed_time(y) for x, y in ev_s]
    ms_hist = [x.elapsed_time(y) for x, y in ev_h]
    ms_sweep = [x[0].elapsed_time(m) for x, m in zip(ev_h, ev_m)]
    it_sum, it_max = g.newton_stats()
    total_s = sum(ms_step) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    res = dict(g=g, w=w, value=world * N * K / total_s, ms_per_step=1e3 * total_s / K,
               hist_ms=statistics.mean(ms_hist), sweep_ms=statistics.mean(ms_sweep), hist_bytes=hist_bytes,
               dev_bytes=dev_bytes,
               clocks=clk, it_sum=it_sum, it_max=it_max,
               slots=int(np.maximum(g.windows() - 1, 0).sum()))
    return res


def _e2e(torch, a, g, w, world):
    """Through the C ABI with host buffers: per step tau_load in, V out (pinned)."""
    N = a.N
    tau_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
    v_h = torch.empty(N, dtype=torch.float64, pin_memory=True)
    tau_np = tau_h.numpy()
    v_np = v_h.numpy()
    fr = w.f0 + w.a * np.log(w.V_init / w.V0) + w.b * np.log(w.theta_init * w.V0 / w.Dc)
    tau_np[:] = np.where(w.prescribed, 0.0, w.sigma_load * fr + w.mu / (2 * w.cs) * w.V_init)
    for _ in range(3):
        g.step_host(tau_load=tau_np, V_out=v_np)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        g.step_host(tau_load=tau_np, V_out=v_np)
    el = time.perf_counter() - t0
    return {"value": N * a.e2e_steps / el * world, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
            "d2h_bytes_per_step": 8 * N + 12}


def _read_ceiling(torch, nbytes: int, flush, reps: int = 20) -> dict:
    """The library's plain streaming read (sbiem_read_probe) of the sweep's byte count, flushed and
    timed like the sweep: what any read of this size reaches on this GPU, beside the large-copy peak."""
    from paper_2107_03550_gb300.sbiem import read_probe
    nb = (nbytes + 15) // 16 * 16
    x = torch.zeros(nb // 4, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for r in range(reps + 3):
        flush()
        e0.record()
        read_probe(x.data_ptr(), nb, sink.data_ptr(), st)
        e1.record()
        torch.cuda.synchronize()
        if r >= 3:
            ms.append(e0.elapsed_time(e1))
    del x
    t = statistics.mean(ms)
    return {"GBps": nb / (t * 1e-3) / 1e9, "ms": t, "bytes": nb,
            "what": "sbiem_read_probe: plain 128-bit streaming read of the sweep's algorithmic bytes, "
                    "L2 flushed the same way"}


def run_ours(a):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and "," not in vis and vis.strip().isdigit():
        dev_index = int(vis)
    flush = _flusher(torch)
    other = "fp64" if a.precision == "fp32" else "fp32"
    # the plain FP64 path and the chosen form, same workload, same timing
    side = None
    if not a.no_side:
        side = _measure(torch, a, other, rank, world, flush, dev_index)
        side["g"].close()
    qd = None
    if not a.no_side:
        # the quasi-dynamic limit (eta_w = 0) of the same workload and form
        import copy
        aq = copy.copy(a)
        aq.steps = min(a.steps, 500)
        qd = _measure(torch, aq, a.precision, rank, world, flush, dev_index, extra={"eta_w": 0.0})
        qd["g"].close()
    main = _measure(torch, a, a.precision, rank, world, flush, dev_index,
                    extra={"kcN_L": a.kcN_L} if a.kcN_L > 0 else None)
    e2e = None if a.no_e2e else _e2e(torch, a, main["g"], main["w"], world)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = _oracle_leg(a.N, a.cpu_seconds)
    peak, peak_kind = _peaks()
    achieved = main["hist_bytes"] / (main["sweep_ms"] * 1e-3) / 1e9
    ceiling = _read_ceiling(torch, main["hist_bytes"], flush)
    ceiling["frac_of_peak"] = ceiling["GBps"] / peak
    if rank == 0:
        w = main["w"]
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32/f64",
            "data": "synthetic",
            "config": {"workload": _workload_name(w, a.N) + (f"; normal kernel cut at k_c L = {a.kcN_L:g}"
                                                              if a.kcN_L > 0 else ""), "N": a.N, "dx_m": w.dx,
                       "precision": a.precision + (" (FP32 history convolution and FFTs, FP64 state and Newton)"
                                                   if a.precision == "fp32" else ""),
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed before every timed launch: 256 MiB write, then 256 MiB read, "
                             "outside the timed events",
                       "history_slots": main["slots"], "history_bytes_per_step": main["hist_bytes"],
                       "device_bytes": main["dev_bytes"],
                       "newton_iters_last_step": {"sum": main["it_sum"], "max": main["it_max"]},
                       "history_ms_with_finish": main["hist_ms"],
                       f"{other}_path": None if side is None else {
                           "value": side["value"], "ms_per_step": side["ms_per_step"], "sweep_ms": side["sweep_ms"],
                           "sweep_GBps": side["hist_bytes"] / (side["sweep_ms"] * 1e-3) / 1e9},
                       "quasi_dynamic_path": None if qd is None else {
                           "value": qd["value"], "ms_per_step": qd["ms_per_step"], "steps": min(a.steps, 500),
                           "what": "eta_w = 0: static stiffness plus radiation damping, no history; same "
                                   "workload and form, L2 flushed the same way"}},
            "roofline": {"bound": "hbm", "kernel": "k_sweep", "achieved": achieved, "peak": peak,
                         "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6800 GB/s", "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic(a.precision, a.N), "ms_per_launch": main["sweep_ms"],
                         "algorithmic_bytes_per_launch": main["hist_bytes"],
                         # context: a plain read of the same bytes (the size, not the kernel, caps frac)
                         "same_size_read": ceiling},
            "clocks": main["clocks"],
            "e2e": e2e,
            # per timed step: sweep + finish (side branch), two passes of
            # (spectral, Newton), commit; per timed history launch: sweep + finish
            "gpu_launches": 9 * a.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    main["g"].close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    global _KIND
    a = _args()
    _KIND = a.workload
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
