#!/usr/bin/env python3
"""Throughput of the non-planar spectral BIEM time step on one GB300.

Metric: element-steps/s (N elements x accepted steps / device time) of the
whole step -- history convolution, two passes of predictor / FFTs / spectral
assembly / Newton, commit.

Default workload: the large single fault (N = 262144, dx = 1 m, Hurst-1
roughness alpha = 0.003 plus a 200 m Gaussian seamount, central 70%
rate-and-state, outer 30% at the plate rate) in steady state: every history
window full (311 M ring slots per field), dt = dt_min.  The headline is the
chosen form: FP32 history convolution and FFTs, FP64 state, slip, time and
Newton, with the learned Newton initial guess deployed when a trained network
is present.  The plain FP64 path is timed the same way and reported beside it,
with side records at N = 4096 and N = 65536 and the quasi-dynamic limit.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
                    [--workload large|rough|sinusoidal|ensemble] [--N n]
    python bench.py --impl reference     # the FP64 CPU oracle on the same workload

Timing: each timed step runs as one CUDA-graph launch bracketed by CUDA events
on the launch stream (the step sweeps the next step's history on a side
branch while its passes run); after it, the history convolution alone is
launched and timed the same way, with an event between its sweep kernel and
its per-mode finish (the roofline is the sweep's).  Rings larger than L2 are
streamed from HBM every step; smaller ones are evicted by an L2 flush (256 MiB
written, then 256 MiB read) before every timed launch, outside the events.
Under torchrun every rank runs an independent replica (the path has no
exchange step), the maximum device time over ranks is taken and the value sums
all ranks' element-steps.  One JSON line is printed by rank 0.
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
L2_BYTES = 129 << 20
L2_FLUSH_BYTES = 256 << 20
HIST_AMP = 1e-3   # m/s: slip-rate amplitude of the seeded history (spectral scale amp*sqrt(N))
MLP_PATH = os.path.join(ROOT, "paper_2107_03550_gb300", "data", "newton_guess_mlp.f32")
DEFAULT_N = {"large": 262144, "rough": 4096, "sinusoidal": 4096, "ensemble": 0}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp32")
    ap.add_argument("--N", type=int, default=0, help="elements (0: the workload's own size)")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mlp", action="store_true", help="plain Newton in the headline (no learned guess)")
    ap.add_argument("--no-side", action="store_true", help="skip the side records (profiling runs)")
    ap.add_argument("--workload", choices=["large", "rough", "sinusoidal", "ensemble"], default="large",
                    help="large: the N = 262144 fault (headline); rough: the rough-fault cycle; sinusoidal: "
                         "the paper's own cycle setup; ensemble: 256 rough-fault realizations of uneven N")
    ap.add_argument("--kcN-L", type=float, default=0.0,
                    help="k_c * eta * L of the normal-traction kernel (the second cutting plane); 0: one plane")
    ap.add_argument("--members", type=int, default=256,
                    help="ensemble members (a multiple of 4; 256 is the ensemble workload, fewer for profiling runs)")
    ap.add_argument("--sweep-only", action="store_true",
                    help="profiling runs: only W + K launches of the history convolution on the workload's handle "
                         "(no tuning unless --weights tune), one JSON line with their times")
    ap.add_argument("--weights", choices=["tune", "generated", "streamed"], default="tune",
                    help="history sweep weights: autotuned (default), evaluated on chip where the modes allow, "
                         "or streamed")
    a = ap.parse_args()
    if a.N == 0:
        a.N = DEFAULT_N[a.workload]
    return a


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload(kind: str, N: int):
    from paper_2107_03550_gb300.workloads import large_fault, rough_cycle, sinusoidal_cycle
    if kind == "sinusoidal":
        return sinusoidal_cycle(N=N)
    if kind == "large":
        return large_fault(N=N, dx=262144.0 / N)
    if N == 65536:
        return rough_cycle(N=65536, dx=2.0, seed=3)
    return rough_cycle(N=N, lam_max=min(40e3, N * 10.0))


def _workload_name(kind: str, w) -> str:
    N = w.N
    tail = "; dt = dt_min = 0.25 dx/cs; every history window full"
    if kind == "sinusoidal":
        return (f"sinusoidal-fault cycle (Table 1), steady state: N={N}, dx={w.dx:g} m, fault "
                f"{w.extra['fault_length'] / 1e3:g} km of a 4L periodic domain, null slip rate on 1.5L each "
                f"side, h = {w.extra['amp']:g} m sin(2 pi x / {w.extra['wavelength'] / 1e3:g} km)" + tail)
    if kind == "large":
        e = w.extra
        return (f"large single fault, steady state: N={N}, dx={w.dx:g} m, Hurst-1 roughness alpha={e['alpha']:g}, "
                f"lambda in [{e['lam_min']:g} m, {e['lam_max'] / 1e3:g} km] plus a {e['seamount'][0]:g} m Gaussian "
                f"seamount (sigma {e['seamount'][1] / 1e3:g} km), central 70% rate-and-state, outer 30% at V_pl"
                + tail)
    lam = 40.0 if N * w.dx >= 40e3 else N * w.dx / 1e3
    return (f"rough-fault cycle, steady state: N={N}, dx={w.dx:g} m, Hurst-1 roughness alpha=0.005, "
            f"lambda in [20 m, {lam:g} km], central 70% rate-and-state, outer 30% at V_pl" + tail)


def _fill_history(torch, g, seed: int, precision: str):
    """Seeded random history drawn on the device (every window full)."""
    from paper_2107_03550_gb300.workloads import random_history_device
    R = np.maximum(g.windows() - 1, 0)
    if R.sum() == 0:
        return   # no history (the quasi-dynamic limit)
    dt = torch.float32 if precision == "fp32" else torch.float64
    HT, HN = random_history_device(R, seed, HIST_AMP * np.sqrt(g.N), torch, dtype=dt)
    g.set_history_device(HT, HN)
    del HT, HN
    torch.cuda.empty_cache()


def _mlp_params():
    if os.path.exists(MLP_PATH):
        return np.fromfile(MLP_PATH, dtype=np.float32)
    return None


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
def _sum_worker(args):
    """Time the oracle's per-mode history sums over modes drawn at random (one process)."""
    N, dx, cs, cp, mu, dt_min, modes, seed, budget = args
    import time as _t
    from oracle import Params
    from oracle.sbiem import mode_history_sum, weights, windows
    p = Params(N=N, dx=dx, mu=mu, cs=cs, cp=cp, dt_min=dt_min)
    M = windows(p)
    rng = np.random.default_rng(seed)
    done, slots, el = 0, 0, 0.0
    w0 = _t.perf_counter()
    for n in modes:
        wT, wN, off = weights(p, M, modes=[n])
        w = slice(off[n], off[n + 1])
        R = max(int(M[n]) - 1, 0)
        HT = rng.standard_normal(R) + 1j * rng.standard_normal(R)
        HN = rng.standard_normal(R) + 1j * rng.standard_normal(R)
        t0 = _t.perf_counter()
        mode_history_sum(wT[w], wN[w], HT, HN, 1)
        el += _t.perf_counter() - t0
        done += 1
        slots += R
        if el >= budget or _t.perf_counter() - w0 >= 3 * budget:
            break
    return done, slots, el


def _oracle_leg(kind: str, N: int, seconds: float, max_steps: int | None = None) -> dict:
    """The FP64 oracle, as it stands, on the same workload in steady state.

    Small faults (whole weight tables under ~3e7 lags): the oracle's own
    steps with every window full, timed whole.  Larger faults, whose weight
    tables the oracle cannot build in a bounded sample: the step is timed in
    its two parts -- the history sums of sampled modes (the oracle's
    per-mode sum, on all host cores, one process per core) extrapolated to
    every ring slot, plus the rest of the step (FFTs, spectral assembly, the
    two Newton passes) timed whole on the quasi-dynamic oracle (no history),
    which runs exactly that rest.
    """
    from oracle import Oracle, Params
    from oracle.sbiem import windows
    w = _workload(kind, N)
    p = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min)
    M = windows(p)
    R = np.maximum(M - 1, 0)
    total = int(R.sum())
    if M.sum() < 3e7:
        from paper_2107_03550_gb300.workloads import random_history
        o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init,
                   prescribed=w.prescribed, V_presc=w.V_presc)
        HT, HN, off = random_history(R, 11, HIST_AMP * np.sqrt(N))
        o.set_history([HT[off[n]:off[n + 1]] for n in range(M.size)],
                      [HN[off[n]:off[n + 1]] for n in range(M.size)])
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
                "sample": f"{steps} whole steady-state steps of the N={N} workload (numpy FP64, single "
                          f"thread), {el:.1f} s"}
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    cores = max(1, min(os.cpu_count() or 1, 72))
    # modes drawn uniformly at random (each process its own share of one
    # seeded permutation): the mean time per mode times the number of modes
    # estimates the whole sweep, short and long windows alike
    perm = np.random.default_rng(7).permutation(np.arange(1, M.size))
    jobs = [(w.N, w.dx, w.cs, w.cp, w.mu, w.dt_min, perm[i::cores].tolist(), 100 + i, seconds / 2)
            for i in range(cores)]
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_sum_worker, jobs))
    nmodes = sum(r[0] for r in res)
    slots = sum(r[1] for r in res)
    t_mode = sum(r[2] for r in res) / max(nmodes, 1)
    t_sums = (M.size - 1) * t_mode / cores                  # all modes, spread over the processes
    rate = slots / max(sum(r[2] for r in res), 1e-12)
    pq = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min, eta_w=0.0)
    oq = Oracle(pq, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init,
                prescribed=w.prescribed, V_presc=w.V_presc)
    steps = 0
    t0 = time.perf_counter()
    while True:
        if oq.step() != 0:
            raise RuntimeError("oracle step failed")
        steps += 1
        el = time.perf_counter() - t0
        if el >= max(1.0, seconds / 4) or steps >= 50:
            break
    t_rest = el / steps
    t_step = t_sums + t_rest
    return {"value": N / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"extrapolated: the oracle's history sums of {nmodes} of the {M.size - 1} modes drawn at "
                       f"random ({slots} of the {total} ring slots, {cores} processes, {rate:.3g} slots/s per "
                       f"process), mean time per mode x modes / processes = {t_sums:.2f} s per step, plus {steps} "
                       f"whole quasi-dynamic oracle steps at N={N} for the FFTs, assembly and Newton "
                       f"({t_rest:.3f} s per step, one thread)")}


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


def _persist_source_sha() -> str:
    """Hash of the ensemble's persistent history kernel: the sweep section and the persistent-launch section."""
    src = open(os.path.join(ROOT, "paper_2107_03550_gb300", "csrc", "kernels.cu")).read()
    a = src.index("// ---------------------------------------------- history sweep (bulk-async)")
    b = src.index("// Per-mode sums of the sweep's segment partials")
    c = src.index("// Ensemble form of k_sweep_finish")
    d = src.index("// ------------------------------------------------------------ friction")
    return hashlib.sha256((src[a:b] + src[c:d]).encode()).hexdigest()[:16]


def _traffic_ensemble(precision: str, slots: int):
    """ncu DRAM bytes of the ensemble's persistent history launch, scaled by ring slots from a smaller
    ensemble of the same family, if recorded for the current source (else None)."""
    sha = _persist_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not (fn.startswith(f"k_sweep_persist_{precision}_") and fn.endswith(".md")):
            continue
        fields = {}
        for line in open(os.path.join(pdir, fn)):
            if ": " in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(": ", 1)
                fields[k.strip()] = v.strip()
        if fields.get("k_sweep_persist source sha256[:16]") != sha:
            continue
        try:
            dram = float(fields["dram bytes per launch"])
            s = float(fields["ring slots"])
        except (KeyError, ValueError):
            continue
        return {"bytes": dram * slots / s, "from": fn, "scaled_by_slots": slots / s}
    return None


def _traffic(precision: str, kind: str, slots: int):
    """ncu DRAM bytes per sweep launch, if recorded for the current sweep source (else None).

    The profile of the same workload is used when present; otherwise one of a
    smaller fault of the same family, scaled by ring slots (the sweep reads
    each slot once, so its traffic grows in proportion to the slots).
    """
    sha = _sweep_source_sha()
    pdir = os.path.join(ROOT, "profiles")
    found = []
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not (fn.startswith(f"k_sweep_{precision}_") and fn.endswith(".md")):
            continue
        fields = {}
        for line in open(os.path.join(pdir, fn)):
            if ": " in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(": ", 1)
                fields[k.strip()] = v.strip()
        if fields.get("k_sweep source sha256[:16]") != sha or fields.get("workload family") != kind:
            continue
        try:
            dram = float(fields["dram bytes per launch"])
            s = float(fields["ring slots"])
        except (KeyError, ValueError):
            continue
        found.append({"bytes": dram * slots / s, "from": fn, "scaled_by_slots": slots / s})
    # a profile of the same size first
    found.sort(key=lambda r: abs(r["scaled_by_slots"] - 1.0))
    return found[0] if found else None


# -------------------------------------------------------------- reference
def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    if a.workload == "ensemble":
        print(json.dumps({"impl": "reference", "unavailable": "the ensemble is not a single oracle workload"}))
        return
    cpu = _oracle_leg(a.workload, a.N, 30.0, max_steps=max(a.steps, 1))
    w = _workload(a.workload, a.N)
    line = {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(a.workload, w), "N": a.N, "precision": "fp64"},
            "cpu_baseline": {"value": cpu["value"], "unit": UNIT, "cores": cpu["cores"], "kind": "oracle",
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


def _max_over_ranks(torch, seconds: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's time (replicas: every rank runs its own fault; the job's time is the maximum)."""
    if world <= 1:
        return seconds
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_rate(world: int, elements_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job element-steps/s: every rank's elements times the steps, over the slowest rank's time."""
    return world * elements_per_rank * steps / seconds


def _measure(torch, a, kind, N, precision: str, rank: int, world: int, flush, clock_index: int, steps: int,
             extra=None, mlp=None):
    """Time `steps` steps (and as many history-only launches) back to back on one stream."""
    from paper_2107_03550_gb300.sbiem import Fault
    w = _workload(kind, N)
    g = Fault.from_workload(w, precision=1 if precision == "fp32" else 0, **(extra or {}))
    g.set_stream(torch.cuda.current_stream())
    _fill_history(torch, g, 11 + rank, precision)
    if mlp is not None:
        g.set_mlp(mlp)
    tuned = _sweep_setup(g, a)
    hist_bytes, dev_bytes = g.footprint()
    slots = int(np.maximum(g.windows() - 1, 0).sum())
    ring_bytes = slots * (16 if precision == "fp32" else 32)
    flushed = hist_bytes < 2 * L2_BYTES
    fl = flush if flushed else (lambda: None)
    for _ in range(max(a.warmup, 3)):
        fl()
        g.enqueue(1)
        fl()
        g.history_enqueue(1)
    torch.cuda.synchronize()
    flags, _ = g.status(clear=True)
    if flags:
        raise RuntimeError(f"warm-up step failed, status {flags}")
    K = steps
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
    torch.cuda.nvtx.range_push("timed")  # profiling runs capture inside this range (ncu --nvtx-include timed/)
    for k in range(K):
        fl()
        ev_s[k][0].record()
        g.enqueue(1)
        ev_s[k][1].record()
        fl()
        ev_h[k][0].record()
        g.history_enqueue(1, sweep_done=ev_m[k])
        ev_h[k][1].record()
    torch.cuda.nvtx.range_pop()
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
    total_s = _max_over_ranks(torch, sum(ms_step) / 1e3, world)
    return dict(g=g, w=w, N=N, value=_job_rate(world, N, K, total_s), ms_per_step=1e3 * total_s / K,
                hist_ms=statistics.mean(ms_hist), sweep_ms=statistics.mean(ms_sweep),
                sweep_ms_median=statistics.median(ms_sweep), hist_bytes=hist_bytes, ring_bytes=ring_bytes,
                weight_bytes=hist_bytes - ring_bytes, dev_bytes=dev_bytes, clocks=clk, it_sum=it_sum,
                it_max=it_max, slots=slots, flushed=flushed, step_kernels=g.step_kernels(), steps=K,
                sweep=dict(tuned, table_err=g.get_sweep()["table_err"],
                           lag_ctas_per_sm=g.get_sweep()["lag_ctas_per_sm"]))


def _sweep_setup(g, a) -> dict:
    """The history sweep's configuration: the library's autotuner (shape, weight form, CTAs per SM), or a
    weight form forced for profiling (shape 3, as many CTAs as fit)."""
    if a.weights == "tune" or g.get_sweep()["table_err"] < 0:
        return g.tune(reps=5)
    g.set_sweep(4, 1.0 / 64 if a.weights == "generated" else 0.0, 0)
    sw = g.get_sweep()
    return {"shape": sw["shape"], "gen_ds_max": sw["gen_ds_max"], "ctas_per_sm": sw["ctas_per_sm"], "ms": None}


def _sweep_only(torch, a):
    """W + K launches of the history convolution alone (profiling runs)."""
    from paper_2107_03550_gb300.sbiem import Fault
    w = _workload(a.workload, a.N)
    g = Fault.from_workload(w, precision=1 if a.precision == "fp32" else 0)
    g.set_stream(torch.cuda.current_stream())
    _fill_history(torch, g, 11, a.precision)
    cfg = _sweep_setup(g, a)
    slots = int(np.maximum(g.windows() - 1, 0).sum())
    for _ in range(a.warmup):
        g.history_enqueue(1)
    ms = []
    for _ in range(a.steps):
        e0, e1, em = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        em.record()
        e0.record()
        g.history_enqueue(1, sweep_done=em)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(em))
    g.close()
    ring = slots * (16 if a.precision == "fp32" else 32)
    print(json.dumps({"sweep_only": True, "workload": _workload_name(a.workload, w), "N": a.N, "sweep": cfg,
                      "ring_slots": slots, "ring_bytes": ring, "sweep_ms": ms,
                      "ring_GBps_median": ring / (statistics.median(ms) * 1e-3) / 1e9}), flush=True)


def _side(res: dict, what: str) -> dict:
    return {"N": res["N"], "value": res["value"], "ms_per_step": res["ms_per_step"], "sweep_ms": res["sweep_ms"],
            "ring_GBps": res["ring_bytes"] / (res["sweep_ms"] * 1e-3) / 1e9, "steps": res["steps"],
            "sweep": res["sweep"],
            "l2": "flushed before every timed launch" if res["flushed"] else "rings larger than L2",
            "what": what}


def _e2e(torch, a, g, w, world):
    """Through the C ABI with host buffers: per step tau_load in, V out (pinned)."""
    N = g.N
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
    el = _max_over_ranks(torch, time.perf_counter() - t0, world)
    return {"value": _job_rate(world, N, a.e2e_steps, el), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
            "d2h_bytes_per_step": 8 * N + 12}


def _read_ceiling(torch, nbytes: int, flush, reps: int = 20) -> dict:
    """The library's plain streaming read (sbiem_read_probe) of the sweep's ring bytes, timed like the
    sweep: what any read of this size reaches on this GPU, beside the large-copy peak."""
    from paper_2107_03550_gb300.sbiem import read_probe
    nb = (nbytes + 15) // 16 * 16
    x = torch.zeros(nb // 4, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    fl = flush if nb < 2 * L2_BYTES else (lambda: None)
    for r in range(reps + 3):
        fl()
        e0.record()
        read_probe(x.data_ptr(), nb, sink.data_ptr(), st)
        e1.record()
        torch.cuda.synchronize()
        if r >= 3:
            ms.append(e0.elapsed_time(e1))
    del x
    torch.cuda.empty_cache()
    t = statistics.mean(ms)
    return {"GBps": nb / (t * 1e-3) / 1e9, "ms": t, "bytes": nb,
            "what": "sbiem_read_probe: plain 128-bit streaming read of the sweep's ring bytes"}


def _ensemble(torch, a, rank, world, clock_index):
    """256 rough-fault realizations (64 each of N = 1024, 2048, 4096, 8192; dx = 10 m; alpha ~ U[0.001, 0.01])
    in one batch: the history sweep over every member's rings in one launch, per-size pass launches."""
    from paper_2107_03550_gb300.sbiem import Batch, Fault
    from paper_2107_03550_gb300.workloads import rough_fault
    rng = np.random.default_rng(1000)
    Ns = [1024, 2048, 4096, 8192]
    members = []
    nm = max(4, a.members // 4 * 4)
    for r in range(nm):
        N = Ns[r // (nm // 4)]
        w = rough_fault(N, 10.0, float(rng.uniform(1e-3, 1e-2)), seed=1000 + r)
        g = Fault.from_workload(w, precision=1 if a.precision == "fp32" else 0)
        _fill_history(torch, g, 5000 + r + 1000 * rank, a.precision)
        members.append(g)
    b = Batch(members)
    b.set_stream(torch.cuda.current_stream())
    chunk, blocks, tune_ms = b.tune(reps=5)
    slots = sum(int(np.maximum(g.windows() - 1, 0).sum()) for g in members)
    elems = sum(g.N for g in members)
    for _ in range(max(a.warmup, 3)):
        b.enqueue(1)
    torch.cuda.synchronize()
    fl, _ = b.status()
    if np.any(fl):
        raise RuntimeError("ensemble warm-up failed")
    K = a.steps
    info = b.get_sweep()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(clock_index)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    torch.cuda.nvtx.range_push("timed")  # profiling runs capture inside this range (ncu --nvtx-include timed/)
    e0.record()
    b.enqueue(K)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    fl, done = b.status()
    if np.any(fl):
        raise RuntimeError("ensemble step failed")
    total_s = e0.elapsed_time(e1) / 1e3
    # the same batch with the history convolution in the other form: two
    # launches (sweep, then the per-(member, mode) sums) or one persistent
    # launch with a grid barrier, whichever the autotuner did not keep
    b.set_persistent(not info["persistent"])
    K2 = max(10, K // 5)
    b.enqueue(3)
    torch.cuda.synchronize()
    e0.record()
    b.enqueue(K2)
    e1.record()
    torch.cuda.synchronize()
    fl, _ = b.status()
    if np.any(fl):
        raise RuntimeError("ensemble step (two-launch form) failed")
    two_s = e0.elapsed_time(e1) / 1e3 / K2
    b.set_persistent(info["persistent"])
    total_s = _max_over_ranks(torch, total_s, world)
    bytes_ring = slots * (16 if a.precision == "fp32" else 32)
    peak, peak_kind = _peaks()
    traffic = _traffic_ensemble(a.precision, slots)
    line = {
        "metric": METRIC, "value": _job_rate(world, elems, K, total_s), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": a.warmup, "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64" if a.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"ensemble of {nm} rough-fault realizations: {nm // 4} each of N = 1024, 2048, "
                               "4096, 8192, dx = 10 m, Hurst-1 alpha ~ U[0.001, 0.01], seeds 1000 + r; every "
                               "history window full; dt = dt_min", "elements_per_step": elems, "history_slots": slots,
                   "ring_bytes_per_step": bytes_ring, "precision": a.precision,
                   "parallelism": f"replicas x{world}", "l2": "rings larger than L2 (no flush)",
                   "tuned": {"chunk_slots": chunk, "sweep_ctas_per_sm": blocks, "sweep_ms": tune_ms,
                             "shape": info["shape"], "gen_ds_max": info["gen_ds_max"], "overlap": info["overlap"],
                             "distinct_weight_arrays": info["distinct_weights"]},
                   "history_form": "one persistent launch" if info["persistent"] else "two launches",
                   "side": {"other_history_form": {
                       "value": world * elems / two_s, "ms_per_step": 1e3 * two_s, "steps": K2,
                       "what": ("history convolution as a sweep launch and a sum launch (no grid barrier)"
                                if info["persistent"] else
                                "history convolution as one persistent launch with a grid barrier")
                               + "; the rest of the step unchanged"}}},
        "roofline": {"bound": "hbm", "kernel": "k_sweep_persist" if info["persistent"] else "k_sweep", "achieved": bytes_ring / (tune_ms * 1e-3) / 1e9,
                     "peak": peak, "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst)", "unit": "GB/s",
                     "frac": bytes_ring / (tune_ms * 1e-3) / 1e9 / peak,
                     # both forms sweep with the same code and copy policy: the same DRAM bytes
                     "traffic": traffic["bytes"] if traffic else None,
                     "traffic_source": traffic,
                     "algorithmic_bytes": "ring slots x 2 fields x complex", "ms_per_launch": tune_ms,
                     "timing": "median of the autotuner's event-timed launches of the history convolution alone"},
        "ring_GBps_over_step": bytes_ring / (total_s / K) / 1e9,
        "clocks": clk, "e2e": None, "gpu_launches": None, "cpu_baseline": None,
    }
    for g in members:
        g.close()
    b.close()
    return line


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
    if a.sweep_only:
        _sweep_only(torch, a)
        return
    if a.workload == "ensemble":
        line = _ensemble(torch, a, rank, world, dev_index)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    flush = _flusher(torch)
    kind, N = a.workload, a.N
    other = "fp64" if a.precision == "fp32" else "fp32"
    mlp = None if (a.no_mlp or a.precision == "fp64") else _mlp_params()
    side = {}
    if not a.no_side:
        # the plain path of the other precision on the same workload (the comparison of the metric)
        r = _measure(torch, a, kind, N, other, rank, world, flush, dev_index, min(a.steps, 1000))
        side[f"{other}_path"] = _side(r, f"{other} form, same workload, plain Newton")
        r["g"].close()
        r = _measure(torch, a, kind, N, a.precision, rank, world, flush, dev_index, min(a.steps, 500),
                     extra={"eta_w": 0.0})
        side["quasi_dynamic_path"] = _side(r, "eta_w = 0: static stiffness plus radiation damping, no history; "
                                              "same workload and form")
        r["g"].close()
        if mlp is not None:
            # the same form with plain Newton (the learned guess off)
            r = _measure(torch, a, kind, N, a.precision, rank, world, flush, dev_index, min(a.steps, 1000))
            side[f"{a.precision}_plain_newton"] = _side(r, "the chosen form without the learned Newton guess")
            r["g"].close()
        for n2 in (4096, 65536):
            if n2 == N:
                continue
            r = _measure(torch, a, "rough", n2, a.precision, rank, world, flush, dev_index, min(a.steps, 1000))
            side[f"rough_cycle_N{n2}"] = _side(r, _workload_name("rough", r["w"]))
            r["g"].close()
        torch.cuda.empty_cache()
    main = _measure(torch, a, kind, N, a.precision, rank, world, flush, dev_index, a.steps,
                    extra={"kcN_L": a.kcN_L} if a.kcN_L > 0 else None, mlp=mlp)
    e2e = None if a.no_e2e else _e2e(torch, a, main["g"], main["w"], world)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = _oracle_leg(kind, N, a.cpu_seconds)
    peak, peak_kind = _peaks()
    achieved = main["ring_bytes"] / (main["sweep_ms"] * 1e-3) / 1e9
    ceiling = _read_ceiling(torch, main["ring_bytes"], flush)
    ceiling["frac_of_peak"] = ceiling["GBps"] / peak
    traffic = _traffic(a.precision, kind, main["slots"])
    if rank == 0:
        w = main["w"]
        line = {
            "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32/f64",
            "data": "synthetic",
            "config": {"workload": _workload_name(kind, w) + (f"; normal kernel cut at k_c L = {a.kcN_L:g}"
                                                                if a.kcN_L > 0 else ""), "N": N, "dx_m": w.dx,
                       "precision": a.precision + (" (FP32 history convolution and FFTs, FP64 state and Newton)"
                                                   if a.precision == "fp32" else ""),
                       "newton_guess": ("learned (5-64-64-1 BF16 network, " + os.path.relpath(MLP_PATH, ROOT) + ")"
                                        if mlp is not None else "plain (previous slip rate)"),
                       "parallelism": f"replicas x{world}",
                       "l2": ("flushed before every timed launch: 256 MiB write, then 256 MiB read, outside the "
                              "timed events") if main["flushed"] else
                             f"rings ({main['ring_bytes'] / 1e9:.2f} GB) larger than L2: no flush",
                       "history_slots": main["slots"], "ring_bytes_per_step": main["ring_bytes"],
                       "weight_bytes_per_step": main["weight_bytes"], "device_bytes": main["dev_bytes"],
                       "device_bytes_limit": 180e9,
                       "newton_iters_last_step": {"sum": main["it_sum"], "max": main["it_max"]},
                       "history_ms_with_finish": main["hist_ms"], "sweep": main["sweep"], "side": side},
            "roofline": {"bound": "hbm", "kernel": "k_sweep", "achieved": achieved, "peak": peak,
                         "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs, burst: the sweep is timed alone)"
                         if peak_kind == "measured" else "fallback 6800 GB/s", "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": None if traffic is None else traffic["bytes"],
                         "traffic_source": traffic,
                         "ms_per_launch": main["sweep_ms"], "ms_per_launch_median": main["sweep_ms_median"],
                         "algorithmic_bytes_per_launch": main["ring_bytes"],
                         "algorithmic_bytes": "ring slots x 2 fields x complex (16 B per slot FP32, 32 B FP64)",
                         "weight_bytes_per_launch": main["weight_bytes"],
                         "same_size_read": ceiling},
            "clocks": main["clocks"],
            "e2e": e2e,
            # per timed step: the step graph's kernels; per timed history launch: sweep + finish
            "gpu_launches": (main["step_kernels"] + 2) * a.steps,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    main["g"].close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
