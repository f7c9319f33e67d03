"""Benchmark of the adaptive MR-LBM step on GB300: leaf-cell updates per second.

A step is one adaptive time step (multiresolution analysis, mesh update, data
transfer, leaves collision, reconstructed-flux stream) of every instance of the
workload.  The default workload is the mixed batch of 4096 independent
instances (D1Q2 advection / Burgers, vectorial D1Q2^2 shallow water, vectorial
D1Q2^3 Euler; Jmax uniform in 8..14; eps log-uniform in [1e-5, 1e-2];
piecewise-constant data with 1..6 jumps).  The headline `value` is the FP64
path (the paper's precision); the FP32 path on the same inputs sits beside it
under "fp32".  Timed: exactly K steps as replays of a CUDA graph holding one
persistent launch of G steps, bracketed by a barrier and a device
synchronisation, CUDA events on the solver's stream; the per-GPU state (GBs)
is far larger than L2.  Clocks are sampled over at least a second of the same
graph replays run on a saved copy of the state just before the timed region
(the state is restored, so the timed steps are steps W+1..W+K).

Beside the batch: "singles" times the four single-instance configurations
(advection Jmax 10, Burgers Jmax 13, shallow water Jmax 15, Sod Jmax 18) in
both precisions against a latency floor (dependent passes per step times the
measured cost of one warp-to-warp hand-over through memory and a barrier);
"accuracy" compares the FP64 and FP32 paths with the FP64 oracle on those
configurations and on 64 batch instances; "cpu_baseline" times the oracle on
the host cores.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload batch|batch_sw|advection|burgers|shallow|sod|...]

Under torchrun every rank runs its own seeded batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "adaptive LBM leaf-cell updates/s at 1 GB300, FP32 vs FP64, at matched L1 error"
UNIT = "leaf-cell updates/s"
GRAPH_STEPS = 64  # adaptive steps per persistent launch, captured once in a CUDA graph and replayed
HBM_FALLBACK = 6800.0
CLOCK_PREROLL_S = 1.2
SINGLES = ("advection", "burgers", "shallow", "sod")
# single-instance timing: (warm-up steps, timed steps in one launch)
SINGLE_STEPS = {"advection": (4, 64), "burgers": (64, 256), "shallow": (64, 256), "sod": (64, 256)}
# accuracy against the FP64 oracle: steps compared (the configurations' full T where the oracle
# finishes in seconds; a fixed window from the initial state otherwise)
ACCURACY_STEPS = {"advection": None, "burgers": None, "shallow": 2048, "sod": 128}


# --------------------------------------------------------------------------- helpers

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2102_12163_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def host_cores():
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:
        usable = os.cpu_count() or 1
    return usable, os.cpu_count() or usable


def profiled_traffic(workload: str, precision: str, graph_steps: int):
    """DRAM bytes per leaf update from the committed ncu record
    (profiles/traffic.json) of a launch of the same number of steps, if it was
    taken on the current kernel source.  The steps per launch are part of the
    key because an instance's values stay in L2 between the steps of one launch:
    the DRAM bytes per update fall as the launch grows."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            j = json.load(fh)
        e = j[f"{workload}:{precision}:g{graph_steps}"]
        if e.get("source_hash") != source_hash():
            return None
        return e
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling (every 50 ms) while the GPU runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []  # (host time, line)
        self.marks = {}

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons, inside = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = self.marks.get("load_start"), self.marks.get("timed_end")
        ts, te = self.marks.get("timed_start"), self.marks.get("timed_end")
        for t, line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or (t0 is not None and t < t0) or (t1 is not None and t > t1 + 0.06):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            if ts is not None and ts <= t <= te + 0.06:
                inside += 1
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": inside,
               "window": "the same graph replays on a saved copy of the state for >= 1 s, then the timed region"}
        if t0 is not None and t1 is not None:
            out["window_s"] = round(t1 - t0, 3)
        return out


def make_workload(name: str, rank: int, n_batch: int = 4096):
    from paper_2102_12163_gb300 import workloads as W

    if name == "batch":
        insts = W.batch(n=n_batch, seed=12163 + rank)
        desc = (f"batch of {n_batch} mixed D1Q2 advection/Burgers, D1Q2^2 shallow water, D1Q2^3 Euler; "
                f"Jmax 8..14; eps 1e-5..1e-2; Euler density U[0.4, 1] (sound speed below lambda = 3)")
    elif name == "batch_sw":
        insts = W.batch_sw(n=n_batch, seed=5202 + rank)
        desc = f"batch of {n_batch} shallow water instances, D1Q3 / D1Q5 (Section 5.2); Jmax 8..14; eps 1e-5..1e-2"
    else:
        insts = [W.WORKLOADS[name]()]
        i = insts[0]
        desc = f"{name} single instance, Jmin {i.Jmin} Jmax {i.Jmax} eps {i.eps:g}"
    return insts, desc


# --------------------------------------------------------------------------- oracle (CPU) work

def _params(inst):
    import oracle as O

    return O.Params(Jmin=inst.Jmin, Jmax=inst.Jmax, eq=inst.eq, lam=inst.lam, eps=inst.eps, gamma=inst.gamma,
                    mu_bar=inst.mu_bar, bc=inst.bc, a=inst.a, b=inst.b, s=inst.s, eqp=inst.eqp,
                    collision=inst.collision)


def _oracle_task(args):
    inst, warm, n = args
    sys.path.insert(0, ROOT)
    import oracle as O

    o = O.Oracle(_params(inst))
    o.set_initial(inst.m0)
    o.step(warm)
    upd = 0
    t0 = time.perf_counter()
    for _ in range(n):
        o.step()
        upd += len(o.leaves()[0])
    return upd, time.perf_counter() - t0


def _oracle_run_task(args):
    """Oracle adaptive run and uniform reference scheme over `steps` steps:
    (finest conserved moments of the adaptive run, of the reference)."""
    inst, steps = args
    sys.path.insert(0, ROOT)
    import oracle as O

    p = _params(inst)
    o = O.Oracle(p)
    o.set_initial(inst.m0)
    o.step(steps)
    F = O.uniform_step(p, O.equilibrium(p, inst.m0), steps)
    return o.finest_moments(), O.moments(p, F)


def _pool(cores):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    return ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn"))


def oracle_throughput(insts, target_s: float = 15.0, warm: int = 4):
    """The oracle as it stands on a bounded sample of the workload, spread over
    all usable host cores with a spawned process pool; returns (value, cores,
    sample description, ms per step of the whole workload at that rate)."""
    cores, total = host_cores()
    stride = max(1, len(insts) // (8 * cores))
    sample = insts[::stride][: 8 * cores]
    cal = [_oracle_task((i, warm, 1))[1] for i in sample[: min(8, len(sample))]]
    per_step = max(sum(cal) / len(cal), 1e-5)
    n = int(max(1, min(2048, target_s * cores / (per_step * len(sample)))))
    t0 = time.perf_counter()
    with _pool(cores) as ex:
        res = list(ex.map(_oracle_task, [(i, warm, n) for i in sample]))
    wall = time.perf_counter() - t0
    upd = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    value = upd / busy * cores
    desc = (f"{len(sample)} of {len(insts)} instances (every {stride}th), {warm} untimed + {n} timed steps each, "
            f"{cores} worker processes on {cores} usable of {total} host cores, {wall:.1f} s wall")
    # the sample's mean leaves per instance-step, for all instances of the workload
    ms_step = upd / (len(sample) * n) * len(insts) / value * 1e3
    return value, cores, desc, ms_step


# --------------------------------------------------------------------------- GPU legs

def reduce_over_ranks(dt: float, upd: float, dist, device):
    """Weak scaling: the job's time is the slowest rank's, its work the sum of
    the ranks' leaf updates (every rank advances its own batch)."""
    import torch

    t = torch.tensor([dt, float(upd)], dtype=torch.float64, device=device)
    tmax, tsum = t[:1].clone(), t[1:].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def run_gpu(insts, precision: int, steps: int, warmup: int, dist, block=None):
    import numpy as np
    import torch

    from paper_2102_12163_gb300 import MRLBM

    dev = torch.cuda.current_device()
    s = MRLBM(insts, precision=precision, device=f"cuda:{dev}", block=block)
    s.set_initial()
    s.advance(warmup)
    s.sync()
    # the timed steps replay a CUDA graph holding one persistent launch of G steps;
    # launch shape from the autotuner over launches of the same G steps (state
    # restored afterwards) unless fixed
    G = GRAPH_STEPS if steps % GRAPH_STEPS == 0 else steps
    tune = s.autotune(G) if block is None else {"block": block, "fixed": True}
    l0 = s.launches()
    graph = s.capture(G)
    kernels_per_graph = s.launches() - l0  # one kernel per variant group the batch holds
    saved = torch.empty_like(s.ws)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk, torch.cuda.stream(s.stream):
        # clock pre-roll: the same replays on the same state for >= CLOCK_PREROLL_S, then the
        # state is restored, so the timed region runs steps W+1..W+K on a GPU under this load
        saved.copy_(s.ws)
        torch.cuda.synchronize()
        clk.mark("load_start")
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < CLOCK_PREROLL_S:
            for _ in range(4):
                graph.replay()
            s.stream.synchronize()
        s.ws.copy_(saved)
        torch.cuda.synchronize()
        u0, _, _ = s.stats()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clk.mark("timed_start")
        ev0.record(s.stream)
        for _ in range(steps // G):
            graph.replay()
        ev1.record(s.stream)
        ev1.synchronize()
        clk.mark("timed_end")
    torch.cuda.synchronize()
    del saved
    s.sync()
    dt = ev0.elapsed_time(ev1) / 1e3
    launches = (steps // G) * kernels_per_graph
    u1, _, _ = s.stats()
    upd = u1 - u0
    q = np.array([i.q for i in insts], dtype=np.float64)
    # algorithmic bytes: each leaf's q populations read and written once per step
    # (the batch mean q over the current leaves)
    _, nleaf = s.summary()
    qmean = float((q * nleaf).sum() / max(1, nleaf.sum()))
    vb = 4 if precision == 1 else 8
    if dist:
        dt, upd = reduce_over_ranks(dt, upd, dist, "cuda")
    return {
        "solver": s, "dt": dt, "updates": upd, "launches": launches, "clocks": clk.summary(), "tune": tune,
        "graph_steps": G, "kernels_per_graph": kernels_per_graph,
        "bytes_alg": 2.0 * qmean * vb * upd, "qmean": qmean,
    }


def e2e(s, steps: int):
    """Same metric through the public API with host buffers: pinned initial data
    uploaded, K steps, per-instance summary read back, all inside the timer."""
    import torch

    host = torch.from_numpy(s.initial_data()).pin_memory()
    n = len(s.instances)
    mass = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    nleaf = torch.empty(n, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.set_initial(host)
    s.advance(steps)
    s.summary(mass, nleaf)
    t = time.perf_counter() - t0
    upd, _, _ = s.stats()
    return {"value": upd / t, "unit": UNIT, "h2d_bytes_per_step": host.numel() * 8 / steps,
            "d2h_bytes_per_step": (mass.numel() * 8 + nleaf.numel() * 4) / steps, "seconds": t}


def singles(latency):
    """Configurations 1-4 as single instances, both precisions: one launch of
    the timed steps after a warm-up, CUDA events; the floor is the step's chain
    of dependent passes (team barriers per step, counted on the device) times
    the measured cost of one warp-to-warp hand-over through global memory and
    a barrier, at the maximum SM clock."""
    import torch

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, MRLBM
    from paper_2102_12163_gb300 import workloads as W

    sm_max = 2070.0
    out = {}
    for name in SINGLES:
        warm, K = SINGLE_STEPS[name]
        inst = W.WORKLOADS[name]()
        row = {"Jmax": inst.Jmax, "steps_timed": K, "after_steps": warm}
        for key, prec in (("fp64", MR_FP64), ("fp32", MR_FP32_MIXED)):
            s = MRLBM(inst, precision=prec)
            s.set_initial()
            s.advance(warm)
            s.sync()
            u0, _, _ = s.stats()
            st0, ps0 = s.step_passes()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.advance(K)
            e1.record(s.stream)
            e1.synchronize()
            s.sync()
            dt = e0.elapsed_time(e1) / 1e3
            u1, _, _ = s.stats()
            st1, ps1 = s.step_passes()
            # the kernel variants of the large instances count their barriers; the batch
            # variants (Jmax < 15 here) do not (it cost them 7 %), so these get no floor
            passes = (ps1 - ps0) / max(1, st1 - st0) if ps1 > ps0 else None
            floor_us = passes * latency["global_handover_cycles"] / sm_max if passes else None
            row[key] = {"us_per_step": dt / K * 1e6, "updates_per_s": (u1 - u0) / dt,
                        "leaves_per_step": (u1 - u0) / K, "passes_per_step": passes,
                        "floor_us_per_step": floor_us,
                        "step_over_floor": dt / K * 1e6 / floor_us if floor_us else None}
            s.close()
        out[name] = row
    out["floor_model"] = {"handover": latency, "sm_clock_mhz": sm_max,
                          "meaning": "passes per step x one warp-to-warp hand-over through global memory and a "
                                     "block barrier (mr_probe_latency), at the maximum SM clock; passes are counted "
                                     "by the kernel variant of instances with >= 2048 mask words per bitmask "
                                     "(Jmax >= 15), null for the others"}
    return out


# --------------------------------------------------------------------------- accuracy (untimed)

def _moment_errors(a, b, dx):
    import numpy as np

    d = np.abs(a - b)
    return {"l1": [float(dx * r.sum()) for r in d], "linf": [float(r.max()) for r in d],
            "linf_rel": [float(r.max() / max(np.abs(bb).max(), 1e-300)) for r, bb in zip(d, b)]}


def accuracy(insts, batch_every: int = 64, batch_steps: int = 64):
    """FP64 and FP32 paths against the FP64 oracle (finest reconstruction of the
    conserved moments, per moment: L1 weighted by dx and Linf) on configurations
    1-4 and on a sample of the batch; perturbation errors delta (L1 over the
    conserved moments against the uniform reference scheme run by the oracle)
    of FP32 at eps and FP64 at eps and 2 eps, and the matched-error check FP32
    at eps <= FP64 at 2 eps, with the same check of FP64 at eps as control."""
    import numpy as np

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, MRLBM
    from paper_2102_12163_gb300 import workloads as W

    cases = []
    for name in SINGLES:
        inst = W.WORKLOADS[name]()
        n = ACCURACY_STEPS[name] or inst.nsteps
        cases.append((name, inst, n))
    sample = insts[::batch_every] if len(insts) > batch_every else insts
    cores, _ = host_cores()
    t0 = time.perf_counter()
    with _pool(cores) as ex:
        futs = [ex.submit(_oracle_run_task, (inst, n)) for _, inst, n in cases]
        bfuts = [ex.submit(_oracle_run_task, (inst, batch_steps)) for inst in sample]

        def gpu_finest(ins, prec, n, scale=1.0):
            ins = ins if isinstance(ins, list) else [ins]
            run = [i.with_(eps=i.eps * scale) for i in ins]
            for a, b in zip(run, ins):
                a.m0 = b.m0
            s = MRLBM(run if len(run) > 1 else run[0], precision=prec)
            s.set_initial()
            s.advance(n)
            s.sync()
            out = [s.finest(i) for i in range(len(run))]
            s.close()
            return out

        gpu = {}
        for name, inst, n in cases:
            gpu[name] = {"fp64": gpu_finest(inst, MR_FP64, n)[0], "fp32": gpu_finest(inst, MR_FP32_MIXED, n)[0],
                         "fp64_2eps": gpu_finest(inst, MR_FP64, n, 2.0)[0]}
        b64 = gpu_finest(sample, MR_FP64, batch_steps)
        b32 = gpu_finest(sample, MR_FP32_MIXED, batch_steps)
        b64x2 = gpu_finest(sample, MR_FP64, batch_steps, 2.0)
        orc = [f.result() for f in futs]
        borc = [f.result() for f in bfuts]
    out = {}
    for (name, inst, n), (m_orc, m_ref) in zip(cases, orc):
        g = gpu[name]
        dl = lambda m: float(inst.dx * np.abs(m - m_ref).sum())  # noqa: E731
        d32, d64, d64x2 = dl(g["fp32"]), dl(g["fp64"]), dl(g["fp64_2eps"])
        out[name] = {"steps": n, "full_T": ACCURACY_STEPS[name] is None,
                     "fp64_vs_oracle": _moment_errors(g["fp64"], m_orc, inst.dx),
                     "fp32_vs_oracle": _moment_errors(g["fp32"], m_orc, inst.dx),
                     "delta_fp32_eps": d32, "delta_fp64_eps": d64, "delta_fp64_2eps": d64x2,
                     "delta_oracle_eps": dl(m_orc),
                     "fp32_within_fp64_at_2eps": bool(d32 <= d64x2 * (1 + 1e-12))}
    ok32 = ok64 = 0
    l1_64, l1_32, lr_64, lr_32, deltas = [], [], [], [], []
    for i, inst in enumerate(sample):
        m_orc, m_ref = borc[i]
        dl = lambda m: float(inst.dx * np.abs(m - m_ref).sum())  # noqa: E731
        d32, d64, d64x2 = dl(b32[i]), dl(b64[i]), dl(b64x2[i])
        ok32 += d32 <= d64x2 * (1 + 1e-12)
        ok64 += d64 <= d64x2 * (1 + 1e-12)
        e64, e32 = _moment_errors(b64[i], m_orc, inst.dx), _moment_errors(b32[i], m_orc, inst.dx)
        l1_64.append(max(e64["l1"]))
        l1_32.append(max(e32["l1"]))
        lr_64.append(max(e64["linf_rel"]))
        lr_32.append(max(e32["linf_rel"]))
        deltas.append((d32, d64, d64x2))
    dd = np.array(deltas)
    out["batch_sample"] = {
        "instances": len(sample), "steps": batch_steps,
        "fp64_vs_oracle": {"l1_max": max(l1_64), "linf_rel_max": max(lr_64)},
        "fp32_vs_oracle": {"l1_max": max(l1_32), "l1_median": float(np.median(l1_32)), "linf_rel_max": max(lr_32)},
        "delta_fp32_eps_median": float(np.median(dd[:, 0])), "delta_fp64_eps_median": float(np.median(dd[:, 1])),
        "delta_fp64_2eps_median": float(np.median(dd[:, 2])),
        "fp32_within_fp64_at_2eps": f"{ok32}/{len(sample)}",
        "control_fp64_eps_within_fp64_at_2eps": f"{ok64}/{len(sample)}",
    }
    out["reference"] = "FP64 oracle (oracle/) on the same inputs; delta against the oracle's uniform finest-lattice scheme"
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def accuracy_scalar(inst, name: str):
    """Tests I-IV of Table 1 at their final time: E = reference scheme (the FP64
    path at eps = 0) against the exact solution, delta = adaptive against the
    reference, for both precisions, with the paper's Table 2 ratio at s = 1."""
    import numpy as np

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, MRLBM
    from paper_2102_12163_gb300 import workloads as W

    test = {"test1": "I", "test2": "II", "test3": "III", "test4": "IV", "sw_d1q3": "SW", "sw_d1q5": "SW"}[name]
    table2_s1 = {"I": 59.4, "II": 2310.0, "III": 37.1, "IV": 341.0}.get(test)
    N = inst.nsteps

    def run(prec, eps):
        i = inst.with_(eps=eps)
        s = MRLBM(i, precision=prec)
        s.set_initial()
        s.advance(N)
        s.sync()
        out, nl = s.finest(), len(s.leaves()[0])
        s.close()
        return out, nl

    edges = W.cell_edges(inst.a, inst.b, inst.Jmax)
    if test == "SW":  # dam break of Section 5.2: both conserved moments (h, hu)
        M, _ = run(MR_FP64, 0.0)
        exact = W.sw_riemann_exact(edges, N * inst.dx / inst.lam)
    else:
        M, _ = run(MR_FP64, 0.0)
        M, exact = M[:1], W.scalar_exact(test, edges, N * inst.dx / inst.lam)[None, :]
    E = float(inst.dx * np.abs(exact - M).sum())
    out = {"test": test if test != "SW" else f"dam break, {name[3:].upper()}", "s": inst.s[0], "steps": N,
           "E_reference_vs_exact": E, "table2_E_over_delta_at_s1": table2_s1}
    for key, prec in (("fp64", MR_FP64), ("fp32", MR_FP32_MIXED)):
        f, nl = run(prec, inst.eps)
        d = float(inst.dx * np.abs(M - f[: M.shape[0]]).sum())
        out[key] = {"delta": d, "E_over_delta": E / d if d > 0 else None,
                    "compression_percent": 100.0 * (1.0 - nl / (1 << inst.Jmax))}
    return out


# --------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1024)
    ap.add_argument("--warmup", type=int, default=16)
    ap.add_argument("--instances", type=int, default=4096, help="batch size (smaller only for profiling)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "batch_sw", "advection", "burgers", "shallow", "sod", "test1", "test2", "test3",
                             "test4", "sw_d1q3", "sw_d1q5"])
    ap.add_argument("--block", type=int, default=None)
    ap.add_argument("--gamma", type=int, default=1, choices=[1, 2, 3],
                    help="prediction stencil half-width of every instance (Section 3.1)")
    ap.add_argument("--collision", default="leaves", choices=["leaves", "reconstructed"],
                    help="collision of the adaptive scheme (Section 4.5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="same as --precision fp32")
    ap.add_argument("--precision", default="both", choices=["both", "fp32", "fp64"],
                    help="legs to time: the FP64 headline with FP32 beside it, or one of them")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-singles", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    insts, desc = make_workload(args.workload, rank, args.instances)
    if args.gamma != 1 or args.collision != "leaves":
        coll = 1 if args.collision == "reconstructed" else 0
        for i in range(len(insts)):
            insts[i] = insts[i].with_(gamma=args.gamma, collision=coll)
        if args.gamma != 1:
            desc += f"; prediction stencil gamma = {args.gamma}"
        if coll:
            desc += "; reconstructed collision"
    hbm, hbm_src = peaks()

    if args.impl == "reference":
        # the reference arm is the oracle as it stands, on the host cores, rank 0 only
        if rank != 0:
            return
        K, W = args.steps, args.warmup
        value, cores, sample, ms_step = oracle_throughput(insts, target_s=max(5.0, 60.0 / max(1, K)) * K / 4)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": W,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": desc},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as td

        torch.cuda.set_device(local)
        td.init_process_group("nccl")
        dist = td
    else:
        torch.cuda.set_device(0)

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, probe_latency

    if args.no_fp64:
        args.precision = "fp32"
    r32 = r64 = None
    if args.precision in ("both", "fp64"):
        r64 = run_gpu(insts, MR_FP64, args.steps, args.warmup, dist, args.block)
    if args.precision in ("both", "fp32"):
        r32 = run_gpu(insts, MR_FP32_MIXED, args.steps, args.warmup, dist, args.block)
    head = r64 if r64 is not None else r32
    head_prec = "fp64" if r64 is not None else "fp32"
    ee = e2e(head["solver"], args.steps)
    for r in (r32, r64):
        if r is not None:
            r["solver"].close()

    sing = None
    if rank == 0 and not args.no_singles and args.workload in ("batch", "batch_sw"):
        sing = singles(probe_latency(f"cuda:{torch.cuda.current_device()}"))

    acc = None
    if rank == 0 and not args.no_accuracy and args.workload == "batch":
        acc = accuracy(insts)
    elif rank == 0 and not args.no_accuracy and (args.workload.startswith("test") or args.workload.startswith("sw_")):
        acc = accuracy_scalar(insts[0], args.workload)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_throughput(insts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if dist:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    def roof(r, prec):
        achieved = r["bytes_alg"] / r["dt"] / 1e9
        tr = (profiled_traffic(args.workload, prec, r["graph_steps"])
              if len(insts) == 4096 or args.workload != "batch" else None)
        launches = max(1, r["launches"])
        per_launch_updates = r["updates"] / launches
        out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
               "traffic": (tr["dram_bytes_per_update"] * per_launch_updates if tr else None),
               "traffic_unit": "DRAM bytes per launch (ncu DRAM bytes per leaf update x this run's leaf updates "
                               "per launch)",
               "algorithmic_bytes_per_launch": r["bytes_alg"] / launches,
               "launch_ms": r["dt"] * 1e3 / launches,
               "peak_source": f"{hbm_src} HBM copy bandwidth (MEASURED_PEAKS.json)" if hbm_src == "measured"
               else "fallback 6.8 TB/s",
               "algorithmic_bytes_per_update": 2 * r["qmean"] * (4 if prec == "fp32" else 8)}
        if tr:
            out["dram_bytes_per_update"] = tr["dram_bytes_per_update"]
            if "fp64_pipe_active_pct" in tr:
                # GB300's FP64 units are the other roof of this kernel (two FP64 operations per SM per cycle)
                out["fp64_pipe_active_pct"] = tr["fp64_pipe_active_pct"]
        return out

    def leg(r, prec):
        return {"value": r["updates"] / r["dt"], "ms_per_step": r["dt"] * 1e3 / args.steps,
                "roofline": roof(r, prec), "gpu_launches": r["launches"], "clocks": r["clocks"],
                "autotune": r["tune"]}

    line = {
        "metric": METRIC, "value": head["updates"] / head["dt"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["dt"] * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head_prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": desc, "instances_per_gpu": len(insts), "steps_per_launch": head["graph_steps"],
                   "launch": f"CUDA graph of {head['graph_steps']} steps: one persistent launch per kernel "
                             f"variant the batch needs ({head['kernels_per_graph']}"
                             f"{', on forked streams' if head['kernels_per_graph'] > 1 else ''}), replayed",
                   "autotune": head["tune"],
                   "l2": "inputs larger than L2 (per-GPU workspace of several GB)",
                   "precision": "headline: FP64 throughout; 'fp32': FP32 populations, FP64 detail test near the "
                                "thresholds, mass audit in float-float partials with FP64 totals"},
        "roofline": roof(head, head_prec),
        "cpu_baseline": cpu,
        "e2e": ee,
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
    }
    if r32 is not None and r64 is not None:
        line["fp32"] = leg(r32, "fp32")
    line["singles"] = sing
    line["accuracy"] = acc
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
