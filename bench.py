"""Benchmark of the adaptive MR-LBM step on GB300: leaf-cell updates per second.

A step is one adaptive time step (multiresolution analysis, mesh update, data
transfer, leaves collision, reconstructed-flux stream) of every instance of the
workload.  The default workload is the mixed batch of 4096 independent
instances (D1Q2 advection / Burgers, vectorial D1Q2^2 shallow water, vectorial
D1Q2^3 Euler; Jmax uniform in 8..14; eps log-uniform in [1e-5, 1e-2];
piecewise-constant data with 1..6 jumps), run in FP32 (the headline) and in
FP64 on the same inputs.  Timed: exactly K steps in one persistent launch,
bracketed by a barrier and a device synchronisation, CUDA events on the
solver's stream; the per-GPU state (several GB) is far larger than L2.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--workload batch|burgers|sod|shallow|advection]

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


def profiled_traffic(workload: str, precision: str, graph_steps: int, instances: int):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.json),
    if it was taken on the current kernel source and the same launch (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            j = json.load(fh)
        e = j[f"{workload}:{precision}"]
        if e.get("source_hash") != source_hash() or e.get("graph_steps") != graph_steps:
            return None
        if e.get("instances") != instances:
            return None
        return e
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

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
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(name: str, rank: int, n_batch: int = 4096):
    from paper_2102_12163_gb300 import workloads as W

    if name == "batch":
        insts = W.batch(n=n_batch, seed=12163 + rank)
        desc = f"batch of {n_batch} mixed D1Q2 advection/Burgers, D1Q2^2 shallow water, D1Q2^3 Euler; Jmax 8..14; eps 1e-5..1e-2"
    elif name == "batch_sw":
        insts = W.batch_sw(n=n_batch, seed=5202 + rank)
        desc = f"batch of {n_batch} shallow water instances, D1Q3 / D1Q5 (Section 5.2); Jmax 8..14; eps 1e-5..1e-2"
    else:
        insts = [W.WORKLOADS[name]()]
        i = insts[0]
        desc = f"{name} single instance, Jmin {i.Jmin} Jmax {i.Jmax} eps {i.eps:g}"
    return insts, desc


# --------------------------------------------------------------------------- oracle (CPU) timing

def _oracle_task(args):
    inst, warm, n = args
    sys.path.insert(0, ROOT)
    import oracle as O

    p = O.Params(Jmin=inst.Jmin, Jmax=inst.Jmax, eq=inst.eq, lam=inst.lam, eps=inst.eps, gamma=inst.gamma,
                 mu_bar=inst.mu_bar, bc=inst.bc, a=inst.a, b=inst.b, s=inst.s, eqp=inst.eqp,
                    collision=inst.collision)
    o = O.Oracle(p)
    o.set_initial(inst.m0)
    o.step(warm)
    upd = 0
    t0 = time.perf_counter()
    for _ in range(n):
        o.step()
        upd += len(o.leaves()[0])
    return upd, time.perf_counter() - t0


def oracle_throughput(insts, target_s: float = 15.0, warm: int = 4):
    """The oracle as it stands on a bounded sample of the workload, spread over
    the host cores with a spawned process pool; returns (value, cores, sample)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    cores = max(1, min(os.cpu_count() or 1, 16))
    stride = max(1, len(insts) // (8 * cores))
    sample = insts[::stride][: 8 * cores]
    # calibrate the step cost on a few sampled instances
    cal = [_oracle_task((i, warm, 1))[1] for i in sample[: min(8, len(sample))]]
    per_step = max(sum(cal) / len(cal), 1e-5)
    n = int(max(1, min(2048, target_s * cores / (per_step * len(sample)))))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ProcessPoolExecutor(cores, mp_context=ctx) as ex:
        res = list(ex.map(_oracle_task, [(i, warm, n) for i in sample]))
    wall = time.perf_counter() - t0
    upd = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    value = upd / busy * cores
    desc = (f"{len(sample)} of {len(insts)} instances (every {stride}th), {warm} untimed + {n} timed steps each, "
            f"{cores} worker processes, {wall:.1f} s wall")
    return value, cores, desc


# --------------------------------------------------------------------------- GPU leg

def reduce_over_ranks(dt: float, upd: float, dist, device):
    """Weak scaling: the job's time is the slowest rank's, its work the sum of
    the ranks' leaf updates (every rank advances its own batch)."""
    import torch

    t = torch.tensor([dt, float(upd)], dtype=torch.float64, device=device)
    tmax, tsum = t[:1].clone(), t[1:].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


def run_gpu(insts, precision: int, steps: int, warmup: int, rank: int, world: int, dist, block=None):
    import numpy as np
    import torch

    from paper_2102_12163_gb300 import MRLBM

    s = MRLBM(insts, precision=precision, device=f"cuda:{torch.cuda.current_device()}", block=block)
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
    u0, _, _ = s.stats()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk, torch.cuda.stream(s.stream):
        t_wall = time.perf_counter()
        ev0.record(s.stream)
        for _ in range(steps // G):
            graph.replay()
        ev1.record(s.stream)
        ev1.synchronize()
        t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    s.sync()
    dt = ev0.elapsed_time(ev1) / 1e3
    launches = (steps // G) * kernels_per_graph
    u1, _, _ = s.stats()
    upd = u1 - u0
    q = np.array([i.q for i in insts], dtype=np.float64)
    # algorithmic bytes: each leaf's q populations read and written once per step
    # (the per-instance mean q weighted by that instance's updates is not
    # tracked on the device, so the batch mean q over leaves is used)
    _, nleaf = s.summary()
    qmean = float((q * nleaf).sum() / max(1, nleaf.sum()))
    vb = 4 if precision == 1 else 8
    if dist:
        dt, upd = reduce_over_ranks(dt, upd, dist, "cuda")
    res = {
        "solver": s, "dt": dt, "updates": upd, "launches": launches, "clocks": clk.summary(), "tune": tune,
        "graph_steps": G, "kernels_per_graph": kernels_per_graph,
        "bytes_alg": 2.0 * qmean * vb * upd, "qmean": qmean, "t_wall": t_wall,
    }
    return res


def e2e(s, steps: int):
    """Same metric through the public API with host buffers: pinned initial data
    uploaded, K steps, per-instance summary read back, all inside the timer."""
    import numpy as np
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
    del np
    return {"value": upd / t, "unit": UNIT, "h2d_bytes_per_step": host.numel() * 8 / steps,
            "d2h_bytes_per_step": (mass.numel() * 8 + nleaf.numel() * 4) / steps, "seconds": t}


# --------------------------------------------------------------------------- accuracy (untimed)

def accuracy(insts, steps: int, every: int = 256):
    """L1 error of the conserved moments against the uniform reference scheme,
    FP32 at eps versus FP64 at eps and at 2 eps, on a sample of the workload.
    The reference is the FP64 path at eps = 0 (the adaptive scheme on the full
    tree is the reference scheme on the finest lattice)."""
    import numpy as np

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64, MRLBM

    sample = insts[::every] if len(insts) > every else insts

    def run(prec, scale):
        ins = [i.with_(eps=i.eps * scale) for i in sample]
        for a, b in zip(ins, sample):
            a.m0 = b.m0
        s = MRLBM(ins, precision=prec)
        s.set_initial()
        s.advance(steps)
        s.sync()
        out = [s.finest(i) for i in range(len(ins))]
        s.close()
        return out

    ref = run(MR_FP64, 0.0)
    f64, f64x2, f32 = run(MR_FP64, 1.0), run(MR_FP64, 2.0), run(MR_FP32_MIXED, 1.0)
    rows = []
    for i, inst in enumerate(sample):
        d = lambda m: float(inst.dx * np.abs(m - ref[i]).sum())  # noqa: E731  (weighted l1, all fields)
        rows.append((d(f32[i]), d(f64[i]), d(f64x2[i]), float(np.max(np.abs(f32[i] - f64[i])))))
    r = np.array(rows)
    ok = r[:, 0] <= r[:, 2] * (1 + 1e-12) + 1e-15
    return {
        "instances": len(sample), "steps": steps,
        "delta_l1_fp32_eps_median": float(np.median(r[:, 0])),
        "delta_l1_fp64_eps_median": float(np.median(r[:, 1])),
        "delta_l1_fp64_2eps_median": float(np.median(r[:, 2])),
        "fp32_within_fp64_at_2eps": f"{int(ok.sum())}/{len(sample)}",
        "fp32_vs_fp64_linf_max": float(r[:, 3].max()),
        "reference": "uniform finest-lattice scheme (FP64 path at eps = 0)",
    }


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
                    help="legs to time: the FP32 headline with FP64 beside it, or one of them")
    ap.add_argument("--no-accuracy", action="store_true")
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
        value, cores, sample = oracle_throughput(insts, target_s=max(5.0, 60.0 / max(1, K)) * K / 4)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": W,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
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

    from paper_2102_12163_gb300 import MR_FP32_MIXED, MR_FP64

    if args.no_fp64:
        args.precision = "fp32"
    r32 = r64 = None
    if args.precision in ("both", "fp32"):
        r32 = run_gpu(insts, MR_FP32_MIXED, args.steps, args.warmup, rank, world, dist, args.block)
    if args.precision in ("both", "fp64"):
        r64 = run_gpu(insts, MR_FP64, args.steps, args.warmup, rank, world, dist, args.block)
    head = r32 if r32 is not None else r64
    head_prec = "fp32" if r32 is not None else "fp64"
    ee = e2e(head["solver"], args.steps)

    acc = None
    if rank == 0 and not args.no_accuracy and args.workload == "batch":
        acc = accuracy(insts, min(args.steps, 64))
    elif rank == 0 and not args.no_accuracy and (args.workload.startswith("test") or args.workload.startswith("sw_")):
        acc = accuracy_scalar(insts[0], args.workload)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_throughput(insts)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if dist:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return

    def roof(r, prec):
        achieved = r["bytes_alg"] / r["dt"] / 1e9
        tr = profiled_traffic(args.workload, prec, r["graph_steps"], len(insts))
        out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                "traffic_unit": f"DRAM bytes per graph replay ({r['graph_steps']} steps of every instance, "
                                f"{r['kernels_per_graph']} kernels), ncu",
                "peak_source": f"{hbm_src} HBM copy bandwidth (MEASURED_PEAKS.json)" if hbm_src == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_update": 2 * r["qmean"] * (4 if prec == "fp32" else 8)}
        if tr and "fp64_pipe_active_pct" in tr:
            # GB300's FP64 units are the other roof of this kernel (two FP64 operations per SM per cycle)
            out["fp64_pipe_active_pct"] = tr["fp64_pipe_active_pct"]
        return out

    line = {
        "metric": METRIC, "value": head["updates"] / head["dt"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["dt"] * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if head_prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": desc, "instances_per_gpu": len(insts), "steps_per_launch": head["graph_steps"],
                   "launch": f"CUDA graph of {head['graph_steps']} steps: one persistent launch per kernel "
                             f"variant the batch needs ({head['kernels_per_graph']}"
                             f"{', on forked streams' if head['kernels_per_graph'] > 1 else ''}), replayed",
                   "autotune": head["tune"],
                   "l2": "inputs larger than L2 (per-GPU workspace of several GB)",
                   "precision": "FP32 populations; FP64 detail test near the thresholds; mass audit in "
                                "float-float partials with FP64 totals"},
        "roofline": roof(head, head_prec),
        "cpu_baseline": cpu,
        "e2e": ee,
        "gpu_launches": head["launches"],
        "clocks": head["clocks"],
        "accuracy": acc,
    }
    if r64 is not None and r32 is not None:
        line["fp64"] = {"value": r64["updates"] / r64["dt"], "ms_per_step": r64["dt"] * 1e3 / args.steps,
                        "roofline": roof(r64, "fp64"), "gpu_launches": r64["launches"], "clocks": r64["clocks"],
                        "autotune": r64["tune"]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
