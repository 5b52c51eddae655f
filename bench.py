#!/usr/bin/env python
"""Benchmark of the GB300 market-split lattice solver.

One step = the whole hot path over one batch: lattice of Eq. (2), LLL,
kernel extraction and Gram-Schmidt, top-level split and exhaustive
enumeration of all solutions (Algorithm 1) for 64 synthetic instances with m
uniform in {4,5,6,7}, n = 10(m-1), D cycling over {50, 100, 200} (the batch
workload).  The metric is evaluated nodes per second (a node = one candidate
(t, u_t) whose norm is computed).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  `value` is device-timed with inputs resident
in HBM; `e2e` is the same metric through the C ABI from host buffers, with
the host->device copy of the instances and the device->host read of the
statistics and solutions inside the timed region.  L2 is flushed between
timed steps.  The reference arm is the CPU oracle (oracle/), timed on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "enum nodes/s; time to all sols (m=9) & first sol (m=12), learned vs plain order"
# the autotuner's grid for the batch (coordinate descent, library defaults first)
TUNE_GRID = {"lanes": (8, 16), "warps_per_block": (8, 4), "blocks_per_sm": (0, 1),
             "split_target": (0, 256, 4096, 16384)}
DRAM_BYTES_PER_NODE = (126.395648e6 + 516.611072e6) / 268321291   # enum_kernel<8, 8, 0>, ncu
# FP64 lane operations the same capture executed, per evaluated node (ncu
# sm__sass_thread_inst_executed_op_fp64_pred_on): the counter-based FP64 work
FP64_LANE_OPS_PER_NODE = 7249881043 / 268321291
UNIT = "nodes/s"
WORKLOAD = "batch of 64 fMSP instances, m~U{4..7}, n=10(m-1), D in {50,100,200}, all solutions"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--lanes", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=30.0)
    p.add_argument("--instances", type=int, default=64,
                   help="run only the first K instances of the batch (small profiling cases)")
    p.add_argument("--workload", default="batch64", choices=["batch64"] + sorted(WORKLOADS),
                   help="batch64: the nodes/s benchmark; the others time the paper's all- and "
                        "first-solution configurations once (one GPU)")
    p.add_argument("--bkz", type=int, default=None, help="BKZ block size (default: 0 for batch64, 10 otherwise)")
    p.add_argument("--cap", type=float, default=None, help="time cap in seconds for the other workloads")
    p.add_argument("--orders", default="plain,learned,lds,lds_learned",
                   help="first-solution workloads: orders to time")
    p.add_argument("--no-tune", action="store_true", help="batch64: library defaults instead of the autotuner")
    p.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                   help="other workloads: set an msp_opts field (e.g. replicas=4, lds_rank=0)")
    p.add_argument("--no-headline", action="store_true",
                   help="batch64: skip the m=9 all-solutions and m=12 first-solution runs")
    return p.parse_args()


# The paper's larger configurations (synthetic stand-ins, seeds in instances.py):
# name -> (generator spec, mode, default time cap in seconds); a spec is the
# name of a generator of instances.py, or (name, positional arguments)
WORKLOADS = {
    "m8_all": ("m8_n70", "all", 300.0),     # m=8, n=70, D=200, 16 instances
    "m9_all": ("m9_n80", "all", 1200.0),    # m=9, n=80, D=100, 8 instances, 40 ones planted
    "m8_first": ("m8_n70", "first", 120.0),
    "m12_first": ("m12_n110", "first", 60.0),   # m=12, n=110, D=100, 4 instances
    "m10d50_first": ("m10_n90_d50", "first", 30.0),    # m=10, n=90, D=50, 4 planted instances
    "m11d50_first": ("m11_n100_d50", "first", 30.0),   # m=11, n=100, D=50, 4 planted instances
    "m12d50_first": ("m12_n110_d50", "first", 60.0),   # m=12, n=110, D=50, 4 planted instances
    "cd8_all": (("cd_batch", (8, 16)), "all", 600.0),   # Cornuejols-Dawande m=8 (nothing planted), 16 instances
    # centred right-hand sides (the paper's instance library's solution counts), D = 50
    "m7c50_all": (("centred", (7, 50)), "all", 120.0),
    "m8c50_all": (("centred", (8, 50)), "all", 300.0),
    "m9c100_all": (("centred", (9, 100)), "all", 1200.0),
    "m10c50_first": (("centred", (10, 50)), "first", 30.0),
    "m11c50_first": (("centred", (11, 50)), "first", 60.0),
    "m12c50_first": (("centred", (12, 50)), "first", 120.0),
}


def make_instances(spec):
    """The instances of a WORKLOADS generator spec."""
    from paper_2508_08702_gb300 import instances as I
    if isinstance(spec, str):
        return getattr(I, spec)()
    name, args = spec
    return getattr(I, name)(*args)


def _verified(ctx, i, inst):
    """Every reported x solves A x = d exactly; is the planted x among them?"""
    import numpy as np
    xs = ctx.msp_solutions(i).astype(np.int64)
    ok = all(np.array_equal(x @ inst.A.T.astype(np.int64), inst.d) for x in xs)
    planted = inst.planted is not None and any(np.array_equal(inst.planted, x) for x in xs)
    return ok, planted, len(xs)


def run_all_solutions(insts, cap, **opts):
    """Wall time from the reduction to the verified solutions of the whole
    batch (the paper's timings include the reduction), one launch."""
    import torch
    from paper_2508_08702_gb300 import instances as I
    from paper_2508_08702_gb300 import msp as M
    pk = I.pack(insts)
    ctx = M.Context(max_seconds=cap + 60, **opts)
    ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.msp_reduce()
    res = ctx.msp_enumerate(M.MSP_ALL, M.MSP_PLAIN, cap, allow=(M.MSP_OK, M.MSP_ETIMEOUT))
    wall = time.perf_counter() - t0
    ph = ctx.msp_phase_ms()
    checks = [_verified(ctx, i, x) for i, x in enumerate(insts)]
    out = {"wall_s": round(wall, 3), "complete": res.status == M.MSP_OK, "status": res.status,
           "lanes": ctx.lanes, "phase_ms": {k: round(v, 1) for k, v in ph.items()},
           "nodes": res.total["nodes"], "nodes_per_s": res.total["nodes"] / max(ph["enumerate"] / 1e3, 1e-9),
           "solutions": [c[2] for c in checks], "all_verified": all(c[0] for c in checks),
           "planted_found": sum(c[1] for c in checks),
           "proved_infeasible": sum(1 for c in checks if c[2] == 0) if res.status == M.MSP_OK else 0}
    ctx.close()
    return out


def train_scorer():
    """The subtree scorer, trained on the device on 256 generated m = 5..7
    instances (seeds disjoint from every evaluation set)."""
    from paper_2508_08702_gb300 import instances as I
    from paper_2508_08702_gb300 import learn
    t0 = time.perf_counter()
    data = learn.collect(I.training_set(256))
    theta, _ = learn.train(data, steps=4000)
    return theta, round(time.perf_counter() - t0, 2)


def run_first_solution(insts, cap, orders, theta=None, **opts):
    """Per order: wall time of reduction + search, and each instance's time
    to its first verified solution from the start of the enumeration."""
    import numpy as np
    import torch
    from paper_2508_08702_gb300 import instances as I
    from paper_2508_08702_gb300 import msp as M
    pk = I.pack(insts)
    names = {"plain": M.MSP_PLAIN, "learned": M.MSP_LEARNED, "lds": M.MSP_LDS, "lds_learned": M.MSP_LDS_LEARNED}
    runs = {}
    for name in orders:
        ctx = M.Context(max_seconds=cap + 60, **opts)
        if name in ("learned", "lds_learned"):
            ctx.msp_set_scorer(theta)
        ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.msp_reduce()
        res = ctx.msp_enumerate(M.MSP_FIRST, names[name], cap, allow=(M.MSP_OK, M.MSP_ETIMEOUT, M.MSP_ECAP))
        wall = time.perf_counter() - t0
        ph = ctx.msp_phase_ms()
        fm = [s["first_ms"] for s in res.stats]
        solved = [f for f in fm if f >= 0]
        checks = [_verified(ctx, i, x) for i, x in enumerate(insts)]
        runs[name] = {"wall_s": round(wall, 3), "reduce_ms": round(ph["reduce"], 1),
                      "solved": len(solved), "of": len(fm),
                      "first_s": [round(f / 1e3, 3) if f >= 0 else None for f in fm],
                      "median_first_s": round(float(np.median(fm)) / 1e3, 3) if len(solved) == len(fm) else None,
                      "nodes": res.total["nodes"], "all_verified": all(c[0] for c in checks)}
        if name.startswith("lds"):
            runs[name]["lds_budget"] = [s["lds_budget"] for s in res.stats]
        ctx.close()
    return runs


def extended(args):
    """One timed run of a paper configuration: wall time from the reduction
    to the verified solutions (the paper's timings include the reduction),
    per instance and for the batch; first-solution workloads compare the
    queue orders."""
    import torch
    from paper_2508_08702_gb300 import build as B
    from paper_2508_08702_gb300 import instances as I

    B.build()
    gen, mode, cap = WORKLOADS[args.workload]
    cap = args.cap or cap
    bkz = 10 if args.bkz is None else args.bkz
    insts = make_instances(gen)
    opts = dict(bkz_beta=bkz)
    if args.lanes:
        opts["lanes"] = args.lanes
    for kv in args.opt:
        k, v = kv.split("=", 1)
        opts[k] = float(v) if "." in v else int(v)
    data = ("synthetic, centred right-hand side d = floor(sum a / 2), nothing planted" if insts[0].planted is None
            else "synthetic (planted instances of the paper's shapes)")
    out = {"workload": args.workload, "instances": len(insts), "m": insts[0].m, "n": insts[0].n, "D": insts[0].D,
           "bkz_beta": bkz, "cap_s": cap, "data": data, "opts": opts,
           "gpu": torch.cuda.get_device_name()}
    clocks = Clocks(torch.cuda.current_device())
    if mode == "all":
        clocks.start()
        r = run_all_solutions(insts, cap, **opts)
        out["clocks"] = clocks.stop()
        out.update({"metric": "time to all solutions (reduction + enumeration), whole batch",
                    "value": r["wall_s"], "unit": "s", "higher_is_better": False}, **r)
    else:
        theta = None
        orders = args.orders.split(",")
        if any("learned" in o for o in orders):
            theta, out["scorer_training_s"] = train_scorer()
        clocks.start()
        runs = run_first_solution(insts, cap, orders, theta, **opts)
        out["clocks"] = clocks.stop()
        med = [r["median_first_s"] for r in runs.values() if r["median_first_s"] is not None]
        out.update({"metric": "median time to an instance's first solution (from the enumeration start), "
                              "best queue order", "value": min(med) if med else None, "unit": "s",
                    "higher_is_better": False, "orders": runs})
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------
def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7], pcap=f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# --------------------------------------------------------------------------
def oracle_nodes_per_s(instances, seconds: float, lanes: int = 32, min_seconds: float = 0.0):
    """The CPU oracle as it stands, one thread, on instances taken in order
    until `seconds` of work (whole passes over the list are repeated until
    `min_seconds` have passed); returns (nodes/s, nodes, seconds, count)."""
    from oracle import oracle as O
    nodes = 0
    t0 = time.perf_counter()
    done = 0
    while True:
        for inst in instances:
            r = O.solve(inst.A, inst.d, lanes=lanes).result
            nodes += r.nodes
            done += 1
            if time.perf_counter() - t0 > seconds:
                break
        dt = time.perf_counter() - t0
        if dt > seconds or dt >= min_seconds or not instances:
            break
    return nodes / dt, nodes, dt, done


def cpu_sample(instances):
    """Bounded sample of the batch for the oracle: the instances with m <= 6
    (about 2.5 s of one core in all; the m = 7 instances take the oracle 2
    to 70 s each).  The GPU's nodes/s is reported on the same sample."""
    return [x for x in instances if x.m <= 6]


def cpu_baseline_sample(instances):
    """The instances with m <= 6 and the m = 7 ones with D >= 100 (2 to 7 s
    each; with D = 50 they take 30 to 70 s)."""
    return [x for x in instances if x.m <= 6 or (x.m == 7 and getattr(x, "D", 0) >= 100)]


def cpu_baseline(sample, seconds: float, lanes: int):
    """The oracle, one thread, repeated passes over the sample (10 to
    `seconds` s of CPU work), and the same instances one per core."""
    v, nodes, dt, cnt = oracle_nodes_per_s(sample, seconds, lanes=lanes, min_seconds=10.0)
    host = host_cpu()
    out = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"the {len(sample)} batch instances with m<=6, {cnt} runs in order ({nodes} nodes, "
                     f"{dt:.1f} s), LLL + enumeration, one thread, |w|_1 order of {lanes}-lane walkers",
           "host": host}
    if host["nproc"] and host["nproc"] > 1:
        pv, pn, pdt = oracle_parallel_nodes_per_s(sample, host["nproc"])
        out["parallel"] = {"value": pv, "unit": UNIT, "cores": host["nproc"],
                           "sample": f"the same {len(sample)} instances, one instance per core "
                                     f"({pn} nodes, {pdt:.1f} s wall)"}
    return out


def gpu_nodes_per_s(instances, opts, steps, flush):
    """Device-timed nodes/s of whole steps on a batch (after one warm-up
    step, L2 flushed before each step); returns (nodes/s, nodes per step)."""
    import torch
    from paper_2508_08702_gb300 import instances as I
    from paper_2508_08702_gb300 import msp as M
    pk = I.pack(instances)
    ctx = M.Context(**opts)
    A_dev = torch.from_numpy(pk.A).cuda()
    d_dev = torch.from_numpy(pk.d).cuda()
    stream = torch.cuda.current_stream()
    ms, nodes = 0.0, 0
    for k in range(max(1, min(steps, 5)) + 1):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.msp_build_lattice(pk.dims, A_dev, d_dev)
        ctx.msp_run_async()
        e1.record(stream)
        res = ctx.msp_wait()
        if k > 0:
            ms += e0.elapsed_time(e1)
            nodes += res.total["nodes"]
    per_step = res.total["nodes"]
    ctx.close()
    return nodes / (ms / 1e3), per_step


def launch_desc(opts, lanes):
    """The enumeration launch in effect: the options given and the lanes chosen."""
    d = {k: v for k, v in opts.items()}
    d["lanes"] = lanes
    return d


# the headline's paper configurations (synthetic stand-ins, seeds in instances.py)
HEADLINE_FIRST = (
    # key, generator spec, runs (orders, cap in seconds, extra options), description
    ("m12_n110_d100", "m12_n110", (("plain,learned,lds,lds_learned", 15.0, {}),),
     "m=12, n=110, D=100, 4 planted instances (seeds 5000..5003)"),
    ("m12_n110_d50_centred", ("centred", (12, 50)),
     (("plain,learned", 30.0, {}), ("lds,lds_learned", 150.0, {"replicas": 4})),
     "m=12, n=110, D=50, 4 instances with the centred right-hand side (seeds 61250..61253): the paper's m=12 row"),
)


def headline(args, clocks_index=0):
    """The metric's two headline times, measured in the same run as the node
    rate: all solutions of the m = 9, n = 80, D = 100 batch (8 instances,
    BKZ-10; one warm-up on one m = 8 instance, which runs the same kernels),
    and the time to the first solution at m = 12 under the plain, learned and
    limited-discrepancy orders (BKZ-10, a cap per run; the discrepancy
    searches run 4 shuffled replicas per instance, Sec. 4)."""
    from paper_2508_08702_gb300 import instances as I
    out = {}
    clocks = Clocks(clocks_index)
    run_all_solutions(I.m8_n70(1), 120.0, bkz_beta=10)   # warm-up
    clocks.start()
    r = run_all_solutions(I.m9_n80(8), 1200.0, bkz_beta=10)
    r["clocks"] = clocks.stop()
    r["workload"] = "m=9, n=80, D=100, 8 instances, planted x with 40 ones (seeds 4000..4007), BKZ-10, all solutions"
    out["m9_all"] = r
    theta, train_s = train_scorer()
    first = {"scorer_training_s": train_s, "bkz_beta": 10, "workloads": {}}
    clocks.start()
    for key, gen, runs_spec, desc in HEADLINE_FIRST:
        insts = make_instances(gen)
        runs = {}
        for orders, cap, extra in runs_spec:
            for name, r in run_first_solution(insts, cap, orders.split(","), theta, bkz_beta=10, **extra).items():
                runs[name] = dict(r, cap_s=cap, **extra)
        first["workloads"][key] = {"workload": desc, "orders": runs}
    first["clocks"] = clocks.stop()
    out["first_solution"] = first
    return out


def _oracle_solve_nodes(Ad):
    """One instance through the oracle (a worker of the parallel leg)."""
    from oracle import oracle as O
    A, d = Ad
    return O.solve(A, d).result.nodes


def oracle_parallel_nodes_per_s(instances, workers: int):
    """The oracle one instance per core (a spawned process pool: started
    after GPU work, so no fork); returns (nodes/s, nodes, wall seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_solve_nodes, [(instances[0].A, instances[0].d)] * workers)   # workers up
        t0 = time.perf_counter()
        nodes = sum(pool.map(_oracle_solve_nodes, [(x.A, x.d) for x in instances], chunksize=1))
        dt = time.perf_counter() - t0
    return nodes / dt, nodes, dt


def host_cpu():
    """Core count and model of the host, as lscpu reports them."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.processor(), "machine": platform.machine()}


def reference_arm(args, rank, world):
    from paper_2508_08702_gb300 import instances as I
    if rank != 0:
        return
    # the same sample as the main arm's cpu_baseline and its gpu_same_sample
    insts = cpu_sample(I.batch_m4_7(64))
    for _ in range(args.warmup):
        oracle_nodes_per_s(insts[:4], 1e9, lanes=8)
    vals, nodes_tot, t_tot = [], 0, 0.0
    for _ in range(args.steps):
        v, nodes, dt, _ = oracle_nodes_per_s(insts, 1e9, lanes=8)
        vals.append(v)
        nodes_tot += nodes
        t_tot += dt
    value = nodes_tot / t_tot
    sample = (f"{len(insts)} of the 64 batch instances (those with m<=6), LLL + enumeration, one thread, "
              f"|w|_1 order of 8-lane walkers")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------
def algorithmic_fp64_ops(stats, dims, lanes):
    """FP64 lane operations the canonical arithmetic needs inside the
    enumeration kernel: 3 per evaluated node (x, x^2, rho), 2 dim + log2 G + 1
    per node passing the norm test above level 0 (w update, |w|_1 partial
    sums and tree, slack add), plus the centre-fold fmas."""
    ops = 0
    for s, (m, n) in zip(stats, dims):
        dim = int(n) + 1
        nodes = s["nodes"] - s["split_nodes"]
        inner = s["passed"] - s["split_passed"] - s["leaves"]
        ops += 3 * nodes + (2 * dim + int(math.log2(lanes)) + 1) * inner + s["center_fma"]
    return ops


def main():
    args = parse()
    rank, world, local = dist_init(args.gpus)
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload != "batch64":
        if rank == 0:
            extended(args)
        return
    import numpy as np
    import torch
    from paper_2508_08702_gb300 import build as B
    from paper_2508_08702_gb300 import instances as I
    from paper_2508_08702_gb300 import msp as M

    B.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    # weak scaling: every rank runs its own batch of 64 (seeds shifted by rank)
    insts = I.batch_m4_7(64, first_seed=2000 + 64 * rank)[:args.instances]
    pk = I.pack(insts)
    kw = {} if args.lanes is None else {"lanes": args.lanes}
    tuning = None
    if not args.no_tune:
        # the launch shape and split of this batch, picked by the autotuner
        # (coordinate descent over lanes, warps per block, blocks per SM and
        # the split target; device time of whole steps)
        from paper_2508_08702_gb300 import tune
        grid = dict(TUNE_GRID)
        if args.lanes is not None:
            grid["lanes"] = (args.lanes,)
        t0 = time.perf_counter()
        tuning = tune.tune(insts, grid=grid, strategy="descent", repeats=1)
        tuning["seconds"] = round(time.perf_counter() - t0, 1)
        kw.update(tuning["opts"])
    ctx = M.Context(**kw)
    A_dev = torch.from_numpy(pk.A).to(dev)
    d_dev = torch.from_numpy(pk.d).to(dev)
    A_pin = torch.from_numpy(pk.A).pin_memory()
    d_pin = torch.from_numpy(pk.d).pin_memory()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)   # 512 MB > L2
    stream = torch.cuda.current_stream()

    def step_device():
        ctx.msp_build_lattice(pk.dims, A_dev, d_dev)
        ctx.msp_run_async()

    for _ in range(args.warmup):
        step_device()
        ctx.msp_wait()
    peak_dfma = ctx.msp_fp64_peak()
    lanes = ctx.lanes   # in effect for this batch (automatic unless --lanes)

    # ---- device-timed steps, inputs resident in HBM ----
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.kernel_launches
    times, nodes_all, enum_ms, ops_all, last = [], 0, [], 0, None
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_device()
        e1.record(stream)
        res = ctx.msp_wait()
        times.append(e0.elapsed_time(e1))
        nodes_all += res.total["nodes"]
        ph = ctx.msp_phase_ms()
        enum_ms.append(ph["enumerate"])
        ops_all += algorithmic_fp64_ops(res.stats, pk.dims, lanes)
        last = (res, ph)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    launches = ctx.kernel_launches - launches0
    t_step = sum(times) / len(times)
    t_max = max_over_ranks(sum(times), world)
    nodes_sum = sum_over_ranks(nodes_all, world)
    value = nodes_sum / (t_max / 1e3)

    # ---- end to end through the C ABI from host buffers ----
    torch.cuda.synchronize()
    barrier(world)
    e2e_t, h2d, d2h = [], 0, 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.msp_build_lattice(pk.dims, A_pin.numpy(), d_pin.numpy())
        ctx.msp_run_async()
        res_h = ctx.msp_wait()
        sols = [ctx.msp_solutions(i) for i in range(len(insts))]
        e2e_t.append(time.perf_counter() - t0)
        h2d = pk.A.nbytes + pk.d.nbytes
        d2h = sum(s.nbytes for s in sols) + len(insts) * 8 * 16
    e2e_s = max_over_ranks(sum(e2e_t), world)
    e2e_value = sum_over_ranks(res_h.total["nodes"] * len(e2e_t), world) / e2e_s

    # ---- roofline of the dominant kernel (the enumerator) ----
    res, ph = last
    ops = algorithmic_fp64_ops(res.stats, pk.dims, lanes)
    achieved = ops / (ph["enumerate"] / 1e3)
    # DRAM bytes per launch: ncu's dram read + write per evaluated node on a
    # 4-instance capture of the same kernel (profiles/enum_kernel_batch4.md),
    # scaled by this launch's nodes
    traffic = None
    if lanes == 8:
        traffic = DRAM_BYTES_PER_NODE * res.total["nodes"]
    counted = FP64_LANE_OPS_PER_NODE * (res.total["nodes"] - sum(s["split_nodes"] for s in res.stats))
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_dfma / 1e9,
            "unit": "Gop/s (FP64 lane ops)", "frac": achieved / peak_dfma, "traffic": traffic,
            "frac_kind": "FP64-equivalent: the method's algorithmic FP64 operations per launch over the FP64 FMA "
                         "peak; most of them run as exact int64 fixed-point arithmetic",
            "fp64_counted_frac": (counted / (ph["enumerate"] / 1e3)) / peak_dfma if lanes == 8 else None,
            "fp64_counted_source": "FP64 lane instructions per node from ncu (profiles/enum_kernel_batch4.md) x "
                                   "this launch's nodes / enumeration time / peak",
            "traffic_source": "ncu dram bytes per node of a 4-instance capture, scaled by nodes",
            "peak_source": "measured FP64 fma throughput (msp_fp64_peak) on this GPU; the nominal "
                           "GB300 FP64 rate 1.25 TFLOP/s is 625 G fma/s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if len(insts) == 64 else f"first {len(insts)} instances of: {WORKLOAD}",
                   "instances": len(insts), "lanes": lanes,
                   "l2": "flushed between steps (512 MB write)",
                   "nodes_per_step": res.total["nodes"], "solutions_per_step": res.total["solutions"],
                   "phase_ms": {k: round(v, 3) for k, v in ph.items()},
                   "split_levels_median": float(np.median([s["kernel_rank"] - s["split_level"] for s in res.stats])),
                   "launch": launch_desc(kw, ctx.lanes),
                   "wall_s_timed_region": round(wall, 3)},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if tuning is not None:
        line["config"]["autotuned"] = {
            "strategy": tuning["strategy"], "seconds": tuning["seconds"], "chosen": tuning["opts"],
            "table": [dict(r["opts"], ms=round(r["ms"], 2) if math.isfinite(r["ms"]) else None)
                      for r in tuning["table"]]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the GPU on exactly the oracle's sample, so that the two divide like for like
        sample = cpu_sample(insts)
        gv, gnodes = gpu_nodes_per_s(sample, kw, args.steps, flush)
        line["cpu_baseline"] = cpu_baseline(sample, args.cpu_seconds, ctx.lanes)
        line["cpu_baseline"]["gpu_same_sample"] = {
            "value": gv, "unit": UNIT, "nodes_per_step": gnodes,
            "sample": f"the same {len(sample)} instances on the GPU, device time of whole steps"}
    ctx.close()
    if rank == 0 and world == 1 and not args.no_headline:
        line.update(headline(args, clocks_index=local))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
