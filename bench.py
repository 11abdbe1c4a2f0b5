#!/usr/bin/env python
"""Benchmark of the dual APG on the 512-scenario Barcelona-sized tree.

One step = one solve (rapidnet_solve_device) of ``--iters`` APG iterations
on the synthetic 512-scenario tree (63 tanks, 114 flows, 88 demand
sectors, 17 mixing nodes, N = 24, branching [8,4,4,2,2,1,...], 10,664
decision nodes) with its inputs resident in HBM.  L2 is flushed (512 MB
write) between steps, outside the timed events.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W --precision fp64|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle, same metric

Multi-GPU (torchrun, one rank per GPU): independent replicas of the same
solve, no collective on the data path ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dual-APG iters/s & solve time to 1e-4 residual @512 scen; serving p50/p99"
MODES = ("fp64_path", "batched", "serving", "closed_loop", "scenario_tree", "dense_wu",
         "per_node")
CONFIG_NAME = "barcelona512"
WORKLOAD = ("barcelona512: synthetic Barcelona-sized network (63 tanks, 114 flows, 88 demand "
            "sectors, 17 mixing nodes, A = I), N = 24, branching [8,4,4,2,2,1,...], "
            "512 scenarios, 10,664 decision nodes, 2,559,360 duals")
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--iters", type=int, default=1000, help="APG iterations per step (solve)")
    ap.add_argument("--tol-iters", type=int, default=20000,
                    help="cap of the time-to-1e-4 solve (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-modes", action="store_true",
                    help="skip every section after the headline solve")
    ap.add_argument("--modes", default=",".join(MODES),
                    help="comma-separated sections to run after the headline solve")
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--batch-iters", type=int, default=2000)
    ap.add_argument("--serve-iters", type=int, default=2000)
    ap.add_argument("--loop-hours", type=int, default=168)
    ap.add_argument("--tree-paths", type=int, default=10000)
    ap.add_argument("--tree-oracle-paths", type=int, default=2000)
    ap.add_argument("--loop-iters", type=int, default=500)
    ap.add_argument("--pn-iters", type=int, default=200,
                    help="APG iterations of the timed per-node FP32 solve")
    ap.add_argument("--mode-tol", type=float, default=10.0,
                    help="stopping tolerance of the batched and served solves (and of the "
                         "FP64 solves they are compared with)")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    return ap.parse_args()


# ---------------------------------------------------------------------------
# per-node accounting of the persistent APG kernel: values a node reads and writes per
# iteration and the flops of the sparse-Schur form
# ---------------------------------------------------------------------------
def node_counts(net):
    import numpy as np
    nnzB = int(np.count_nonzero(net.B))
    nnzE = int(np.count_nonzero(net.E))
    nx, nu, ne = net.nx, net.nu, net.ne
    # values moved per decision node per iteration in the fused two-sweep
    # design: w read twice, y read, y+ and w+ written (5 (2nx+nu)), data
    # terms c0, ubar, Gd d (2nu + nx)
    values = 5 * (2 * nx + nu) + 2 * nu + nx
    # FP64/FP32 flops per node per iteration of the sparse-Schur form
    flops = 31 * nx + 18 * nu + 4 * nnzB + 5 * nnzE + 2 * ne * ne + 6
    return values, flops


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6780.0), "measured"
    return 6800.0, "fallback"


# FP64 peak: the nominal 1.25 TFLOP/s of the GB300 (FMA = 2 flops); FP32
# SIMT: 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s nominal.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.device), "-lms", "200"], stdout=self.file,
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
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample, single thread, in a fresh process
# ---------------------------------------------------------------------------
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import oracle as O
from synthetic import make_problem
pb = make_problem({cfg!r})
P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
F = O.factor(P)
S = O.solve_consts(P, F, pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha)
gamma = O.step_size(O.power_iteration(P, F, 3))
O.apg(P, F, S, 1, gamma)
times = []
w0 = time.time()
t_end = time.perf_counter() + {seconds}
while True:
    t0 = time.perf_counter()
    O.apg(P, F, S, {per}, gamma)
    times.append(time.perf_counter() - t0)
    if time.perf_counter() > t_end or len(times) >= {max_steps}:
        break
print(json.dumps(dict(times=times, per=int({per}), wall=[w0, time.time()])))
"""


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def run_oracle_sample(seconds: float, per: int = 1, max_steps: int = 1000, procs: int = 1):
    """The oracle as it stands, one thread per process.  procs > 1 runs that
    many independent copies of the same solve at once, one per host core,
    and returns each copy's record (the all-cores throughput is their
    iterations over the span of their timed loops)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SAMPLE.format(root=ROOT, cfg=CONFIG_NAME, seconds=seconds, per=per,
                                max_steps=max_steps)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=env) for _ in range(procs)]
    outs = []
    for p in ps:
        so, se = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed:\n" + se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1]))
    return outs[0] if procs == 1 else outs


def all_cores_rate(recs) -> float:
    """Iterations of all copies over the span from the first copy's start to
    the last copy's end of its timed loop."""
    iters = sum(r["per"] * len(r["times"]) for r in recs)
    span = max(r["wall"][1] for r in recs) - min(r["wall"][0] for r in recs)
    return iters / span


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    total = args.warmup + args.steps
    d = run_oracle_sample(seconds=1e9, per=1, max_steps=total)
    times = d["times"][args.warmup:]
    iters = d["per"] * len(times)
    secs = sum(times)
    value = iters / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one APG iteration of the FP64 CPU oracle "
                   "(general per-node Riccati recursion, numpy, one thread)"},
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(times)} oracle APG iterations on {CONFIG_NAME} "
                                   f"after {args.warmup} warm-up iterations; host {cpu_model()}"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))



# ---------------------------------------------------------------------------
# DRAM traffic of the dominant kernel from a committed ncu summary, used only
# while the kernel sources are the ones the counters were taken on
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ["paper_1904_10548_gb300/csrc/kernels.cuh",
                  "paper_1904_10548_gb300/csrc/solve_device.cuh",
                  "paper_1904_10548_gb300/csrc/dense_f.cuh",
                  "paper_1904_10548_gb300/csrc/solve_kernels.cu",
                  "paper_1904_10548_gb300/csrc/mixed_kernels.cu"]


PERNODE_SOURCES = ["paper_1904_10548_gb300/csrc/pernode.h",
                   "paper_1904_10548_gb300/csrc/pernode.cu"]


def kernel_source_hash(sources=None) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kind: str, sources=None):
    """Per-iteration DRAM bytes of a persistent kernel from
    profiles/traffic.json, or None when its sources changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f).get(kind)
    except (OSError, ValueError):
        return None
    if not d or d.get("source_hash") != kernel_source_hash(sources):
        return None
    return d["dram_bytes_per_iter"]


# ---------------------------------------------------------------------------
# time to tolerance and accuracy of the mixed path
# ---------------------------------------------------------------------------
TOL_LADDER = (100.0, 30.0, 10.0, 5.0, 1.0, 5e-2, 1e-4)


def time_to_tol(rn, name, gamma, max_iters):
    """One solve per path to 1e-4 (or max_iters) with the residual history:
    the first check at or below each tolerance of the ladder, its iteration
    and time (iterations x the launch's device time per iteration)."""
    from synthetic import make_problem
    pb = make_problem(name)
    d = pb.data
    out = {}
    for prec, label in ((rn.RN_PREC_FP64, "fp64"), (rn.RN_PREC_MIXED, "mixed")):
        f = rn.Factor(pb.net, pb.cost, pb.tree, precision=prec, gamma=gamma)
        gamma = f.info()["gamma"]
        r = f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=max_iters, tol=1e-4,
                    res_hist_len=max_iters // 10 + 1)
        f.close()
        h = r["res_hist"]
        us = r["apg_ms"] * 1e3 / r["iters"]
        reached = {}
        for tol in TOL_LADDER:
            k = next((i for i, v in enumerate(h) if v <= tol), None)
            reached[f"{tol:g}"] = (None if k is None else
                                   {"iters": 10 * (k + 1), "ms": 10 * (k + 1) * us / 1e3})
        kmin = int(h.argmin())
        out[label] = {"converged_1e-4": r["status"] == rn.RN_OK, "iters": r["iters"],
                      "ms": r["apg_ms"], "us_per_iter": us, "final_residual": r["primal_res"],
                      "min_residual": float(h[kmin]), "min_at_iter": 10 * (kmin + 1),
                      "ubox_viol": r["ubox_viol"], "reached": reached,
                      "trace": [float(h[i]) for i in range(0, len(h), max(1, len(h) // 40))]}
    out["gamma"] = gamma
    return out


def accuracy_vs_fp64(rn, pb, tensors, gamma, iters):
    import numpy as np
    d = pb.data

    def run(prec, g):
        f = rn.Factor(pb.net, pb.cost, pb.tree, precision=prec, gamma=g)
        r = f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
        f.close()
        return r

    rel = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    def cmp(a, b):
        return {"cost_rel": abs(a["cost"] - b["cost"]) / abs(b["cost"]),
                "u_rel": rel(a["u"], b["u"]), "x_rel": rel(a["x"], b["x"]),
                "y_rel": rel(a["y"], b["y"]), "residual": [a["primal_res"], b["primal_res"]],
                "ubox_viol": [a["ubox_viol"], b["ubox_viol"]]}

    ref = run(rn.RN_PREC_FP64, gamma)
    mixed = run(rn.RN_PREC_MIXED, gamma)
    ulp = run(rn.RN_PREC_FP64, gamma * (1.0 + 2.0 ** -23))
    return {"iters": iters, "mixed_vs_fp64_gpu": cmp(mixed, ref),
            "fp64_envelope": cmp(ulp, ref),
            "note": "fp64_envelope: FP64 path with the step size changed by one FP32 ulp "
                    "against the FP64 path"}


# ---------------------------------------------------------------------------
# the other modes: plain FP64 path, batched, serving
# ---------------------------------------------------------------------------
def run_fp64_path(rn, pb, tensors, gamma, iters=300, steps=3):
    import torch
    f = rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_FP64, gamma=gamma)
    x0, q, dem, alp, u, x, y = tensors
    f.solve_device(x0, q, dem, alp, iters, 0.0, u, x, y)
    ms = []
    for _ in range(steps):
        r = f.solve_device(x0, q, dem, alp, iters, 0.0, u, x, y)
        ms.append(r["apg_ms"])
    f.close()
    us = sum(ms) / len(ms) * 1e3 / iters
    return {"iters_per_s": 1e6 / us, "us_per_iter": us, "iters_per_step": iters,
            "precision": "fp64"}


def batch_problems(n):
    from synthetic import make_cost, make_data, make_network, random_branching
    from synthetic.configs import Problem
    dims = {16: (16, 29, 22, 4), 63: (63, 114, 88, 17), 128: (128, 230, 179, 35)}
    out = []
    for i in range(n):
        nx = (16, 63, 128)[i % 3]
        net = make_network(*dims[nx], seed=1000 + i)
        tree = random_branching(24, seed=2000 + i, s_min=16, s_max=512)
        out.append(Problem(net=net, cost=make_cost(net, seed=1000 + i), tree=tree,
                           data=make_data(net, tree, seed=3000 + i)))
    return out


def max_over_ranks(ms, dist, device):
    """The job's time: the slowest rank's (all ranks get it)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(total_ms, world, steps, iters):
    """Whole-job throughput: the iterations of all ranks over the job's time."""
    return world * steps * iters / (total_ms / 1e3)


def run_batched(rn, n, iters, tol):
    """256 problems (nx 16/63/128, uneven trees of 16-512 scenarios, N = 24)
    in one persistent launch (mixed precision) vs a sample of the same
    problems solved one by one on the FP64 path, both with the same stopping
    rule (residual <= tol, at most iters iterations)."""
    import numpy as np
    import torch
    pbs, facs, declined = [], [], 0
    for pb in batch_problems(n):
        try:
            facs.append(rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_MIXED,
                                  power_iters=50))
            pbs.append(pb)
        except rn.RapidNetError as e:  # layouts the library refuses (reported)
            if e.status != rn.RN_ERR_UNSUPPORTED:
                raise
            declined += 1
    n = len(pbs)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    data = [(dev(pb.data.x0), dev(pb.data.q), dev(pb.data.demand), dev(pb.data.alpha))
            for pb in pbs]
    rn.solve_batch(facs, data, iters, tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = rn.solve_batch(facs, data, iters, tol)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    conv = sum(1 for o in outs if o["primal_res"] <= tol)
    # solo FP64 solves of a sample, same step sizes and stopping rule
    solo, k, solo_conv = 0.0, 0, 0
    for i in range(0, n, max(1, n // 12)):
        pb = pbs[i]
        f = rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_FP64,
                      gamma=facs[i].info()["gamma"])
        nn = pb.tree.n_nodes
        u = torch.empty((nn, pb.net.nu), dtype=torch.float64, device="cuda")
        x = torch.empty((nn, pb.net.nx), dtype=torch.float64, device="cuda")
        y = torch.empty((nn, 2 * pb.net.nx + pb.net.nu), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = f.solve_device(*data[i], iters, tol, u, x, y)
        torch.cuda.synchronize()
        solo += time.perf_counter() - t1
        k += 1
        solo_conv += int(r["status"] == rn.RN_OK)
        f.close()
    for f in facs:
        f.close()
    nodes = sum(pb.tree.n_nodes - 1 for pb in pbs)
    return {"problems": n, "declined_unsupported": declined, "decision_nodes": nodes,
            "max_iters": iters, "tol": tol, "converged_fraction": conv / n,
            "mean_iters": sum(o["iters"] for o in outs) / n,
            "solves_per_s": n / wall, "kernel_ms": outs[0]["apg_ms"],
            "fp64_solo": {"sample": k, "solves_per_s": k / solo,
                          "converged_fraction": solo_conv / k},
            "speedup_vs_fp64_solo": (n / wall) / (k / solo), "precision": "mixed"}


def run_serving(rn, seconds, rate, max_iters, tol):
    """Poisson arrivals (mean `rate` per second) over three models: the 32-
    and 512-scenario Barcelona-sized trees and an nx = 128 network on a
    32-scenario tree; warm-started duals kept per slot."""
    import numpy as np
    from synthetic import make_cost, make_data, make_network, make_problem, make_tree
    from synthetic.configs import Problem
    net128 = make_network(128, 230, 179, 35, seed=7)
    tree128 = make_tree([4, 2, 2, 2] + [1] * 20, seed=8)
    models = [make_problem("barcelona32"), make_problem("barcelona512"),
              Problem(net=net128, cost=make_cost(net128, seed=7), tree=tree128,
                      data=make_data(net128, tree128, seed=9))]
    srv = rn.Server(workers=16, slots_per_model=4, budget_bytes=24 << 30, max_queue=256)
    keys = [srv.add_model(pb.net, pb.cost, pb.tree) for pb in models]
    rng = np.random.default_rng(4)
    n = int(seconds * rate)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    which = rng.integers(0, 3, size=n)
    tickets, rejected, results = [], 0, []
    t0 = time.perf_counter()
    for k in range(n):
        now = time.perf_counter() - t0
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        pb = models[which[k]]
        d = pb.data
        try:
            tickets.append((which[k], srv.submit(keys[which[k]], d.x0, d.q, d.demand, d.alpha,
                                                 max_iters, tol, warm=True)))
        except Exception:
            rejected += 1
    for key, t in tickets:
        results.append(srv.wait(keys[key], t))
    wall = time.perf_counter() - t0
    conv = sum(1 for r in results if r["status"] == rn.RN_OK)
    st = srv.stats()
    srv.close()
    return {"offered_per_s": rate, "seconds": seconds, "submitted": int(st["submitted"]),
            "completed": int(st["completed"]), "rejected": rejected,
            "solves_per_s": st["completed"] / wall, "p50_ms": st["p50_s"] * 1e3,
            "p99_ms": st["p99_s"] * 1e3, "mean_ms": st["mean_s"] * 1e3, "slots": st["slots"],
            "max_iters": max_iters, "tol": tol, "warm_start": True,
            "converged_fraction": conv / max(1, len(results)),
            "models": ["barcelona32", "barcelona512", "nx128 on 32 scenarios"],
            "precision": "mixed"}

def run_closed_loop(rn, hours, max_iters):
    """A week of hourly closed-loop operation (paper §6.3 experiment shape) of
    the Barcelona-sized network on a 32-scenario tree with one stage-1 node
    ([1,4,2,2,2,1,...], N = 24), mixed precision, warm-started duals; the
    three indices of §6.3."""
    import numpy as np

    from paper_1904_10548_gb300.closed_loop import simulate
    from synthetic import make_cost, make_data, make_network, make_tree
    from synthetic.configs import CONFIGS
    nx, nu, nd, ne = CONFIGS["barcelona32"]["dims"]
    net = make_network(nx, nu, nd, ne, seed=1)
    cost = make_cost(net, seed=1)
    tree = make_tree([1, 4, 2, 2, 2] + [1] * 19, seed=2)
    fac = rn.Factor(net, cost, tree, precision=rn.RN_PREC_MIXED)
    start = make_data(net, tree, seed=3)
    out = simulate(fac, net, cost,
                   lambda k: (lambda d: (d.demand, d.alpha))(make_data(net, tree, 1000 + k, k)),
                   start.x0, start.q, steps=hours, max_iters=max_iters)
    fac.close()
    return {"hours": hours, "max_iters": max_iters, "tree": "[1,4,2,2,2,1,...] N=24, 32 scenarios",
            "kpi_e": out.kpi_e, "kpi_s": out.kpi_s, "kpi_tau_s": out.kpi_tau,
            "kpi_tau_device_s": out.kpi_tau_device, "mean_solve_s": float(out.tau_s.mean()),
            "final_residual_median": float(np.median(out.residual)), "precision": "mixed"}


MIXED_REFRESH = 40  # FP64 refresh period of RN_PREC_MIXED (rn_opts.refresh_every = 0)


def run_per_node(rn, gamma, iters32, iters64):
    """The per-node factor form (paper §4.4 general recursion; §5.2 streams
    per-node matrices): barcelona512, Phi_nu and K_nu streamed from HBM at
    every iteration.  Algorithmic bytes per node and iteration: the 1,491
    vector values of the shared form plus the 2 nu^2 matrix entries, in the
    iteration's precision; the mixed precision adds one FP64 evaluation
    (the same bytes at 8 B) per refresh of its base, every MIXED_REFRESH
    iterations (the library's default period, passed explicitly).
    FP32 and mixed against FP64 of the same form at the same iteration
    count for the error; the factor step (host, FP64) timed."""
    import numpy as np
    from synthetic import make_problem
    pb = make_problem(CONFIG_NAME)
    d = pb.data
    nu, n = pb.net.nu, int(pb.tree.stage_ptr[-1]) - 1
    hbm_peak, hbm_src = load_peaks()
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    out = {"workload": WORKLOAD.split(":")[0] + " (A = I), per-node matrices", "nodes": n}
    res = {}
    per_val = (1491 + 2 * nu * nu) * n
    for key, prec, iters, bytes_it in (("fp32", rn.RN_PREC_FP32, iters32, per_val * 4),
                                       ("fp64", rn.RN_PREC_FP64, iters64, per_val * 8),
                                       ("mixed", rn.RN_PREC_MIXED, iters32,
                                        per_val * 4 + per_val * 8 / MIXED_REFRESH)):
        t0 = time.perf_counter()
        f = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=prec,
                      factor_form=rn.RN_FACTOR_PER_NODE,
                      refresh_every=MIXED_REFRESH if key == "mixed" else 0)
        factor_s = time.perf_counter() - t0
        info = f.info()
        f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=10)
        r = f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
        acc = f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters64)
        f.close()
        us = r["apg_ms"] * 1e3 / iters
        gbs = bytes_it / (us * 1e-6) / 1e9
        res[key] = acc
        out[key] = {"iters": iters, "us_per_iter": us, "iters_per_s": 1e6 / us,
                    "algorithmic_bytes_per_iter": bytes_it, "achieved_gbs": gbs,
                    "frac_hbm": gbs / hbm_peak, "peak_source": f"{hbm_src} copy bandwidth",
                    "traffic_per_iter": (measured_traffic(f"k_pn_{key}", PERNODE_SOURCES)
                                         if key != "mixed" else None),
                    "factor_step_s": factor_s, "grid_ctas": info["grid_ctas"],
                    "block_threads": info["block_threads"],
                    "device_bytes": info["device_bytes"]}
    for key in ("fp32", "mixed"):
        out[f"{key}_vs_fp64"] = {"iters": iters64,
                                 "cost_rel": abs(res[key]["cost"] - res["fp64"]["cost"])
                                 / abs(res["fp64"]["cost"]),
                                 "u_rel": rel(res[key]["u"], res["fp64"]["u"]),
                                 "x_rel": rel(res[key]["x"], res["fp64"]["x"]),
                                 "y_rel": rel(res[key]["y"], res["fp64"]["y"])}
    return out


def run_dense_wu(rn, iters):
    """The benchmark tree with a dense symmetric positive definite W_u: F is
    a dense matrix, applied with FMAs in the FP64 steps and on the tensor
    cores (TF32 head/tail split) in the FP32 steps of the mixed path."""
    import numpy as np
    from synthetic import make_cost, make_problem
    pb = make_problem(CONFIG_NAME)
    cost = make_cost(pb.net, seed=1, dense_wu=True)
    d = pb.data
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    out = {"workload": "barcelona512 with a dense SPD W_u", "iters": iters}
    f64 = rn.Factor(pb.net, cost, pb.tree, precision=rn.RN_PREC_FP64, power_iters=100)
    gamma = f64.info()["gamma"]
    f64.solve(d.x0, d.q, d.demand, d.alpha, max_iters=20)
    a = f64.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    f64.close()
    mx = rn.Factor(pb.net, cost, pb.tree, precision=rn.RN_PREC_MIXED, gamma=gamma)
    mx.solve(d.x0, d.q, d.demand, d.alpha, max_iters=20)
    b = mx.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    mx.close()
    out.update(fp64_us_per_iter=a["apg_ms"] * 1e3 / iters,
               mixed_us_per_iter=b["apg_ms"] * 1e3 / iters,
               mixed_vs_fp64={"cost_rel": abs(a["cost"] - b["cost"]) / abs(a["cost"]),
                              "u_rel": rel(b["u"], a["u"]), "y_rel": rel(b["y"], a["y"])},
               tensor_cores="mma.sync m16n8k8 TF32, head/tail split (FP32 steps)")
    return out


def run_scenario_tree(rn, S, oracle_S):
    """Scenario-tree construction (paper §6.2: 10^4 Monte-Carlo price paths
    reduced into a tree) with the 512-scenario shape [8,4,4,2,2,1,...],
    N = 24, on the GPU; the oracle (numpy, one thread) on a smaller sample
    of the same kind for scale."""
    import numpy as np
    from synthetic import make_price_paths
    br = [8, 4, 4, 2, 2] + [1] * 19
    paths = make_price_paths(S, 24, 1, seed=6)
    rn.scenario_tree(paths[:2000], br)  # warm-up (module load, allocations)
    t0 = time.perf_counter()
    t = rn.scenario_tree(paths, br)
    gpu_s = time.perf_counter() - t0
    # the selection steps stream the S x S distance matrix once per choice
    # at the root: 8 choices x S^2 x 8 bytes
    root_bytes = 8 * S * S * 8
    out = {"paths": S, "stages": 24, "branching": "[8,4,4,2,2,1,...]",
           "nodes": int(t["n_nodes"]), "leaves": int(np.diff(t["stage_ptr"])[-1]),
           "gpu_s": gpu_s, "root_selection_bytes": root_bytes}
    if oracle_S > 0:
        code = (f"import sys, time, numpy as np; sys.path.insert(0, {ROOT!r}); "
                "from synthetic import make_price_paths; "
                "from oracle.scenario_tree import build_tree; "
                f"P = make_price_paths({oracle_S}, 24, 1, seed=6); "
                "t = time.perf_counter(); "
                f"build_tree(P, np.full({oracle_S}, 1.0 / {oracle_S}), {br!r}); "
                "print(time.perf_counter() - t)")
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
        if r.returncode == 0:
            cpu_s = float(r.stdout.strip().splitlines()[-1])
            t2 = rn.scenario_tree(paths[:oracle_S], br)
            t0 = time.perf_counter()
            rn.scenario_tree(paths[:oracle_S], br)
            out["oracle_sample"] = {"paths": oracle_S, "cpu_s": cpu_s, "cores": 1,
                                    "gpu_s": time.perf_counter() - t0,
                                    "nodes": int(t2["n_nodes"])}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # the oracle's CPU samples run first, in fresh processes, before any GPU
    # work: one thread, then one copy per host core
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle_sample(args.cpu_seconds)
        ncores = os.cpu_count() or 1
        if ncores > 1:
            cpu_all = run_oracle_sample(args.cpu_seconds, procs=ncores)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1904_10548_gb300 as rn
    from synthetic import make_problem

    pb = make_problem(CONFIG_NAME)
    net, tree, data = pb.net, pb.tree, pb.data
    n = tree.n_nodes
    nx, nu, nd = net.nx, net.nu, net.nd
    ny = 2 * nx + nu
    prec = rn.RN_PREC_FP64 if args.precision == "fp64" else rn.RN_PREC_MIXED
    stream = torch.cuda.Stream()
    fac = rn.Factor(net, pb.cost, tree, precision=prec, device=local, stream=stream)
    info = fac.info()

    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x0, q, dem, alp = dev(data.x0), dev(data.q), dev(data.demand), dev(data.alpha)
    u = torch.empty((n, nu), dtype=torch.float64, device="cuda")
    x = torch.empty((n, nx), dtype=torch.float64, device="cuda")
    y = torch.empty((n, ny), dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        return fac.solve_device(x0, q, dem, alp, args.iters, 0.0, u, x, y)

    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            flush.zero_()
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    apg_ms = []
    launches = 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = step()
        e1.record(stream)
        evs.append((e0, e1))
        apg_ms.append(r["apg_ms"])
        # kq, prep, x*(0) step, init, APG, gather (+ dual gather in mixed), reduce, final reduce
        launches += 9 if args.precision == "mixed" else 8
        assert r["iters"] == args.iters
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, "cuda")
    value = job_value(total_ms, world, args.steps, args.iters)

    # end to end through the host entry point: pinned host inputs and outputs
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    hx0, hq, hdem, halp = pin(data.x0), pin(data.q), pin(data.demand), pin(data.alpha)
    hu = torch.empty((n, nu), dtype=torch.float64).pin_memory()
    hx = torch.empty((n, nx), dtype=torch.float64).pin_memory()
    hy = torch.empty((n, ny), dtype=torch.float64).pin_memory()
    e2e_s = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fac.solve(hx0.numpy(), hq.numpy(), hdem.numpy(), halp.numpy(), args.iters,
                  out=(hu.numpy(), hx.numpy(), hy.numpy()))
        if k > 0:
            e2e_s.append(time.perf_counter() - t0)
    e2e_val = args.iters / (sum(e2e_s) / len(e2e_s)) * world if e2e_s else None
    h2d = 8 * (nx + nu + n * nd + n * nu)
    d2h = 8 * n * (nu + nx + ny)

    # time to tolerance: the metric's 1e-4 and the paper's 5e-2, plus a
    # ladder of looser ones, for both paths and both Barcelona-sized trees
    tol_run = None
    if args.tol_iters > 0:
        tol_run = {"check_every": 10, "residual": "|H x*(w) - t|_inf, absolute (state units; "
                   "tank capacities 50-150)", "trees": {}}
        for name, cap in (("barcelona512", args.tol_iters), ("barcelona32", 2 * args.tol_iters)):
            tol_run["trees"][name] = time_to_tol(rn, name, info["gamma"] if name == CONFIG_NAME
                                                 else 0.0, cap)

    # accuracy of the timed mixed solve against the FP64 path at the same
    # iteration count, beside the spread of two FP64 solves whose step sizes
    # differ by one FP32 ulp (how far the iteration itself carries an
    # FP32-sized perturbation after this many iterations)
    accuracy = None
    if args.precision == "mixed" and world == 1 and not args.no_accuracy:
        accuracy = accuracy_vs_fp64(rn, pb, (x0, q, dem, alp), info["gamma"], args.iters)

    modes = {}
    want = set() if args.no_modes or world > 1 else set(args.modes.split(",")) - {""}
    unknown = want - set(MODES)
    if unknown:
        raise SystemExit(f"unknown --modes entries {sorted(unknown)}; known: {list(MODES)}")
    if "fp64_path" in want:
        modes["fp64_path"] = run_fp64_path(rn, pb, (x0, q, dem, alp, u, x, y), info["gamma"])
    if "batched" in want:
        modes["batched"] = run_batched(rn, args.batch_problems, args.batch_iters, args.mode_tol)
    if "serving" in want:
        modes["serving"] = run_serving(rn, args.serve_seconds, args.serve_rate,
                                       args.serve_iters, args.mode_tol)
    if "closed_loop" in want:
        modes["closed_loop"] = run_closed_loop(rn, args.loop_hours, args.loop_iters)
    if "scenario_tree" in want:
        modes["scenario_tree"] = run_scenario_tree(rn, args.tree_paths, args.tree_oracle_paths)
    if "dense_wu" in want:
        modes["dense_wu"] = run_dense_wu(rn, 300)
    if "per_node" in want:
        modes["per_node"] = run_per_node(rn, info["gamma"], args.pn_iters, 40)

    # roofline of the dominant kernel (the persistent APG launch)
    values, flops = node_counts(net)
    nodes = n - 1
    bpv = 8 if args.precision == "fp64" else 4
    apg_avg_s = sum(apg_ms) / len(apg_ms) / 1e3
    hbm_peak, hbm_src = load_peaks()
    bytes_launch = values * bpv * nodes * args.iters
    flops_launch = flops * nodes * args.iters
    gbs = bytes_launch / apg_avg_s / 1e9
    tfl = flops_launch / apg_avg_s / 1e12
    traffic_iter = measured_traffic("k_mixed" if args.precision == "mixed" else "k_solve_fp64")
    traffic = traffic_iter * args.iters if traffic_iter else None
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tfl / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "nominal GB300 FP64 (recipe table)",
                "hbm_view": {"achieved_gbs": gbs, "peak_gbs": hbm_peak,
                             "frac": gbs / hbm_peak, "peak_source": hbm_src}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "traffic": traffic,
                "peak_source": f"{hbm_src} copy bandwidth (of measured)"}
    roof.update(bytes_per_launch=bytes_launch, flops_per_launch=flops_launch,
                kernel_ms=apg_avg_s * 1e3, us_per_iter=apg_avg_s * 1e6 / args.iters,
                per_node={"values": values, "bytes": values * bpv, "flops": flops})

    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "iters_per_step": args.iters,
                   "precision": args.precision, "l2": "flushed between steps (512 MB write)",
                   "fp64_refresh_every": MIXED_REFRESH if args.precision == "mixed" else None,
                   "grid_ctas": info["grid_ctas"], "block_threads": info["block_threads"],
                   "gamma": info["gamma"], "parallelism": f"replicas x{world}"},
        "e2e": ({"value": e2e_val, "unit": "iters/s", "h2d_bytes_per_step": h2d,
                 "d2h_bytes_per_step": d2h} if e2e_val else None),
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "time_to_tol": tol_run,
        "accuracy": accuracy,
        "modes": modes or None,
    }
    if "fp64_path" in modes:
        modes["fp64_path"]["mixed_speedup"] = value / modes["fp64_path"]["iters_per_s"]
    if cpu is not None:
        cv = cpu["per"] * len(cpu["times"]) / sum(cpu["times"])
        one = {"value": cv, "unit": "iters/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(cpu['times'])} FP64 oracle APG iterations on "
                         f"{CONFIG_NAME}, one thread, host {cpu_model()} "
                         f"({os.cpu_count()} cores present)"}
        line["cpu_baseline"] = one
        if cpu_all:
            its = sum(r["per"] * len(r["times"]) for r in cpu_all)
            line["cpu_baseline"] = {
                "value": all_cores_rate(cpu_all), "unit": "iters/s", "cores": len(cpu_all),
                "kind": "oracle",
                "sample": f"{len(cpu_all)} independent copies of the FP64 oracle's solve of "
                          f"{CONFIG_NAME} at once, one per host core ({its} APG iterations "
                          f"in all; value = their iterations over the span of their timed "
                          f"loops), host {cpu_model()}",
                "single_thread": one}
    if rank == 0:
        print(json.dumps(line))
    fac.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
