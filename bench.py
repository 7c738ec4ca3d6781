#!/usr/bin/env python
"""Benchmark: node-updates/s of sequence-form DCFR on one large seeded game.

One step = one CFR iteration (both players, alternating; every step of the
hot path: regret matching, top-down sequence form, payoff products, bottom-up
counterfactual values, regret / variant / average updates) over the whole
game.  Workload (default): the depth-12 random game with chance at depths 0
and 6 (4 outcomes each), 3-4 actions, N(0,1) payoffs, seed 3: 6.22e6 nodes.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the workload (games are
independent units; no collective on the data path); value = node-updates of
all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_14277_b300 import games as G  # noqa: E402

METRIC = "node-updates/s per CFR iteration (DCFR, single large game)"
UNIT = "node-updates/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def workload(name):
    if name == "large":
        return G.large_random_game(3), "dcfr"
    if name == "poker":
        return G.poker_game(), "dcfr"
    if name == "small":
        return G.small_random_game(1), "cfr"
    raise ValueError(name)


def sources_sha256():
    """sha256 over the kernel sources (file name, then contents, in name order)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2605_14277_b300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(os.path.basename(f).encode())
            h.update(open(f, "rb").read())
    return h.hexdigest()


def profiled_traffic(kernel_slot):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when that summary was taken on other sources."""
    path = os.path.join(ROOT, "profiles", "k_up_staged_large.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    want = None
    for line in txt.splitlines():
        line = line.strip().strip("`")
        if "sources_sha256:" in line:
            want = line.split("sources_sha256:")[1].strip().strip("`").split()[0]
    if want != sources_sha256():
        return None
    key = f"traffic_bytes_per_launch_{kernel_slot}:"
    for line in txt.splitlines():
        if line.startswith(key):
            return int(line[len(key):].strip())
    return None


def alg_bytes(sz):
    """Algorithmic bytes per launch (forest totals include one root per game).

    up(p):   8 Z (payoff col + val) + 4 S_p (row pointers) + 16 S_p (regret
             float-float read + write) + 8 S_p (strategy read + write)
             + 4 S_p (child pointers) + 4 J_p (segment pointers) + 4 S_o (gather
             of the other player's x, each entry once)
    down(p): 16 S_p (average sums read + write) + 8 S_p (x read + write)
             + 4 S_p (strategy) + 8 J_p (parent and segment pointers)
    """
    S1, S2 = sz["S1"] + 1, sz["S2"] + 1
    J1, J2 = sz["J1"] + 1, sz["J2"] + 1
    Z = sz["nnz"]
    up1 = 8 * Z + 32 * S1 + 4 * J1 + 4 * S2
    up2 = 8 * Z + 32 * S2 + 4 * J2 + 4 * S1
    dn1 = 28 * S1 + 8 * J1
    dn2 = 28 * S2 + 8 * J2
    return {"up_p1": up1, "down_p1": dn1, "up_p2": up2, "down_p2": dn2}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.gpu_id)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(tree, variant, budget_s=15.0):
    """The FP64 oracle as it stands, single-threaded, on a bounded number of
    iterations of the same game."""
    from oracle.oracle import Oracle
    o = Oracle(tree)
    t0 = time.perf_counter()
    o.iterate(1, variant)
    one = time.perf_counter() - t0
    n = int(max(1, min(200, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.iterate(n, variant)
    el = time.perf_counter() - t0
    return {"value": tree.n_nodes * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} {variant} iterations of the full {tree.n_nodes}-node game (after 1 untimed)",
            "sec_per_iteration": el / n}


def dist_setup():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def run_reference(args):
    """The oracle, as it stands, on the host cores: same workload and metric."""
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    tree, variant = workload(args.workload)
    from oracle.oracle import Oracle
    o = Oracle(tree)
    t0 = time.perf_counter()
    o.iterate(max(1, args.warmup), variant)
    per = (time.perf_counter() - t0) / max(1, args.warmup)
    k = int(min(args.steps, max(3, 150.0 / max(per, 1e-9))))
    t0 = time.perf_counter()
    o.iterate(k, variant)
    el = time.perf_counter() - t0
    value = tree.n_nodes * k / el
    sample = f"{k} of {args.steps} requested {variant} iterations of the full {tree.n_nodes}-node game"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / k, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": tree.name, "nodes": tree.n_nodes, "variant": variant},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_14277_b300 import cfr as C

    tree, variant = workload(args.workload)
    stream = torch.cuda.Stream()
    s = C.Solver(tree, stream=stream)
    sz = s.sizes()
    s.iterate(args.warmup, variant)   # untimed: graphs captured, caches warm
    s.sync()
    props = torch.cuda.get_device_properties(local)
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_id)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.iterate(args.steps, variant)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    s.sync()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # per-kernel device time (events between eager launches, same stream)
    n_prof = max(50, min(2000, args.steps // 5))
    kms = s.profile(n_prof, variant)
    kbytes = alg_bytes(sz)
    names = ["up_p1", "down_p1", "up_p2", "down_p2"]
    avg_ms = {n: kms[i] / n_prof for i, n in enumerate(names)}
    dom = max(names, key=lambda n: avg_ms[n])
    hbm, src = peaks()
    achieved = kbytes[dom] / (avg_ms[dom] * 1e-3) / 1e9
    iter_bytes = sum(kbytes.values())
    value = tree.n_nodes * args.steps * world / (ms * 1e-3)
    if rank == 0:
        # end to end through the public API from host buffers: load (compile +
        # upload), the config's iterations, exploitability and both average
        # strategies back to the host
        e2e_iters = args.e2e_iters
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = C.Solver(tree, stream=stream)
        s2.iterate(e2e_iters, variant)
        expl = s2.exploitability()
        a1 = s2.average_strategy(1)
        a2 = s2.average_strategy(2)
        el = time.perf_counter() - t0
        sz2 = s2.sizes()
        s2.close()
        d2h = a1.nbytes + a2.nbytes + 3 * 8
        e2e = {"value": tree.n_nodes * e2e_iters / el, "unit": UNIT,
               "h2d_bytes_per_step": sz2["h2d_bytes"] / e2e_iters, "d2h_bytes_per_step": d2h / e2e_iters,
               "iterations": e2e_iters, "seconds": el, "exploitability": expl[0],
               "what": "Solver(host tree) + iterate + exploitability + average strategies, wall clock"}
        cpu = cpu_baseline(tree, variant, budget_s=args.cpu_budget) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 passes, f32+f32 (Kahan) accumulators, f64 best response",
            "data": "synthetic",
            "config": {"workload": tree.name, "nodes": tree.n_nodes, "terminals": int((tree.kind == 3).sum()),
                       "S1": sz["S1"], "S2": sz["S2"], "J1": sz["J1"], "J2": sz["J2"], "nnz": sz["nnz"],
                       "variant": variant + "(1.5,0,2)" if variant == "dcfr" else variant,
                       "updates": "alternating" if variant != "cfr" else "simultaneous",
                       "l2": f"inputs larger than L2: {sz['device_bytes'] / 2**20:.0f} MiB resident vs 126 MiB L2",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": 4 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": profiled_traffic(dom),
                         "kernel": f"{'k_up_staged' if dom.startswith('up') else 'k_down_staged'} ({dom})",
                         "alg_bytes_per_launch": kbytes[dom], "avg_launch_us": avg_ms[dom] * 1e3,
                         "peak_source": src},
            "iteration": {"alg_bytes": iter_bytes, "alg_GBps": iter_bytes / (ms / args.steps * 1e-3) / 1e9,
                          "frac_of_peak": iter_bytes / (ms / args.steps * 1e-3) / 1e9 / hbm,
                          "kernel_us": {n: avg_ms[n] * 1e3 for n in names}},
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "poker", "small"])
    ap.add_argument("--e2e-iters", type=int, default=10000)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
