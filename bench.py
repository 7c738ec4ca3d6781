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

import numpy as np

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


def workload(name, variant=None):
    """(tree, variant) of a single-game workload; `variant` overrides the
    workload's own (DCFR for the large game and poker, vanilla CFR for the
    small game)."""
    tree, v = _workload(name)
    return tree, (variant or v)


def workload_config(tree, variant):
    """The keys that name a single-game workload, shared by both arms' lines."""
    return {"workload": tree.name, "nodes": tree.n_nodes, "terminals": int((tree.kind == 3).sum()),
            "variant": variant + "(1.5,0,2)" if variant == "dcfr" else variant,
            "updates": "alternating" if variant != "cfr" else "simultaneous"}


def _workload(name):
    if name == "large":
        return G.large_random_game(3), "dcfr"
    if name == "poker":
        return G.poker_game(), "dcfr"
    if name == "small":
        return G.small_random_game(1), "cfr"
    raise ValueError(name)


TWO_PLAYER_SOURCES = ("capi.cu", "compiler.cpp", "kernels.cuh", "layout.h", "staged.cuh")
NPLAYER_SOURCES = ("kernels.cuh", "layout.h", "nplayer.cu")


def sources_sha256(files=TWO_PLAYER_SOURCES):
    """sha256 over the sources a path's kernels are built from (file name,
    then contents, in name order): by default the two-player passes'."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(files):
        h.update(name.encode())
        h.update(open(os.path.join(ROOT, "paper_2605_14277_b300", "csrc", name), "rb").read())
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


def graph_length(steps, cap=64):
    """Iterations per CUDA graph for the timed run: the largest k <= cap that
    divides the step count (the timed region is whole replays).  Each replay
    starts with a parameter-table refill and cannot overlap the previous
    replay's last pass (~16 us per replay on the large game), so longer graphs
    win even when the warm-up cannot replay the same graph (it is captured and
    uploaded to the device before the warm-up)."""
    steps = max(1, steps)
    return max(d for d in range(1, min(cap, steps) + 1) if steps % d == 0)


def alg_bytes(sz):
    """Algorithmic bytes per launch (forest totals include one root per game).

    up(p):   8 Z (payoff col + val) + 4 S_p (row pointers) + 16 S_p (regret
             float-float read + write) + 8 S_p (strategy read + write)
             + 4 S_p (child pointers) + 4 J_p (segment pointers) + 4 S_o (the
             other player's x, each entry once); then the average update in
             the same launch: 16 S_p (average sums read + write) + 4 S_p (x)
    down(p): 4 S_p (strategy) + 4 S_p (x written) + 8 J_p (parent and
             segment pointers)
    """
    S1, S2 = sz["S1"] + 1, sz["S2"] + 1
    J1, J2 = sz["J1"] + 1, sz["J2"] + 1
    Z = sz["nnz"]
    up1 = 8 * Z + 52 * S1 + 4 * J1 + 4 * S2
    up2 = 8 * Z + 52 * S2 + 4 * J2 + 4 * S1
    dn1 = 8 * S1 + 8 * J1
    dn2 = 8 * S2 + 8 * J2
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


def cpu_info():
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return model, n


def _oracle_timed(job):
    """One oracle process: build the game of `job`, run `warm` untimed
    iterations, then as many timed iterations as fit the budget (at most
    `cap`).  Returns (node-updates, seconds, iterations)."""
    name, variant, budget_s, cap, warm = (tuple(job) + (1,))[:5]
    from oracle.oracle import Oracle
    tree, _ = workload(name)
    o = Oracle(tree)
    t0 = time.perf_counter()
    o.iterate(max(1, warm), variant)
    one = (time.perf_counter() - t0) / max(1, warm)
    n = int(max(1, min(cap, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.iterate(n, variant)
    el = time.perf_counter() - t0
    return tree.n_nodes * n, el, n


def cpu_baseline(tree, variant, budget_s=15.0, name="large", cores=None):
    """The FP64 oracle as it stands on the host's cores: one process per core
    (spawned), each iterating its own copy of the same game for a bounded
    time; the aggregate node-updates/s over all of them, and the
    single-process figure beside it.  The oracle is sequential, so more cores
    means more independent copies, not a faster single game."""
    import multiprocessing as mp
    model, nproc = cpu_info()
    cores = int(cores or min(nproc, 16))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_timed, [(name, variant, budget_s, 200, 1)] * cores)
    work = sum(r[0] for r in res)
    span = max(r[1] for r in res)
    one = res[0]
    return {"value": work / span, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each {min(r[2] for r in res)}-{max(r[2] for r in res)} {variant} "
                      f"iterations of its own copy of the full {tree.n_nodes}-node game (after 1 untimed)",
            "single_core": {"value": one[0] / one[1], "unit": UNIT, "sec_per_iteration": one[1] / one[2]},
            "cpu_model": model, "nproc": nproc}


def oracle_parity(s, tree, variant):
    """The timed run's parity against the FP64 oracle, taken in the CPU leg:
    the oracle picks up the GPU's final state.  Both sides evaluate the FP64
    exploitability of the GPU's average strategies, then each runs one more
    iteration from that state.  Reported: the relative difference of the two
    exploitabilities, and the largest element-wise one-step errors of the
    regrets (against the regret update's own magnitude) and of the average
    sums (against the vector's RMS), beside the tests' one-step bound."""
    from oracle.oracle import Oracle
    from tests.parity_util import ONE_STEP_RTOL, elementwise, oracle_values, regret_scale
    t0 = time.perf_counter()
    o = Oracle(tree)
    for p in (1, 2):
        st = s.get_state(p)
        o.set_state(p, st["r"], st["b"], st["xbar"], st["t"])
    e_o = o.exploitability()[0]
    e_g = s.exploitability()[0]
    init = {p: (o.get_state(p)["r"], o.get_state(p)["b"]) for p in (1, 2)}
    o.iterate(1, variant)
    s.iterate(1, variant)
    vals = oracle_values(o, init, s.get_state(1)["b"], alternating=(variant != "cfr"))
    err_r = err_x = 0.0
    for p in (1, 2):
        g_, o_ = s.get_state(p), o.get_state(p)
        sc = regret_scale(o, p, init[p][0], o_["r"], vals[p][0], vals[p][1])
        err_r = max(err_r, float(np.max(np.abs(g_["r"] - o_["r"]) / np.maximum(sc, 1e-300))))
        err_x = max(err_x, elementwise(g_["xbar"], o_["xbar"]))
    return {"t": s.sizes()["t"] - 1, "exploitability": e_g, "oracle_exploitability": e_o,
            "exploitability_rel_diff": abs(e_g - e_o) / max(abs(e_o), 1e-300),
            "one_step_r_err": err_r, "one_step_xbar_err": err_x, "one_step_tol": ONE_STEP_RTOL,
            "seconds": time.perf_counter() - t0,
            "what": "FP64 exploitability of the GPU's averages on both sides; then one iteration each from "
                    "the GPU's state, element-wise errors"}


def max_over_ranks(x, dist):
    """The largest value over all ranks (the slowest rank's time), on every rank."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist):
    """The sum over all ranks (work done by the whole job), on every rank."""
    if not dist:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_setup():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def run_reference_batch(args):
    """The oracle on the batched workload: a bounded sample of the games."""
    from oracle.oracle import Oracle
    trees = G.batch_games(args.batch_games)[:: max(1, args.batch_games // 64)]
    os_ = [Oracle(t) for t in trees]
    t0 = time.perf_counter()
    for o in os_:
        o.iterate(max(1, args.warmup), "cfr+")
    per = (time.perf_counter() - t0) / max(1, args.warmup)
    k = int(min(args.steps, max(3, 120.0 / max(per, 1e-9))))
    t0 = time.perf_counter()
    for o in os_:
        o.iterate(k, "cfr+")
    el = time.perf_counter() - t0
    nodes = sum(t.n_nodes for t in trees)
    value = nodes * k / el
    sample = f"{k} cfr+ iterations of {len(trees)} of the {args.batch_games} games (every 64th)"
    line = {"metric": "node-updates/s per CFR iteration (CFR+, 4096-game batch)", "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / k,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": f"batch of {args.batch_games} random games, nodes log-uniform in [1e2, 1e5]",
                                               "games": args.batch_games, "variant": "cfr+", "updates": "alternating"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_serve(args):
    """The oracle on the serving workload: requests solved one at a time, in
    arrival order, until the time budget is spent."""
    from oracle.oracle import Oracle
    from paper_2605_14277_b300 import serving as SV
    n = max(1, int(round(args.serve_rate * args.serve_seconds)))
    seed0 = 500000
    arrivals = G.poisson_arrivals(seed0, args.serve_rate, n)
    t0 = time.perf_counter()
    lat, done = [], 0
    for k in range(n):
        if time.perf_counter() - t0 > 120.0:
            break
        tree = G.serving_request(seed0 + 1 + k)
        rng = SV.payoff_range(tree)
        o = Oracle(tree)
        it = 0
        while True:
            o.iterate(64, "dcfr", alpha=1.5, beta=0.0, gamma=2.0)
            it += 64
            if o.exploitability()[0] <= 1e-3 * rng or it >= 100000:
                break
        done += 1
        lat.append(time.perf_counter() - t0 - arrivals[k])
    el = time.perf_counter() - t0
    value = done / el
    line = {"metric": "solves/s at exploitability <= 1e-3 of the payoff range (serving, Poisson arrivals)",
            "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": done, "warmup": 0,
            "ms_per_step": 1e3 * el / max(done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{n} requests, Poisson {args.serve_rate:g}/s, nodes log-uniform in [1e3, 1e6]",
                       "variant": "dcfr(1.5,0,2)"},
            "latency": {"p50_s": float(np.percentile(lat, 50)) if lat else None,
                        "p99_s": float(np.percentile(lat, 99)) if lat else None},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"the first {done} of {n} requests, one at a time, 120 s budget"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference(args):
    """The oracle, as it stands, on the host cores: same workload and metric."""
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    if args.workload == "batch":
        return run_reference_batch(args)
    if args.workload == "serve":
        return run_reference_serve(args)
    if args.workload == "nplayer":
        return run_reference_nplayer(args)
    tree, variant = workload(args.workload, args.variant)
    # the oracle is sequential: the host's cores each run their own copy of
    # the game (spawned processes), and the job's rate is their sum
    import multiprocessing as mp
    model, nproc = cpu_info()
    cores = min(nproc, 16)
    warm = min(args.warmup, 3)
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_timed, [(args.workload, variant, 60.0, args.steps, warm)] * cores)
    work = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    k = min(r[2] for r in res)
    value = work / el
    sample = (f"{cores} processes, each {k}-{max(r[2] for r in res)} of {args.steps} requested {variant} "
              f"iterations of its own copy of the full {tree.n_nodes}-node game (after {max(1, warm)} untimed)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / k, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(tree, variant),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "single_core": {"value": res[0][0] / res[0][1], "unit": UNIT},
                             "cpu_model": model, "nproc": nproc},
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

    tree, variant = workload(args.workload, args.variant)
    stream = torch.cuda.Stream()
    s = C.Solver(tree, stream=stream)
    sz = s.sizes()
    # the product path: the timed steps replay CUDA graphs of k iterations,
    # k = the step count up to 64 (or the largest divisor of it up to 64),
    # captured before the timed region; every k computes the same iterations
    k_graph = graph_length(args.steps)
    s.set_graph_iterations(k_graph)
    s.prepare_graph(variant)
    props = torch.cuda.get_device_properties(local)
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_id)
    sampler.start()
    # untimed warm-up right before the timed region (caches, clocks up after
    # the sampler's start-up pause)
    s.iterate(args.warmup, variant)
    s.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n_launch0 = s.kernel_launches()
    e0.record(stream)
    s.iterate(args.steps, variant)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    n_launch = s.kernel_launches() - n_launch0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    s.sync()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    # per-kernel device time (events between eager launches, same stream)
    n_prof = max(50, min(2000, args.steps // 5))
    kms = s.profile(n_prof, variant)
    kbytes = alg_bytes(sz)
    # launch slots in schedule order: alternating p1 up, p1 down, p2 up, p2
    # down; simultaneous (vanilla CFR's default) both up passes first
    if variant == "cfr":
        names = ["up_p1", "up_p2", "down_p1", "down_p2"]
    else:
        names = ["up_p1", "down_p1", "up_p2", "down_p2"]
    avg_ms = {n: kms[i] / n_prof for i, n in enumerate(names)}
    # the dominant kernel: the kernel function with the most device time per
    # iteration (each runs once per player); its achieved rate is its
    # algorithmic bytes over its time, summed over both players' launches
    kern = {"k_up_staged": ["up_p1", "up_p2"], "k_down_staged": ["down_p1", "down_p2"]}
    dom_fn = max(kern, key=lambda f: sum(avg_ms[n] for n in kern[f]))
    dom = kern[dom_fn]
    dom_ms = sum(avg_ms[n] for n in dom) / len(dom)          # per launch
    dom_bytes = sum(kbytes[n] for n in dom) / len(dom)       # per launch
    hbm, src = peaks()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    tr = [profiled_traffic(n) for n in dom]
    traffic = (sum(tr) / len(tr)) if all(t is not None for t in tr) else None
    iter_bytes = sum(kbytes.values())
    value = sum_over_ranks(tree.n_nodes * args.steps, dist) / (ms * 1e-3)
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
        cpu = (cpu_baseline(tree, variant, budget_s=args.cpu_budget, name=args.workload)
               if (world == 1 and not args.no_cpu) else None)
        parity = oracle_parity(s, tree, variant) if (world == 1 and not args.no_cpu) else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 passes, f32+f32 (Kahan) accumulators, f64 best response",
            "data": "synthetic",
            "config": {**workload_config(tree, variant),
                       "S1": sz["S1"], "S2": sz["S2"], "J1": sz["J1"], "J2": sz["J2"], "nnz": sz["nnz"],
                       "l2": f"inputs larger than L2: {sz['device_bytes'] / 2**20:.0f} MiB resident vs 126 MiB L2",
                       "parallelism": f"replicas x{world}",
                       "cuda_graph_iterations": k_graph},
            "gpu_launches": n_launch,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "dram_GBps": (traffic / (dom_ms * 1e-3) / 1e9) if traffic else None,
                         "dram_frac": (traffic / (dom_ms * 1e-3) / 1e9 / hbm) if traffic else None,
                         "kernel": f"{dom_fn} ({' + '.join(dom)}, per launch)",
                         "alg_bytes_per_launch": dom_bytes, "avg_launch_us": dom_ms * 1e3,
                         "per_launch": {n: {"alg_bytes": kbytes[n], "us": avg_ms[n] * 1e3,
                                            "frac": kbytes[n] / (avg_ms[n] * 1e-3) / 1e9 / hbm} for n in dom},
                         "peak_source": src},
            "iteration": {"alg_bytes": iter_bytes, "alg_GBps": iter_bytes / (ms / args.steps * 1e-3) / 1e9,
                          "frac_of_peak": iter_bytes / (ms / args.steps * 1e-3) / 1e9 / hbm,
                          "kernel_us": {n: avg_ms[n] * 1e3 for n in names}},
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "parity": parity,
        }
        if not args.no_sub and world == 1:
            # the batched, served and n-player workloads, bounded, in the same run
            line["batch"] = batch_summary(args, stream)
            line["serve"] = serve_summary(args, local)
            line["nplayer"] = nplayer_summary(args, stream)
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def solve_batch(s, trees, variant, target_rel=1e-3, cap=8192):
    """Rounds of 64 iterations with solved games masked off, until every game
    is at or below target_rel of its payoff range (or `cap` iterations).
    Returns (seconds, iterations per game, final exploitabilities)."""
    import torch
    from paper_2605_14277_b300 import serving as SV
    G_ = len(trees)
    rng = np.array([SV.payoff_range(t) for t in trees])
    active = np.ones(G_, np.uint8)
    its = np.zeros(G_, np.int64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while active.any() and its.max() < cap:
        s.iterate(64, variant, active=active)
        its[active.astype(bool)] += 64
        e = s.exploitability_batch()[0]
        active &= (e > target_rel * rng).astype(np.uint8)
    return time.perf_counter() - t0, its, e


def batch_summary(args, stream):
    """The 4096-game batch (CFR+, 64-iteration graphs, the launch shape and
    layout the autotuner picks on every 8th game within a few seconds):
    iteration time and node-updates/s against one launch sequence per game,
    and solves/s to exploitability <= 1e-3 of the payoff range against
    solving the games one at a time (on a sample)."""
    import torch
    from paper_2605_14277_b300 import autotune
    from paper_2605_14277_b300 import cfr as C
    variant = "cfr+"
    trees = G.batch_games(args.batch_games)
    nodes = sum(t.n_nodes for t in trees)
    t0 = time.perf_counter()
    tuned = autotune.tune(trees[::8], variant=variant, iterations=64, repeats=2, stream=stream,
                          budget_s=args.batch_tune_seconds)
    tune_s = time.perf_counter() - t0
    layout = {"shape": tuned["shape"], "flat": tuned["flat"], "passes": tuned["passes"]}
    s = C.Solver(trees, stream=stream, **layout)
    sizes = [s.sizes(g) for g in range(len(trees))]
    s.iterate(64, variant)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n_it = 256
    n0 = s.kernel_launches()
    e0.record(stream)
    s.iterate(n_it, variant)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n_it
    launches = (s.kernel_launches() - n0) / n_it
    s.close()
    hbm, _ = peaks()
    iter_bytes = batch_alg_bytes(sizes)
    # one context per game, the same 64 iterations, on a sample
    sample = trees[:: max(1, len(trees) // 64)][:64]
    solos = [C.Solver(t, stream=stream) for t in sample]
    for x in solos:
        x.iterate(64, variant)
    torch.cuda.synchronize()
    e0.record(stream)
    for x in solos:
        x.iterate(64, variant)
    e1.record(stream)
    e1.synchronize()
    solo_rate = sum(t.n_nodes for t in sample) * 64 / (e0.elapsed_time(e1) * 1e-3)
    for x in solos:
        x.close()
    # solves: the whole batch in one context, against a sample one at a time
    s = C.Solver(trees, stream=stream, **layout)
    sec, its, e = solve_batch(s, trees, variant)
    s.close()
    one_sec = 0.0
    one_its = []
    for t in sample[:32]:
        x = C.Solver(t, stream=stream)
        sec1, it1, _ = solve_batch(x, [t], variant)
        one_sec += sec1
        one_its.append(int(it1[0]))
        x.close()
    return {"workload": f"{len(trees)} random games, nodes log-uniform in [1e2, 1e5], CFR+", "nodes": nodes,
            "layout": {**layout, "shape_info": C.shapes()[layout["shape"]], "tune_seconds": tune_s,
                       "candidates_timed": len(tuned["table"]),
                       "default_shape": C.pick_shape(len(trees), nodes)},
            "us_per_iteration": ms * 1e3, "node_updates_per_s": nodes / (ms * 1e-3),
            "roofline_frac_of_measured_hbm": iter_bytes / (ms * 1e-3) / 1e9 / hbm,
            "alg_bytes_per_iteration": iter_bytes, "gpu_launches_per_iteration": launches,
            "per_game_launches_node_updates_per_s": solo_rate,
            "batched_over_per_game": nodes / (ms * 1e-3) / solo_rate,
            "solves_per_s": len(trees) / sec, "solve_seconds": sec, "solved": int((its < 8192).sum()),
            "iterations_to_target": {"median": float(np.median(its)), "max": int(its.max())},
            "one_at_a_time_solves_per_s": len(one_its) / one_sec,
            "one_at_a_time_sample": f"{len(one_its)} of the games, each alone in rounds of 64",
            "solves_batched_over_one_at_a_time": (len(trees) / sec) / (len(one_its) / one_sec),
            "target": "exploitability <= 1e-3 of the payoff range"}


def serve_workload(args, local, n, seed0=500000):
    """Poisson arrivals of subgame-solve requests through the continuous
    batching server; returns (server stats, one-at-a-time stats, nodes)."""
    import torch
    from paper_2605_14277_b300 import cfr as C
    from paper_2605_14277_b300 import serving as SV
    arrivals = G.poisson_arrivals(seed0, args.serve_rate, n)
    trees = [G.serving_request(seed0 + 1 + k) for k in range(n)]
    factory = lambda ts, st: C.Solver(ts, stream=st)   # noqa: E731
    # warm-up: one small cohort through the whole path (library load, graphs)
    warm = SV.make_requests(trees[:4], [0.0] * 4)
    SV.Server(factory, stream_factory=torch.cuda.Stream, max_iterations=256).run(warm)
    reqs = SV.make_requests(trees, arrivals)
    # every loader thread started, with its device set, before the server runs
    with SV.loader_pool(args.serve_loaders, initializer=torch.cuda.set_device, initargs=(local,)) as pool:
        srv = SV.Server(factory, hbm_budget=args.serve_budget_gb * 1e9, round_iters=64, variant="dcfr",
                        target_rel=1e-3, max_cohort_nodes=args.serve_cohort_nodes,
                        stream_factory=torch.cuda.Stream, loader=pool.submit)
        st = srv.run(reqs, time_limit=args.serve_time_limit)
    base_n = min(n, args.serve_baseline)
    base = SV.make_requests(trees[:base_n], arrivals[:base_n])
    bst = SV.serve_one_at_a_time(factory, base, round_iters=64, variant="dcfr", target_rel=1e-3,
                                 time_limit=args.serve_time_limit)
    return st, bst, sum(t.n_nodes for t in trees)


def serve_summary(args, local):
    n = max(1, int(round(args.serve_rate * args.serve_sub_seconds)))
    st, bst, nodes = serve_workload(args, local, n)
    return {"workload": f"{n} requests, Poisson {args.serve_rate:g}/s, nodes log-uniform in [1e3, 1e6], "
                        f"DCFR to exploitability <= 1e-3 of the payoff range", "nodes": nodes,
            "solves_per_s": st["solves_per_s"], "p50_latency_s": st["p50_latency_s"],
            "p99_latency_s": st["p99_latency_s"], "completed": st["completed"], "cohorts": st["cohorts"],
            "moved_games": st["moved_games"], "peak_bytes": st["peak_bytes"],
            "one_at_a_time": {"requests": bst["requests"], "completed": bst["completed"],
                              "solves_per_s": bst["solves_per_s"]},
            "served_over_one_at_a_time": st["solves_per_s"] / max(bst["solves_per_s"], 1e-12)}


def gpu_uuid(local):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        return local


def batch_alg_bytes(sizes):
    """Algorithmic bytes of one iteration over a batch: the per-launch formula
    of alg_bytes on the forest totals (one root per game)."""
    tot = {k: sum(z[k] for z in sizes) for k in ("S1", "S2", "J1", "J2", "nnz")}
    G_ = len(sizes)
    S1, S2, J1, J2, Z = tot["S1"] + G_, tot["S2"] + G_, tot["J1"] + G_, tot["J2"] + G_, tot["nnz"]
    return (8 * Z + 52 * S1 + 4 * J1 + 4 * S2) + (8 * S1 + 8 * J1) + (8 * Z + 52 * S2 + 4 * J2 + 4 * S1) + \
        (8 * S2 + 8 * J2)


def run_batch(args):
    """4096 seeded games of 10^2-10^5 nodes advanced together by CFR+: one
    launch per pass for all games, 64 iterations per CUDA graph, layout and
    launch shape from the autotuner; against per-game launches on a sample."""
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
    from paper_2605_14277_b300 import autotune
    from paper_2605_14277_b300 import cfr as C

    variant = "cfr+"
    n_games = args.batch_games
    trees = G.batch_games(n_games, seed0=1000 + rank * n_games)
    nodes = sum(t.n_nodes for t in trees)
    stream = torch.cuda.Stream()
    # autotune on a sample of the batch (every 8th game)
    tuned = autotune.tune(trees[::8], variant=variant, iterations=64, repeats=2, stream=stream,
                          cache=args.tune_cache, budget_s=args.tune_budget)
    s = C.Solver(trees, stream=stream, shape=tuned["shape"], flat=tuned["flat"], passes=tuned["passes"])
    s.set_graph_iterations(64)
    sizes = [s.sizes(g) for g in range(n_games)]
    s.iterate(max(args.warmup, 64), variant)
    s.sync()
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n_launch0 = s.kernel_launches()
    e0.record(stream)
    s.iterate(args.steps, variant)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    n_launch = s.kernel_launches() - n_launch0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    n_prof = 64
    kms = s.profile(n_prof, variant)
    names = ["up_p1", "down_p1", "up_p2", "down_p2"]
    s.close()
    value = sum_over_ranks(nodes * args.steps, dist) / (ms * 1e-3)
    iter_bytes = batch_alg_bytes(sizes)
    hbm, src = peaks()
    if rank == 0:
        # per-game launches: the same iterations, one context per game, each
        # game's 64-iteration graph replayed in turn on the same stream
        sample = trees[:: max(1, n_games // args.per_game_sample)][: args.per_game_sample]
        solos = [C.Solver(t, stream=stream) for t in sample]
        for x in solos:
            x.set_graph_iterations(64)
            x.iterate(64, variant)
        torch.cuda.synchronize()
        e0.record(stream)
        for x in solos:
            x.iterate(64, variant)
        e1.record(stream)
        e1.synchronize()
        solo_ms = e0.elapsed_time(e1)
        solo_nodes = sum(t.n_nodes for t in sample)
        for x in solos:
            x.close()
        per_game = {"value": solo_nodes * 64 / (solo_ms * 1e-3), "unit": UNIT,
                    "sample": f"{len(sample)} of the {n_games} games, 64 CFR+ iterations each, one context per game"}
        # end to end from host arrays: load, the iterations, exploitability back
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = C.Solver(trees, stream=stream, shape=tuned["shape"], flat=tuned["flat"], passes=tuned["passes"])
        s2.iterate(args.e2e_iters, variant)
        expl, _, _ = s2.exploitability_batch()
        el = time.perf_counter() - t0
        h2d = s2.sizes()["h2d_bytes"]
        s2.close()
        e2e = {"value": nodes * args.e2e_iters / el, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.e2e_iters, "d2h_bytes_per_step": expl.nbytes / args.e2e_iters,
               "iterations": args.e2e_iters, "seconds": el, "max_exploitability": float(expl.max()),
               "what": "Solver(host trees) + iterate + exploitability of every game, wall clock"}
        cpu = None
        if world == 1 and not args.no_cpu:
            cpu = cpu_baseline_batch(trees[:: max(1, n_games // 64)], variant, budget_s=args.cpu_budget)
        line = {
            "metric": "node-updates/s per CFR iteration (CFR+, 4096-game batch)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 passes, f32+f32 (Kahan) accumulators, f64 best response", "data": "synthetic",
            "config": {"workload": f"batch of {n_games} random games, nodes log-uniform in [1e2, 1e5]",
                       "games": n_games, "nodes": nodes, "variant": "cfr+", "updates": "alternating",
                       "graph_iterations": 64, "shape": tuned["shape"], "flat": tuned["flat"],
                       "launches_per_player": 1 if tuned["passes"] == 1 else 2,
                       "shape_info": C.shapes()[tuned["shape"]],
                       "l2": f"inputs larger than L2: {iter_bytes / 2**20:.0f} MiB streamed per iteration vs 126 MiB L2",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": n_launch,
            "roofline": {"bound": "hbm", "achieved": iter_bytes / (ms / args.steps * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": iter_bytes / (ms / args.steps * 1e-3) / 1e9 / hbm, "traffic": None,
                         "kernel": "whole iteration (every pass launch)", "alg_bytes_per_iteration": iter_bytes,
                         "peak_source": src},
            "iteration": {"kernel_us": {n: kms[i] / n_prof * 1e3 for i, n in enumerate(names)}},
            "autotune": {"table": [[a, b, c, round(d, 2)] for a, b, c, d in tuned["table"]],
                         "sample": "every 8th game of the batch"},
            "per_game_launches": per_game,
            "batched_over_per_game": value / world / per_game["value"],
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_serve(args):
    """Subgame-solve requests (nodes log-uniform in [1e3, 1e6], N(0,1)
    payoffs) arriving as a Poisson process, served with continuous batching
    under a 120 GB budget and solved by DCFR to exploitability <= 1e-3 of the
    payoff range; against the one-at-a-time loop on a sample."""
    import torch
    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    n = max(1, int(round(args.serve_rate * args.serve_seconds)))
    sampler = ClockSampler(gpu_uuid(local))
    sampler.start()
    st, bst, nodes = serve_workload(args, local, n, seed0=500000 + rank * 100000)
    clocks = sampler.stop()
    if rank == 0:
        line = {
            "metric": "solves/s at exploitability <= 1e-3 of the payoff range (serving, Poisson arrivals)",
            "value": st["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": n, "warmup": 4,
            "ms_per_step": 1e3 / st["solves_per_s"] if st["solves_per_s"] else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 passes, f32+f32 (Kahan) accumulators, f64 best response", "data": "synthetic",
            "config": {"workload": f"{n} requests, Poisson {args.serve_rate:g}/s, nodes log-uniform in [1e3, 1e6]",
                       "nodes": nodes, "variant": "dcfr(1.5,0,2)", "round_iterations": 64,
                       "cohort_nodes_max": args.serve_cohort_nodes, "loader_threads": args.serve_loaders,
                       "hbm_budget_gb": args.serve_budget_gb, "parallelism": f"replicas x{world}"},
            "latency": {"p50_s": st["p50_latency_s"], "p99_s": st["p99_latency_s"]},
            "serving": st,
            "node_updates_per_s": st["node_iterations"] / max(st["elapsed_s"], 1e-9),
            "one_at_a_time": {"requests": bst["requests"], "solves_per_s": bst["solves_per_s"],
                              "p50_s": bst["p50_latency_s"], "p99_s": bst["p99_latency_s"],
                              "completed": bst["completed"]},
            "clocks": clocks,
            "e2e": {"value": st["solves_per_s"], "unit": "solves/s",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                    "what": "request trees from host memory: compile, upload, iterate, exploitability checks"},
            "gpu_launches": None, "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line))
    return 0


NP_METRIC = "node-updates/s per CFR iteration (DCFR, three-player game, payoff tensors)"


def nplayer_alg_bytes(sizes, deepest_seqs=None):
    """Algorithmic bytes of one n-player iteration, per kind of pass, summed
    over the players (S_i sequences with the empty one, J_i decision points,
    Z_i tensor entries of player i; each array element counted once):

    rows(i): 4 (S_i + 1) row pointers + Z_i (4 value + 4 (n - 1) columns)
             + 4 (S_k + 1) for every other player's x (each entry once)
             + 4 (S_i + 1) u written; the average update in the same kernel:
             per sequence 4 x + 8 + 8 average sums read and written
    up(i):   per sequence 4 u + 8 + 8 regret read and written + 4 + 4
             strategy read and written + 4 child pointers (none on the
             player's deepest level, whose sequences have no children:
             deepest_seqs[i] of them); per decision point 4 segment start
             + 4 ev written + 4 ev read by its parent
    down(i): per sequence 4 b + 4 x written; per decision point 4 parent,
             4 segment start, 4 parent's x
    """
    n = len(sizes)
    S = [z["S"] + 1 for z in sizes]
    out = {"rows": 0, "up": 0, "down": 0}
    for i, z in enumerate(sizes):
        out["rows"] += 8 * S[i] + z["nnz"] * 4 * n + 4 * sum(S[k] for k in range(n) if k != i) + 20 * S[i]
        out["up"] += 32 * S[i] + 12 * z["J"] - 4 * (deepest_seqs[i] if deepest_seqs else 0)
        out["down"] += 8 * S[i] + 12 * z["J"]
    return out


def nplayer_config(tree, variant):
    """The keys that name the n-player workload, shared by both arms' lines."""
    return {"workload": tree.name, "nodes": tree.n_nodes, "players": tree.n_players,
            "terminals": int((tree.kind == G.N_TERMINAL).sum()),
            "variant": variant + "(1.5,0,2)" if variant == "dcfr" else variant,
            "updates": "alternating"}


NP_KERNELS = {"rows": "k_np_rows and k_np_rows_long (with the average update)",
              "up": "k_np_up2, k_np_up_wide and k_np_up_top",
              "down": "k_np_down_walk (k_np_down and k_np_down_top for players it does not take)"}


def nplayer_timed(NP, tree, variant, steps, warmup, stream, dist=None, sampler=None):
    """Load the n-player game, warm up, time `steps` iterations (CUDA graphs,
    events on the solver's stream, barriers and the max over ranks), then
    each kind of pass eagerly.  Returns the solver and the figures."""
    import torch
    s = NP.NSolver(tree, stream=stream)
    sizes = [s.size(i) for i in range(tree.n_players)]
    k_graph = graph_length(steps)
    s.set_graph_iterations(k_graph)
    s.prepare_graph(variant)   # captured before the timed region
    if sampler:
        sampler.start()
    s.iterate(warmup, variant)
    s.sync()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = s.launches
    e0.record(stream)
    s.iterate(steps, variant)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    n_launch = s.launches - n0
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    # per kind of pass: CUDA events around its launches (eager, same stream)
    us = s.time_passes(max(10, min(200, steps // 10)), variant)
    kb = nplayer_alg_bytes(sizes, [lv[-1][1] if lv else 0 for lv in (s.level_sizes(i) for i in range(tree.n_players))])
    hbm, src = peaks()
    dom = max(us, key=lambda k: us[k])
    achieved = kb[dom] / (us[dom] * 1e-6) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": f"{NP_KERNELS[dom]} (all its launches of one iteration)",
                "alg_bytes_per_iteration": kb[dom], "us_per_iteration": us[dom],
                "per_kind": {k: {"alg_bytes": kb[k], "us": us[k], "frac": kb[k] / (us[k] * 1e-6) / 1e9 / hbm}
                             for k in us},
                "peak_source": src}
    return s, {"sizes": sizes, "k_graph": k_graph, "ms": ms, "n_launch": n_launch, "clocks": clocks,
               "roofline": roofline, "iter_bytes": sum(kb.values()), "hbm": hbm}


def nplayer_summary(args, stream):
    """The n-player row, bounded, for the default line: the same game and
    timing as `--workload nplayer` with 512 iterations, and the FP64 NashConv
    parity of the timed run (the oracle evaluates the GPU's averages)."""
    from oracle.nplayer import NOracle
    from paper_2605_14277_b300 import nplayer as NP
    tree = G.large_nplayer_game(3)
    variant = "dcfr"
    s, f = nplayer_timed(NP, tree, variant, 512, 64, stream)
    o = NOracle(tree)
    for i in range(tree.n_players):
        st = s.get_state(i)
        o.r[i][1:], o.b[i][1:], o.xbar[i], o.t = st["r"], st["b"], st["xbar"].copy(), st["t"]
    nc_g, _ = s.nash_conv()
    nc_o, _ = o.nash_conv()
    s.close()
    ms = f["ms"]
    return {"metric": NP_METRIC, "workload": nplayer_config(tree, variant),
            "value": tree.n_nodes * 512 / (ms * 1e-3), "unit": UNIT, "us_per_iteration": ms / 512 * 1e3,
            "steps": 512, "warmup": 64, "cuda_graph_iterations": f["k_graph"], "gpu_launches": f["n_launch"],
            "iteration_frac_of_peak": f["iter_bytes"] / (ms / 512 * 1e-3) / 1e9 / f["hbm"],
            "roofline": f["roofline"],
            "parity": {"t": o.t, "nash_conv": nc_g, "oracle_nash_conv": nc_o,
                       "nash_conv_rel_diff": abs(nc_g - nc_o) / max(abs(nc_o), 1e-300)}}


def run_nplayer(args):
    """The n-player row: the 4.84M-node three-player game (payoff tensors)
    under DCFR, node-updates/s over the timed CUDA-graph iterations."""
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
    from paper_2605_14277_b300 import nplayer as NP
    tree = G.large_nplayer_game(3)
    variant = args.variant or "dcfr"
    stream = torch.cuda.Stream()
    s, f = nplayer_timed(NP, tree, variant, args.steps, args.warmup, stream, dist, ClockSampler(gpu_uuid(local)))
    sizes, k_graph, ms, n_launch, clocks = f["sizes"], f["k_graph"], f["ms"], f["n_launch"], f["clocks"]
    value = sum_over_ranks(tree.n_nodes * args.steps, dist) / (ms * 1e-3)
    iter_bytes, hbm = f["iter_bytes"], f["hbm"]
    if rank == 0:
        e2e_iters = min(args.e2e_iters, 2000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = NP.NSolver(tree, stream=stream)
        s2.set_graph_iterations(64)
        s2.iterate(e2e_iters, variant)
        nc, gains = s2.nash_conv()
        avgs = [s2.average_strategy(i) for i in range(tree.n_players)]
        el = time.perf_counter() - t0
        s2.close()
        h2d = sum(a.nbytes for a in (tree.parent, tree.kind, tree.actor, tree.infoset, tree.action,
                                     tree.chance_prob, tree.payoff))
        d2h = sum(a.nbytes for a in avgs) + 8 * (1 + tree.n_players)
        e2e = {"value": tree.n_nodes * e2e_iters / el, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_iters,
               "d2h_bytes_per_step": d2h / e2e_iters, "iterations": e2e_iters, "seconds": el, "nash_conv": nc,
               "what": "NSolver(host tree) + iterate + NashConv + average strategies, wall clock"}
        cpu = parity = None
        if world == 1 and not args.no_cpu:
            cpu, parity = nplayer_cpu_leg(tree, variant, s, args.cpu_budget)
        line = {
            "metric": NP_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 passes, f32+f32 (Kahan) accumulators, f64 NashConv",
            "data": "synthetic",
            "config": {**nplayer_config(tree, variant),
                       "S": [z["S"] for z in sizes], "J": [z["J"] for z in sizes], "nnz": [z["nnz"] for z in sizes],
                       "levels": [z["levels"] for z in sizes],
                       "l2": "inputs larger than L2: tensors and state of about 0.3 GB resident vs 126 MiB L2",
                       "parallelism": f"replicas x{world}", "cuda_graph_iterations": k_graph},
            "gpu_launches": n_launch,
            "roofline": f["roofline"],
            "iteration": {"alg_bytes": iter_bytes, "alg_GBps": iter_bytes / (ms / args.steps * 1e-3) / 1e9,
                          "frac_of_peak": iter_bytes / (ms / args.steps * 1e-3) / 1e9 / hbm},
            "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "parity": parity,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def nplayer_cpu_leg(tree, variant, s, budget_s):
    """The n-player oracle on the host: its rate on a bounded number of
    iterations of the full game, and the timed run's parity (both sides'
    FP64 NashConv of the GPU's averages)."""
    from oracle.nplayer import NOracle
    from paper_2605_14277_b300.cfr import DEFAULT_PARAMS, VARIANTS
    v = VARIANTS[variant]
    a, b, g = DEFAULT_PARAMS[v]
    o = NOracle(tree)
    t0 = time.perf_counter()
    o.iterate(1, v, a, b, g)
    one = time.perf_counter() - t0
    n = int(max(1, min(50, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    o.iterate(n, v, a, b, g)
    el = time.perf_counter() - t0
    model, nproc = cpu_info()
    cpu = {"value": tree.n_nodes * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} {variant} iterations of the full {tree.n_nodes}-node game (after 1 untimed), "
                     "one process (numpy)", "cpu_model": model, "nproc": nproc}
    for i in range(tree.n_players):
        st = s.get_state(i)
        o.r[i][1:] = st["r"]
        o.b[i][1:] = st["b"]
        o.xbar[i] = st["xbar"].copy()
        o.t = st["t"]
    nc_g, _ = s.nash_conv()
    nc_o, _ = o.nash_conv()
    parity = {"t": o.t, "nash_conv": nc_g, "oracle_nash_conv": nc_o,
              "nash_conv_rel_diff": abs(nc_g - nc_o) / max(abs(nc_o), 1e-300),
              "what": "FP64 NashConv of the GPU's averages on both sides"}
    return cpu, parity


def run_reference_nplayer(args):
    """The n-player oracle as it stands, on the same game and metric."""
    from oracle.nplayer import NOracle
    from paper_2605_14277_b300.cfr import DEFAULT_PARAMS, VARIANTS
    tree = G.large_nplayer_game(3)
    variant = args.variant or "dcfr"
    v = VARIANTS[variant]
    a, b, g = DEFAULT_PARAMS[v]
    o = NOracle(tree)
    o.iterate(max(1, min(args.warmup, 1)), v, a, b, g)
    t0 = time.perf_counter()
    k = 0
    while k < args.steps and time.perf_counter() - t0 < 60.0:
        o.iterate(1, v, a, b, g)
        k += 1
    el = time.perf_counter() - t0
    value = tree.n_nodes * k / el
    model, nproc = cpu_info()
    sample = f"{k} of {args.steps} requested {variant} iterations of the full {tree.n_nodes}-node game, one process"
    line = {"metric": NP_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / k, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": nplayer_config(tree, variant),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": model, "nproc": nproc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline_batch(trees, variant, budget_s=15.0):
    """The FP64 oracle, single-threaded, on a bounded sample of the batch."""
    from oracle.oracle import Oracle
    os_ = [Oracle(t) for t in trees]
    t0 = time.perf_counter()
    for o in os_:
        o.iterate(1, variant)
    one = time.perf_counter() - t0
    n = int(max(1, min(200, budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    for o in os_:
        o.iterate(n, variant)
    el = time.perf_counter() - t0
    nodes = sum(t.n_nodes for t in trees)
    return {"value": nodes * n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} {variant} iterations of {len(trees)} of the batch's games (every 64th)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "poker", "small", "batch", "serve", "nplayer"])
    ap.add_argument("--variant", default=None, choices=["cfr", "cfr+", "dcfr", "pcfr+", "pcfr"],
                    help="regret minimiser for the single-game workloads (default: the workload's own)")
    ap.add_argument("--serve-rate", type=float, default=1000.0)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-sub-seconds", type=float, default=1.0,
                    help="arrival window of the serving summary in the default line (rate x seconds requests)")
    ap.add_argument("--no-sub", action="store_true",
                    help="leave the batched and served summaries out of the default line")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--serve-time-limit", type=float, default=120.0)
    ap.add_argument("--serve-baseline", type=int, default=16)
    ap.add_argument("--serve-cohort-nodes", type=float, default=4e6)
    ap.add_argument("--serve-loaders", type=int, default=max(2, min(8, (os.cpu_count() or 4) // 2)),
                    help="host threads compiling and uploading admitted cohorts (default: half the cores, "
                         "at most 8)")
    ap.add_argument("--batch-games", type=int, default=4096)
    ap.add_argument("--per-game-sample", type=int, default=128)
    ap.add_argument("--tune-budget", type=float, default=60.0)
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file keeping the autotuner's choice per layout signature (--workload batch)")
    ap.add_argument("--batch-tune-seconds", type=float, default=8.0,
                    help="autotuning budget of the batch summary in the default line")
    ap.add_argument("--e2e-iters", type=int, default=10000)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "nplayer":
        return run_nplayer(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
