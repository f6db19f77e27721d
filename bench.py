"""Benchmark: particles/s per force step of the tree-code on a 1M-body Plummer sphere.

One "step" is the whole hot path on one batch: FP64 leapfrog predict,
frame + Morton keys, radix sort, move, cells + links + groups, moments, the
group walk (theta = 0.5, eps = 0.005) and the FP64 correct, replayed as one
CUDA graph per step.  Inputs are resident in HBM when the timed region
starts; L2 is flushed (a 512 MB write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own 1M-body system (weak scaling, no
collective on the data path); the value is the bodies of all ranks divided
by the slowest rank's time.  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s per force step (1M Plummer, θ=0.5), batched vs plain, same error"
UNIT = "particles/s"
N_BODIES = 1 << 20
THETA, EPS, DT = 0.5, 0.005, 1.0 / 64
SEED = 2
# flops per interaction: FMA = 2, rsqrt = 1, add/sub/mul = 1 (counted from k_walk.cu)
FLOPS_PP = 20
FLOPS_PC = 54  # the work unit fixed from the first particle-cell sequence
FLOPS_PC_IMPLEMENTED = 53  # what the current pc2() performs by the same rule
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
# Algorithmic HBM bytes of the build phases and the leapfrog of one step:
# what each kernel must read and write once.  Per body: predict 112 (x, v,
# a_old read; x, v written), bbox 32 (x, m), keys 36 (x; key, index), sort
# histogram 8 + eight passes of 24 (key and index, read and written), move 188
# (80 gathered, 108 written: two-float positions, state, ids), levels + scan +
# emit 14 (key, flags, per-warp counts), moments 32 (two-float positions),
# correct 96 (v, a, a_old read; v, a written): 710.  Per cell: emit 20, link
# 36, moments 128 (record written, children's records read): 184 (the opening
# radii belong to the walk phase).  Per group: begin and system, 8.
BUILD_BYTES_PER_BODY = 710
BUILD_BYTES_PER_CELL = 184
BUILD_BYTES_PER_GROUP = 8
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_BODIES)
    ap.add_argument("--theta", type=float, default=THETA)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eager", action="store_true", help="launch kernel by kernel instead of the graph")
    ap.add_argument("--flush-mb", type=int, default=512, help="L2 flush buffer written between timed steps")
    ap.add_argument("--untuned", action="store_true", help="use the paper's N_leaf = 16, N_crit = 64")
    ap.add_argument("--mac", type=int, default=0, choices=[0, 1],
                    help="opening criterion: 0 Eq. 1 (default), 1 minimal distance")
    ap.add_argument("--block", action="store_true", help="add the block time-step measurement")
    ap.add_argument("--block-eta", type=float, default=0.05, help="time-step accuracy parameter eta")
    ap.add_argument("--split", action="store_true",
                    help="split walk (lists through a pool, then a separate evaluation kernel)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-vs-plain ensemble comparison")
    ap.add_argument("--shard", action="store_true",
                    help="one system with its groups shared out among the ranks (strong scaling) instead of "
                         "an independent system per rank")
    ap.add_argument("--ensemble-steps", type=int, default=100,
                    help="steps of each arm of the batched-vs-plain ensemble comparison")
    ap.add_argument("--key-levels", type=int, default=20,
                    help="key depth D (20: the paper's 60-bit keys; up to 30: 90-bit keys)")
    ap.add_argument("--list-capacity", type=int, default=0,
                    help="split walk: longest interaction list (0: library default)")
    ap.add_argument("--list-buffer", type=int, default=0,
                    help="fused walk: entries of each list buffer of a walking warp (0: library default)")
    ap.add_argument("--workload", default="plummer", choices=["plummer", "galaxy", "nested"],
                    help="plummer: N-body Plummer sphere (--n); galaxy: Hernquist sphere + exponential disk, "
                         "8,388,608 bodies")
    ap.add_argument("--galaxy-n", type=int, default=8388608,
                    help="galaxy bodies, half sphere and half disk (smaller cases for profiling)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def walk_traffic(summary="walk_plummer_1m.md"):
    """Per-launch DRAM bytes of the dominant walk kernel from the committed ncu
    summary, if it was taken from the current source of the kernel."""
    src = open(os.path.join(ROOT, "paper_1106_1900_gb300", "csrc", "k_walk.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if m_sha and m_b and m_sha.group(1) == sha:
        return float(m_b.group(1))
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(pos, mass, theta, eps, n_leaf=16, n_crit=64, target_s=15.0, gpu=None):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload
    (same N_leaf, N_crit): the whole tree build plus the walk of every k-th group.
    With ``gpu`` = (acc, pot, group stats) of the library's force evaluation of
    the same input, also the parity report of the sampled groups (the policy
    of the parity tests: 1e-5 per body, clauses counted and bounded)."""
    import numpy as np

    import oracle

    t0 = time.perf_counter()
    t = oracle.build_tree(pos, mass, n_leaf, n_crit)
    t_build = time.perf_counter() - t0
    # size the sample from a short probe so that the walk takes ~target_s
    probe = np.arange(0, t.G, max(1, t.G // 64))
    t0 = time.perf_counter()
    oracle.walk(t, theta, eps, probe)
    t_probe = time.perf_counter() - t0
    per_group = t_probe / len(probe)
    k = max(1, int(t.G * per_group / max(target_s - t_build, 1.0)))
    groups = np.arange(0, t.G, k)
    t0 = time.perf_counter()
    acc_s, pot_s, st = oracle.walk(t, theta, eps, groups)
    t_walk = time.perf_counter() - t0
    bodies = int(sum(t.gend[g] - t.gbeg[g] for g in groups))
    secs = t_walk + t_build * bodies / t.n
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": bodies / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"FP64 tree build of all {t.n} bodies ({t_build:.2f} s, charged pro rata) + walk of "
                     f"every {k}-th group ({len(groups)} groups, {bodies} bodies, {t_walk:.2f} s), "
                     f"theta={theta}, eps={eps}, N_leaf={n_leaf}, N_crit={n_crit}"}
    if gpu is not None:
        from tests import _parity

        acc_g, pot_g, gst = gpu
        try:
            rep = _parity.group_forces_report(acc_g, pot_g, t, groups, acc_s, pot_s, st,
                                              {k_: v[groups] for k_, v in gst.items()})
            rep["ok"] = True
        except AssertionError as e:
            rep = {"ok": False, "error": str(e)[:500]}
        rep["what"] = (f"library forces vs the FP64 oracle on the same tree, the {len(groups)} sampled groups "
                       f"({bodies} bodies) of the initial state: tolerance 1e-5 per body")
        out["parity"] = rep
    return out


def block_compare(bh, dev, pos, vel, mass, theta, eps, params, dt_max=1.0 / 64, k_max=6, eta=0.05,
                  rebuild_every=False):
    """Block time-steps on the same workload: one synchronised interval of
    dt_max (a rebuild at every block step, or at the interval's start with
    moment refreshes inside it), against stepping every body with the
    smallest step any body used in it (what a shared step needs for the same
    per-body accuracy), timed by one shared step."""
    import torch

    n = pos.shape[0]
    tc = bh.TreeCode(n, device=dev.index, **params)
    tc.set_state(pos, vel, mass)
    tc.block_start(dt_max, k_max, eta, theta, eps)
    sync = 2 ** k_max
    # one warm interval, then the timed one
    for rep in range(2):
        t0 = tc.block_info()["tick"]
        torch.cuda.synchronize()
        start = time.perf_counter()
        steps = updates = rebuilds = 0
        deepest = 0
        tick = t0
        while tick < t0 + sync:
            rebuild = rebuild_every or tick % sync == 0
            tc.block_step(theta, eps, rebuild=rebuild)
            info = tc.block_info()  # (the one host synchronisation of a block step)
            tick = info["tick"]
            steps += 1
            updates += info["active"]
            rebuilds += int(rebuild)
            deepest = max(deepest, info["deepest"])
        torch.cuda.synchronize()
        wall = time.perf_counter() - start
    tc.check()
    # a shared step of the same system (graph replay), for the comparison
    ts = bh.TreeCode(n, device=dev.index, **params)
    ts.set_state(pos, vel, mass)
    for _ in range(3):
        ts.step(dt_max / 2 ** deepest, theta, eps, graph=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        ts.step(dt_max / 2 ** deepest, theta, eps, graph=True)
    b.record()
    torch.cuda.synchronize()
    shared_ms = a.elapsed_time(b) / 5
    shared_interval_s = shared_ms * 1e-3 * 2 ** deepest
    policy = "a rebuild at every block step" if rebuild_every else "rebuild at its start, moment refresh inside"
    return {"what": f"block time-steps, dt_max = 1/{round(1 / dt_max)}, k_max = {k_max}, eta = {eta}: one "
                    f"synchronised dt_max interval (host-driven block steps, {policy}) against shared steps of "
                    "the smallest step used",
            "block_steps": steps, "rebuilds": rebuilds, "deepest_level": deepest,
            "body_updates": updates, "updates_per_s": updates / wall, "interval_s": wall,
            "shared_step_ms": shared_ms, "shared_interval_s": shared_interval_s,
            "speedup_vs_shared": shared_interval_s / wall}


def ensemble_compare(bh, dev, theta, eps, steps, warmup, n_sys=512, params=None):
    """512 independent Plummer clusters (sizes log-uniform in [1024, 65536],
    scale radii U(0.5, 2)): one forest stepped as one CUDA graph per step
    against one context per cluster, each stepping its own graph, all from
    the same initial state.

    The plain arm runs the paper's N_leaf = 16, N_crit = 64.  The batched arm
    runs (a) the autotuner's parameters for this workload (`params`), whose
    99th-percentile force error is no larger than the paper pair's times
    1.05 (the autotuner's rule), and (b) the paper pair itself: the same
    trees, lists and forces as the plain arm (a forest's systems share
    nothing), so the two end in the same states, which is checked."""
    import numpy as np
    import torch

    import ics

    pos, vel, m, off = ics.ensemble(n_sys, 5)
    N = len(pos)
    P, V, M = (torch.from_numpy(a).to(dev) for a in (pos, vel, m))
    ev = lambda: torch.cuda.Event(enable_timing=True)
    paper = {"n_leaf": 16, "n_crit": 64}

    def batched(prm):
        # one forest, one graph per step
        tf = bh.TreeCode(N, n_sys, device=dev.index, **prm)
        tf.set_state(P, V, M, offsets=off)
        for _ in range(warmup):
            tf.step(DT, theta, eps, graph=True)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record()
        for _ in range(steps):
            tf.step(DT, theta, eps, graph=True)
        b.record()
        torch.cuda.synchronize()
        tf.check()
        xf = torch.empty_like(P)
        tf.get_state(xf)
        tf.close()
        return a.elapsed_time(b) * 1e-3, xf

    t_tuned, _ = batched(dict(params or paper))
    t_batched, xf = batched(paper)
    # plain: one context and graph per system, launched one after another
    ctxs = []
    for s_ in range(n_sys):
        lo, hi = int(off[s_]), int(off[s_ + 1])
        tc = bh.TreeCode(hi - lo, device=dev.index, stack_capacity=2048, **paper)
        tc.set_state(P[lo:hi], V[lo:hi], M[lo:hi])
        ctxs.append((lo, hi, tc))
    for _ in range(warmup):
        for _, _, tc in ctxs:
            tc.step(DT, theta, eps, graph=True)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(steps):
        for _, _, tc in ctxs:
            tc.step(DT, theta, eps, graph=True)
    b.record()
    torch.cuda.synchronize()
    t_plain = a.elapsed_time(b) * 1e-3
    maxdiff = 0.0
    for lo, hi, tc in ctxs:
        tc.check()
        xs = torch.empty((hi - lo, 3), dtype=torch.float64, device=dev)
        tc.get_state(xs)
        maxdiff = max(maxdiff, float((xs - xf[lo:hi]).abs().max()))
        tc.close()
    return {"workload": f"{n_sys} Plummer clusters, N={N} (sizes log-uniform 1024..65536, seeds 5000+s), "
                        f"theta={theta}, eps={eps}, dt=1/64",
            "steps": steps,
            "batched_params": params or paper, "batched_particles_per_s": N * steps / t_tuned,
            "batched_ms_per_step": 1e3 * t_tuned / steps,
            "plain_params": paper, "plain_particles_per_s": N * steps / t_plain,
            "plain_ms_per_step": 1e3 * t_plain / steps,
            "speedup": t_plain / t_tuned,
            "same_params": {"params": paper, "batched_particles_per_s": N * steps / t_batched,
                            "speedup": t_plain / t_batched, "max_state_difference": maxdiff}}


def run_reference(args):
    """The oracle as the reference arm: each step builds the full tree and walks a sample of groups."""
    import numpy as np

    import ics
    import oracle

    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    pos, vel, m = ics.plummer(args.n, SEED)
    from paper_1106_1900_gb300 import autotune  # (the cached parameters only: no GPU, no library)

    tuned = None if args.untuned else autotune.tuned_params(args.n, args.theta, "plummer")
    nl, nc = (tuned["n_leaf"], tuned["n_crit"]) if tuned else (16, 64)
    t0 = time.perf_counter()
    t = oracle.build_tree(pos, m, nl, nc)
    t_build = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)  # whole run within a few minutes
    probe = np.arange(0, t.G, max(1, t.G // 32))
    t0 = time.perf_counter()
    oracle.walk(t, args.theta, EPS, probe)
    per_group = (time.perf_counter() - t0) / len(probe)
    k = max(1, int(t.G * per_group / max(budget - t_build, 0.5)))
    groups = np.arange(0, t.G, k)
    bodies = int(sum(t.gend[g] - t.gbeg[g] for g in groups))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        tt = oracle.build_tree(pos, m, nl, nc)
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.walk(tt, args.theta, EPS, groups)
        tw = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(tw + tb * bodies / tt.n)
    secs = sum(times)
    value = bodies * len(times) / secs
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"per step: FP64 tree build of all {args.n} bodies (charged pro rata) + walk of every {k}-th "
              f"group ({len(groups)} groups, {bodies} bodies), N_leaf={nl}, N_crit={nc}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(times) * args.n / bodies,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"Plummer N={args.n}, theta={args.theta}, eps={EPS}, seed={SEED}",
                   "global_batch": args.n, "parallelism": "oracle on host cores", "n_leaf": nl, "n_crit": nc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_sharded(args):
    """One system shared out among the ranks (paper_1106_1900_gb300.shard):
    every rank builds the same tree, walks its range of groups, and one
    all-gather per step exchanges the walked bodies' forces (strong scaling:
    the same bodies whatever the number of ranks)."""
    import torch

    import ics
    import paper_1106_1900_gb300 as bh
    from paper_1106_1900_gb300 import autotune, shard

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bh.load()
    pos, vel, m = ics.plummer(args.n, SEED)  # the same system on every rank
    n = len(pos)
    tuned = None if args.untuned else autotune.tuned_params(n, args.theta, "plummer")
    tc = bh.TreeCode(n, device=local, **(tuned or {}))
    tc.set_state(*(torch.from_numpy(a).to(dev) for a in (pos, vel, m)))
    st = shard.ShardedStep(tc, rank, world)
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        st.step(DT, args.theta, EPS)
    tc.check()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total = 0.0
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            if args.flush_mb > 0:
                flush.fill_(k & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            st.step(DT, args.theta, EPS)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
    if world > 1:
        torch.distributed.barrier()
    tc.check()
    t_max = max_over_ranks(total, world, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * args.steps / (t_max * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Plummer N={n} (seed {SEED}), theta={args.theta}, eps={EPS}, dt=1/64, one system",
                       "global_batch": n, "parallelism": f"groups shared out over {world} ranks, tree on every rank",
                       "exchange": "one all-gather of the walked bodies' forces (16 B per body) and one of the "
                                   "groups' interaction counts per step",
                       "l2": f"flushed between timed steps ({args.flush_mb} MB write)" if args.flush_mb else "not flushed",
                       "params": tuned or "library defaults", "last_split": st.last_ranges},
            "clocks": clk.summary(),
        }), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.shard:
        run_sharded(args)
        return
    import numpy as np
    import torch

    import ics
    import paper_1106_1900_gb300 as bh

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    bh.load()
    eps, dt = EPS, DT
    if args.workload == "galaxy":
        pos, vel, m = ics.galaxy(args.galaxy_n // 2, args.galaxy_n - args.galaxy_n // 2, 3 + rank)
        eps = 0.01
        workload = (f"galaxy: Hernquist sphere (a=1, M=1) + exponential disk (R_d=1, z0=0.1, M=0.2), "
                    f"N={len(pos)} per GPU (seed 3+rank), theta={args.theta}, eps={eps}, dt=1/64")
    elif args.workload == "nested":
        n_core = args.n // 16
        pos, vel, m = ics.nested(args.n, SEED + rank, n_core)
        eps, dt = 1e-7, 2.0 ** -32  # a step well below the cluster's crossing time (~1e-8)
        workload = (f"nested: Plummer N={args.n} per GPU holding a Plummer cluster of {n_core} bodies shrunk "
                    f"by 1e-6 (seeds {SEED}+rank, +1), theta={args.theta}, eps={eps}, dt=2^-32")
    else:
        pos, vel, m = ics.plummer(args.n, SEED + rank)
        workload = (f"Plummer N={args.n} per GPU (virial units, seed {SEED}+rank), theta={args.theta}, "
                    f"eps={EPS}, dt=1/64")
    n = len(pos)
    from paper_1106_1900_gb300 import autotune

    tuned = None if args.untuned else autotune.tuned_params(n, args.theta, args.workload)
    kw = dict(tuned or {}, walk_split=int(args.split), mac=args.mac, key_levels=args.key_levels)
    if args.list_capacity:
        kw["list_capacity"] = args.list_capacity
    if args.list_buffer:
        kw["list_buffer"] = args.list_buffer
    tc = bh.TreeCode(n, device=local, **kw)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(max(args.flush_mb, 1) << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        P = torch.from_numpy(pos).to(dev)
        V = torch.from_numpy(vel).to(dev)
        M = torch.from_numpy(m).to(dev)
        tc.set_state(P, V, M)
        tc.set_profiling(True)
        for _ in range(args.warmup):
            tc.step(dt, args.theta, eps, graph=not args.eager)
        tc.check()
        torch.cuda.synchronize()
        tc.reset_counters()
        c0 = tc.counts()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        step_ms, walk_ms, eval_ms, phases = [], [], [], []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                if args.flush_mb > 0:
                    flush.fill_(k & 0xff)
                ev[k][0].record(stream)
                tc.step(dt, args.theta, eps, graph=not args.eager)
                ev[k][1].record(stream)
                ph = tc.phase_times()  # synchronises on this step's events
                walk_ms.append(ph["walk"])
                eval_ms.append(ph["walk eval"])
                phases.append(ph)
            torch.cuda.synchronize()
        wall1 = time.perf_counter()
        if world > 1:
            torch.distributed.barrier()
        tc.check()
        c1 = tc.counts()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    t_max = max_over_ranks(total_ms, world, dev)
    bodies_all = sum_over_ranks(float(n * args.steps), world, dev)
    value = bodies_all / (t_max * 1e-3)
    launches = c1["launches"] - c0["launches"]
    # ---- roofline of the dominant kernel (the walk): algorithmic flops / its device time
    pp, pc = c1["pp"] - c0["pp"], c1["pc"] - c0["pc"]
    flops = FLOPS_PP * pp + FLOPS_PC * pc
    walk_s = sum(walk_ms) * 1e-3
    eval_s = sum(eval_ms) * 1e-3
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
    achieved = flops / eval_s if eval_s > 0 else 0.0  # the dominant kernel: k_eval
    achieved_walk = flops / walk_s if walk_s > 0 else 0.0
    # the committed counters are of the 1M Plummer step at theta = 0.5 with the default options
    profiled = (args.workload == "plummer" and args.n == N_BODIES and args.theta == THETA and args.mac == 0
                and args.key_levels == 20 and not args.untuned and not args.list_capacity
                and not args.list_buffer)
    traffic = walk_traffic("eval_plummer_1m.md" if args.split else "walk_plummer_1m.md") if profiled else None
    clocks = clk.summary()
    mean_phase = {k: statistics.mean(p[k] for p in phases) for k in bh.PHASES if k != "call"}
    # build phases against HBM bandwidth
    cnt0 = tc.counts()
    build_ms = sum(mean_phase[k] for k in ("frame+keys", "sort", "move", "cells+link+groups", "moments",
                                           "leapfrog"))
    build_bytes = (BUILD_BYTES_PER_BODY * n + BUILD_BYTES_PER_CELL * cnt0["cells"]
                   + BUILD_BYTES_PER_GROUP * cnt0["groups"])
    hbm = float(measured_peaks().get("hbm_gbs", HBM_FALLBACK_GBS))
    build_gbs = build_bytes / (build_ms * 1e-3) / 1e9 if build_ms > 0 else 0.0
    build = {"ms_per_step": build_ms, "algorithmic_bytes_per_step": build_bytes, "achieved_GBs": build_gbs,
             "peak_GBs": hbm, "frac": build_gbs / hbm,
             "peak_source": "measured" if "hbm_gbs" in measured_peaks() else "fallback"}
    # ---- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        hp = torch.from_numpy(pos).pin_memory()
        hm = torch.from_numpy(m).pin_memory()
        ha = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        hq = torch.empty(n, dtype=torch.float32).pin_memory()
        tc2 = bh.TreeCode(n, device=local, **kw)
        for _ in range(max(1, args.warmup)):
            tc2.forces_host(hp, hm, args.theta, eps, ha, hq, stream=stream)
        if world > 1:
            torch.distributed.barrier()
        e0 = time.perf_counter()
        for _ in range(args.steps):
            tc2.forces_host(hp, hm, args.theta, eps, ha, hq, stream=stream)
        e_s = max_over_ranks(time.perf_counter() - e0, world, dev)
        e2e = {"value": bodies_all / e_s, "unit": UNIT, "h2d_bytes_per_step": n * (24 + 8),
               "d2h_bytes_per_step": n * (12 + 4)}
        tc2.close()
    ens = None
    if not args.no_ensemble and args.workload == "plummer":
        ens_params = None if args.untuned else autotune.tuned_params(7672972, args.theta, "ensemble")
        ens = ensemble_compare(bh, dev, args.theta, 0.01, steps=args.ensemble_steps, warmup=3, params=ens_params)
    blk = None
    if args.block:
        blk = {"rebuild_every_step": block_compare(bh, dev, P, V, M, args.theta, eps, kw, eta=args.block_eta,
                                                   rebuild_every=True),
               "refresh_inside": block_compare(bh, dev, P, V, M, args.theta, eps, kw, eta=args.block_eta)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the library's forces on the initial state, for the parity report of the sampled groups
        tcp = bh.TreeCode(n, device=local, **kw)
        tcp.build(torch.from_numpy(pos).to(dev), torch.from_numpy(m).to(dev))
        acc0, pot0 = tcp.compute_forces(args.theta, eps)
        tcp.check()
        gpu0 = (acc0.cpu().numpy(), pot0.cpu().numpy(), tcp.group_stats())
        tcp.close()
        del acc0, pot0
        cpu = cpu_baseline(pos, m, args.theta, eps, tc.params.n_leaf, tc.params.n_crit, gpu=gpu0)
    if rank != 0:
        return
    cnt = tc.counts()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload + ", full leapfrog step as one CUDA graph",
                   "global_batch": n * world, "parallelism": f"independent system per GPU x{world}",
                   "l2": f"flushed between timed steps ({args.flush_mb} MB write)" if args.flush_mb else "not flushed",
                   "n_leaf": tc.params.n_leaf, "n_crit": tc.params.n_crit,
                   "params": "autotuned (paper_1106_1900_gb300/tuned.json)" if tuned else "paper defaults",
                   "cells": cnt["cells"], "groups": cnt["groups"], "graph": not args.eager,
                   "opening": "Eq. 1" if args.mac == 0 else "minimal distance",
                   "key_levels": args.key_levels, "deepest_level": cnt["deepest"],
                   "walk": "split" if args.split else "fused"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": ("k_eval (interaction lists -> accelerations, potentials)" if args.split else
                                "k_walk (per group: breadth-first walk into the warp's scratch, then the "
                                "evaluation of its lists)"),
                     "peak_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                    f"{SM_MAX_MHZ:.0f} MHz (unit counts and max clock)",
                     "flops_per_pp": FLOPS_PP, "flops_per_pc_unit": FLOPS_PC,
                     "flops_per_pc_implemented": FLOPS_PC_IMPLEMENTED,
                     "flops_per_step": flops / args.steps, "pp_per_step": pp / args.steps,
                     "pc_per_step": pc / args.steps, "eval_ms_mean": statistics.mean(eval_ms),
                     "walk_phase": {"ms_mean": statistics.mean(walk_ms), "achieved": achieved_walk / 1e12,
                                    "frac": achieved_walk / peak if peak else None,
                                    "what": ("opening radii + k_traverse + k_order + k_eval" if args.split
                                             else "opening radii + group order + k_walk")}},
        "phase_ms_mean": mean_phase,
        "build": build,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": {k_: v for k_, v in cpu.items() if k_ != "parity"} if cpu else None,
        "parity": cpu.get("parity") if cpu else None,
        "ensemble": ens,
        "block": blk,
        "wall_s_timed": wall1 - wall0,
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
