"""Autotuner of the tree-code's group and leaf sizes (N_crit, N_leaf).

The paper fixes N_leaf = 16 (§2.1) and N_crit "typically 64" (§2.2) for its
GPUs.  On a GB300 the best pair depends on the workload: smaller groups
shorten every body's interaction lists, larger ones share one walk among
more bodies (groups of more than 64 bodies are evaluated in several passes
over their lists).  For one workload (bodies on the device) and (theta, eps)
this module:

* times the full leapfrog step (one CUDA graph replay per step) for each
  (n_leaf, n_crit) of a grid;
* measures each pair's acceleration error against direct summation
  (``bh_direct_forces``) on a fixed subsample of bodies;
* keeps the fastest pair whose 99th-percentile error is no worse than the
  paper's pair (16, 64) times ``slack`` -- faster at equal error.

Results are cached in ``tuned.json`` beside this file, keyed by workload class
(log2 N, theta); :func:`tuned_params` looks them up.

    python -m paper_1106_1900_gb300.autotune --n 1048576 --theta 0.5 --eps 0.005
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

TUNED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
PAPER_PAIR = (16, 64)
DEFAULT_GRID = [(nl, nc) for nc in (16, 32, 48, 64, 96, 128, 192, 256) for nl in (4, 8, 16) if nl <= nc]


def key_for(n: int, theta: float, kind: str = "plummer") -> str:
    return f"{kind}/log2n={round(math.log2(max(n, 1)))}/theta={theta:.2f}"


def load_table(path: str = TUNED) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_params(n: int, theta: float, kind: str = "plummer", path: str = TUNED):
    """The cached (n_leaf, n_crit) for this workload class, or None."""
    e = load_table(path).get(key_for(n, theta, kind))
    return None if e is None else {"n_leaf": e["n_leaf"], "n_crit": e["n_crit"]}


def _errors(acc, ref):
    import torch

    a = acc.double()
    r = ref.double()
    e = (torch.linalg.norm(a - r, dim=1) / torch.linalg.norm(r, dim=1)).cpu()
    q = torch.quantile(e, torch.tensor([0.5, 0.99], dtype=e.dtype))
    return {"p50": float(q[0]), "p99": float(q[1]), "rms": float(torch.sqrt((e * e).mean()))}


def measure(pos, vel, mass, theta, eps, dt, n_leaf, n_crit, steps, targets, ref_acc, device=0, pool_per_body=None):
    """Error against the reference and the mean step time of one (n_leaf, n_crit)."""
    import torch

    from . import TreeCode

    n = pos.shape[0]
    extra = {} if pool_per_body is None else {"pool_per_body": pool_per_body}
    tc = TreeCode(n, device=device, n_leaf=n_leaf, n_crit=n_crit, **extra)
    try:
        tc.build(pos, mass)
        acc, _ = tc.compute_forces(theta, eps)
        tc.check()
        err = _errors(acc[targets.long()], ref_acc)
        tc.set_state(pos, vel, mass)
        for _ in range(2):
            tc.step(dt, theta, eps, graph=True)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(steps):
            tc.step(dt, theta, eps, graph=True)
        t1.record()
        torch.cuda.synchronize()
        tc.check()
        ms = t0.elapsed_time(t1) / steps
    finally:
        tc.close()
    out = {"n_leaf": n_leaf, "n_crit": n_crit, "ms_per_step": ms, **err}
    if pool_per_body is not None:
        out["pool_per_body"] = pool_per_body
    return out


def measure_or_skip(*args, **kw):
    """measure(), retried once with a four times larger list pool when the
    interaction lists overflow it (small groups at small theta); None when the
    pair does not fit at all."""
    from . import STATUS_CAPACITY, BHError, default_params

    try:
        return measure(*args, **kw)
    except BHError as e:
        if e.code != STATUS_CAPACITY:
            raise
    try:
        return measure(*args, **kw, pool_per_body=4 * default_params().pool_per_body)
    except BHError as e:
        if e.code != STATUS_CAPACITY:
            raise
        return None


def autotune(pos, vel, mass, theta, eps, dt=1.0 / 64, grid=None, steps=5, subsample=4096, seed=40, slack=1.05,
             device=0, log=None):
    """Returns (best, trials).  pos/vel/mass are float64 CUDA tensors."""
    import numpy as np
    import torch

    from . import direct_forces

    grid = list(grid or DEFAULT_GRID)
    if PAPER_PAIR not in grid:
        grid.append(PAPER_PAIR)
    n = pos.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n, size=min(subsample, n), replace=False)).astype(np.int32)
    targets = torch.from_numpy(idx).to(pos.device)
    ref_acc, _ = direct_forces(pos, mass, targets, eps)
    trials = []
    for nl, nc in grid:
        r = measure_or_skip(pos, vel, mass, theta, eps, dt, nl, nc, steps, targets, ref_acc, device)
        if r is None:
            r = {"n_leaf": nl, "n_crit": nc, "skipped": "interaction lists exceed the capacities"}
        else:
            trials.append(r)
        if log:
            log(r)
    paper = next(r for r in trials if (r["n_leaf"], r["n_crit"]) == PAPER_PAIR)
    ok = [r for r in trials if r["p99"] <= paper["p99"] * slack]
    best = min(ok, key=lambda r: r["ms_per_step"])
    return best, trials


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=0.005)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--workload", default="plummer", choices=["plummer", "galaxy"],
                    help="galaxy: Hernquist sphere + exponential disk, 8,388,608 bodies (--n ignored)")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--out", default=TUNED)
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import ics

    if args.workload == "galaxy":
        pos, vel, m = ics.galaxy(4194304, 4194304, 3)
    else:
        pos, vel, m = ics.plummer(args.n, args.seed)
    dev = torch.device("cuda", 0)
    P, V, M = (torch.from_numpy(a).to(dev) for a in (pos, vel, m))
    best, trials = autotune(P, V, M, args.theta, args.eps, steps=args.steps,
                            log=lambda r: print(json.dumps(r), flush=True))
    table = load_table(args.out)
    table[key_for(len(pos), args.theta, args.workload)] = {**best, "eps": args.eps, "trials": trials}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps({"best": best}))


if __name__ == "__main__":
    main()
