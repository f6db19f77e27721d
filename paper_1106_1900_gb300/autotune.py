"""Autotuner of the tree-code's group and leaf sizes and of the walk's buffers.

The paper fixes N_leaf = 16 (§2.1) and N_crit "typically 64" (§2.2) for its
GPUs.  On a GB300 the best pair depends on the workload: smaller groups
shorten every body's interaction lists, larger ones share one walk among
more bodies (groups of more than 64 bodies are evaluated in several passes
over their lists).  For one workload (bodies on the device, or a forest of
independent systems) and (theta, eps) this module:

* times the full leapfrog step (one CUDA graph replay per step) for each
  (n_leaf, n_crit) of a grid;
* measures each pair's acceleration error against direct summation
  (``bh_direct_forces``, system by system for a forest) on a fixed
  subsample of bodies;
* keeps the fastest pair whose 99th-percentile error is no worse than the
  paper's pair (16, 64) times ``slack`` -- faster at equal error;
* then, for that pair, times the walk's list-buffer size (the entries a
  walking warp buffers before it evaluates, ``list_buffer``) and the number
  of walking warps per SM (``walk_blocks_per_sm`` blocks of four warps; one
  warp walks and evaluates a group, its 64 slots shared out among the
  group's bodies), which change the speed, not the lists.

Results are cached in ``tuned.json`` beside this file, keyed by workload class
(log2 N, theta); :func:`tuned_params` looks them up.

    python -m paper_1106_1900_gb300.autotune --n 1048576 --theta 0.5 --eps 0.005
    python -m paper_1106_1900_gb300.autotune --workload ensemble --theta 0.5 --eps 0.01
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


WALK_GRID = [(lb, wb) for lb in (1024, 2048, 4096, 8192) for wb in (4, 5, 6)]
WALK_KEYS = ("list_buffer", "walk_blocks_per_sm")


def tuned_params(n: int, theta: float, kind: str = "plummer", path: str = TUNED):
    """The cached parameters (n_leaf, n_crit and, when tuned, list_buffer and
    walk_blocks_per_sm) for this workload class, or None."""
    e = load_table(path).get(key_for(n, theta, kind))
    if e is None:
        return None
    out = {"n_leaf": e["n_leaf"], "n_crit": e["n_crit"]}
    for k in WALK_KEYS:
        if k in e:
            out[k] = e[k]
    return out


def _errors(acc, ref):
    import torch

    a = acc.double()
    r = ref.double()
    e = (torch.linalg.norm(a - r, dim=1) / torch.linalg.norm(r, dim=1)).cpu()
    q = torch.quantile(e, torch.tensor([0.5, 0.99], dtype=e.dtype))
    return {"p50": float(q[0]), "p99": float(q[1]), "rms": float(torch.sqrt((e * e).mean()))}


def measure(pos, vel, mass, theta, eps, dt, params, steps, targets, ref_acc, device=0, offsets=None):
    """Error against the reference and the mean step time of one parameter set."""
    import torch

    from . import TreeCode

    n = pos.shape[0]
    nsys = 1 if offsets is None else len(offsets) - 1
    tc = TreeCode(n, nsys, device=device, **params)
    try:
        tc.build(pos, mass, offsets=offsets)
        acc, _ = tc.compute_forces(theta, eps)
        tc.check()
        err = _errors(acc[targets.long()], ref_acc)
        tc.set_state(pos, vel, mass, offsets=offsets)
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
    return {**params, "ms_per_step": ms, **err}


def measure_or_skip(*args, **kw):
    """measure(), None when the parameters do not fit (a capacity error)."""
    from . import STATUS_CAPACITY, BHError

    try:
        return measure(*args, **kw)
    except BHError as e:
        if e.code != STATUS_CAPACITY:
            raise
        return None


def reference(pos, mass, eps, targets, offsets=None):
    """Direct-summation accelerations on the targets (sorted body indices): of
    the whole system, or of each target's own system in a forest."""
    import numpy as np
    import torch

    from . import direct_forces

    if offsets is None:
        return direct_forces(pos, mass, targets, eps)[0]
    tg = targets.cpu().numpy()
    out = torch.empty((len(tg), 3), dtype=torch.float32, device=pos.device)
    sys_of = np.searchsorted(np.asarray(offsets), tg, side="right") - 1
    for s in np.unique(sys_of):
        lo, hi = int(offsets[s]), int(offsets[s + 1])
        sel = np.nonzero(sys_of == s)[0]
        local = torch.from_numpy((tg[sel] - lo).astype(np.int32)).to(pos.device)
        acc, _ = direct_forces(pos[lo:hi], mass[lo:hi], local, eps)
        out[torch.from_numpy(sel).to(pos.device)] = acc
    return out


def autotune(pos, vel, mass, theta, eps, dt=1.0 / 64, grid=None, steps=5, subsample=4096, seed=40, slack=1.05,
             device=0, log=None, offsets=None, walk_grid=None):
    """Returns (best, trials).  pos/vel/mass are float64 CUDA tensors;
    ``offsets`` (host, n_sys + 1) makes the bodies a forest of systems."""
    import numpy as np
    import torch

    grid = list(grid or DEFAULT_GRID)
    if PAPER_PAIR not in grid:
        grid.append(PAPER_PAIR)
    n = pos.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(n, size=min(subsample, n), replace=False)).astype(np.int32)
    targets = torch.from_numpy(idx).to(pos.device)
    ref_acc = reference(pos, mass, eps, targets, offsets)
    trials = []
    for nl, nc in grid:
        r = measure_or_skip(pos, vel, mass, theta, eps, dt, {"n_leaf": nl, "n_crit": nc}, steps, targets, ref_acc,
                            device, offsets)
        if r is None:
            r = {"n_leaf": nl, "n_crit": nc, "skipped": "does not fit the capacities"}
        else:
            trials.append(r)
        if log:
            log(r)
    paper = next(r for r in trials if (r["n_leaf"], r["n_crit"]) == PAPER_PAIR)
    ok = [r for r in trials if r["p99"] <= paper["p99"] * slack]
    best = min(ok, key=lambda r: r["ms_per_step"])
    # the walk's buffers and resident warps for the chosen pair (same lists, other speed)
    for lb, wb in (walk_grid if walk_grid is not None else WALK_GRID):
        params = {"n_leaf": best["n_leaf"], "n_crit": best["n_crit"], "list_buffer": lb, "walk_blocks_per_sm": wb}
        r = measure_or_skip(pos, vel, mass, theta, eps, dt, params, steps, targets, ref_acc, device, offsets)
        if r is None:
            continue
        r["stage"] = "walk"
        trials.append(r)
        if log:
            log(r)
        if r["ms_per_step"] < best["ms_per_step"] and r["p99"] <= paper["p99"] * slack:
            best = r
    return best, trials


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=0.005)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--workload", default="plummer", choices=["plummer", "galaxy", "ensemble"],
                    help="galaxy: Hernquist sphere + exponential disk, 8,388,608 bodies; ensemble: 512 Plummer "
                         "clusters of 1,024..65,536 bodies as one forest (--n ignored for both)")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--out", default=TUNED)
    args = ap.parse_args(argv)
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import ics

    off = None
    if args.workload == "galaxy":
        pos, vel, m = ics.galaxy(4194304, 4194304, 3)
    elif args.workload == "ensemble":
        pos, vel, m, off = ics.ensemble(512, 5)
    else:
        pos, vel, m = ics.plummer(args.n, args.seed)
    dev = torch.device("cuda", 0)
    P, V, M = (torch.from_numpy(a).to(dev) for a in (pos, vel, m))
    best, trials = autotune(P, V, M, args.theta, args.eps, steps=args.steps, offsets=off,
                            log=lambda r: print(json.dumps(r), flush=True))
    table = load_table(args.out)
    table[key_for(len(pos), args.theta, args.workload)] = {**best, "eps": args.eps, "trials": trials}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps({"best": best}))


if __name__ == "__main__":
    main()
