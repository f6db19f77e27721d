"""Comparison helpers for the CUDA-vs-oracle parity tests.

Integer results (keys, permutation, cell and group tables) must be identical.
Forces follow this policy:

* A group's interaction lists are compared through their lengths and index
  sums.  Where they match, every body of the group must satisfy
  |a_gpu - a_oracle| <= TOL * max(|a_oracle|, KAPPA * sum_j |a_ij|) and
  |phi_gpu - phi_oracle| <= TOL * |phi_oracle|, TOL = 1e-5.  The second
  term of the max only matters for bodies whose force nearly cancels (at the
  centre of a cluster |a| -> 0 while its terms do not): FP32 terms carry
  errors proportional to their own size, not to the sum's; KAPPA follows
  from the FP32 error bound of one term (see U_TERM).
* Where they differ, an opening decision flipped between FP32 and FP64; the
  oracle must have met a decision that close to its threshold (relative
  margin < MARGIN), and those bodies are held to FLIP_TOL = 1e-3 (the tree's
  own approximation error).
* Neither exception may be common: the bodies that needed the conditioning
  term and the groups with a flipped decision are counted and bounded.
"""
import numpy as np

TOL = 1e-5
# One FP32 interaction term carries a relative error of at most about
# U_TERM = 8 * 2^-24 (rsqrtf <= 2 ulp plus ~6 further roundings, each <= 1/2 ulp).
# If those errors line up, a sum's error reaches U_TERM * sum_j |a_ij|, so a
# body can only be held to TOL relative to max(|a|, U_TERM/TOL * sum_j |a_ij|).
U_TERM = 8 * 2.0 ** -24
KAPPA = U_TERM / TOL  # ~0.048
MARGIN = 1e-5
FLIP_TOL = 1e-3
# At most this fraction of the compared bodies may need the conditioning clause
# (their |a| below KAPPA * sum_j |a_ij|: near the centre of a cluster), and at
# most this fraction of the compared groups may have a flipped decision; the
# absolute floors serve small inputs.
MAX_COND_FRAC = 1e-3
MIN_COND = 4
MAX_FLIP_FRAC = 5e-3
MIN_FLIP = 2


def group_of_sorted(gbeg, n):
    g = np.searchsorted(np.asarray(gbeg), np.arange(n), side="right") - 1
    return g


def compare_tree(tree_gpu, t):
    """Bit-exact comparison of the integer tree with the oracle's ``Tree``."""
    assert np.array_equal(tree_gpu["skey"], t.skey), "sorted keys differ"
    assert np.array_equal(tree_gpu["perm"].astype(np.int64), t.perm), "sort permutation differs"
    assert len(tree_gpu["level"]) == t.C, f"cell count {len(tree_gpu['level'])} != {t.C}"
    assert np.array_equal(tree_gpu["level"], t.level), "cell levels differ"
    assert np.array_equal(tree_gpu["pbeg"], t.pbeg), "cell first bodies differ"
    assert np.array_equal(tree_gpu["pend"], t.pend), "cell body ends differ"
    assert np.array_equal(tree_gpu["is_leaf"], t.is_leaf), "leaf flags differ"
    assert np.array_equal(tree_gpu["parent"], t.parent), "parents differ"
    assert np.array_equal(tree_gpu["first_child"], t.first_child), "first children differ"
    assert np.array_equal(tree_gpu["n_children"], t.n_children), "child counts differ"
    assert np.array_equal(tree_gpu["gbeg"], t.gbeg), "group starts differ"
    assert np.array_equal(tree_gpu["gend"], t.gend), "group ends differ"


def compare_moments(mom, t, tol=2e-6):
    """Moments against the oracle's FP64 values, scaled by each cell's size."""
    M = t.M
    assert np.allclose(mom["mass"], M, rtol=tol, atol=0), "cell masses differ"
    l = t.size
    com_err = np.abs(mom["com"] - t.com).max(axis=1) / l
    assert com_err.max() < tol, f"centre of mass off by {com_err.max():.2e} cell sizes"
    q_scale = np.maximum(M * l * l, 1e-300)
    q_err = np.abs(mom["quad"].astype(np.float64) - t.Q).max(axis=1) / q_scale
    assert q_err.max() < 10 * tol, f"quadrupole off by {q_err.max():.2e} M l^2"
    assert np.allclose(mom["size"], l, rtol=1e-7, atol=0)
    d_err = np.abs(mom["delta"] - t.delta) / l
    assert d_err.max() < tol, f"delta off by {d_err.max():.2e} cell sizes"
    return {"com": float(com_err.max()), "quad": float(q_err.max()), "delta": float(d_err.max())}


def group_forces_report(acc_in, pot_in, t, groups, acc_s, pot_s, st_o, st_g, tol=TOL):
    """Forces of the listed groups under the policy above.

    ``acc_in``/``pot_in``: the GPU's results in input order; ``acc_s``,
    ``pot_s``, ``st_o``: the oracle's walk of ``groups`` (sorted order, stats
    per listed group); ``st_g``: the GPU's group statistics of the same groups.
    Besides the per-body bounds it bounds how many bodies needed the
    conditioning clause (at most MAX_COND_FRAC of the compared bodies) and how
    many groups had an opening decision flip (at most MAX_FLIP_FRAC of them),
    so that neither clause can cover a systematic error."""
    groups = np.asarray(groups, dtype=np.int64)
    same = ((st_g["nc"] == st_o["nc"]) & (st_g["np"] == st_o["np"]) & (st_g["csum"] == st_o["csum"])
            & (st_g["psum"] == st_o["psum"]))
    flipped = np.nonzero(~same)[0]
    assert np.all(st_o["margin"][flipped] < MARGIN), (
        f"groups {groups[flipped[st_o['margin'][flipped] >= MARGIN][:10]]} have different lists without a near-tie")
    sizes = t.gend[groups] - t.gbeg[groups]
    bodies = np.concatenate([np.arange(t.gbeg[g], t.gend[g]) for g in groups]) if len(groups) else np.zeros(0, int)
    ok_body = np.repeat(same, sizes)
    inp = t.perm[bodies]
    ao = acc_s[bodies]
    an = np.linalg.norm(ao, axis=1)
    amag = st_o["amag"][bodies]
    scale = np.maximum(an, KAPPA * amag)
    da = np.linalg.norm(acc_in[inp].astype(np.float64) - ao, axis=1)
    rel = da / np.maximum(scale, 1e-300)
    po = pot_s[bodies]
    prel = np.abs(pot_in[inp].astype(np.float64) - po) / np.maximum(np.abs(po), 1e-300)
    plain = da / np.maximum(an, 1e-300)
    any_ok = bool(ok_body.any())
    rep = {
        "groups": int(len(groups)), "bodies": int(len(bodies)), "flipped_groups": int(len(flipped)),
        "max_rel": float(rel[ok_body].max()) if any_ok else 0.0,
        "max_prel": float(prel[ok_body].max()) if any_ok else 0.0,
        "p99_plain": float(np.percentile(plain[ok_body], 99)) if any_ok else 0.0,
        "max_plain": float(plain[ok_body].max()) if any_ok else 0.0,
        "n_conditioned": int(np.sum(ok_body & (plain > tol))),
        "worst_cond": float((an / np.maximum(amag, 1e-300))[ok_body][np.argmax(rel[ok_body])]) if any_ok else 0.0,
        "flip_max": float(rel[~ok_body].max()) if (~ok_body).any() else 0.0,
    }
    assert rep["max_rel"] <= tol, f"acceleration error {rep}"
    assert rep["max_prel"] <= tol, f"potential error {rep}"
    assert rep["flip_max"] <= FLIP_TOL, f"flipped-group error {rep}"
    assert rep["n_conditioned"] <= max(MIN_COND, MAX_COND_FRAC * rep["bodies"]), f"conditioning clause overused {rep}"
    assert rep["flipped_groups"] <= max(MIN_FLIP, MAX_FLIP_FRAC * rep["groups"]), f"too many flipped groups {rep}"
    return rep


def compare_forces(acc_g, pot_g, acc_o, pot_o, t, st_o, st_g, tol=TOL):
    """Accelerations and potentials of every group (GPU and oracle results in
    input order, ``st_o`` from ``oracle.tree_forces``)."""
    acc_s = np.empty_like(acc_o)
    pot_s = np.empty_like(pot_o)
    acc_s[np.arange(t.n)] = acc_o[t.perm]
    pot_s[np.arange(t.n)] = pot_o[t.perm]
    return group_forces_report(acc_g, pot_g, t, np.arange(t.G), acc_s, pot_s, st_o, st_g, tol)
