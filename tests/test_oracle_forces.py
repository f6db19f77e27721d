"""Pins of the oracle's floating-point path (moments, walk, direct sum, leapfrog).

Closed forms and invariants that a dropped term, a wrong sign or a wrong index
would break: two-body quadrupole, the octupole-order far-field error of the
quadrupole expansion, theta -> 0 giving the direct sum (§3.3), momentum
conservation, the lists partitioning the system, the Plummer potential, the
virial ratio and a two-body circular orbit.
"""
import math

import numpy as np
import pytest

import ics
import oracle


# ------------------------------------------------------------- §3.2 moments
def test_two_body_moments_closed_form():
    x1, x2 = np.array([0.1, 0.2, 0.3]), np.array([0.35, 0.1, 0.31])
    m1, m2 = 0.3, 0.7
    t = oracle.build_tree(np.array([x1, x2]), np.array([m1, m2]), n_leaf=4, n_crit=4)
    assert t.C == 1 and t.is_leaf[0] == 1
    M = m1 + m2
    assert t.M[0] == pytest.approx(M, rel=1e-15)
    assert np.allclose(t.com[0], (m1 * x1 + m2 * x2) / M, rtol=0, atol=1e-15)
    # traceless quadrupole of two bodies: mu (3 d d^T - d^2 I), mu the reduced mass
    d = x2 - x1
    mu = m1 * m2 / M
    Qf = mu * (3 * np.outer(d, d) - d @ d * np.eye(3))
    want = [Qf[0, 0], Qf[1, 1], Qf[2, 2], Qf[0, 1], Qf[0, 2], Qf[1, 2]]
    assert np.allclose(t.Q[0], want, rtol=0, atol=1e-15)


def test_symmetric_cell_has_no_quadrupole():
    h = 0.01
    pos = np.array([[h, 0, 0], [-h, 0, 0], [0, h, 0], [0, -h, 0], [0, 0, h], [0, 0, -h]]) + 0.5
    t = oracle.build_tree(pos, np.full(6, 1 / 6), n_leaf=16, n_crit=16)
    assert np.max(np.abs(t.Q[0])) < 1e-18
    assert np.allclose(t.com[0], [0.5, 0.5, 0.5], atol=1e-16)


def test_geometry_and_containment():
    pos, _, m = ics.plummer(3000, 21)
    t = oracle.build_tree(pos, m)
    assert np.all(t.size == t.frame[0, 3] / 2.0 ** t.level)
    for c in range(t.C):
        p = t.spos[t.pbeg[c]:t.pend[c]]
        assert np.all(p >= t.ctr[c] - t.size[c] / 2 - 1e-12)
        assert np.all(p <= t.ctr[c] + t.size[c] / 2 + 1e-12)
    assert np.allclose(t.delta, np.linalg.norm(t.com - t.ctr, axis=1), rtol=0, atol=1e-15)


def test_quadrupole_far_field_order():
    # relative error of mono+quad at distance R falls like R^-3 (octupole order);
    # the monopole alone falls like R^-2 (no dipole about the centre of mass)
    rng = np.random.default_rng(2)
    pos = rng.uniform(size=(12, 3)) * np.array([1.0, 0.6, 0.3])
    m = rng.uniform(0.5, 1.5, 12)
    t = oracle.build_tree(pos, m, n_leaf=16, n_crit=16)
    u = np.array([0.48, -0.64, 0.6])
    u /= np.linalg.norm(u)
    err_q, err_m = [], []
    for R in [20.0, 40.0, 80.0]:
        x = t.com[0] + R * u
        a_ex, p_ex = oracle.cell_exact(t, 0, x)
        a_mp, p_mp = oracle.cell_multipole(t, 0, x)
        err_q.append(np.linalg.norm(a_mp - a_ex) / np.linalg.norm(a_ex))
        mono = -t.M[0] * (x - t.com[0]) / np.linalg.norm(x - t.com[0]) ** 3
        err_m.append(np.linalg.norm(mono - a_ex) / np.linalg.norm(a_ex))
        assert abs(p_mp - p_ex) / abs(p_ex) < err_m[-1]
    for i in range(2):
        assert 6.0 < err_q[i] / err_q[i + 1] < 10.5
        assert 3.0 < err_m[i] / err_m[i + 1] < 5.2
    assert err_q[0] < 0.2 * err_m[0]


# ---------------------------------------------------------- direct summation
def test_direct_matches_numpy_brute_force():
    pos, _, m = ics.plummer(64, 5)
    eps = 0.01
    a, p = oracle.direct(pos, m, eps)
    d = pos[None, :, :] - pos[:, None, :]
    r2 = (d * d).sum(-1) + eps * eps
    np.fill_diagonal(r2, np.inf)
    inv = 1.0 / np.sqrt(r2)
    a_ref = (m[None, :, None] * d * (inv ** 3)[:, :, None]).sum(1)
    p_ref = -(m[None, :] * inv).sum(1)
    assert np.allclose(a, a_ref, rtol=1e-13, atol=0)
    assert np.allclose(p, p_ref, rtol=1e-13, atol=0)


def test_direct_momentum_conservation():
    pos, _, m = ics.plummer(2000, 6)
    a, _ = oracle.direct(pos, m, 0.0)
    f = (m[:, None] * a).sum(0)
    assert np.max(np.abs(f)) < 1e-13 * np.abs(m[:, None] * a).sum()


def test_direct_plummer_closed_form_potential():
    n = 8192
    pos, vel, m = ics.plummer(n, 8)
    _, p = oracle.direct(pos, m, 0.0)
    b = 3 * math.pi / 16
    r = np.linalg.norm(pos, axis=1)
    closed = -1.0 / np.sqrt(r * r + b * b)
    order = np.argsort(r)
    for chunk in np.array_split(order[: int(0.95 * n)], 8):
        rel = np.mean(p[chunk] - closed[chunk]) / abs(np.mean(closed[chunk]))
        assert abs(rel) < 0.03
    # virial ratio 2K/|W| = 1 within a few 1/sqrt(N)
    ek, ep, _ = oracle.energy(vel, m, p)
    assert abs(2 * ek / abs(ep) - 1.0) < 3.0 / math.sqrt(n)
    assert ep == pytest.approx(-0.5, rel=0.03)  # virial units: W = -1/2


# ----------------------------------------------------------------- §2.2 walk
@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_theta_zero_is_direct_sum(eps):
    pos, _, m = ics.plummer(1500, 12)
    acc, pot, t, st = oracle.tree_forces(pos, m, theta=0.0, eps=eps, n_leaf=8, n_crit=32)
    assert np.all(st["nc"] == 0)
    assert np.all(st["np"] == 1500)
    ad, pd = oracle.direct(pos, m, eps)
    assert np.allclose(acc, ad, rtol=1e-11, atol=1e-13 * np.abs(ad).max())
    assert np.allclose(pot, pd, rtol=1e-12)


def test_walk_lists_partition_the_system():
    # with a huge softening every interaction is ~ -m/eps, so phi*eps sums the
    # mass on both lists: it must be the system mass minus the body's own, and
    # a*eps^3 must be M (COM - x) (the monopole reproduces the first moment)
    pos, _, m = ics.plummer(3000, 13)
    m = m * np.random.default_rng(0).uniform(0.5, 1.5, 3000)
    eps = 1e6
    acc, pot, t, st = oracle.tree_forces(pos, m, theta=0.6, eps=eps)
    assert st["nc"].sum() > 0
    Mtot = m.sum()
    assert np.max(np.abs(pot * eps + (Mtot - m))) < 1e-9
    com = (m[:, None] * pos).sum(0) / Mtot
    want = Mtot * (com[None, :] - pos)
    assert np.max(np.abs(acc * eps ** 3 - want)) < 1e-8 * np.abs(want).max()


def test_tree_error_vs_direct_by_theta():
    pos, _, m = ics.plummer(16384, 1)
    ad, _ = oracle.direct(pos, m, 0.01)
    med = []
    for th in [0.3, 0.5, 0.75]:
        acc, _, _, _ = oracle.tree_forces(pos, m, th, 0.01)
        err = np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)
        med.append(np.median(err))
    assert med[0] < med[1] < med[2]
    assert 1e-6 < med[1] < 1e-3  # quadrupole tree at theta = 0.5: ~1e-4


# --------------------------------------- §2.3 minimal-distance criterion (mac = 1)
@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_min_distance_theta_zero_is_direct_sum(eps):
    pos, _, m = ics.plummer(1500, 12)
    acc, pot, t, st = oracle.tree_forces(pos, m, theta=0.0, eps=eps, n_leaf=8, n_crit=32, mac=1)
    assert np.all(st["nc"] == 0) and np.all(st["np"] == 1500)
    ad, pd = oracle.direct(pos, m, eps)
    assert np.allclose(acc, ad, rtol=1e-11, atol=1e-13 * np.abs(ad).max())
    assert np.allclose(pot, pd, rtol=1e-12)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.75])
def test_min_distance_is_more_accurate_and_costlier(theta):
    # §2.3: the minimal-distance criterion gives smaller acceleration errors
    # than Eq. 1 at the same theta, at the price of more interactions
    pos, _, m = ics.plummer(8192, 7)
    sub = ics.subsample(8192, 1024, 41)
    ad, _ = oracle.direct(pos, m, 0.005, targets=sub)
    rms, inter = [], []
    for mac in (0, 1):
        acc, _, t, st = oracle.tree_forces(pos, m, theta, 0.005, mac=mac)
        e = np.linalg.norm(acc[sub] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        rms.append(np.sqrt(np.mean(e * e)))
        inter.append(((t.gend - t.gbeg) * (st["nc"] + st["np"])).sum())
    assert rms[1] < 0.95 * rms[0]
    assert inter[1] > 1.1 * inter[0]


def test_opening_margin_reported():
    pos, _, m = ics.plummer(4000, 14)
    _, _, _, st = oracle.tree_forces(pos, m, 0.5, 0.01)
    assert np.all(st["margin"] >= 0) and np.all(np.isfinite(st["margin"]))


def test_single_and_pair():
    a, p, _, _ = oracle.tree_forces(np.array([[1.0, 2.0, 3.0]]), np.array([2.0]), 0.5, 0.0)
    assert a.tolist() == [[0.0, 0.0, 0.0]] and p.tolist() == [0.0]
    pos = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    a, p, _, _ = oracle.tree_forces(pos, np.array([1.0, 3.0]), 0.5, 0.0)
    assert np.allclose(a, [[0.75, 0, 0], [-0.25, 0, 0]]) and np.allclose(p, [-1.5, -0.5])


# ------------------------------------------------------------ §3.1 leapfrog
def test_leapfrog_two_body_circular_orbit():
    m = np.array([0.25, 0.75])
    d = 1.0
    pos = np.array([[-0.75 * d, 0, 0], [0.25 * d, 0, 0]])
    omega = 1.0  # omega^2 = G (m1 + m2) / d^3
    vel = np.array([[0, -0.75 * omega, 0], [0, 0.25 * omega, 0]])
    accel = lambda x: oracle.direct(x, m, 0.0)
    a, p = accel(pos)
    e0 = oracle.energy(vel, m, p)[2]
    assert e0 == pytest.approx(-m[0] * m[1] / (2 * d), rel=1e-14)
    steps = 1000
    dt = 2 * math.pi / steps
    x, v = pos.copy(), vel.copy()
    emax = 0.0
    for _ in range(steps):
        x, v, a, p = oracle.leapfrog_step(x, v, a, dt, accel)
        emax = max(emax, abs(oracle.energy(v, m, p)[2] / e0 - 1))
    assert emax < 1e-5
    assert np.max(np.abs(x - pos)) < 1e-3  # back after one period 2 pi
    assert np.max(np.abs(oracle.momentum(v, m))) < 1e-14
