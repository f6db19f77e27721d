"""The block time-step oracle (NEXT-1 of the hot path: per-body power-of-two
steps, the walk of the groups that hold active bodies, moment refresh on an
unchanged tree), pinned without the GPU."""
import numpy as np
import pytest

import ics
import oracle


def test_level_rule_at_power_of_two_boundaries():
    # dt_max 2^-k <= eta sqrt(eps/|a|)  <=>  2^k >= r = dt_max sqrt(|a|/eps) / eta
    eps, eta, dt_max = 0.01, 0.5, 0.25
    def acc_for(r):  # |a| giving exactly r
        return np.array([[eps * (r * eta / dt_max) ** 2, 0.0, 0.0]])
    for j in range(0, 6):
        r = 2.0 ** j
        assert oracle.block_level(acc_for(r), eps, eta, dt_max, 30)[0] == j
        assert oracle.block_level(acc_for(r * (1 + 1e-9)), eps, eta, dt_max, 30)[0] == j + 1
    assert oracle.block_level(acc_for(0.3), eps, eta, dt_max, 30)[0] == 0
    assert oracle.block_level(np.zeros((1, 3)), eps, eta, dt_max, 30)[0] == 0
    assert oracle.block_level(acc_for(1e9), eps, eta, dt_max, 7)[0] == 7


def test_refresh_without_motion_is_the_build():
    pos, _, m = ics.plummer(3000, 5)
    t = oracle.build_tree(pos, m, 16, 64)
    r = oracle.refresh_tree(t, t.spos.copy())
    for f in ("M", "com", "Q", "ctr", "size", "delta"):
        assert np.array_equal(getattr(r, f), getattr(t, f)), f


def test_refresh_cubes_hold_their_bodies_and_children():
    pos, vel, m = ics.plummer(3000, 6)
    t = oracle.build_tree(pos, m, 16, 64)
    moved = t.spos + 0.05 * np.random.default_rng(1).standard_normal(t.spos.shape)
    r = oracle.refresh_tree(t, moved)
    assert np.all(r.size >= t.size)
    assert np.any(r.size > t.size)
    for c in range(t.C):
        half = 0.5 * r.size[c]
        if t.is_leaf[c]:
            x = moved[t.pbeg[c]:t.pend[c]]
            assert np.all(np.abs(x - r.ctr[c]) <= half * (1 + 1e-12))
        else:
            for ch in range(t.first_child[c], t.first_child[c] + t.n_children[c]):
                assert np.all(np.abs(r.ctr[ch] - r.ctr[c]) + 0.5 * r.size[ch] <= half * (1 + 1e-12))
    # moments from the moved bodies, as a build at the moved positions would give
    M = np.array([m[t.perm][t.pbeg[c]:t.pend[c]].sum() for c in range(t.C)])
    assert np.allclose(r.M, M)


def test_single_level_is_the_shared_step_leapfrog():
    # k_max = 0: every body steps with dt_max every block step, all groups are
    # active, and the block step is the shared-step leapfrog bit for bit
    pos, vel, m = ics.plummer(1500, 8)
    dt, theta, eps = 1.0 / 64, 0.5, 0.01
    st = oracle.block_start(oracle.BlockState(pos, vel, m, dt, 0, 1.0), theta, eps)
    accel = lambda x: oracle.tree_forces(x, m, theta, eps)[:2]
    x, v = pos.copy(), vel.copy()
    a, _ = accel(x)
    for _ in range(3):
        act = oracle.block_step(st, theta, eps, rebuild=True)
        assert act.all()
        x, v, a, _ = oracle.leapfrog_step(x, v, a, dt, accel)
    assert np.array_equal(st.x, x) and np.array_equal(st.v, v) and np.array_equal(st.a, a)
    assert st.T == 3


@pytest.mark.parametrize("rebuild", [True, False])
def test_block_steps_conserve_energy(rebuild):
    pos, vel, m = ics.plummer(2000, 3)
    theta, eps = 0.4, 0.01
    st = oracle.block_start(oracle.BlockState(pos, vel, m, 1.0 / 32, 5, 0.05), theta, eps)
    e0 = oracle.energy(st.v, m, st.pot)[2]
    assert len(np.unique(st.k)) >= 3  # the bodies spread over several levels
    updates = 0
    while st.T < 8 * 2 ** 5:  # eight synchronisation intervals of dt_max
        act = oracle.block_step(st, theta, eps, rebuild=rebuild or st.T % 2 ** 5 == 0)
        updates += act.sum()
    assert np.all(st.t == st.T)  # synchronised again
    _, pot, _, _ = oracle.tree_forces(st.x, m, theta, eps)
    e1 = oracle.energy(st.v, m, pot)[2]
    assert abs((e1 - e0) / e0) < 2e-4
    # fewer force evaluations than stepping every body with the smallest step used
    assert updates < len(m) * 8 * 2 ** int(st.k.max())
