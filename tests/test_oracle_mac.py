"""Pins of the oracle's opening decision (§3.3, Eq. 1) and of its
particle-cell potential (§3.2).

The opening test is pinned on a five-body system built by hand, where every
quantity Eq. 1 reads is a short dyadic fraction, so that the FP64 arithmetic
is exact and the decision can be placed exactly on, just inside and just
outside its threshold:

    frame: origin (0, 0, 0), side L = 1 (largest extent 0.7)
    cell P = the level-2 cell [0, 1/4)^3 holding the pair P1 = (0, 0, 0),
             P2 = (1/8, 0, 0), masses 1/4 each:
             centre of mass (1/16, 0, 0), geometric centre (1/8, 1/8, 1/8),
             delta = |(-1/16, -1/8, -1/8)| = 3/16, side l = 1/4
    X = (3/8, 3/8, 3/8): the other level-2 child of P's parent [0, 1/2)^3
    group g = the level-1 leaf holding A = (3/16, 9/20, 9/16) and
             B = (3/10, 3/8, 7/10); its box is [3/16, 3/10] x [3/8, 9/20]
             x [9/16, 7/10], whose point nearest to P's centre of mass is
             the corner (3/16, 3/8, 9/16) -- a corner that is no body
    theta = 1/2:  l/theta + delta = 1/2 + 3/16 = 11/16
    d = |(3/16, 3/8, 9/16) - (1/16, 0, 0)| = |(2, 6, 9)/16| = 11/16

With N_leaf = N_crit = 2 the walk of g opens the root, P's parent and g's own
leaf (margins far from any threshold) and meets P with d = l/theta + delta
exactly: a tie, which opens (the test is strict).  Moving the box by 2^-30
along z puts d just outside (accepted) or just inside (opened) the
threshold.  A decision that measured d from P's geometric centre, dropped
delta, accepted ties, multiplied by theta, took the wrong level's side, or
measured to the group's centre or to its nearest body instead of its box
changes the lists in at least one of these cases.
"""
import numpy as np
import pytest

import oracle

P1, P2 = (0.0, 0.0, 0.0), (0.125, 0.0, 0.0)
X = (0.375, 0.375, 0.375)
A0, B0 = (0.1875, 0.45, 0.5625), (0.3, 0.375, 0.7)
THETA = 0.5


def _system(dz=0.0):
    A = (A0[0], A0[1], A0[2] + dz)
    B = (B0[0], B0[1], B0[2] + dz)
    pos = np.array([P1, P2, X, A, B])
    m = np.array([0.25, 0.25, 0.2, 0.15, 0.15])
    return pos, m


def _walk_of_group(dz, mac=0):
    pos, m = _system(dz)
    t = oracle.build_tree(pos, m, n_leaf=2, n_crit=2)
    inv = np.empty(5, dtype=np.int64)
    inv[t.perm] = np.arange(5)  # sorted position of each input body
    # the group holding A and B
    g = [j for j in range(t.G) if t.gbeg[j] <= inv[3] < t.gend[j]]
    assert len(g) == 1
    g = g[0]
    assert sorted(range(t.gbeg[g], t.gend[g])) == sorted([inv[3], inv[4]])
    _, _, st = oracle.walk(t, THETA, 0.0, groups=[g], mac=mac)
    return t, inv, st


def _cell_of_pair(t, inv):
    c = [c for c in range(t.C) if t.pbeg[c] == min(inv[0], inv[1]) and t.pend[c] == max(inv[0], inv[1]) + 1]
    assert len(c) == 1
    return c[0]


def test_hand_built_cell_geometry():
    # the quantities Eq. 1 reads, for the pair's cell, as derived above
    t, inv, _ = _walk_of_group(0.0)
    c = _cell_of_pair(t, inv)
    assert t.frame[0].tolist() == [0.0, 0.0, 0.0, 1.0]
    assert t.level[c] == 2 and t.is_leaf[c] == 1
    assert t.size[c] == 0.25
    assert t.com[c].tolist() == [0.0625, 0.0, 0.0]
    assert t.ctr[c].tolist() == [0.125, 0.125, 0.125]
    assert t.delta[c] == 0.1875
    corner = np.array([A0[0], B0[1], A0[2]])
    assert np.linalg.norm(corner - t.com[c]) == 11 / 16 == 0.25 / THETA + 0.1875


def _expect(t, inv, st, pair_accepted):
    c = _cell_of_pair(t, inv)
    own = [inv[3], inv[4], inv[2]]  # the group's own leaf, and X (always opened)
    if pair_accepted:
        assert st["nc"][0] == 1 and st["csum"][0] == c
        assert st["np"][0] == 3 and st["psum"][0] == sum(own)
    else:
        assert st["nc"][0] == 0 and st["csum"][0] == 0
        assert st["np"][0] == 5 and st["psum"][0] == sum(own) + inv[0] + inv[1]


def test_eq1_tie_opens():
    t, inv, st = _walk_of_group(0.0)
    _expect(t, inv, st, pair_accepted=False)
    assert st["margin"][0] == 0.0  # the decision sat exactly on the threshold


def test_eq1_just_outside_accepts():
    t, inv, st = _walk_of_group(2.0 ** -30)
    _expect(t, inv, st, pair_accepted=True)


def test_eq1_just_inside_opens():
    t, inv, st = _walk_of_group(-(2.0 ** -30))
    _expect(t, inv, st, pair_accepted=False)


@pytest.mark.parametrize("dz", [0.0, 2.0 ** -30, -(2.0 ** -30)])
def test_eq1_by_the_definition(dz):
    # the same three cases against Eq. 1 written out on the hand values:
    # accept iff |COM - box| > l/theta + delta
    t, inv, st = _walk_of_group(dz)
    near = np.array([A0[0], B0[1], A0[2] + dz])
    d = np.linalg.norm(near - np.array([0.0625, 0.0, 0.0]))
    _expect(t, inv, st, pair_accepted=bool(d > 0.25 / THETA + 0.1875))


def test_min_distance_gap_on_hand_system():
    # §2.3's criterion on the same system: the gap between the pair's cube
    # [0, 1/4]^3 and the group's box is (0, 3/8 - 1/4, 9/16 - 1/4), of length
    # sqrt(1/64 + 25/256) < l/theta = 1/2, so the pair's cell is opened, as
    # Eq. 1 opens it at the tie; far along z the box is accepted
    t, inv, st = _walk_of_group(0.0, mac=1)
    _expect(t, inv, st, pair_accepted=False)
    gap = np.array([0.0, 0.375 - 0.25, 0.5625 - 0.25])
    assert np.linalg.norm(gap) < 0.5


# ----------------------------------------------- §3.2 particle-cell potential
class _Cell:
    """Stand-in tree of one cell with a given mass, centre and quadrupole."""

    def __init__(self, M, com, Q):
        self.M = np.array([float(M)])
        self.com = np.array([com], dtype=np.float64)
        self.Q = np.array([Q], dtype=np.float64)


def _random_traceless_q(rng):
    a = rng.normal(size=(3, 3))
    S = a + a.T
    S -= np.trace(S) / 3 * np.eye(3)
    return [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]


@pytest.mark.parametrize("M", [0.0, 1.3])
@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_pc_acceleration_is_minus_gradient_of_potential(M, eps):
    # the particle-cell force of §3.2 derives from its potential, softened or
    # not: a = -grad(phi), checked by central differences; with M = 0 both
    # sides are the quadrupole terms alone
    rng = np.random.default_rng(11)
    for _ in range(6):
        Q = _random_traceless_q(rng)
        cell = _Cell(M, [0.2, -0.1, 0.4], Q)
        x = np.array([0.2, -0.1, 0.4]) + rng.normal(size=3) * 1.5
        a, _ = oracle.cell_multipole(cell, 0, x, eps)
        h = 1e-5
        g = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            g[k] = -(oracle.cell_multipole(cell, 0, x + e, eps)[1] - oracle.cell_multipole(cell, 0, x - e, eps)[1]) / (
                2 * h)
        assert np.linalg.norm(a) > 1e-3
        assert np.linalg.norm(a - g) < 1e-7 * np.linalg.norm(a)


def test_pc_potential_far_field_order():
    # the potential of the monopole + quadrupole expansion is off by octupole
    # order, R^-3 relative; the monopole alone by quadrupole order, R^-2
    rng = np.random.default_rng(2)
    pos = rng.uniform(size=(12, 3)) * np.array([1.0, 0.6, 0.3])
    m = rng.uniform(0.5, 1.5, 12)
    t = oracle.build_tree(pos, m, n_leaf=16, n_crit=16)
    err_q, err_m = [], []
    for u in ([0.48, -0.64, 0.6], [1.0, 0.0, 0.0], [0.0, 0.6, 0.8]):
        u = np.array(u) / np.linalg.norm(u)
        eq, em = [], []
        for R in [20.0, 40.0, 80.0]:
            x = t.com[0] + R * u
            _, p_ex = oracle.cell_exact(t, 0, x)
            _, p_mp = oracle.cell_multipole(t, 0, x)
            p_mono = -t.M[0] / R
            eq.append(abs(p_mp - p_ex) / abs(p_ex))
            em.append(abs(p_mono - p_ex) / abs(p_ex))
        for i in range(2):
            assert 6.0 < eq[i] / eq[i + 1] < 10.5
            assert 3.0 < em[i] / em[i + 1] < 5.2
        assert eq[0] < 0.25 * em[0]
        err_q.append(eq)
        err_m.append(em)


def test_pc_potential_quadrupole_term_closed_form():
    # two bodies m1, m2 at separation s along z: about the centre of mass the
    # quadrupole is mu (3 s s^T - s^2 I), and on the axis at distance R the
    # exact potential is -m1/|R - z1| - m2/|R - z2|, whose expansion is
    # -M/R - mu s^2/R^3 + O(R^-4); the oracle's expansion must carry exactly
    # that R^-3 term: -(1/2) r.Q.r / R^5 = -(1/2) mu 2 s^2 R^2 / R^5
    m1, m2, s = 0.3, 0.7, 0.2
    M = m1 + m2
    mu = m1 * m2 / M
    z1, z2 = -m2 / M * s, m1 / M * s
    pos = np.array([[0.5, 0.5, 0.5 + z1], [0.5, 0.5, 0.5 + z2]])
    t = oracle.build_tree(pos, np.array([m1, m2]), n_leaf=4, n_crit=4)
    assert t.C == 1
    for R in (3.0, 7.0):
        x = np.array([0.5, 0.5, 0.5 + R])
        _, p = oracle.cell_multipole(t, 0, x)
        assert p == pytest.approx(-M / R - mu * s * s / R ** 3, rel=1e-13)
        # off the axis, in the plane z = 0.5: r.Q.r = -mu s^2 R^2
        x = np.array([0.5 + R, 0.5, 0.5])
        _, p = oracle.cell_multipole(t, 0, x)
        assert p == pytest.approx(-M / R + 0.5 * mu * s * s / R ** 3, rel=1e-13)
