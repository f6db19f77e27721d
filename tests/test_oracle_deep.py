"""Pins of the oracle's deeper keys (App. B: 90-bit keys for 30 levels).

The paper's keys have 60 bits, so its trees stop at level 20; App. B names
longer keys as the way past that limit.  Here the key depth D runs from 20
to 30.  The pins tie the D-level oracle to closed forms (bit layout), to the
20-level keys (the quantisation to 2^D cells refines the one to 2^20 cells
exactly), to numpy's stable sort, and to the brute-force recursive octree.
"""
import numpy as np
import pytest

import ics
import oracle
from test_oracle_build import _check_tree


def _full(hi, lo, D):
    return (int(hi) << (3 * (D - 20))) | int(lo)


def test_deep_key_bit_layout():
    # extent 1 - 2^-20: L = 1 and level-30 cells of side 2^-30; one set bit
    # per axis -> the key's lowest bits
    step, top = 2.0 ** -30, 1 - 2.0 ** -20
    pos = np.array([[0, 0, 0], [step * 1.5, 0, 0], [0, step * 1.5, 0], [0, 0, step * 1.5],
                    [top, top, top]], dtype=np.float64)
    assert oracle.frames(pos)[0, 3] == 1.0
    q, hi, lo, _ = oracle.keys_split(pos, levels=30)
    assert q[1].tolist() == [1, 0, 0]
    assert lo[:4].tolist() == [0, 1, 2, 4] and hi[:4].tolist() == [0, 0, 0, 0]
    # the top corner: q = 2^30 - 2^10, the top 20 bits set on every axis
    assert q[4].tolist() == [2 ** 30 - 2 ** 10] * 3
    assert int(hi[4]) == (1 << 60) - 1 and int(lo[4]) == 0
    # 1.5 2^-21: bits 9 and 8 of q_x (levels 21 and 22) -> key bits 27 and 24
    q, hi, lo, _ = oracle.keys_split(np.array([[0, 0, 0], [2.0 ** -21 * 1.5, 0, 0], [top, 0, 0]]), levels=30)
    assert q[1, 0] == 3 << 8 and int(hi[1]) == 0 and int(lo[1]) == (1 << 27) | (1 << 24)


@pytest.mark.parametrize("D", [21, 25, 30])
def test_deep_keys_refine_the_60_bit_keys(D):
    # floor(floor(d 2^D) / 2^(D-20)) = floor(d 2^20): the top 20 levels are the 60-bit key
    pos, _, _ = ics.plummer(3000, 12)
    q20, key20, _ = oracle.keys(pos)
    q, hi, lo, _ = oracle.keys_split(pos, levels=D)
    assert np.array_equal(q >> (D - 20), q20)
    assert np.array_equal(hi, key20)
    assert q.min() >= 0 and q.max() <= 2 ** D - 1
    assert int(lo.max()) < 1 << (3 * (D - 20))


def test_deep_key_is_the_bit_interleave():
    rng = np.random.default_rng(4)
    pos = rng.uniform(size=(300, 3))
    D = 30
    q, hi, lo, _ = oracle.keys_split(pos, levels=D)
    for i in range(300):
        want = 0
        for b in range(D):
            for a in range(3):
                want |= ((int(q[i, a]) >> b) & 1) << (3 * b + a)
        assert _full(hi[i], lo[i], D) == want


def test_deep_key_prefix_is_octree_cell():
    rng = np.random.default_rng(13)
    pos = rng.uniform(size=(400, 3)) * np.array([1.0, 1e-6, 1.0])  # also close pairs in y
    D = 28
    q, hi, lo, _ = oracle.keys_split(pos, levels=D)
    for _ in range(3000):
        i, j = rng.integers(0, 400, 2)
        k = int(rng.integers(0, D + 1))
        sh = 3 * (D - k)
        same_key = (_full(hi[i], lo[i], D) >> sh) == (_full(hi[j], lo[j], D) >> sh)
        same_q = all((int(q[i, a]) >> (D - k)) == (int(q[j, a]) >> (D - k)) for a in range(3))
        assert same_key == same_q


def test_deep_sort_matches_numpy_stable():
    rng = np.random.default_rng(6)
    n = 5000
    hi = rng.integers(0, 6, n).astype(np.uint64)  # many ties in both words
    lo = rng.integers(0, 6, n).astype(np.uint64)
    sys_ = np.sort(rng.integers(0, 3, n)).astype(np.int32)
    perm = oracle.sort_perm(hi, sys_, lo, levels=24)
    want = np.lexsort((np.arange(n), lo, hi, sys_))
    assert np.array_equal(perm, want)


@pytest.mark.parametrize("D", [21, 26, 30])
def test_deep_tree_matches_brute_force_nested(D):
    # 300 of 2000 bodies in one level-20 cell: the D-level tree splits it
    pos, _, m = ics.nested(2000, 5, 300)
    t = oracle.build_tree(pos, m, n_leaf=8, n_crit=32, levels=D)
    assert t.levels == D
    _check_tree(t, 8, 32)
    assert t.level.max() > 20
    t20 = oracle.build_tree(pos, m, n_leaf=8, n_crit=32)
    _check_tree(t20, 8, 32)
    crowded = (t20.level == 20) & (t20.pend - t20.pbeg > 8)
    assert crowded.any()
    # every leaf below level D holds at most N_leaf bodies
    deep_leaf = (t.is_leaf == 1) & (t.level < D)
    assert np.all(t.pend[deep_leaf] - t.pbeg[deep_leaf] <= 8)


def test_deep_tree_adversarial():
    rng = np.random.default_rng(2)
    cases = [np.zeros((40, 3)) + 0.3]  # coincident: a chain to level D and one leaf
    p = rng.uniform(size=(200, 3)) * 1e-9
    p[0] = [1e3, 1e3, 1e3]  # far outlier: a long single-child chain below level 20
    cases.append(p)
    cases.append(np.concatenate([rng.uniform(size=(60, 3)), np.zeros((30, 3)) + 0.5]))
    for pos in cases:
        m = np.full(len(pos), 1.0 / len(pos))
        t = oracle.build_tree(pos, m, n_leaf=16, n_crit=8, levels=30)
        _check_tree(t, 16, 8)
    t = oracle.build_tree(cases[0], np.full(40, 0.025), n_leaf=16, n_crit=8, levels=30)
    assert t.level.tolist() == list(range(31))
    assert list(zip(t.gbeg, t.gend)) == [(0, 8), (8, 16), (16, 24), (24, 32), (32, 40)]


def test_deep_tree_equals_the_20_level_tree_when_uncrowded():
    # no level-20 cell holds more than N_leaf bodies: nothing changes
    pos, _, m = ics.plummer(3000, 8)
    a = oracle.build_tree(pos, m, 16, 64)
    b = oracle.build_tree(pos, m, 16, 64, levels=30)
    assert a.level.max() < 20
    for f in ("perm", "level", "pbeg", "pend", "is_leaf", "parent", "first_child", "n_children", "gbeg", "gend"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    for f in ("M", "com", "Q", "ctr", "size", "delta"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_deep_forest_equals_plain_systems():
    pa, _, ma = ics.nested(700, 1, 150)
    pb, _, mb = ics.plummer(400, 2)
    pos, m = np.concatenate([pa, pb, pa[:90] * 3.0]), np.concatenate([ma, mb, ma[:90]])
    off = np.array([0, 700, 700, 1100, 1190])
    t = oracle.build_tree(pos, m, 8, 32, offsets=off, levels=30)
    _check_tree(t, 8, 32)
    for s in range(4):
        b, e = off[s], off[s + 1]
        if e == b:
            continue
        ts = oracle.build_tree(pos[b:e], m[b:e], 8, 32, levels=30)
        sel = t.csys == s
        assert np.array_equal(t.perm[b:e] - b, ts.perm)
        assert np.array_equal(t.level[sel], ts.level)
        assert np.array_equal(t.pbeg[sel] - b, ts.pbeg)


def test_deep_geometry_and_moments():
    # level-k cells have side L 2^-k and hold their bodies; moments straight from the bodies
    pos, _, m = ics.nested(1500, 7, 400)
    t = oracle.build_tree(pos, m, 8, 32, levels=30)
    L = t.frame[0, 3]
    assert np.array_equal(t.size, L / 2.0 ** t.level)
    for c in range(t.C):
        b, e = t.pbeg[c], t.pend[c]
        x = t.spos[b:e]
        assert np.all(np.abs(x - t.ctr[c]) <= 0.5 * t.size[c] * (1 + 1e-12) + 1e-300)
        assert t.M[c] == pytest.approx(m[t.perm[b:e]].sum(), rel=1e-14)


def test_deep_walk_theta_to_zero_is_direct():
    pos, _, m = ics.nested(1200, 9, 300)
    acc, pot, t, _ = oracle.tree_forces(pos, m, theta=1e-6, eps=1e-7, n_leaf=8, n_crit=32, levels=30)
    assert t.level.max() > 20
    ad, pd = oracle.direct(pos, m, eps=1e-7)
    assert np.allclose(acc, ad, rtol=1e-9, atol=1e-9 * np.abs(ad).max())
    assert np.allclose(pot, pd, rtol=1e-12)


def test_deep_levels_out_of_range():
    pos, _, m = ics.plummer(10, 1)
    for D in (19, 31):
        with pytest.raises(ValueError):
            oracle.build_tree(pos, m, levels=D)
