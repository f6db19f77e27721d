"""Pins of the oracle's integer path (frame, keys, sort, cells, links, groups).

Each test ties the oracle to something other than itself: the paper's worked
examples (tests/golden), hand-computed closed forms, numpy's stable sort, and
a brute-force recursive octree written here from the definition of an octree.
"""
import os

import numpy as np
import pytest

import ics
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            out[k] = v
    return out


# ------------------------------------------------------------------ App. B
def test_dilate_worked_example():
    g = _golden("dilate_example.txt")
    v = int(g["input"], 2)
    want = int(g["output"].replace(" ", ""), 2)
    assert oracle.dilate10(v) == want


def test_dilate_round_trip():
    for v in range(1024):
        d = oracle.dilate10(v)
        assert d & ~0x09249249 == 0  # only every third bit
        back = sum(((d >> (3 * b)) & 1) << b for b in range(10))
        assert back == v


def test_mask_footnote():
    g = _golden("mask_example.txt")
    assert int(g["key"], 2) & int(g["mask"], 2) == int(g["output"], 2)


def test_frame_closed_form():
    # extent 1 along x -> E*(1+2^-20) > 1 -> L = 2; origin = minimum corner
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.25, -0.5], [0.75, 0.0, 0.0]])
    fr = oracle.frames(pos)
    assert fr[0].tolist() == [0.0, 0.0, -0.5, 2.0]
    q, key, _ = oracle.keys(pos)
    # q = floor((x - origin) * 2^20 / L): exact values by hand
    assert q[1].tolist() == [524288, 131072, 0]
    assert q[2].tolist() == [393216, 0, 262144]
    # a single body and coincident bodies: E = 0 -> L = 1, q = 0
    fr0 = oracle.frames(np.array([[3.0, -2.0, 7.5]] * 3))
    assert fr0[0].tolist() == [3.0, -2.0, 7.5, 1.0]


def test_frame_is_smallest_power_of_two():
    rng = np.random.default_rng(7)
    for scale in [1e-9, 1e-3, 0.37, 1.0, 5.5, 1e4]:
        pos = rng.normal(size=(50, 3)) * scale
        fr = oracle.frames(pos)[0]
        E = float(np.max(pos.max(0) - pos.min(0)))
        v = E * (1.0 + 2.0 ** -20)
        L = fr[3]
        m, e = np.frexp(L)
        assert m == 0.5  # a power of two
        assert L >= v > L / 2
        assert fr[:3].tolist() == pos.min(0).tolist()


def test_key_bit_layout():
    # extent 1 - 2^-20: E (1 + 2^-20) = 1 - 2^-40 < 1, so L = 1 and a cell of
    # level 20 has side 2^-20; one set bit per axis -> the key's lowest three bits
    step = 2.0 ** -20
    pos = np.array([[0, 0, 0], [step * 1.5, 0, 0], [0, step * 1.5, 0], [0, 0, step * 1.5],
                    [1 - step, 1 - step, 1 - step]], dtype=np.float64)
    assert oracle.frames(pos)[0, 3] == 1.0
    q, key, _ = oracle.keys(pos)
    assert q[1].tolist() == [1, 0, 0]
    assert key[:4].tolist() == [0, 1, 2, 4]
    # the top corner: every bit set
    assert int(key[4]) == (1 << 60) - 1


def test_key_prefix_is_octree_cell():
    # two bodies share the top 3k key bits iff their q share the top k bits on every axis
    rng = np.random.default_rng(3)
    pos = rng.uniform(size=(400, 3))
    q, key, _ = oracle.keys(pos)
    for _ in range(2000):
        i, j = rng.integers(0, 400, 2)
        k = int(rng.integers(0, 21))
        same_key = (int(key[i]) >> (60 - 3 * k)) == (int(key[j]) >> (60 - 3 * k))
        same_q = all((int(q[i, a]) >> (20 - k)) == (int(q[j, a]) >> (20 - k)) for a in range(3))
        assert same_key == same_q


def test_quantisation_range_and_order():
    pos, _, _ = ics.plummer(3000, 11)
    q, _, _ = oracle.keys(pos)
    assert q.min() >= 0 and q.max() <= 2 ** 20 - 1
    for a in range(3):
        o = np.argsort(pos[:, a], kind="stable")
        assert np.all(np.diff(q[o, a]) >= 0)


# ------------------------------------------------------------------- sort
def test_sort_matches_numpy_stable():
    rng = np.random.default_rng(5)
    key = rng.integers(0, 40, 5000).astype(np.uint64)  # many ties
    sys_ = np.sort(rng.integers(0, 4, 5000)).astype(np.int32)
    perm = oracle.sort_perm(key, sys_)
    want = np.lexsort((np.arange(5000), key, sys_))
    assert np.array_equal(perm, want)


# ------------------------------------------------- brute-force octree (§2.1)
def brute_octree(t, n_leaf):
    """Recursive insertion-free octree over the sorted bodies, straight from the
    definition: split a cell into its occupied octants (by the next bit of the
    quantised coordinates) until it holds <= N_leaf bodies or is at the key
    depth (level 20 for the paper's 60-bit keys)."""
    q = t.sq
    depth = getattr(t, "levels", 20)
    cells = []

    def rec(b, e, k, parent, s):
        n = e - b
        leaf = n <= n_leaf or k == depth
        me = len(cells)
        cells.append({"level": k, "sys": s, "pbeg": b, "pend": e, "leaf": leaf, "parent": parent, "kids": []})
        if parent >= 0:
            cells[parent]["kids"].append(me)
        if leaf:
            return
        sh = depth - 1 - k
        octant = ((q[b:e, 0] >> sh) & 1) | (((q[b:e, 1] >> sh) & 1) << 1) | (((q[b:e, 2] >> sh) & 1) << 2)
        assert np.all(np.diff(octant) >= 0), "sorted order must list octants in order"
        for o in range(8):
            idx = np.nonzero(octant == o)[0]
            if len(idx):
                assert idx[-1] - idx[0] + 1 == len(idx)
                rec(b + int(idx[0]), b + int(idx[-1]) + 1, k + 1, me, s)

    for s in range(len(t.offsets) - 1):
        b, e = int(t.offsets[s]), int(t.offsets[s + 1])
        if e > b:
            rec(b, e, 0, -1, s)
    order = sorted(range(len(cells)), key=lambda c: (cells[c]["level"], cells[c]["sys"], cells[c]["pbeg"]))
    rank = {c: r for r, c in enumerate(order)}
    out = [cells[c] for c in order]
    for c in out:
        c["parent"] = rank[c["parent"]] if c["parent"] >= 0 else -1
        c["kids"] = sorted(rank[k] for k in c["kids"])
    return out


def brute_groups(cells, n_crit):
    groups = []

    def rec(c):
        cc = cells[c]
        n = cc["pend"] - cc["pbeg"]
        if n <= n_crit or cc["leaf"]:
            for b in range(cc["pbeg"], cc["pend"], n_crit):
                groups.append((b, min(b + n_crit, cc["pend"])))
        else:
            for k in cc["kids"]:
                rec(k)

    for c, cc in enumerate(cells):
        if cc["level"] == 0:
            rec(c)
    return groups


def _check_tree(t, n_leaf, n_crit):
    cells = brute_octree(t, n_leaf)
    assert t.C == len(cells)
    assert t.level.tolist() == [c["level"] for c in cells]
    assert t.csys.tolist() == [c["sys"] for c in cells]
    assert t.pbeg.tolist() == [c["pbeg"] for c in cells]
    assert t.pend.tolist() == [c["pend"] for c in cells]
    assert t.is_leaf.astype(bool).tolist() == [c["leaf"] for c in cells]
    assert t.parent.tolist() == [c["parent"] for c in cells]
    assert t.n_children.tolist() == [len(c["kids"]) for c in cells]
    for c, cc in enumerate(cells):
        if cc["kids"]:
            assert cc["kids"] == list(range(t.first_child[c], t.first_child[c] + len(cc["kids"])))
        else:
            assert t.first_child[c] == -1
    g = brute_groups(cells, n_crit)
    assert list(zip(t.gbeg.tolist(), t.gend.tolist())) == g
    # groups tile [0, N) in order
    if t.G:
        assert t.gbeg[0] == 0 and t.gend[-1] == t.n and np.all(t.gbeg[1:] == t.gend[:-1])


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (17, 2), (300, 3), (2000, 4)])
def test_tree_matches_brute_force_plummer(n, seed):
    pos, _, m = ics.plummer(n, seed)
    t = oracle.build_tree(pos, m, n_leaf=16, n_crit=64)
    _check_tree(t, 16, 64)


@pytest.mark.parametrize("n_leaf,n_crit", [(1, 1), (4, 8), (8, 32), (16, 16), (32, 64), (16, 128), (8, 256)])
def test_tree_parameters(n_leaf, n_crit):
    pos, _, m = ics.plummer(700, 9)
    t = oracle.build_tree(pos, m, n_leaf=n_leaf, n_crit=n_crit)
    _check_tree(t, n_leaf, n_crit)


def test_tree_adversarial():
    rng = np.random.default_rng(1)
    cases = []
    cases.append(np.zeros((40, 3)) + 0.3)  # coincident -> depth-20 leaf, chunked groups
    p = rng.uniform(size=(200, 3)) * 1e-3
    p[0] = [1e3, 1e3, 1e3]  # one body far away -> long single-child chain
    cases.append(p)
    cases.append(rng.uniform(size=(100, 3)) * np.array([1e-7, 1.0, 1.0]))  # flat in x
    cases.append(np.concatenate([rng.uniform(size=(60, 3)), np.zeros((30, 3)) + 0.5]))
    for pos in cases:
        m = np.full(len(pos), 1.0 / len(pos))
        t = oracle.build_tree(pos, m, n_leaf=16, n_crit=8)
        _check_tree(t, 16, 8)
    # the coincident case: a chain to level 20 ending in one leaf of 40 bodies
    t = oracle.build_tree(cases[0], np.full(40, 0.025), n_leaf=16, n_crit=8)
    assert t.level.tolist() == list(range(21))
    assert t.is_leaf.tolist() == [0] * 20 + [1]
    assert list(zip(t.gbeg, t.gend)) == [(0, 8), (8, 16), (16, 24), (24, 32), (32, 40)]


def test_forest_equals_plain_systems():
    # a forest's tables restricted to system s equal the plain tree of s (offset)
    pos, _, m, off = ics.ensemble(n_sys=5, seed=9, n_min=1, n_max=900)
    off = off.copy()
    t = oracle.build_tree(pos, m, 16, 64, offsets=off)
    _check_tree(t, 16, 64)
    for s in range(5):
        b, e = off[s], off[s + 1]
        ts = oracle.build_tree(pos[b:e], m[b:e], 16, 64)
        sel = t.csys == s
        assert np.array_equal(t.perm[b:e] - b, ts.perm)
        assert np.array_equal(t.pbeg[sel] - b, ts.pbeg)
        assert np.array_equal(t.pend[sel] - b, ts.pend)
        assert np.array_equal(t.level[sel], ts.level)
        assert np.array_equal(t.frame[s], ts.frame[0])


def test_forest_with_empty_systems():
    pos, _, m = ics.plummer(100, 4)
    off = np.array([0, 0, 30, 30, 100, 100])
    t = oracle.build_tree(pos, m, 16, 64, offsets=off)
    _check_tree(t, 16, 64)
    assert t.sys_root.tolist()[0] == -1 and t.sys_root[2] == -1 and t.sys_root[4] == -1
