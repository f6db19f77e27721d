"""Deeper keys on the GPU against the oracle (App. B: 90-bit keys for 30
levels lift the 20-level limit of 60-bit keys).  Needs a GB300.

Integer tables (both key words, permutation, cells, links, groups) are
compared bit for bit, moments and forces under the policy of tests/_parity.py.
"""
import numpy as np
import pytest

import ics
import oracle
from tests import _parity as P
from tests.test_gpu_parity import _dev, _run

pytestmark = pytest.mark.gpu


def _deep_parity(bh, pos, m, theta, eps, D, n_leaf=8, n_crit=64, offsets=None, **kw):
    tc, acc, pot = _run(bh, pos, m, theta, eps, n_leaf, n_crit, offsets, key_levels=D, **kw)
    acc_o, pot_o, t, st_o = oracle.tree_forces(pos, m, theta, eps, n_leaf, n_crit, offsets, mac=kw.get("mac", 0),
                                               levels=D)
    tr = tc.tree()
    P.compare_tree(tr, t)
    assert np.array_equal(tr["skey_lo"], t.skey_lo), "sorted low key words differ"
    if t.C:
        P.compare_moments(tc.moments(), t)
    rep = P.compare_forces(acc, pot, acc_o, pot_o, t, st_o, tc.group_stats())
    return tc, t, rep


@pytest.mark.parametrize("D", [21, 25, 30])
def test_deep_keys_nested_cluster(cuda_lib, D):
    # 3000 of 20000 bodies inside one level-20 cell (ragged sort tiles)
    pos, _, m = ics.nested(20001, 5, 3000)
    _, t, rep = _deep_parity(cuda_lib, pos, m, 0.5, 1e-7, D)
    print(f"nested D={D}:", rep, "deepest", int(t.level.max()))
    assert t.level.max() > 20


def test_crowded_level20_leaf_small_buffers(cuda_lib):
    # with 20-level keys most of the 3000-body cluster is one level-20 leaf
    # (2,839 bodies): every group near it opens that leaf, whose bodies pass
    # through a 128-entry particle buffer in parts (no list length limit)
    pos, _, m = ics.nested(20001, 5, 3000)
    tc, t, rep = _deep_parity(cuda_lib, pos, m, 0.5, 1e-7, 20, list_buffer=128)
    leaf = t.is_leaf == 1
    assert (t.pend[leaf] - t.pbeg[leaf]).max() > 2000  # one crowded level-20 leaf
    assert tc.group_stats()["np"].max() > 2000


def test_deep_keys_equal_20_levels_when_uncrowded(cuda_lib):
    # no level-20 cell holds more than N_leaf bodies: the same tree and moments
    # bit for bit; the walks differ in rounding (30-level keys round each
    # offset once, and also read the low part of each cell position in the
    # opening test), so both are held to the oracle's forces
    pos, _, m = ics.plummer(16384, 1)
    acc_o, pot_o, t, st_o = oracle.tree_forces(pos, m, 0.5, 0.01, 16, 64)
    out = []
    for D in (20, 30):
        tc, acc, pot = _run(cuda_lib, pos, m, 0.5, 0.01, 16, 64, key_levels=D)
        out.append((tc.tree(), tc.moments()))
        P.compare_forces(acc, pot, acc_o, pot_o, t, st_o, tc.group_stats())
    (ta, ma), (tb, mb) = out
    for k in ("skey", "perm", "level", "pbeg", "pend", "parent", "first_child", "n_children", "is_leaf", "gbeg",
              "gend"):
        assert np.array_equal(ta[k], tb[k]), k
    assert ta["level"].max() < 20 and tb["skey_lo"].any()  # low words exist but split no cell
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k


def test_deep_keys_forest(cuda_lib):
    # deep and shallow systems, an empty one; 4 + 8 + 1 = 13 digit passes (odd)
    pa, _, ma = ics.nested(7000, 1, 1500)
    pb, _, mb = ics.plummer(5000, 2)
    pos = np.concatenate([pa, pb, pa[:900] * 3.0])
    m = np.concatenate([ma, mb, ma[:900]])
    off = np.array([0, 7000, 7000, 12000, 12900])
    _, t, rep = _deep_parity(cuda_lib, pos, m, 0.5, 1e-7, 30, offsets=off)
    print("deep forest:", rep)
    assert t.level.max() > 20


def test_deep_keys_edge_cases(cuda_lib):
    rng = np.random.default_rng(3)
    # coincident bodies: a chain of single children down to level 30, one leaf cut into groups
    pos = np.zeros((300, 3)) + 0.25
    _, t, _ = _deep_parity(cuda_lib, pos, np.full(300, 1 / 300), 0.5, 0.01, 30, n_leaf=16, n_crit=32)
    assert t.level.tolist() == list(range(31)) and t.G == 10
    # a far outlier and a cluster of 1e-6: deep single-child chains
    p = rng.uniform(size=(5000, 3)) * 1e-6
    p[0] = [1e3, -1e3, 1e3]
    _, t, _ = _deep_parity(cuda_lib, p, np.full(5000, 2e-4), 0.5, 1e-9, 30, n_leaf=4, n_crit=16)
    assert t.level.max() > 25
    # one body
    _deep_parity(cuda_lib, np.array([[1.0, 2.0, 3.0]]), np.array([1.0]), 0.5, 0.01, 30)


@pytest.mark.parametrize("theta,split", [(0.5, 0), (0.75, 1)])
def test_deep_keys_min_distance_mac(cuda_lib, theta, split):
    pos, _, m = ics.nested(12000, 7, 2000)
    _deep_parity(cuda_lib, pos, m, theta, 1e-7, 30, mac=1, walk_split=split)


def test_deep_keys_steps_graph_equals_eager(cuda_lib):
    import torch

    pos, vel, m = ics.nested(9000, 11, 1500)
    res = []
    for graph in (False, True):
        tc = cuda_lib.TreeCode(len(pos), n_leaf=8, n_crit=64, key_levels=30)
        tc.set_state(_dev(pos), _dev(vel), _dev(m))
        for _ in range(3):
            tc.step(2.0 ** -32, 0.5, 1e-7, graph=graph)  # below the cluster's crossing time
        tc.check()
        x = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
        v = torch.empty_like(x)
        a = torch.empty((len(pos), 3), dtype=torch.float32, device="cuda")
        tc.get_state(x, v, a)
        res.append((x.cpu().numpy(), v.cpu().numpy()))
        assert tc.counts()["deepest"] > 20
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_deep_keys_refreshed_moments(cuda_lib):
    # a block step on the unchanged tree refreshes the moments of cells below level 20 too
    pos, vel, m = ics.nested(8000, 13, 1200)
    dt = 2.0 ** -32
    tc = cuda_lib.TreeCode(len(pos), n_leaf=8, n_crit=64, key_levels=30)
    tc.set_state(_dev(pos), _dev(vel), _dev(m))
    tc.block_start(dt, 0, 1.0, 0.5, 1e-7)
    tc.block_step(0.5, 1e-7, rebuild=False)
    tc.check()
    st = oracle.block_start(oracle.BlockState(pos, vel, m, dt, 0, 1.0, n_leaf=8, n_crit=64, levels=30), 0.5, 1e-7)
    assert st.tree.level.max() > 20
    xp = st.x + st.v * dt + 0.5 * st.a * dt * dt
    r = oracle.refresh_tree(st.tree, xp[st.tree.perm])
    mom = tc.moments()
    l = r.size
    assert np.allclose(mom["mass"], r.M, rtol=2e-6, atol=0)
    assert (np.abs(mom["com"] - r.com).max(axis=1) / l).max() < 2e-5
    assert np.allclose(mom["size"], l, rtol=2e-5, atol=0)


def test_deep_keys_1m_nested_sampled(cuda_lib):
    """A 2^20-body Plummer sphere holding a 65,536-body cluster shrunk by 10^6
    (one level-20 cell would hold all of it): every table bit-exact, every
    200th group's forces against the oracle."""
    pos, _, m = ics.nested(1 << 20, 2, 1 << 16)
    D, n_leaf, n_crit = 30, 16, 96
    tc, acc, pot = _run(cuda_lib, pos, m, 0.5, 1e-7, n_leaf, n_crit, key_levels=D)
    t = oracle.build_tree(pos, m, n_leaf, n_crit, levels=D)
    tr = tc.tree()
    P.compare_tree(tr, t)
    assert np.array_equal(tr["skey_lo"], t.skey_lo)
    assert t.level.max() > 20
    groups = np.arange(0, t.G, 200)
    acc_s, pot_s, st = oracle.walk(t, 0.5, 1e-7, groups)
    gst = tc.group_stats()
    sub = {k: v[groups] for k, v in gst.items()}
    same = (sub["nc"] == st["nc"]) & (sub["np"] == st["np"]) & (sub["csum"] == st["csum"]) & (
        sub["psum"] == st["psum"])
    assert np.all(st["margin"][~same] < P.MARGIN)
    bodies = np.concatenate([np.arange(t.gbeg[g], t.gend[g]) for g in groups[same]])
    inp = t.perm[bodies]
    an = np.linalg.norm(acc_s[bodies], axis=1)
    scale = np.maximum(an, P.KAPPA * st["amag"][bodies])
    rel = np.linalg.norm(acc[inp] - acc_s[bodies], axis=1) / scale
    prel = np.abs(pot[inp] - pot_s[bodies]) / np.abs(pot_s[bodies])
    assert rel.max() <= P.TOL and prel.max() <= P.TOL


@pytest.mark.parametrize("D", [19, 31])
def test_key_levels_out_of_range(cuda_lib, D):
    with pytest.raises(Exception):
        cuda_lib.TreeCode(100, key_levels=D)
