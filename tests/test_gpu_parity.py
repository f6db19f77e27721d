"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Integer work (keys, sort permutation, cells, links, groups) is compared bit
for bit; moments and forces within the tolerances of tests/_parity.py.
Inputs are seeded and synthetic, sized so the oracle finishes in seconds
while spanning several sort tiles and ragged tails.
"""
import numpy as np
import pytest

import ics
import oracle
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _run(bh, pos, mass, theta, eps, n_leaf=16, n_crit=64, offsets=None, **kw):
    import torch

    n = len(pos)
    nsys = 1 if offsets is None else len(offsets) - 1
    tc = bh.TreeCode(max(n, 1), max(nsys, 1), n_leaf=n_leaf, n_crit=n_crit, **kw)
    p, m = _dev(pos), _dev(mass)
    tc.build(p, m, offsets=offsets)
    acc = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    tc.compute_forces(theta, eps, acc, pot)
    tc.check()
    return tc, acc.cpu().numpy(), pot.cpu().numpy()


def _full_parity(bh, pos, mass, theta, eps, n_leaf=16, n_crit=64, offsets=None, **kw):
    tc, acc, pot = _run(bh, pos, mass, theta, eps, n_leaf, n_crit, offsets, **kw)
    acc_o, pot_o, t, st_o = oracle.tree_forces(pos, mass, theta, eps, n_leaf, n_crit, offsets, mac=kw.get("mac", 0))
    P.compare_tree(tc.tree(), t)
    if t.C:
        P.compare_moments(tc.moments(), t)
    rep = P.compare_forces(acc, pot, acc_o, pot_o, t, st_o, tc.group_stats())
    return tc, t, rep


# ------------------------------------------------------------- App. A scan
def test_scan_worked_example(cuda_lib):
    import torch

    import os

    g = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "scan_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split(None, 1)
                g[k] = [int(w) for w in v.split()]
    tc = cuda_lib.TreeCode(1 << 16)
    x = torch.tensor(g["input"], dtype=torch.int32, device="cuda")
    ex, total = tc.exclusive_scan(x)
    inclusive = (ex + x).cpu().numpy().tolist()
    assert inclusive == g["output"]
    assert total == g["output"][-1]


@pytest.mark.parametrize("n", [1, 4095, 4096, 4097, 60001])
def test_scan_random(cuda_lib, n):
    import torch

    tc = cuda_lib.TreeCode(1 << 16)
    x = np.random.default_rng(n).integers(0, 50, n).astype(np.int32)
    ex, total = tc.exclusive_scan(torch.from_numpy(x).cuda())
    want = np.concatenate([[0], np.cumsum(x)[:-1]])
    assert np.array_equal(ex.cpu().numpy(), want) and total == int(x.sum())


# ----------------------------------------------------------- plain systems
def test_plummer_16k_parity(cuda_lib):
    pos, _, m = ics.plummer(16384, 1)
    _, t, rep = _full_parity(cuda_lib, pos, m, 0.5, 0.01)
    print("plummer 16384:", rep)
    assert rep["flipped_groups"] <= max(2, t.G // 100)


@pytest.mark.parametrize("theta", [0.3, 0.75])
def test_plummer_ragged_theta(cuda_lib, theta):
    pos, _, m = ics.plummer(10007, 17)
    _full_parity(cuda_lib, pos, m, theta, 0.005)


def test_eps_zero(cuda_lib):
    pos, _, m = ics.plummer(5000, 3)
    _full_parity(cuda_lib, pos, m, 0.5, 0.0)


@pytest.mark.parametrize("n_leaf,n_crit", [(1, 1), (4, 8), (8, 32), (16, 16), (32, 64), (64, 64), (16, 96),
                                           (16, 128), (8, 256)])
def test_parameters(cuda_lib, n_leaf, n_crit):
    pos, _, m = ics.plummer(3000, 9)
    _full_parity(cuda_lib, pos, m, 0.6, 0.01, n_leaf=n_leaf, n_crit=n_crit)


def test_theta_zero_is_direct(cuda_lib):
    pos, _, m = ics.plummer(2000, 12)
    _, acc, pot = _run(cuda_lib, pos, m, 0.0, 0.01, n_leaf=8, n_crit=32)
    ad, pd = oracle.direct(pos, m, 0.01)
    err = np.linalg.norm(acc - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert err.max() < 1e-5
    assert np.max(np.abs(pot - pd) / np.abs(pd)) < 1e-5


def test_edge_cases(cuda_lib):
    rng = np.random.default_rng(4)
    cases = [
        np.array([[1.0, 2.0, 3.0]]),
        np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]]),
        rng.uniform(size=(17, 3)),
        rng.uniform(size=(16, 3)),  # root is a leaf
        np.concatenate([rng.uniform(size=(60, 3)), np.zeros((30, 3)) + 0.5]),  # coincident bodies
        np.concatenate([rng.uniform(size=(200, 3)) * 1e-3, [[1e3, 1e3, 1e3]]]),  # one far away
        rng.uniform(size=(300, 3)) * np.array([1e-7, 1.0, 1.0]),  # flat
        np.zeros((100, 3)) + 0.25,  # all coincident: depth-20 leaf, chunked groups
    ]
    for pos in cases:
        m = rng.uniform(0.5, 1.5, len(pos)) / len(pos)
        _full_parity(cuda_lib, pos, m, 0.5, 0.01, n_leaf=16, n_crit=32)


@pytest.mark.parametrize("eps", [1e-4, 0.01])
def test_close_pair_far_from_group_centre(cuda_lib, eps):
    # a sparse group: its centre is the first body, 30 units away from a pair
    # 1e-3 apart; the pair's force must keep FP32 relative accuracy
    rng = np.random.default_rng(8)
    pos = np.array([[0.0, 0.0, 0.0], [30.0, 0.2, -0.1], [30.001, 0.2003, -0.1004]])
    pos = np.concatenate([pos, rng.uniform(-30, 30, size=(5, 3))])
    m = rng.uniform(0.5, 1.5, len(pos))
    _full_parity(cuda_lib, pos, m, 0.5, eps, n_leaf=16, n_crit=16)


def test_nonfinite_input_is_reported(cuda_lib):
    import torch

    pos, _, m = ics.plummer(1000, 2)
    pos[17, 1] = np.nan
    tc = cuda_lib.TreeCode(1000)
    tc.build(_dev(pos), _dev(m))
    assert tc.status() == 3  # BH_ERR_NONFINITE
    pos[17, 1] = 0.0
    tc.build(_dev(pos), _dev(m))
    acc = torch.empty((1000, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty(1000, dtype=torch.float32, device="cuda")
    tc.compute_forces(0.5, 0.01, acc, pot)
    assert tc.status() == 0


def test_stack_overflow_is_reported(cuda_lib):
    import torch

    pos, _, m = ics.plummer(4000, 5)
    tc = cuda_lib.TreeCode(4000, stack_capacity=64)
    tc.build(_dev(pos), _dev(m))
    acc = torch.empty((4000, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty(4000, dtype=torch.float32, device="cuda")
    tc.compute_forces(0.0, 0.01, acc, pot)  # theta = 0 opens everything: a wide frontier
    assert tc.status() == 2  # BH_ERR_CAPACITY
    assert tc.status() == 0  # the status word was cleared


def test_list_pool_above_its_address_range_is_refused(cuda_lib):
    # the split walk addresses its list pool with 32-bit multiples of 4
    # entries: a pool above 2^34 entries is refused before anything is bound
    p = cuda_lib.default_params(walk_split=1, pool_per_body=4096)
    with pytest.raises(cuda_lib.BHError) as e:
        cuda_lib.workspace_bytes(p, 1 << 23)
    assert e.value.code == 2  # BH_ERR_CAPACITY
    cuda_lib.workspace_bytes(cuda_lib.default_params(walk_split=1, pool_per_body=2048), 1 << 23)


def test_bounded_wait_gives_up(cuda_lib):
    # a look-back wait on tiles that nothing publishes gives up, latches the
    # timeout and leaves the context usable
    import torch

    pos, _, m = ics.plummer(4000, 6)
    tc = cuda_lib.TreeCode(4000)
    tc.wait_probe(1000)
    assert tc.status() == 4  # BH_ERR_TIMEOUT
    assert tc.status() == 0  # the status word was cleared
    tc.build(_dev(pos), _dev(m))
    acc = torch.empty((4000, 3), dtype=torch.float32, device="cuda")
    pot = torch.empty(4000, dtype=torch.float32, device="cuda")
    tc.compute_forces(0.5, 0.01, acc, pot)
    tc.check()
    acc_o, _, _, _ = oracle.tree_forces(pos, m, 0.5, 0.01)
    assert np.allclose(acc.cpu().numpy(), acc_o, rtol=1e-3, atol=1e-3 * np.abs(acc_o).max())
    with pytest.raises(Exception):
        tc.wait_probe(0)


# ----------------------------------------------------------------- forest
def test_forest_parity(cuda_lib):
    pos, _, m, off = ics.ensemble(n_sys=40, seed=9, n_min=1, n_max=3000)
    tc, t, _ = _full_parity(cuda_lib, pos, m, 0.5, 0.01, offsets=off)
    # each system alone gives the same tables and forces (the forest shares nothing across systems)
    for s in [0, 7, 39]:
        b, e = off[s], off[s + 1]
        ts, acc_s, pot_s = _run(cuda_lib, pos[b:e], m[b:e], 0.5, 0.01)
        assert np.array_equal(ts.tree()["perm"], tc.tree()["perm"][b:e] - b)


def test_forest_with_empty_systems(cuda_lib):
    pos, _, m = ics.plummer(500, 4)
    off = np.array([0, 0, 130, 130, 131, 500, 500])
    _full_parity(cuda_lib, pos, m, 0.5, 0.01, offsets=off)


# ---------------------------------------------------------------- host e2e
def test_forces_host_equals_device(cuda_lib):
    import torch

    pos, _, m = ics.plummer(8192, 6)
    tc, acc, pot = _run(cuda_lib, pos, m, 0.5, 0.01)
    hp = torch.from_numpy(pos).pin_memory()
    hm = torch.from_numpy(m).pin_memory()
    ha = torch.empty((8192, 3), dtype=torch.float32).pin_memory()
    hq = torch.empty(8192, dtype=torch.float32).pin_memory()
    tc.forces_host(hp, hm, 0.5, 0.01, ha, hq)
    assert np.array_equal(ha.numpy(), acc) and np.array_equal(hq.numpy(), pot)


# ---------------------------------------------------------------- leapfrog
def _state_run(bh, pos, vel, m, steps, dt, theta, eps, graph=False, offsets=None):
    import torch

    n = len(pos)
    tc = bh.TreeCode(n, 1 if offsets is None else len(offsets) - 1)
    tc.set_state(_dev(pos), _dev(vel), _dev(m), offsets=offsets)
    for _ in range(steps):
        tc.step(dt, theta, eps, graph=graph)
    x = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    a = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    p = torch.empty(n, dtype=torch.float32, device="cuda")
    tc.get_state(x, v, a, p)
    tc.check()
    return tc, x.cpu().numpy(), v.cpu().numpy(), a.cpu().numpy(), p.cpu().numpy()


def test_leapfrog_matches_oracle_steps(cuda_lib):
    pos, vel, m = ics.plummer(3000, 31)
    dt, theta, eps, steps = 1 / 64, 0.5, 0.01, 5
    _, x, v, a, p = _state_run(cuda_lib, pos, vel, m, steps, dt, theta, eps)
    # oracle: same predictor-corrector with its own FP64 tree forces
    accel = lambda xx: oracle.tree_forces(xx, m, theta, eps)[:2]
    ao, _ = accel(pos)
    xo, vo = pos.copy(), vel.copy()
    for _ in range(steps):
        xo, vo, ao, po = oracle.leapfrog_step(xo, vo, ao, dt, accel)
    assert np.max(np.abs(x - xo)) < 1e-8
    assert np.max(np.abs(v - vo)) < 1e-6
    assert np.max(np.linalg.norm(a - ao, axis=1) / np.linalg.norm(ao, axis=1)) < 1e-3


def test_two_body_orbit_energy(cuda_lib):
    m = np.array([0.25, 0.75])
    pos = np.array([[-0.75, 0, 0], [0.25, 0, 0]])
    vel = np.array([[0, -0.75, 0], [0, 0.25, 0]])
    steps = 1000
    tc, x, v, a, p = _state_run(cuda_lib, pos, vel, m, steps, 2 * np.pi / steps, 0.5, 0.0)
    d = tc.diagnostics()
    e0 = -m[0] * m[1] / 2.0
    assert abs((d["ekin"] + d["epot"]) / e0 - 1) < 1e-5
    assert np.max(np.abs(x - pos)) < 1e-3


def test_diagnostics_match_oracle(cuda_lib):
    """Energies and momentum (§4.2.2, Eq. 3) of a 16K Plummer state after one
    step, against the oracle's energy and momentum of the same positions and
    velocities with the oracle tree's potentials (same N_leaf, N_crit)."""
    pos, vel, m = ics.plummer(16384, 34)
    m = m * np.random.default_rng(34).uniform(0.5, 1.5, len(m))
    tc, x, v, a, p = _state_run(cuda_lib, pos, vel, m, 1, 1 / 64, 0.5, 0.01)
    d = tc.diagnostics()
    _, pot_o, _, _ = oracle.tree_forces(x, m, 0.5, 0.01)
    ek, ep, _ = oracle.energy(v, m, pot_o)
    mom = oracle.momentum(v, m)
    assert abs(d["ekin"] - ek) <= 1e-6 * abs(ek)
    assert abs(d["epot"] - ep) <= 1e-5 * abs(ep)
    scale = float(np.sum(m * np.linalg.norm(v, axis=1)))
    assert np.linalg.norm(np.array(d["mom"]) - mom) <= 1e-6 * scale
    # the kinetic energy and momentum are FP64 sums of the state: much closer
    assert abs(d["ekin"] - ek) <= 1e-12 * abs(ek)
    assert np.linalg.norm(np.array(d["mom"]) - mom) <= 1e-12 * scale


def test_graph_step_equals_eager(cuda_lib):
    pos, vel, m = ics.plummer(20000, 32)
    _, x1, v1, a1, _ = _state_run(cuda_lib, pos, vel, m, 4, 1 / 64, 0.5, 0.01, graph=False)
    _, x2, v2, a2, _ = _state_run(cuda_lib, pos, vel, m, 4, 1 / 64, 0.5, 0.01, graph=True)
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2) and np.array_equal(a1, a2)


def test_checkpoint_resume_is_bit_identical(cuda_lib):
    # 6 steps in one run == 3 steps, state copied out, loaded into a new
    # context, 3 more steps (the tree is rebuilt from positions every step)
    import torch

    pos, vel, m = ics.plummer(20000, 33)
    _, x6, v6, a6, _ = _state_run(cuda_lib, pos, vel, m, 6, 1 / 64, 0.5, 0.01)
    _, x3, v3, _, _ = _state_run(cuda_lib, pos, vel, m, 3, 1 / 64, 0.5, 0.01)
    _, xr, vr, ar, _ = _state_run(cuda_lib, x3, v3, m, 3, 1 / 64, 0.5, 0.01)
    assert np.array_equal(x6, xr) and np.array_equal(v6, vr) and np.array_equal(a6, ar)


@pytest.mark.parametrize("variant,n_crit", [(0, 64), (0, 96), (1, 64)])
def test_fused_walk_equals_split_walk(cuda_lib, variant, n_crit):
    """The fused walk (walk and evaluation in one kernel, lists in the warp's
    scratch) and the split walk (lists through the pool) build the same lists
    in the same order and evaluate them with the same code: identical bits."""
    import torch

    pos, _, m = ics.plummer(16384, 1)
    P, M = torch.from_numpy(pos).cuda(), torch.from_numpy(m).cuda()
    out = []
    for split in (0, 1):
        # a list buffer longer than every list: the fused walk evaluates each list once, at its end
        tc = cuda_lib.TreeCode(len(pos), walk_split=split, walk_variant=variant, n_crit=n_crit, list_buffer=16384)
        tc.build(P, M)
        acc, pot = tc.compute_forces(0.5, 0.01)
        tc.check()
        out.append((acc.cpu().numpy(), pot.cpu().numpy(), tc.group_stats(), tc.counts()))
    (a0, p0, g0, c0), (a1, p1, g1, c1) = out
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
    for k in ("nc", "np", "csum", "psum"):
        assert np.array_equal(g0[k], g1[k])
    assert (c0["pp"], c0["pc"]) == (c1["pp"], c1["pc"])


@pytest.mark.parametrize("n_leaf,n_crit,theta", [(8, 64, 0.5), (8, 128, 0.5), (16, 256, 0.3), (4, 40, 0.75)])
def test_small_list_buffers(cuda_lib, n_leaf, n_crit, theta):
    """§2.2, Fig. 3: the fused walk evaluates a list buffer whenever it fills
    and the rest at the end.  With 128-entry buffers every long list is
    evaluated in many parts (one-pass groups keep their sums in shared
    memory between parts, several-pass groups per body in the workspace):
    the results meet the same tolerance against the oracle."""
    pos, _, m = ics.plummer(16384, 1)
    tc, t, rep = _full_parity(cuda_lib, pos, m, theta, 0.01, n_leaf, n_crit, list_buffer=128)
    st = tc.group_stats()
    assert st["nc"].max() > 8 * 128 and st["np"].max() > 2 * 128  # lists many buffers long


def test_small_list_buffers_forest_and_split(cuda_lib):
    pos, _, m, off = ics.ensemble(n_sys=30, seed=19, n_min=1, n_max=4000)
    _full_parity(cuda_lib, pos, m, 0.4, 0.01, offsets=off, list_buffer=192)
    # 1024-entry buffers against whole lists (split walk): same lists, equal within the tolerance
    pos, _, m = ics.plummer(30000, 4)
    tc, acc, pot = _run(cuda_lib, pos, m, 0.3, 0.005, 8, 128, list_buffer=1024)
    tc2, acc2, pot2 = _run(cuda_lib, pos, m, 0.3, 0.005, 8, 128, walk_split=1)
    g, g2 = tc.group_stats(), tc2.group_stats()
    for k in ("nc", "np", "csum", "psum"):
        assert np.array_equal(g[k], g2[k])
    assert g["nc"].max() > 1024  # the buffers were evaluated in parts
    scale = np.linalg.norm(acc2, axis=1)
    assert np.max(np.linalg.norm(acc - acc2, axis=1) / scale) < 2e-6


@pytest.mark.parametrize("theta,split", [(0.5, 0), (0.75, 0), (0.5, 1)])
def test_min_distance_mac_parity(cuda_lib, theta, split):
    """§2.3's minimal-distance criterion against the oracle's: same lists
    (up to near-tie flips), same forces within the tolerance."""
    pos, _, m = ics.plummer(16384, 1)
    _full_parity(cuda_lib, pos, m, theta, 0.01, mac=1, walk_split=split)


def test_min_distance_mac_forest(cuda_lib):
    pos, _, m, off = ics.ensemble(12, 3, n_min=200, n_max=3000)
    _full_parity(cuda_lib, pos, m, 0.6, 0.01, offsets=off, mac=1)


def test_step_in_parts_two_ranks_equal_one_step(cuda_lib):
    """One system's groups shared out among two "ranks" (two contexts on one
    GPU, run one after the other): each builds the same tree, walks its own
    group range, the walked bodies' forces are exchanged and both correct
    every body.  Four steps (the initial evaluation and three leapfrog
    steps, the split balanced by the previous step's counts) equal the
    one-context leapfrog bit for bit, on both ranks."""
    import torch

    from paper_1106_1900_gb300 import shard

    pos, vel, m = ics.plummer(30000, 41)
    n, theta, eps, dt = len(pos), 0.5, 0.01, 1 / 64
    kw = dict(n_leaf=8, n_crit=64, list_buffer=1024)
    ref = cuda_lib.TreeCode(n, **kw)
    ref.set_state(_dev(pos), _dev(vel), _dev(m))
    for _ in range(3):
        ref.step(dt, theta, eps)
    ranks = []
    for _ in range(2):
        tc = cuda_lib.TreeCode(n, **kw)
        tc.set_state(_dev(pos), _dev(vel), _dev(m))
        ranks.append(tc)
    prev = None
    for k in range(4):
        init, h = k == 0, (0.0 if k == 0 else dt)
        for tc in ranks:
            tc.step_begin(h, init=init)
        gbeg = ranks[0].group_begins()
        assert np.array_equal(gbeg, ranks[1].group_begins())
        ranges = shard.split_groups(shard.group_costs(gbeg, prev), 2)
        assert ranges[0][1] > 0 and ranges[1][0] < len(gbeg) - 1  # both ranks walk
        for r, tc in enumerate(ranks):
            tc.walk_groups(theta, eps, *ranges[r])
        f = [tc.sorted_forces() for tc in ranks]
        (a0, a1), (b0, b1) = ((int(gbeg[g0]), int(gbeg[g1])) for g0, g1 in ranges)
        f[0][b0:b1] = f[1][b0:b1]
        f[1][a0:a1] = f[0][a0:a1]
        st = [tc.group_stats() for tc in ranks]
        npp = np.concatenate([st[0]["np"][:ranges[0][1]], st[1]["np"][ranges[1][0]:]])
        npc = np.concatenate([st[0]["nc"][:ranges[0][1]], st[1]["nc"][ranges[1][0]:]])
        prev = shard.body_costs(gbeg, npc, npp)
        for tc in ranks:
            tc.step_end(h, init=init)
    want = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    ref.get_state(*want)
    for tc in ranks:
        tc.check()
        got = [torch.empty((n, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
        tc.get_state(*got)
        assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])


def test_step_in_parts_order_is_checked(cuda_lib):
    pos, vel, m = ics.plummer(2000, 42)
    tc = cuda_lib.TreeCode(2000)
    tc.set_state(_dev(pos), _dev(vel), _dev(m))
    with pytest.raises(cuda_lib.BHError) as e:
        tc.walk_groups(0.5, 0.01, 0, 10)  # no step begun
    assert e.value.code == 6
    with pytest.raises(cuda_lib.BHError):
        tc.step_begin(1 / 64, init=False)  # the initial evaluation first
    tc.step_begin(0.0, init=True)
    with pytest.raises(cuda_lib.BHError):
        tc.step_end(0.0, init=False)  # begun as the initial evaluation
    tc.walk_groups(0.5, 0.01, 0, 1 << 30)  # every group (the end is clamped)
    tc.step_end(0.0, init=True)
    tc.check()


def test_forest_step_equals_systems(cuda_lib):
    pos, vel, m, off = ics.ensemble(n_sys=6, seed=7, n_min=500, n_max=4000)
    _, xf, vf, _, _ = _state_run(cuda_lib, pos, vel, m, 3, 1 / 64, 0.5, 0.01, offsets=off)
    for s in range(6):
        b, e = off[s], off[s + 1]
        _, xs, vs, _, _ = _state_run(cuda_lib, pos[b:e], vel[b:e], m[b:e], 3, 1 / 64, 0.5, 0.01)
        assert np.allclose(xf[b:e], xs, rtol=0, atol=1e-12)
        assert np.allclose(vf[b:e], vs, rtol=0, atol=1e-9)


# --------------------------------------------- full-size workloads
def _workload_parity(bh, pos, m, theta, eps, kind, every=1, offsets=None, **kw):
    """The benchmark's launch configuration (autotuned N_leaf, N_crit of the
    workload class): integer tables bit-exact, moments of every cell, and the
    forces of every `every`-th group (all of them by default) against the
    oracle walking the same groups."""
    from paper_1106_1900_gb300 import autotune

    tp = autotune.tuned_params(len(pos), theta, kind) or {"n_leaf": 16, "n_crit": 64}
    tc, acc, pot = _run(bh, pos, m, theta, eps, offsets=offsets, **tp, **kw)
    t = oracle.build_tree(pos, m, tp["n_leaf"], tp["n_crit"], offsets=offsets)
    P.compare_tree(tc.tree(), t)
    P.compare_moments(tc.moments(), t)
    groups = np.arange(0, t.G, every)
    acc_s, pot_s, st = oracle.walk(t, theta, eps, groups)
    gst = tc.group_stats()
    rep = P.group_forces_report(acc, pot, t, groups, acc_s, pot_s, st, {k: v[groups] for k, v in gst.items()})
    print(kind, tp, rep)
    return t, rep


def test_plummer_1m_all_groups(cuda_lib):
    """The benchmark's workload: 2^20-body Plummer sphere, theta = 0.5, eps =
    0.005, every body compared."""
    pos, _, m = ics.plummer(1 << 20, 2)
    t, rep = _workload_parity(cuda_lib, pos, m, 0.5, 0.005, "plummer")
    assert rep["bodies"] == 1 << 20


def test_galaxy_8m(cuda_lib):
    """Hernquist sphere + exponential disk, 8,388,608 bodies: a sparse, very
    non-uniform tree; every body compared."""
    pos, _, m = ics.galaxy(4194304, 4194304, 3)
    t, rep = _workload_parity(cuda_lib, pos, m, 0.5, 0.01, "galaxy")
    assert np.bincount(t.level).size > 12  # a deep tree
    assert rep["bodies"] == len(pos)


def test_ensemble_7m(cuda_lib):
    """512 Plummer clusters of 1,024..65,536 bodies, ~7.7M bodies in one
    forest; every body compared."""
    pos, _, m, off = ics.ensemble(512, 5)
    t, rep = _workload_parity(cuda_lib, pos, m, 0.5, 0.01, "ensemble", offsets=off)
    assert t.sys_root.min() >= 0
    assert rep["bodies"] == len(pos)


# ------------------------------------------------------- direct summation
@pytest.mark.parametrize("eps", [0.0, 0.01])
def test_direct_forces_match_oracle(cuda_lib, eps):
    import torch

    pos, _, m = ics.plummer(3000, 21)
    tg = ics.subsample(3000, 700, 40).astype(np.int32)
    acc, pot = cuda_lib.direct_forces(_dev(pos), _dev(m), torch.from_numpy(tg).cuda(), eps)
    ad, pd = oracle.direct(pos, m, eps, targets=tg)
    # magnitude of the terms, for bodies whose force nearly cancels
    d = pos[None, :, :] - pos[tg][:, None, :]
    r2 = (d * d).sum(-1) + eps * eps
    r2[np.arange(len(tg)), tg] = np.inf
    amag = (m[None, :] / r2).sum(1)
    scale = np.maximum(np.linalg.norm(ad, axis=1), P.KAPPA * amag)
    assert np.max(np.linalg.norm(acc.cpu().numpy() - ad, axis=1) / scale) <= P.TOL
    assert np.max(np.abs(pot.cpu().numpy() - pd) / np.abs(pd)) <= P.TOL


def test_autotune_keeps_error_and_picks_fastest(cuda_lib):
    import torch

    from paper_1106_1900_gb300 import autotune

    pos, vel, m = ics.plummer(30000, 3)
    P_, V_, M_ = (torch.from_numpy(a).cuda() for a in (pos, vel, m))
    best, trials = autotune.autotune(P_, V_, M_, 0.5, 0.01, grid=[(8, 16), (16, 32)], steps=2, subsample=1024,
                                     walk_grid=[(1024, 6), (4096, 5)])
    paper = next(r for r in trials if (r["n_leaf"], r["n_crit"]) == autotune.PAPER_PAIR)
    assert best["p99"] <= paper["p99"] * 1.05
    assert best["ms_per_step"] == min(r["ms_per_step"] for r in trials if r["p99"] <= paper["p99"] * 1.05)
    assert 1e-6 < paper["p50"] < 1e-3  # a quadrupole tree at theta = 0.5
    # the walk stage keeps the chosen pair and tries the buffer and warp settings
    walk = [r for r in trials if r.get("stage") == "walk"]
    assert len(walk) == 2 and all("list_buffer" in r for r in walk)


def test_autotune_forest_reference_is_per_system(cuda_lib):
    """The forest's error reference sums each target's own system only."""
    import torch

    from paper_1106_1900_gb300 import autotune

    pos, vel, m, off = ics.ensemble(n_sys=8, seed=12, n_min=500, n_max=3000)
    P_, M_ = torch.from_numpy(pos).cuda(), torch.from_numpy(m).cuda()
    tg = np.sort(np.random.default_rng(1).choice(len(pos), 300, replace=False)).astype(np.int32)
    ref = autotune.reference(P_, M_, 0.01, torch.from_numpy(tg).cuda(), off).cpu().numpy()
    ad, _ = oracle.direct(pos, m, 0.01, targets=tg, offsets=off)
    assert np.max(np.linalg.norm(ref - ad, axis=1) / np.linalg.norm(ad, axis=1)) < 1e-4
