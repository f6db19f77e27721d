"""Block time-steps on the GPU against the block-step oracle (needs a GB300).

Levels are integers decided from accelerations, FP32 on the GPU and FP64 in
the oracle: where the wanted-level value r = dt_max sqrt(|a|/eps)/eta lies
within 1e-4 (relative) of a power of two the two sides may decide
differently, and such bodies are left out of the comparison from then on;
every other decision must agree exactly."""
import numpy as np
import pytest

import ics
import oracle

pytestmark = pytest.mark.gpu

THETA, EPS = 0.5, 0.01


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _state(tc, n):
    import torch

    x = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty_like(x)
    a = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    tc.get_state(x, v, a)
    return x.cpu().numpy(), v.cpu().numpy(), a.cpu().numpy().astype(np.float64)


def _levels(tc):
    lv, tk = tc.block_levels()
    return lv.cpu().numpy().astype(np.int64), tk.cpu().numpy()


def _near_tie(acc, dt_max, eta):
    """Bodies whose wanted-level value sits within 1e-4 of a power of two."""
    r = dt_max * np.sqrt(np.linalg.norm(acc, axis=1) / EPS) / eta
    lg = np.log2(np.maximum(r, 1e-300))
    return np.abs(lg - np.round(lg)) < 1e-4 / np.log(2)


def test_single_level_is_the_shared_step(cuda_lib):
    """k_max = 0: three block steps (rebuilding) are three bh_step, bit for bit."""
    pos, vel, m = ics.plummer(8192, 21)
    dt = 1.0 / 64
    out = []
    for block in (False, True):
        tc = cuda_lib.TreeCode(len(pos))
        tc.set_state(_dev(pos), _dev(vel), _dev(m))
        if block:
            tc.block_start(dt, 0, 1.0, THETA, EPS)
            for _ in range(3):
                tc.block_step(THETA, EPS, rebuild=True)
            info = tc.block_info()
            assert info["tick"] == 3 and info["active"] == len(pos) and info["deepest"] == 0
        else:
            for _ in range(3):
                tc.step(dt, THETA, EPS, graph=False)
        tc.check()
        out.append(_state(tc, len(pos)))
    for u, w in zip(*out):
        assert np.array_equal(u, w)


def test_refreshed_moments_match_the_oracle(cuda_lib):
    """One block step on the unchanged tree (k_max = 0: every body moved by one
    step): moments and grown cell sizes against the oracle's refresh."""
    pos, vel, m = ics.plummer(16384, 22)
    dt = 1.0 / 32
    tc = cuda_lib.TreeCode(len(pos))
    tc.set_state(_dev(pos), _dev(vel), _dev(m))
    tc.block_start(dt, 0, 1.0, THETA, EPS)
    tc.block_step(THETA, EPS, rebuild=False)
    tc.check()
    st = oracle.block_start(oracle.BlockState(pos, vel, m, dt, 0, 1.0), THETA, EPS)
    xp = st.x + st.v * dt + 0.5 * st.a * dt * dt
    r = oracle.refresh_tree(st.tree, xp[st.tree.perm])
    mom = tc.moments()
    assert np.all(mom["size"] >= st.tree.size * (1 - 1e-7)) and np.any(r.size > st.tree.size)
    # the predicted positions differ by dt^2/2 times the FP32-vs-FP64 force
    # difference (~1e-5 |a| dt^2 / 2, ~1e-7 here), held to 2e-5 of the cell size
    l = r.size
    assert np.allclose(mom["mass"], r.M, rtol=2e-6, atol=0)
    assert (np.abs(mom["com"] - r.com).max(axis=1) / l).max() < 2e-5
    assert np.allclose(mom["size"], l, rtol=2e-5, atol=0)
    assert (np.abs(mom["delta"] - r.delta) / l).max() < 2e-5
    q_err = np.abs(mom["quad"].astype(np.float64) - r.Q).max(axis=1) / np.maximum(r.M * l * l, 1e-300)
    assert q_err.max() < 2e-4


@pytest.mark.parametrize("refresh", [False, True])
def test_block_steps_follow_the_oracle(cuda_lib, refresh):
    """Block steps with several levels: the same block times, due bodies and
    levels as the oracle, states within the FP32-force tolerance."""
    n, dt_max, k_max, eta = 6000, 1.0 / 32, 4, 0.05
    pos, vel, m = ics.plummer(n, 23)
    tc = cuda_lib.TreeCode(n)
    tc.set_state(_dev(pos), _dev(vel), _dev(m))
    tc.block_start(dt_max, k_max, eta, THETA, EPS)
    st = oracle.block_start(oracle.BlockState(pos, vel, m, dt_max, k_max, eta), THETA, EPS)
    lv, tk = _levels(tc)
    tie = _near_tie(st.a, dt_max, eta)
    ok = ~tie
    assert np.array_equal(lv[ok], st.k[ok])
    assert len(np.unique(st.k)) >= 3
    for step in range(12):
        rebuild = (not refresh) or step % 4 == 0
        tc.block_step(THETA, EPS, rebuild=rebuild)
        act = oracle.block_step(st, THETA, EPS, rebuild=rebuild)
        tc.check()
        info = tc.block_info()
        assert info["tick"] == st.T
        lv, tk = _levels(tc)
        x, v, a = _state(tc, n)
        tie |= _near_tie(st.a, dt_max, eta)
        ok = ~tie
        if ok.all():
            assert info["active"] == int(act.sum())
        assert np.array_equal(tk[ok], st.t[ok]) and np.array_equal(lv[ok], st.k[ok])
        # positions: predicted with FP32-vs-FP64 forces; velocities: kicked with them
        scale_x = np.abs(st.x[ok]).max()
        assert np.abs(x[ok] - st.x[ok]).max() < 1e-6 * scale_x
        # (FP32 forces are held to 1e-5 of max(|a|, kappa sum|a_ij|): near-cancelling
        # bodies get the median |a| as their scale)
        dv = np.linalg.norm(v[ok] - st.v[ok], axis=1)
        an = np.linalg.norm(st.a[ok], axis=1)
        assert np.all(dv <= 1e-4 * (an + np.median(an)) * dt_max * (step + 1))
    assert tie.sum() < 0.01 * n


def test_block_energy_over_synchronised_intervals(cuda_lib):
    n = 1 << 16
    pos, vel, m = ics.plummer(n, 24)
    dt_max, k_max, eta = 1.0 / 32, 5, 0.05
    tc = cuda_lib.TreeCode(n)
    tc.set_state(_dev(pos), _dev(vel), _dev(m))
    tc.block_start(dt_max, k_max, eta, 0.4, EPS)
    d0 = tc.diagnostics()
    e0 = d0["ekin"] + d0["epot"]
    sync = 2 ** k_max
    updates, steps = 0, 0
    while True:
        info_before = tc.block_info()["tick"]
        if info_before >= 8 * sync:
            break
        tc.block_step(0.4, EPS, rebuild=(info_before % sync == 0))
        info = tc.block_info()
        updates += info["active"]
        steps += 1
    tc.check()
    _, tk = _levels(tc)
    assert (tk == 8 * sync).all()
    d1 = tc.diagnostics()
    e1 = d1["ekin"] + d1["epot"]
    assert abs((e1 - e0) / e0) < 2e-4
    assert updates < n * 8 * 2 ** tc.block_info()["deepest"]
    assert max(abs(x) for x in d1["mom"]) < 1e-4


def test_block_steps_on_a_forest(cuda_lib):
    """Block time-steps of a forest: with k_max = 0 they are bh_step bit for
    bit; with several levels, each system's state matches stepping it alone."""
    pos, vel, m, off = ics.ensemble(n_sys=6, seed=7, n_min=500, n_max=3000)
    dt = 1.0 / 64

    def run(p, v, mm, offsets, block, k_max=0, steps=3):
        tc = cuda_lib.TreeCode(len(p), max(1, len(offsets) - 1) if offsets is not None else 1)
        tc.set_state(_dev(p), _dev(v), _dev(mm), offsets=offsets)
        if block:
            tc.block_start(dt, k_max, 0.05, THETA, EPS)
            while tc.block_info()["tick"] < steps * 2 ** k_max:
                tc.block_step(THETA, EPS, rebuild=True)
        else:
            for _ in range(steps):
                tc.step(dt, THETA, EPS, graph=False)
        tc.check()
        return _state(tc, len(p)), (_levels(tc) if block else None)

    (a, _), (b, _) = run(pos, vel, m, off, False), run(pos, vel, m, off, True)
    for u, w in zip(a, b):
        assert np.array_equal(u, w)
    # several levels: a forest's block steps treat each system on its own
    (xf, vf, _), (lf, tf) = run(pos, vel, m, off, True, k_max=3, steps=1)
    for s in (0, 3, 5):
        lo, hi = off[s], off[s + 1]
        (xs, vs, _), (ls, ts) = run(pos[lo:hi], vel[lo:hi], m[lo:hi], None, True, k_max=3, steps=1)
        assert np.array_equal(lf[lo:hi], ls) and np.array_equal(tf[lo:hi], ts)
        assert np.allclose(xf[lo:hi], xs, rtol=0, atol=1e-12) and np.allclose(vf[lo:hi], vs, rtol=0, atol=1e-9)
