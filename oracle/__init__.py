"""FP64 CPU oracle of the sparse-octree tree-code (arXiv:1106.1900).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` use this package.  It shares no code with
the CUDA library (``paper_1106_1900_gb300``) and never imports it.

The arithmetic lives in ``bh_oracle.c`` (plain C, FP64, built with gcc);
this module compiles it on first use and marshals numpy arrays.  Each
function names the passage of the paper it follows; the readings taken where
the paper is silent are listed at the top of ``bh_oracle.c``.

Parity pins (tests marked ``not gpu``) tie it to things other than itself:
the paper's worked examples (App. A scan, §2.1 mask footnote, App. B dilate),
brute-force recursive octrees on tiny inputs, numpy's stable sort, closed
forms (two-body moments, Plummer potential), theta -> 0 reproducing the
direct sum, and momentum conservation of the direct sum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bh_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LEVELS = 20  # the paper's 60-bit keys
LEVELS_MAX = 30  # 90-bit keys (App. B: the way past 20 levels)


def build(force: bool = False) -> str:
    """Compile ``bh_oracle.c`` into ``liboracle.so`` (gcc, OpenMP if available)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, i32, dbl, u32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint32, ctypes.c_void_p
            sig = {
                "or_dilate10": (u32, [u32]),
                "or_frames": (ctypes.c_int, [i64, p, i32, p, p]),
                "or_keys": (ctypes.c_int, [i64, p, i32, p, p, i32, p, p, p, p]),
                "or_sort": (ctypes.c_int, [i64, p, p, i32, p, p]),
                "or_build_levels": (i64, [i64, p, p, i32, p, i32, i64, p, p, p, p, p]),
                "or_link": (ctypes.c_int, [i64, p, p, p, p, p, i32, p, p, p]),
                "or_groups": (i64, [i64, p, p, p, p, p, p, i32, i64, p, p]),
                "or_moments": (ctypes.c_int, [i64, p, p, p, p, p, p, p, p, i32, p, p, p, p, p, p]),
                "or_walk": (ctypes.c_int, [i64, p, p, p, p, p, i64, p, p, p, p, p, p, p, p, p, p, p, i64, p,
                                           p, dbl, dbl, i32, p, p, p, p]),
                "or_direct": (ctypes.c_int, [i64, p, p, i32, p, i64, p, dbl, p, p]),
                "or_cell_exact": (ctypes.c_int, [i64, i64, p, p, p, dbl, p, p]),
                "or_cell_multipole": (ctypes.c_int, [dbl, p, p, p, dbl, p, p]),
                "or_refresh_sizes": (ctypes.c_int, [i64, p, p, p, p, p, p, p, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


def _offsets(n: int, offsets) -> np.ndarray:
    if offsets is None:
        return np.array([0, n], dtype=np.int64)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    return off


# ---------------------------------------------------------------- App. B
def dilate10(v: int) -> int:
    """App. B (Listing 1): bit b of the low 10 bits moved to bit 3b."""
    return int(_load().or_dilate10(v))


def frames(pos: np.ndarray, offsets=None) -> np.ndarray:
    """Per-system frame ``[origin_x, origin_y, origin_z, L]`` (App. B reading)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    off = _offsets(len(pos), offsets)
    fr = np.zeros((len(off) - 1, 4))
    _load().or_frames(len(pos), _p(pos), len(off) - 1, _p(off), _p(fr))
    return fr


def _check_levels(levels: int) -> int:
    levels = int(levels)
    if not LEVELS <= levels <= LEVELS_MAX:
        raise ValueError(f"key depth {levels} outside {LEVELS}..{LEVELS_MAX}")
    return levels


def keys_split(pos: np.ndarray, offsets=None, frame=None, levels: int = LEVELS):
    """Quantised coordinates ``q[N,3]`` (2^levels cells per axis), the
    3*levels-bit Morton keys as two words -- ``key_hi`` (levels 1..20, the
    top 60 bits) and ``key_lo`` (levels 21..``levels``, the low bits; 0 for
    20-level keys) -- and system ids (App. B)."""
    levels = _check_levels(levels)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    off = _offsets(len(pos), offsets)
    fr = frames(pos, off) if frame is None else np.ascontiguousarray(frame, dtype=np.float64)
    n = len(pos)
    q = np.zeros((n, 3), dtype=np.int32)
    key_hi = np.zeros(n, dtype=np.uint64)
    key_lo = np.zeros(n, dtype=np.uint64)
    sys_ = np.zeros(n, dtype=np.int32)
    _load().or_keys(n, _p(pos), len(off) - 1, _p(off), _p(fr), levels, _p(q), _p(key_hi), _p(key_lo), _p(sys_))
    return q, key_hi, key_lo, sys_


def keys(pos: np.ndarray, offsets=None, frame=None):
    """Quantised coordinates ``q[N,3]``, 60-bit Morton keys and system ids."""
    q, key, _, sys_ = keys_split(pos, offsets, frame, LEVELS)
    return q, key, sys_


def sort_perm(key: np.ndarray, sys_: np.ndarray, key_lo=None, levels: int = LEVELS) -> np.ndarray:
    """Stable order by (system, key): ``perm[i]`` = input index of the i-th body (§2.1).
    Deeper keys pass their low word as ``key_lo``."""
    levels = _check_levels(levels)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    lo = np.zeros_like(key) if key_lo is None else np.ascontiguousarray(key_lo, dtype=np.uint64)
    sys_ = np.ascontiguousarray(sys_, dtype=np.int32)
    perm = np.zeros(len(key), dtype=np.int64)
    _load().or_sort(len(key), _p(key), _p(lo), levels, _p(sys_), _p(perm))
    return perm


def cell_bound(n: int, n_leaf: int, n_sys: int = 1, levels: int = LEVELS) -> int:
    """Upper bound on the cell count: at most n/(N_leaf+1) nodes per level
    (levels 0..levels-1) and at most one leaf per body."""
    return levels * (n // (n_leaf + 1)) + n + n_sys + 1


class Tree:
    """The oracle's tree: every array is in sorted (system, key) order."""


def build_tree(pos, mass, n_leaf: int = 16, n_crit: int = 64, offsets=None, levels: int = LEVELS) -> Tree:
    """§2.1 + §2.2 + §3.2: keys, sort, level-by-level cells, link, groups,
    moments; ``levels`` is the key depth (20, or up to 30 with 90-bit keys)."""
    levels = _check_levels(levels)
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = len(pos)
    off = _offsets(n, offsets)
    nsys = len(off) - 1
    t = Tree()
    t.n, t.n_leaf, t.n_crit, t.offsets, t.levels = n, n_leaf, n_crit, off, levels
    t.frame = frames(pos, off)
    t.q, t.key, t.key_lo, t.sys = keys_split(pos, off, t.frame, levels)
    t.perm = sort_perm(t.key, t.sys, t.key_lo, levels)
    t.skey = np.ascontiguousarray(t.key[t.perm])
    t.skey_lo = np.ascontiguousarray(t.key_lo[t.perm])
    t.ssys = np.ascontiguousarray(t.sys[t.perm])
    t.spos = np.ascontiguousarray(pos[t.perm])
    t.smass = np.ascontiguousarray(mass[t.perm])
    t.sq = np.ascontiguousarray(t.q[t.perm])
    cap = cell_bound(n, n_leaf, nsys, levels)
    level = np.zeros(cap, dtype=np.int32)
    pbeg = np.zeros(cap, dtype=np.int64)
    pend = np.zeros(cap, dtype=np.int64)
    is_leaf = np.zeros(cap, dtype=np.int32)
    csys = np.zeros(cap, dtype=np.int32)
    C = lib.or_build_levels(n, _p(t.skey), _p(t.skey_lo), levels, _p(t.ssys), n_leaf, cap, _p(level), _p(pbeg),
                            _p(pend), _p(is_leaf), _p(csys))
    if C < 0:
        raise RuntimeError("oracle: cell capacity exceeded")
    t.C = int(C)
    t.level, t.pbeg, t.pend = level[:C].copy(), pbeg[:C].copy(), pend[:C].copy()
    t.is_leaf, t.csys = is_leaf[:C].copy(), csys[:C].copy()
    t.parent = np.zeros(C, dtype=np.int64)
    t.first_child = np.zeros(C, dtype=np.int64)
    t.n_children = np.zeros(C, dtype=np.int32)
    rc = lib.or_link(C, _p(t.level), _p(t.pbeg), _p(t.csys), _p(t.skey), _p(t.skey_lo), levels, _p(t.parent),
                     _p(t.first_child), _p(t.n_children))
    if rc != 0:
        raise RuntimeError("oracle: link failed")
    gb = np.zeros(n + 1, dtype=np.int64)
    ge = np.zeros(n + 1, dtype=np.int64)
    G = lib.or_groups(C, _p(t.level), _p(t.pbeg), _p(t.pend), _p(t.is_leaf), _p(t.first_child),
                      _p(t.n_children), n_crit, n + 1, _p(gb), _p(ge))
    if G < 0:
        raise RuntimeError("oracle: group capacity exceeded")
    t.G = int(G)
    t.gbeg, t.gend = gb[:G].copy(), ge[:G].copy()
    t.gsys = np.ascontiguousarray(t.ssys[t.gbeg]) if G else np.zeros(0, dtype=np.int32)
    t.sys_root = np.full(nsys, -1, dtype=np.int64)
    roots = np.nonzero(t.level == 0)[0]
    t.sys_root[t.csys[roots]] = roots
    t.M = np.zeros(C)
    t.com = np.zeros((C, 3))
    t.Q = np.zeros((C, 6))
    t.ctr = np.zeros((C, 3))
    t.size = np.zeros(C)
    t.delta = np.zeros(C)
    lib.or_moments(C, _p(t.level), _p(t.pbeg), _p(t.pend), _p(t.csys), _p(t.spos), _p(t.smass), _p(t.sq),
                   _p(t.frame), levels, _p(t.M), _p(t.com), _p(t.Q), _p(t.ctr), _p(t.size), _p(t.delta))
    return t


def walk(t: Tree, theta: float, eps: float, groups=None, mac: int = 0):
    """§2.2 + §3.3 group walk (FP64).  ``mac`` 0: Eq. 1; 1: the minimal-distance
    criterion (cell cube to group box farther than l/theta).

    Returns ``(acc, pot, stats)`` in SORTED order; ``acc``/``pot`` are only
    filled for bodies of the walked groups (NaN elsewhere).  ``stats`` is a
    structured view per walked group: cell-list length ``nc``, particle-list
    length ``np``, index sums ``csum``/``psum`` and the smallest opening
    margin ``margin``; ``stats["amag"]`` holds, per body (sorted order), the
    sum of the magnitudes of its interaction terms.
    """
    lib = _load()
    grp = np.arange(t.G, dtype=np.int64) if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
    acc = np.full((t.n, 3), np.nan)
    pot = np.full(t.n, np.nan)
    raw = np.zeros((len(grp), 5), dtype=np.int64)
    amag = np.full(t.n, np.nan)
    lib.or_walk(len(grp), _p(grp), _p(t.gbeg), _p(t.gend), _p(t.gsys), _p(t.sys_root), t.C, _p(t.is_leaf),
                _p(t.pbeg), _p(t.pend), _p(t.first_child), _p(t.n_children), _p(t.M), _p(t.com), _p(t.Q),
                _p(t.ctr), _p(t.size), _p(t.delta), t.n, _p(t.spos), _p(t.smass), float(theta), float(eps),
                int(mac), _p(acc), _p(pot), _p(raw), _p(amag))
    stats = {
        "nc": raw[:, 0].copy(),
        "np": raw[:, 1].copy(),
        "csum": raw[:, 2].view(np.uint64).copy(),
        "psum": raw[:, 3].view(np.uint64).copy(),
        "margin": raw[:, 4].copy().view(np.float64),
        "amag": amag,
    }
    return acc, pot, stats


def tree_forces(pos, mass, theta: float, eps: float, n_leaf: int = 16, n_crit: int = 64, offsets=None, mac: int = 0,
                levels: int = LEVELS):
    """Build + walk all groups; accelerations and potentials in INPUT order."""
    t = build_tree(pos, mass, n_leaf, n_crit, offsets, levels)
    acc_s, pot_s, stats = walk(t, theta, eps, mac=mac)
    acc = np.empty_like(acc_s)
    pot = np.empty_like(pot_s)
    acc[t.perm] = acc_s
    pot[t.perm] = pot_s
    amag = np.empty_like(pot_s)
    amag[t.perm] = stats["amag"]
    stats["amag_input_order"] = amag
    return acc, pot, t, stats


def direct(pos, mass, eps: float, targets=None, offsets=None):
    """FP64 direct summation over all other bodies of the same system."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = len(pos)
    off = _offsets(n, offsets)
    tg = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.zeros((len(tg), 3))
    pot = np.zeros(len(tg))
    _load().or_direct(n, _p(pos), _p(mass), len(off) - 1, _p(off), len(tg), _p(tg), float(eps), _p(acc), _p(pot))
    return acc, pot


def cell_exact(t: Tree, c: int, x, eps: float = 0.0):
    """Exact force of cell ``c``'s own bodies on point ``x``."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    a = np.zeros(3)
    p = np.zeros(1)
    _load().or_cell_exact(int(t.pbeg[c]), int(t.pend[c]), _p(t.spos), _p(t.smass), _p(x), float(eps), _p(a), _p(p))
    return a, float(p[0])


def cell_multipole(t: Tree, c: int, x, eps: float = 0.0):
    """Monopole + quadrupole approximation of cell ``c`` at point ``x``."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    a = np.zeros(3)
    p = np.zeros(1)
    com = np.ascontiguousarray(t.com[c])
    Q = np.ascontiguousarray(t.Q[c])
    _load().or_cell_multipole(float(t.M[c]), _p(com), _p(Q), _p(x), float(eps), _p(a), _p(p))
    return a, float(p[0])


# ------------------------------------------------------------ §3.1, Eq. 3
def leapfrog_step(x, v, a_old, dt: float, accel):
    """Leapfrog predictor-corrector (§3.1, after Hut et al. 1995), FP64.

    Predict ``x += v dt + a dt^2/2`` and ``v_p = v + a dt`` with the old
    acceleration, evaluate ``a_new = accel(x)``, then correct
    ``v = v_p + (a_new - a_old) dt/2``.  Returns ``(x, v, a_new, pot)``.
    """
    x = x + v * dt + 0.5 * a_old * dt * dt
    vp = v + a_old * dt
    a_new, pot = accel(x)
    v = vp + 0.5 * (a_new - a_old) * dt
    return x, v, a_new, pot


def energy(vel, mass, pot):
    """Kinetic, potential (1/2 sum m phi) and total energy; Eq. 3 uses the total."""
    ek = 0.5 * float(np.sum(mass * np.sum(vel * vel, axis=1)))
    ep = 0.5 * float(np.sum(mass * pot))
    return ek, ep, ek + ep


def momentum(vel, mass):
    return np.sum(mass[:, None] * vel, axis=0)


# ---------------------------------------------------------------- block time-steps
#
# Reading (the paper motivates block time-steps -- §1, §2.2 "active" groups,
# §4 moment refresh and rebuild on degradation -- but prints no scheme):
#   * body i steps with dt_i = dt_max 2^-k_i, k_i in [0, k_max]; times are
#     integer ticks of dt_max 2^-k_max;
#   * the level wanted by a body is the smallest k with
#     dt_max 2^-k <= eta sqrt(eps / |a|) (|a| = 0: level 0);
#   * a block step advances to T = min_i (t_i + s_i), s_i = 2^(k_max - k_i);
#     the bodies with t_i + s_i = T are active;
#   * every body is predicted to T (x + v d + a d^2/2, d = (T - t_i) ticks),
#     the tree is rebuilt at the predicted positions or refreshed on the old
#     tree (refresh_tree), the groups holding an active body are walked, and
#     the active bodies are corrected as in the shared-step leapfrog
#     (v = v + a s + (a_new - a) s/2, x = predicted);
#   * an active body then takes the wanted level if it is deeper, one level
#     shallower if the wanted level is shallower and T is a multiple of the
#     doubled step, else keeps its level.


def refresh_tree(t: Tree, spos_new) -> Tree:
    """The tree with new body positions (sorted order) and the same cells:
    moments recomputed from the bodies, each cell's geometric centre kept and
    its size grown to the smallest cube about that centre holding its bodies
    or children (never below the built size)."""
    import copy

    lib = _load()
    r = copy.copy(t)
    r.spos = np.ascontiguousarray(spos_new, dtype=np.float64)
    C = t.C
    r.M, r.com, r.Q = np.zeros(C), np.zeros((C, 3)), np.zeros((C, 6))
    r.ctr, r.size, r.delta = np.zeros((C, 3)), np.zeros(C), np.zeros(C)
    lib.or_moments(C, _p(t.level), _p(t.pbeg), _p(t.pend), _p(t.csys), _p(r.spos), _p(t.smass), _p(t.sq),
                   _p(t.frame), t.levels, _p(r.M), _p(r.com), _p(r.Q), _p(r.ctr), _p(r.size), _p(r.delta))
    lib.or_refresh_sizes(C, _p(t.is_leaf), _p(t.pbeg), _p(t.pend), _p(t.first_child), _p(t.n_children),
                         _p(r.spos), _p(r.ctr), _p(r.size))
    return r


def block_level(acc, eps: float, eta: float, dt_max: float, k_max: int):
    """Level wanted by each body: the smallest k >= 0 with
    dt_max 2^-k <= eta sqrt(eps / |a|), clamped to k_max (FP64)."""
    a = np.linalg.norm(np.asarray(acc, dtype=np.float64), axis=1)
    r = dt_max * np.sqrt(a / eps) / eta  # need 2^k >= r
    k = np.zeros(len(a), dtype=np.int64)
    big = r > 1.0
    m, e = np.frexp(r[big])  # r = m 2^e, m in [0.5, 1)
    k[big] = np.where(m == 0.5, e - 1, e)
    return np.minimum(k, k_max)


class BlockState:
    """Block time-step state, bodies in the caller's order."""

    def __init__(self, x, v, m, dt_max, k_max, eta, n_leaf=16, n_crit=64, levels=LEVELS):
        self.levels = _check_levels(levels)
        self.x = np.array(x, dtype=np.float64)
        self.v = np.array(v, dtype=np.float64)
        self.m = np.array(m, dtype=np.float64)
        self.dt_max, self.k_max, self.eta = float(dt_max), int(k_max), float(eta)
        self.n_leaf, self.n_crit = n_leaf, n_crit
        self.tick = self.dt_max / 2.0 ** self.k_max
        n = len(self.m)
        self.t = np.zeros(n, dtype=np.int64)
        self.k = np.zeros(n, dtype=np.int64)
        self.a = np.zeros((n, 3))
        self.pot = np.zeros(n)
        self.tree = None
        self.T = 0


def block_start(st: BlockState, theta: float, eps: float):
    """Forces of every body at t = 0 and their first levels."""
    a, pot, t, _ = tree_forces(st.x, st.m, theta, eps, st.n_leaf, st.n_crit, levels=st.levels)
    st.a, st.pot, st.tree = a, pot, t
    st.k = block_level(a, eps, st.eta, st.dt_max, st.k_max)
    return st


def block_step(st: BlockState, theta: float, eps: float, rebuild: bool = True, k_forced=None):
    """One block step (see the reading above).  ``k_forced`` replaces the
    levels the active bodies would take (for parity checks that must follow
    another side's decisions).  Returns the boolean mask of active bodies."""
    s = np.left_shift(np.int64(1), st.k_max - st.k)
    T = int(np.min(st.t + s))
    active = st.t + s == T
    d = ((T - st.t) * st.tick)[:, None]
    xp = st.x + st.v * d + 0.5 * st.a * d * d
    if rebuild or st.tree is None:
        tr = build_tree(xp, st.m, st.n_leaf, st.n_crit, levels=st.levels)
    else:
        tr = refresh_tree(st.tree, xp[st.tree.perm])
    st.tree = tr
    act_sorted = active[tr.perm]
    groups = np.array([g for g in range(tr.G) if act_sorted[tr.gbeg[g]:tr.gend[g]].any()], dtype=np.int64)
    acc_s, pot_s, _ = walk(tr, theta, eps, groups=groups)
    a_new = np.empty_like(acc_s)
    p_new = np.empty_like(pot_s)
    a_new[tr.perm] = acc_s
    p_new[tr.perm] = pot_s
    ds = (s * st.tick)[:, None]
    vp = st.v + st.a * ds
    v_c = vp + 0.5 * (a_new - st.a) * ds
    st.x[active] = xp[active]
    st.v[active] = v_c[active]
    st.a[active] = a_new[active]
    st.pot[active] = p_new[active]
    st.t[active] = T
    want = block_level(a_new, eps, st.eta, st.dt_max, st.k_max) if k_forced is None else np.asarray(k_forced)
    k_old = st.k.copy()
    deeper = want > k_old
    up_ok = (want < k_old) & (k_old > 0) & (T % (2 * s) == 0)
    k_new = np.where(deeper, want, np.where(up_ok, k_old - 1, k_old))
    st.k[active] = k_new[active]
    st.T = T
    return active
