"""Seeded synthetic initial conditions (inputs only).

This module draws particle positions, velocities and masses for the
workloads the tree-code is measured on.  It holds none of the tree-code's
arithmetic: both the CUDA library and the CPU oracle receive these arrays as
plain inputs.  All generators are deterministic functions of their seed
(``numpy.random.default_rng``) and return C-contiguous float64 arrays
``pos[N,3]``, ``vel[N,3]``, ``mass[N]`` in N-body units (G = 1).

Workloads (the paper measures Plummer spheres of 2^15..2^24 bodies, §4.1,
and a galaxy merger whose initial conditions are not public, §4.2.2):

* :func:`plummer` -- Plummer sphere in virial units (M = 1, E = -1/4),
  sampled after Aarseth, Henon & Wielen (1974): radius from the inverse
  cumulative mass, speed by von Neumann rejection on q^2 (1 - q^2)^(7/2).
  Radii are cut at 99.9 % of the mass; the centre of mass is moved to
  the origin and the mean velocity removed.
* :func:`galaxy` -- stand-in for a disk galaxy: a Hernquist (1990) sphere
  (a = 1, M = 1) with isotropic speeds drawn from its closed-form
  distribution function, plus an exponential disk (scale length 1,
  sech^2 height 0.1, M = 0.2) on near-circular orbits.
* :func:`ensemble` -- many independent Plummer clusters of log-uniform
  sizes and uniform scale radii, returned back to back with their
  system offsets.
* :func:`nested` -- a Plummer sphere holding a second, far more compact
  Plummer cluster: more bodies share one cell of the 20th level than any
  leaf may hold, the case deeper keys are for (App. B).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["plummer", "galaxy", "ensemble", "nested", "subsample"]

_VIRIAL_R = 3.0 * math.pi / 16.0  # Plummer scale length in virial units


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def plummer(n: int, seed: int, mass_cut: float = 0.999):
    """Plummer sphere of ``n`` equal-mass bodies (mass 1/n each).

    Returns ``(pos, vel, mass)``.
    """
    rng = np.random.default_rng(seed)
    if n == 0:
        z = np.zeros((0, 3))
        return z, z.copy(), np.zeros(0)
    x1 = rng.uniform(0.0, mass_cut, n)
    with np.errstate(divide="ignore"):
        r = np.where(x1 > 0.0, 1.0 / np.sqrt(np.power(x1, -2.0 / 3.0) - 1.0), 0.0)
    pos = r[:, None] * _isotropic(rng, n)
    # speed in units of the local escape speed: rejection on g(q) = q^2 (1-q^2)^3.5
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.uniform(0.0, 1.0, todo.size)
        x5 = rng.uniform(0.0, 1.0, todo.size)
        ok = 0.1 * x5 < x4 * x4 * np.power(1.0 - x4 * x4, 3.5)
        q[todo[ok]] = x4[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * np.power(1.0 + r * r, -0.25)
    vel = (q * vesc)[:, None] * _isotropic(rng, n)
    pos *= _VIRIAL_R
    vel /= math.sqrt(_VIRIAL_R)
    mass = np.full(n, 1.0 / n)
    pos -= pos.mean(axis=0)
    vel -= vel.mean(axis=0)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def _hernquist_df(eps: np.ndarray) -> np.ndarray:
    """Hernquist (1990) isotropic distribution function, G = M = a = 1, up to a constant.

    ``eps`` is the binding energy -E in (0, 1).
    """
    q = np.sqrt(np.clip(eps, 0.0, 1.0 - 1e-12))
    s = np.sqrt(1.0 - q * q)
    return (3.0 * np.arcsin(q) + q * s * (1.0 - 2.0 * q * q) * (8.0 * q ** 4 - 8.0 * q * q - 3.0)) / s ** 5


def galaxy(n_halo: int, n_disk: int, seed: int):
    """Hernquist sphere (a = 1, M = 1) plus exponential disk (R_d = 1, z0 = 0.1, M = 0.2).

    Returns ``(pos, vel, mass)``; halo bodies come first.
    """
    rng = np.random.default_rng(seed)
    # --- halo: inverse cumulative mass M(<r) = r^2/(r+1)^2, truncated at 0.999
    u = rng.uniform(0.0, 0.999, n_halo)
    su = np.sqrt(u)
    r = su / (1.0 - su)
    pos_h = r[:, None] * _isotropic(rng, n_halo)
    psi = 1.0 / (1.0 + r)
    vesc = np.sqrt(2.0 * psi)
    # rejection on p(v) ~ v^2 f(psi - v^2/2) in [0, vesc]; bound from a coarse grid
    grid = np.linspace(0.0, 1.0, 65)[1:-1]
    pmax = np.zeros(n_halo)
    for g in grid:
        v = g * vesc
        pmax = np.maximum(pmax, v * v * _hernquist_df(psi - 0.5 * v * v))
    pmax *= 1.2
    speed = np.empty(n_halo)
    todo = np.arange(n_halo)
    while todo.size:
        v = rng.uniform(0.0, 1.0, todo.size) * vesc[todo]
        p = v * v * _hernquist_df(psi[todo] - 0.5 * v * v)
        ok = rng.uniform(0.0, 1.0, todo.size) * pmax[todo] < p
        speed[todo[ok]] = v[ok]
        todo = todo[~ok]
    vel_h = speed[:, None] * _isotropic(rng, n_halo)
    # --- disk: R ~ Gamma(2, R_d) (exponential surface density), z ~ sech^2(z/z0)
    m_disk = 0.2
    rr = -np.log(rng.uniform(1e-300, 1.0, n_disk) * rng.uniform(1e-300, 1.0, n_disk))
    rr = np.minimum(rr, 20.0)
    zz = 0.1 * np.arctanh(np.clip(2.0 * rng.uniform(0.0, 1.0, n_disk) - 1.0, -0.999999, 0.999999))
    ph = rng.uniform(0.0, 2.0 * math.pi, n_disk)
    pos_d = np.stack([rr * np.cos(ph), rr * np.sin(ph), zz], axis=1)
    # circular speed from the enclosed mass of both parts (spherical approximation)
    m_enc = rr * rr / (rr + 1.0) ** 2 + m_disk * (1.0 - (1.0 + rr) * np.exp(-rr))
    vc = np.sqrt(m_enc / np.maximum(rr, 1e-6))
    vel_d = np.stack([-vc * np.sin(ph), vc * np.cos(ph), np.zeros(n_disk)], axis=1)
    vel_d += 0.1 * vc[:, None] * rng.standard_normal((n_disk, 3))
    pos = np.concatenate([pos_h, pos_d])
    vel = np.concatenate([vel_h, vel_d])
    mass = np.concatenate([np.full(n_halo, 1.0 / max(n_halo, 1)), np.full(n_disk, m_disk / max(n_disk, 1))])
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def ensemble(n_sys: int = 512, seed: int = 5, n_min: int = 1024, n_max: int = 65536):
    """``n_sys`` independent Plummer clusters, sizes log-uniform in [n_min, n_max].

    Cluster ``s`` has its own seed ``1000 * seed + s`` and a scale radius
    ``b_s ~ U(0.5, 2)``; positions are scaled by ``b_s`` and velocities by
    ``b_s ** -0.5`` (each cluster keeps mass 1).  Returns
    ``(pos, vel, mass, offsets)`` with ``offsets[s]:offsets[s+1]`` the
    bodies of cluster ``s``.
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_sys))).astype(np.int64)
    scales = rng.uniform(0.5, 2.0, n_sys)
    parts = [plummer(int(sizes[s]), 1000 * seed + s) for s in range(n_sys)]
    pos = np.concatenate([p[0] * scales[s] for s, p in enumerate(parts)]) if n_sys else np.zeros((0, 3))
    vel = np.concatenate([p[1] / math.sqrt(scales[s]) for s, p in enumerate(parts)]) if n_sys else np.zeros((0, 3))
    mass = np.concatenate([p[2] for p in parts]) if n_sys else np.zeros(0)
    offsets = np.zeros(n_sys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass, offsets


def nested(n: int, seed: int, n_core: int, core_scale: float = 1e-6, at=(0.3, 0.1, -0.2)):
    """A Plummer sphere of ``n - n_core`` bodies and, centred at ``at``, a
    Plummer cluster of ``n_core`` bodies shrunk by ``core_scale`` (its
    velocities scaled to stay bound: by ``sqrt(f / core_scale)``, f its mass
    fraction).  Equal masses 1/n; the two parts use seeds ``seed`` and
    ``seed + 1``.  Returns ``(pos, vel, mass)``."""
    pa, va, _ = plummer(n - n_core, seed)
    pb, vb, _ = plummer(n_core, seed + 1)
    f = n_core / n
    pos = np.concatenate([pa, pb * core_scale + np.asarray(at, dtype=np.float64)])
    vel = np.concatenate([va, vb * math.sqrt(f / core_scale)])
    mass = np.full(n, 1.0 / n)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def subsample(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct indices of ``range(n)``, drawn without replacement, sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))
