"""Seeded synthetic initial conditions for the direct N-body workloads.

The paper integrates star clusters and galactic nuclei with central black holes
(abstract; introduction) but prints no initial models.  Its stated model class is
a "real core-halo density structure" (abstract), which this module reads as the
Plummer sphere (core + r^-5 halo) and, for the cuspy nucleus, the Dehnen gamma=1
(Hernquist) sphere.  All models are in Henon units: G = 1, stellar mass M = 1 and
total stellar energy E = -1/4 in the N -> infinity limit.

This module is the input generator shared by the oracle tests and the CUDA path.
It samples positions, velocities and masses from their distribution functions
and holds none of the integration method's arithmetic: no pairwise force, no
predictor, corrector, time-step or energy sum.  Scaling to Henon units uses the
analytic energies of the continuous models, never a sum over particles.

Random numbers come from numpy's PCG64 generator with the stated seed, so every
workload is reproducible bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Plummer scale length giving E = -3*pi/64 * G M^2 / a = -1/4.
PLUMMER_A_HENON = 3.0 * math.pi / 16.0
# Hernquist (Dehnen gamma=1) scale length giving E = -G M^2 / (12 a) = -1/4.
HERNQUIST_A_HENON = 1.0 / 3.0
# The Hernquist mass profile has a heavy r^-4 density tail; radii are drawn from
# the innermost 99.9% of the mass so that a handful of far outliers cannot drag
# the centre of mass (r_max = 1998 a).
HERNQUIST_MASS_CUT = 0.999


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """n unit vectors uniform on the sphere."""
    cth = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    return np.stack([sth * np.cos(phi), sth * np.sin(phi), cth], axis=1)


def _to_com(m: np.ndarray, x: np.ndarray, v: np.ndarray) -> None:
    mt = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt


def plummer_enclosed_mass(r, a: float = PLUMMER_A_HENON, mass: float = 1.0):
    """Analytic Plummer mass inside radius r."""
    r = np.asarray(r, dtype=np.float64)
    return mass * r ** 3 / (r * r + a * a) ** 1.5


def hernquist_enclosed_mass(r, a: float = HERNQUIST_A_HENON, mass: float = 1.0):
    """Analytic Hernquist (Dehnen gamma=1) mass inside radius r."""
    r = np.asarray(r, dtype=np.float64)
    return mass * (r / (r + a)) ** 2


def plummer(n: int, seed: int, a: float = PLUMMER_A_HENON):
    """Equal-mass Plummer sphere, Aarseth, Henon & Wielen (1974) sampling.

    Radius from the inverse cumulative mass, speed by rejection from
    g(q) = q^2 (1 - q^2)^(7/2) times the local escape speed, isotropic
    directions, then a shift to the centre-of-mass frame.
    Returns (m[n], x[n,3], v[n,3]) in float64.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = _rng(seed)
    xm = rng.uniform(0.0, 1.0, n)
    xm = np.where(xm <= 0.0, np.finfo(np.float64).tiny, xm)
    r = a / np.sqrt(xm ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        q_try = rng.uniform(0.0, 1.0, todo.size)
        y = rng.uniform(0.0, 0.1, todo.size)
        ok = y < q_try * q_try * (1.0 - q_try * q_try) ** 3.5
        q[todo[ok]] = q_try[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (r * r + a * a) ** -0.25
    v = (q * vesc)[:, None] * _isotropic(rng, n)
    m = np.full(n, 1.0 / n)
    _to_com(m, x, v)
    return m, x, v


def _hernquist_bracket(qv: np.ndarray) -> np.ndarray:
    """3 asin q + q sqrt(1-q^2)(1-2q^2)(8q^4-8q^2-3), series below q = 0.05."""
    qv = np.asarray(qv, dtype=np.float64)
    out = np.empty_like(qv)
    small = qv < 0.05
    qs = qv[small]
    q2 = qs * qs
    out[small] = qs ** 5 * (128.0 / 5 + q2 * (-192.0 / 7 + q2 * (16.0 / 3 + q2 * (8.0 / 11 + q2 * (3.0 / 13 + q2 / 10.0)))))
    ql = qv[~small]
    ql2 = ql * ql
    out[~small] = 3.0 * np.arcsin(ql) + ql * np.sqrt(1.0 - ql2) * (1.0 - 2.0 * ql2) * (8.0 * ql2 * ql2 - 8.0 * ql2 - 3.0)
    return out


def hernquist_df(eps: np.ndarray, a: float = HERNQUIST_A_HENON) -> np.ndarray:
    """Isotropic Hernquist (1990) distribution function up to a constant factor.

    eps is the binding energy per unit mass (>= 0), G = M = 1.
    """
    qq = np.sqrt(np.clip(a * np.asarray(eps, dtype=np.float64), 0.0, 1.0 - 1e-15))
    return _hernquist_bracket(qq) / (1.0 - qq * qq) ** 2.5


def hernquist(n: int, seed: int, a: float = HERNQUIST_A_HENON):
    """Equal-mass Dehnen gamma=1 (Hernquist) sphere.

    Radius from M(r) = (r/(r+a))^2 truncated at HERNQUIST_MASS_CUT, speed by
    rejection from v^2 f(psi - v^2/2) with the closed-form isotropic distribution
    function, isotropic directions; zero total momentum, positions centred on
    the inner half of the mass.
    Returns (m, x, v) in float64.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = _rng(seed)
    xm = rng.uniform(0.0, HERNQUIST_MASS_CUT, n)
    s = np.sqrt(xm)
    r = a * s / (1.0 - s)
    x = r[:, None] * _isotropic(rng, n)
    psi = 1.0 / (r + a)
    ugrid = np.unique(np.concatenate([np.geomspace(1e-5, 1.0, 240), np.linspace(0.0, 1.0, 401)]))
    ugrid = ugrid[(ugrid > 0.0) & (ugrid < 1.0)]
    u = np.empty(n)
    chunk = 8192
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        ps = psi[c0:c1]
        g = ugrid[None, :] ** 2 * hernquist_df(ps[:, None] * (1.0 - ugrid[None, :] ** 2), a)
        env = 1.3 * g.max(axis=1)
        todo = np.arange(c1 - c0)
        while todo.size:
            ut = rng.uniform(0.0, 1.0, todo.size)
            gt = ut * ut * hernquist_df(ps[todo] * (1.0 - ut * ut), a)
            bad = gt > env[todo]
            if np.any(bad):
                env[todo[bad]] = 1.5 * gt[bad]
            y = rng.uniform(0.0, 1.0, todo.size) * env[todo]
            ok = (y < gt) & ~bad
            u[c0 + todo[ok]] = ut[ok]
            todo = todo[~ok]
    vesc = np.sqrt(2.0 * psi)
    v = (u * vesc)[:, None] * _isotropic(rng, n)
    m = np.full(n, 1.0 / n)
    # Zero total momentum; positions centred on the particles inside the median
    # radius, because the tail makes the whole-sample centre of mass wander.
    v -= (m[:, None] * v).sum(axis=0) / m.sum()
    core = r <= np.median(r)
    x -= (m[core, None] * x[core]).sum(axis=0) / m[core].sum()
    return m, x, v


def bh_circular_pair(m_bh: float = 0.005, sep: float = 0.1,
                     enclosed=plummer_enclosed_mass):
    """Two equal black holes on a circular orbit about the centre.

    Each hole sits at radius sep/2 in the x-y plane with opposite velocities.
    The circular speed balances the analytic stellar mass inside sep/2 and the
    other hole: v^2 = (sep/2) * (M_*(<sep/2)/(sep/2)^2 + m_bh/sep^2).
    """
    r = 0.5 * sep
    v2 = r * (float(enclosed(r)) / (r * r) + m_bh / (sep * sep))
    vc = math.sqrt(v2)
    m = np.array([m_bh, m_bh])
    x = np.array([[r, 0.0, 0.0], [-r, 0.0, 0.0]])
    v = np.array([[0.0, vc, 0.0], [0.0, -vc, 0.0]])
    return m, x, v


def bh_binary(m_bh: float = 0.01, a_bin: float = 0.05, ecc: float = 0.5):
    """Equal-mass Keplerian black-hole binary started at apocentre.

    The stellar potential is ignored when setting the orbit.
    """
    mt = 2.0 * m_bh
    r_apo = a_bin * (1.0 + ecc)
    v_apo = math.sqrt(mt * (1.0 - ecc) / (a_bin * (1.0 + ecc)))
    m = np.array([m_bh, m_bh])
    x = np.array([[0.5 * r_apo, 0.0, 0.0], [-0.5 * r_apo, 0.0, 0.0]])
    v = np.array([[0.0, 0.5 * v_apo, 0.0], [0.0, -0.5 * v_apo, 0.0]])
    return m, x, v


def ensemble_sizes(n_clusters: int = 256, lo: int = 1024, hi: int = 32768, seed: int = 0):
    """Cluster sizes drawn log-uniform in [lo, hi]: round(exp(U(ln lo, ln hi)))."""
    rng = _rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), n_clusters)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), lo, hi)


@dataclass
class Workload:
    """One synthetic problem: particles plus the integration parameters."""
    name: str
    m: np.ndarray
    x: np.ndarray
    v: np.ndarray
    eps2: np.ndarray          # per-particle squared softening; pairs use max(eps2_i, eps2_j)
    order: int = 6
    eta: float = 0.2
    eta_s: float = 0.01
    dt_max: float = 1.0 / 16.0
    t_end: float = 0.125
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])


def plummer_cluster(n: int = 1024, seed: int = 1000, eps: float = 1e-4, order: int = 6,
                    t_end: float = 0.125, name: str | None = None) -> Workload:
    """Equal-mass Plummer sphere with uniform Plummer softening."""
    m, x, v = plummer(n, seed)
    return Workload(name or f"plummer_n{n}", m, x, v, np.full(n, eps * eps), order=order,
                    t_end=t_end, meta={"model": "plummer", "seed": seed, "eps": eps})


def plummer_nucleus(n_stars: int = 1 << 20, seed: int = 1002, eps: float = 1e-5,
                    t_end: float = 0.25) -> Workload:
    """Plummer stars (mass 1) plus two 0.005 black holes circling at separation 0.1.

    Star-star softening eps, black holes unsoftened; a pair takes the larger of
    its two particles' softenings.
    """
    m, x, v = plummer(n_stars, seed)
    mb, xb, vb = bh_circular_pair(0.005, 0.1)
    eps2 = np.concatenate([np.full(n_stars, eps * eps), np.zeros(2)])
    return Workload(f"nucleus_plummer_n{n_stars}_2bh", np.concatenate([m, mb]),
                    np.concatenate([x, xb]), np.concatenate([v, vb]), eps2, order=6, t_end=t_end,
                    meta={"model": "plummer+2bh", "seed": seed, "eps": eps, "n_stars": n_stars})


def cusp_nucleus(n_stars: int = 1 << 18, seed: int = 1003, eps: float = 1e-4,
                 t_end: float = 0.25, order: int = 8) -> Workload:
    """Dehnen gamma=1 stars (mass 1) plus a central 0.01+0.01 binary (a=0.05, e=0.5)."""
    m, x, v = hernquist(n_stars, seed)
    mb, xb, vb = bh_binary(0.01, 0.05, 0.5)
    eps2 = np.concatenate([np.full(n_stars, eps * eps), np.zeros(2)])
    return Workload(f"cusp_dehnen1_n{n_stars}_bhb", np.concatenate([m, mb]),
                    np.concatenate([x, xb]), np.concatenate([v, vb]), eps2, order=order, t_end=t_end,
                    meta={"model": "dehnen1+bhb", "seed": seed, "eps": eps, "n_stars": n_stars})


def standard_workload(index: int) -> Workload:
    """The four single-system problems of the benchmark table, by position.

    0: Plummer N=1024, eps 1e-4, order 6, to t=0.125 (exact block-sequence case)
    1: Plummer N=65536, eps 1e-4, order 6, to t=1
    2: Plummer N=2^20 + two 0.005 holes, eps 1e-5 (holes 0), order 6, to t=0.25
    3: Dehnen gamma=1 N=2^18 + 0.01/0.01 binary, eps 1e-4 (holes 0), order 8, to t=0.25
    """
    if index == 0:
        return plummer_cluster(1024, 1000, 1e-4, 6, 0.125)
    if index == 1:
        return plummer_cluster(65536, 1001, 1e-4, 6, 1.0)
    if index == 2:
        return plummer_nucleus(1 << 20, 1002, 1e-5, 0.25)
    if index == 3:
        return cusp_nucleus(1 << 18, 1003, 1e-4, 0.25, 8)
    raise ValueError(f"no standard workload {index}")


def ensemble(n_clusters: int = 256, lo: int = 1024, hi: int = 32768, eps: float = 1e-4):
    """Independent Plummer clusters; cluster i uses seed i, sizes from seed 0."""
    sizes = ensemble_sizes(n_clusters, lo, hi, 0)
    return [plummer_cluster(int(nk), i, eps, 6, 0.5, name=f"ensemble_{i}_plummer_n{nk}")
            for i, nk in enumerate(sizes)]
