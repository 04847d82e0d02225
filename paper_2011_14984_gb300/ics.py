"""Seeded synthetic initial conditions shared by the CUDA path, the oracle tests and the bench.

This module holds no arithmetic of the integrator itself: it only draws particle sets.
Every generator takes an explicit integer seed and uses numpy's PCG64 stream through
``Generator.random`` (uniform doubles) only, with all transformations written out here,
so the same seed gives the same particles on every machine and numpy version that keeps
PCG64's uniform stream.

Recipes (units: Henon units, G = M = 1, E = -1/4, unless stated otherwise):

* Plummer sphere (App. A2, density/potential pair, cumulative mass M(r) and the
  distribution function f(E) ~ E^(7/2)): radii by inverting M(r) with the mass fraction
  clipped to <= 0.999; speeds as a fraction q of the local escape speed by rejection from
  g(q) ~ q^2 (1 - q^2)^(7/2) (the Aarseth-Henon-Wielen 1974 recipe); isotropic directions;
  centre of mass moved to rest at the origin.  Scale radius a = 3 pi / 16 gives E = -1/4.
* Kroupa (2001) mass spectrum (Sec. 5.2): broken power law dN/dm ~ m^-1.3 on
  [0.08, 0.5] and m^-2.3 on [0.5, 100], rescaled to unit total mass.
* Hard binaries: a fraction of the stars paired into Kepler binaries with log-uniform
  semi-major axes and thermal eccentricities (e = sqrt(U)), isotropic orientation and
  uniform mean anomaly, their centres of mass placed on Plummer draws.
* Batches of independent clusters with log-uniform sizes.
"""

from __future__ import annotations

import math

import numpy as np

HENON_PLUMMER_A = 3.0 * math.pi / 16.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere: cos(theta) uniform in [-1, 1], phi uniform."""
    u = rng.random(n)
    w = rng.random(n)
    ct = 2.0 * u - 1.0
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = 2.0 * math.pi * w
    return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)


def _plummer_speed_fraction(rng: np.random.Generator, n: int) -> np.ndarray:
    """q = v / v_esc drawn from g(q) ~ q^2 (1 - q^2)^(7/2) by rejection (max of g < 0.1)."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = max(64, 2 * (n - filled))
        q = rng.random(k)
        y = 0.1 * rng.random(k)
        ok = y < q * q * (1.0 - q * q) ** 3.5
        take = q[ok][: n - filled]
        out[filled : filled + take.size] = take
        filled += take.size
    return out


def plummer(n: int, seed: int, masses: np.ndarray | None = None, *, G: float = 1.0,
            M: float = 1.0, a: float = HENON_PLUMMER_A, max_mass_fraction: float = 0.999,
            recentre: bool = True):
    """Plummer sphere with n particles.  Returns (m[n], x[n,3], v[n,3]) as float64.

    ``masses`` (summing to M) replaces the default equal masses M/n.  Velocities are drawn
    from the isotropic Plummer distribution function independently of the masses.
    """
    rng = _rng(seed)
    if masses is None:
        m = np.full(n, M / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        assert m.shape == (n,)
    X = max_mass_fraction * rng.random(n)
    X = np.maximum(X, 1e-300)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    x = r[:, None] * _isotropic(rng, n)
    q = _plummer_speed_fraction(rng, n)
    vesc = math.sqrt(2.0 * G * M / a) * (1.0 + (r / a) ** 2) ** -0.25
    v = (q * vesc)[:, None] * _isotropic(rng, n)
    if recentre:
        x, v = centre_of_mass_frame(m, x, v)
    return m, x, v


def centre_of_mass_frame(m: np.ndarray, x: np.ndarray, v: np.ndarray):
    mt = m.sum()
    xc = (m[:, None] * x).sum(axis=0) / mt
    vc = (m[:, None] * v).sum(axis=0) / mt
    return x - xc, v - vc


def kroupa_masses(n: int, seed: int, m_lo: float = 0.08, m_br: float = 0.5,
                  m_hi: float = 100.0, alpha1: float = 1.3, alpha2: float = 2.3,
                  total: float = 1.0) -> np.ndarray:
    """Two-segment Kroupa (2001) IMF by inverse-CDF sampling, rescaled to sum ``total``."""
    rng = _rng(seed)
    # Continuous broken power law: k1 m^-a1 on [lo, br], k2 m^-a2 on [br, hi], k2 = k1 br^(a2-a1).
    def seg_int(lo, hi, al):
        return (hi ** (1.0 - al) - lo ** (1.0 - al)) / (1.0 - al)
    w1 = seg_int(m_lo, m_br, alpha1)
    w2 = m_br ** (alpha2 - alpha1) * seg_int(m_br, m_hi, alpha2)
    p1 = w1 / (w1 + w2)
    u = rng.random(n)
    s = rng.random(n)
    m = np.empty(n)
    lo = s < p1
    # inverse CDF inside each segment
    e1 = 1.0 - alpha1
    e2 = 1.0 - alpha2
    m[lo] = (m_lo ** e1 + u[lo] * (m_br ** e1 - m_lo ** e1)) ** (1.0 / e1)
    hi = ~lo
    m[hi] = (m_br ** e2 + u[hi] * (m_hi ** e2 - m_br ** e2)) ** (1.0 / e2)
    return m * (total / m.sum())


def _solve_kepler(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly from mean anomaly by Newton iteration on E - e sin E = M."""
    E = np.where(e < 0.8, M, math.pi * np.ones_like(M))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def kepler_relative_state(a, e, mean_anomaly, G, mtot):
    """Relative position/velocity of a Kepler orbit in its orbital plane (x toward pericentre)."""
    a = np.asarray(a, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    E = _solve_kepler(np.asarray(mean_anomaly, dtype=np.float64), e)
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    r = a * (1.0 - e * cE)
    n_mean = np.sqrt(G * mtot / a ** 3)
    Edot = n_mean / (1.0 - e * cE)
    rel_x = np.stack([a * (cE - e), b * sE, np.zeros_like(a)], axis=-1)
    rel_v = np.stack([-a * sE * Edot, b * cE * Edot, np.zeros_like(a)], axis=-1)
    return rel_x, rel_v, r


def _random_rotation(rng: np.random.Generator, k: int) -> np.ndarray:
    """k isotropic rotation matrices from uniform unit quaternions (Shoemake 1992)."""
    u1, u2, u3 = rng.random(k), rng.random(k), rng.random(k)
    q0 = np.sqrt(1 - u1) * np.sin(2 * math.pi * u2)
    q1 = np.sqrt(1 - u1) * np.cos(2 * math.pi * u2)
    q2 = np.sqrt(u1) * np.sin(2 * math.pi * u3)
    q3 = np.sqrt(u1) * np.cos(2 * math.pi * u3)
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (q2 * q2 + q3 * q3)
    R[:, 0, 1] = 2 * (q1 * q2 - q0 * q3)
    R[:, 0, 2] = 2 * (q1 * q3 + q0 * q2)
    R[:, 1, 0] = 2 * (q1 * q2 + q0 * q3)
    R[:, 1, 1] = 1 - 2 * (q1 * q1 + q3 * q3)
    R[:, 1, 2] = 2 * (q2 * q3 - q0 * q1)
    R[:, 2, 0] = 2 * (q1 * q3 - q0 * q2)
    R[:, 2, 1] = 2 * (q2 * q3 + q0 * q1)
    R[:, 2, 2] = 1 - 2 * (q1 * q1 + q2 * q2)
    return R


def plummer_kroupa_binaries(n: int, seed: int, binary_fraction: float = 0.05,
                            a_min: float = 1e-5, a_max: float = 1e-3, G: float = 1.0):
    """Plummer sphere with Kroupa masses where ``binary_fraction`` of the n stars are
    members of hard binaries (log-uniform a in [a_min, a_max], thermal e, isotropic
    orientation, uniform mean anomaly).  Binary members are stored adjacently."""
    rng = _rng(seed + 7919)
    n_bin = int(round(binary_fraction * n / 2.0))
    n_single = n - 2 * n_bin
    n_sys = n_single + n_bin
    m_star = kroupa_masses(n, seed)
    m_sys = np.concatenate([m_star[:n_single], m_star[n_single::2] + m_star[n_single + 1::2]])
    ms, xs, vs = plummer(n_sys, seed, masses=m_sys, G=G, M=m_sys.sum())
    m = np.empty(n)
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    m[:n_single], x[:n_single], v[:n_single] = m_star[:n_single], xs[:n_single], vs[:n_single]
    if n_bin:
        m1 = m_star[n_single::2]
        m2 = m_star[n_single + 1::2]
        mt = m1 + m2
        la = math.log(a_min) + (math.log(a_max) - math.log(a_min)) * rng.random(n_bin)
        a = np.exp(la)
        e = np.sqrt(rng.random(n_bin))
        Mmean = 2.0 * math.pi * rng.random(n_bin)
        rx, rv, _ = kepler_relative_state(a, e, Mmean, G, mt)
        R = _random_rotation(rng, n_bin)
        rx = np.einsum("kij,kj->ki", R, rx)
        rv = np.einsum("kij,kj->ki", R, rv)
        xc, vc = xs[n_single:], vs[n_single:]
        f1 = (m2 / mt)[:, None]
        f2 = (m1 / mt)[:, None]
        i1 = n_single + 2 * np.arange(n_bin)
        m[i1], m[i1 + 1] = m1, m2
        x[i1], x[i1 + 1] = xc + f1 * rx, xc - f2 * rx
        v[i1], v[i1 + 1] = vc + f1 * rv, vc - f2 * rv
    x, v = centre_of_mass_frame(m, x, v)
    return m, x, v


def binary_pairs(n: int, binary_fraction: float = 0.05) -> np.ndarray:
    """Index pairs [k, 2] of the binary members that plummer_kroupa_binaries(n, ...) stores
    adjacently after the single stars (bookkeeping only)."""
    n_bin = int(round(binary_fraction * n / 2.0))
    i1 = (n - 2 * n_bin) + 2 * np.arange(n_bin)
    return np.stack([i1, i1 + 1], axis=1)


def cluster_batch(n_clusters: int = 256, seed0: int = 1000, n_min: int = 64, n_max: int = 4096):
    """Independent Plummer clusters (each in its own Henon units) with log-uniform sizes
    N_k = floor(n_min * (n_max / n_min)^U).  Returns (offsets[n_clusters+1], m, x, v)."""
    rng = _rng(seed0)
    u = rng.random(n_clusters)
    sizes = np.floor(n_min * (n_max / n_min) ** u).astype(np.int64)
    sizes = np.clip(sizes, n_min, n_max)
    offsets = np.zeros(n_clusters + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    ms, xs, vs = [], [], []
    for k in range(n_clusters):
        m, x, v = plummer(int(sizes[k]), seed0 + k)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    return offsets, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)


def kepler_binary(m1: float, m2: float, a: float, e: float, G: float = 1.0,
                  mean_anomaly: float = 0.0):
    """Two-body Kepler orbit in its centre-of-mass frame, orbit in the x-y plane with
    pericentre along +x.  Returns (m[2], x[2,3], v[2,3])."""
    mt = m1 + m2
    rx, rv, _ = kepler_relative_state(np.array([a]), np.array([e]), np.array([mean_anomaly]), G,
                                      np.array([mt]))
    rx, rv = rx[0], rv[0]
    m = np.array([m1, m2], dtype=np.float64)
    x = np.stack([(m2 / mt) * rx, -(m1 / mt) * rx])
    v = np.stack([(m2 / mt) * rv, -(m1 / mt) * rv])
    return m, x, v


# Named workloads (sizes, seeds and recipes of the benchmarked configurations).
def workload(name: str):
    if name == "plummer_1k":
        return plummer(1024, 1)
    if name == "plummer_64k":
        return plummer(65536, 2)
    if name == "plummer_kroupa_binaries_256k":
        return plummer_kroupa_binaries(262144, 3)
    if name == "plummer_1m":
        return plummer(1048576, 5)
    if name == "plummer_256k":
        # the 1M sphere's recipe and seed at a quarter of its size: the stand-in where a
        # comparison with the FP64 mode does not fit at 1M
        return plummer(262144, 5)
    raise KeyError(name)


def batch_workload(name: str):
    """(offsets, m, x, v) of a named batch of independent clusters."""
    if name == "cluster_batch_256":
        return cluster_batch(256, 1000)
    raise KeyError(name)
