"""Seeded synthetic inputs: Plummer spheres, cluster batches and request streams.

This module holds the random-number generator and the initial-condition
recipes only; it contains none of the force or integrator arithmetic, and it
is the one module that both the CUDA path's tests and the CPU oracle's tests
draw inputs from.

Random numbers come from one counter-based generator: SplitMix64's output
mixer (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to ``key + (counter + 1) * golden_gamma``. Every draw is a
pure function of (key, counter), so arrays of draws are vectorised and the
stream for a given seed is identical on every machine.

The paper (Sect. VI) builds its systems from Plummer spheres; it prints no
sampling recipe, so the standard one is used (Aarseth, Henon & Wielen 1974):
radius by inverting the cumulative mass, speed by von Neumann rejection on
g(q) = q^2 (1 - q^2)^(7/2), isotropic directions, then N-body units
(G = M = 1, E = -1/4: lengths x 3 pi / 16, velocities / sqrt(3 pi / 16)) and
the centre-of-mass frame.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASTER_SEED = 20140920

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S11 = np.uint64(11)
_TWO53 = 2.0 ** -53

# Plummer radius cut, in units of the Plummer scale length.
R_CUT = 22.8


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
        return z ^ (z >> _S31)


def key(seed: int, *tags: int) -> np.uint64:
    """Derive a stream key from a seed and integer tags (hash chain of the mixer)."""
    k = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    with np.errstate(over="ignore"):
        for t in tags:
            k = _mix(k ^ (np.uint64(t & 0xFFFFFFFFFFFFFFFF) * _GAMMA + _GAMMA))
    return k[0]


def u64(k: np.uint64, counters) -> np.ndarray:
    """Raw 64-bit draws number ``counters`` of stream ``k``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(k + (c + np.uint64(1)) * _GAMMA)


def uniform(k: np.uint64, counters) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(k, counters) >> _S11).astype(np.float64) * _TWO53


def uniform_open0(k: np.uint64, counters) -> np.ndarray:
    """Doubles in (0, 1]."""
    return ((u64(k, counters) >> _S11).astype(np.float64) + 1.0) * _TWO53


def normal(k: np.uint64, n: int) -> np.ndarray:
    """n standard normal deviates by the Box-Muller transform on pairs of draws."""
    c = np.arange(n, dtype=np.uint64) * np.uint64(2)
    u1 = uniform_open0(k, c)
    u2 = uniform(k, c + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _isotropic(k: np.uint64, n: int) -> np.ndarray:
    c = np.arange(n, dtype=np.uint64) * np.uint64(2)
    cos_t = 2.0 * uniform(k, c) - 1.0
    phi = 2.0 * math.pi * uniform(k, c + np.uint64(1))
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


@dataclass
class Particles:
    """A system in N-body units: m (n,), pos (n,3), vel (n,3), FP64."""

    m: np.ndarray
    pos: np.ndarray
    vel: np.ndarray

    @property
    def n(self) -> int:
        return int(self.m.shape[0])

    def soa(self):
        """Structure-of-arrays view: (m, x, y, z, vx, vy, vz), contiguous."""
        return (np.ascontiguousarray(self.m),
                *[np.ascontiguousarray(self.pos[:, c]) for c in range(3)],
                *[np.ascontiguousarray(self.vel[:, c]) for c in range(3)])


def to_com_frame(m, pos, vel):
    mt = m.sum()
    pos = pos - (m[:, None] * pos).sum(axis=0) / mt
    vel = vel - (m[:, None] * vel).sum(axis=0) / mt
    return pos, vel


def plummer(n: int, seed: int = MASTER_SEED, masses: str = "equal", sigma: float = 0.5,
            r_cut: float = R_CUT) -> Particles:
    """Plummer sphere of n particles in N-body units (total mass 1).

    masses: "equal" (1/n each) or "lognormal" (m proportional to exp(sigma Z),
    Z standard normal, normalised to total mass 1).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    idx = np.arange(n, dtype=np.uint64)
    # radius: invert M(r) = r^3 / (1 + r^2)^(3/2) on (0, M(r_cut)]
    m_cut = r_cut ** 3 / (1.0 + r_cut * r_cut) ** 1.5
    x = uniform_open0(key(seed, 1), idx) * m_cut
    r = 1.0 / np.sqrt(x ** (-2.0 / 3.0) - 1.0)
    pos = r[:, None] * _isotropic(key(seed, 2), n)
    # speed: von Neumann rejection of q on g(q) = q^2 (1 - q^2)^3.5 (max < 0.1)
    q = np.full(n, np.nan)
    pending = np.arange(n)
    kq, ky = key(seed, 3), key(seed, 4)
    rnd = 0
    batch = 32
    while pending.size:
        cand = (pending.astype(np.uint64)[:, None] * np.uint64(1 << 20)
                + np.uint64(rnd * batch) + np.arange(batch, dtype=np.uint64)[None, :])
        qc = uniform(kq, cand)
        yc = 0.1 * uniform(ky, cand)
        ok = yc < qc * qc * (1.0 - qc * qc) ** 3.5
        has = ok.any(axis=1)
        first = ok.argmax(axis=1)
        sel = pending[has]
        q[sel] = qc[has, first[has]]
        pending = pending[~has]
        rnd += 1
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25
    vel = (q * vesc)[:, None] * _isotropic(key(seed, 5), n)
    if masses == "equal":
        m = np.full(n, 1.0 / n)
    elif masses == "lognormal":
        w = np.exp(sigma * normal(key(seed, 6), n))
        m = w / w.sum()
    else:
        raise ValueError("masses must be 'equal' or 'lognormal'")
    scale = 3.0 * math.pi / 16.0
    pos = pos * scale
    vel = vel / math.sqrt(scale)
    pos, vel = to_com_frame(m, pos, vel)
    return Particles(m, np.ascontiguousarray(pos), np.ascontiguousarray(vel))


def galaxy(n: int, seed: int, bh_fraction: float = 0.01) -> Particles:
    """Plummer sphere of n-1 stars plus a central point mass holding bh_fraction of
    the total mass (particle 0, at rest at the centre before the centre-of-mass shift)."""
    if n < 2:
        raise ValueError("a galaxy needs n >= 2")
    stars = plummer(n - 1, seed)
    m = np.concatenate([[bh_fraction], stars.m * (1.0 - bh_fraction)])
    pos = np.concatenate([np.zeros((1, 3)), stars.pos])
    vel = np.concatenate([np.zeros((1, 3)), stars.vel])
    pos, vel = to_com_frame(m, pos, vel)
    return Particles(m, np.ascontiguousarray(pos), np.ascontiguousarray(vel))


def cluster_sizes(n_clusters: int, n_lo: int, n_hi: int, seed: int = MASTER_SEED) -> np.ndarray:
    """Cluster sizes log-uniform in [n_lo, n_hi], rounded to integers."""
    u = uniform(key(seed, 7), np.arange(n_clusters, dtype=np.uint64))
    n = np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo))))
    return np.clip(n, n_lo, n_hi).astype(np.int64)


def cluster_eps(n) -> np.ndarray:
    """Per-cluster softening eps = 1 / (4 N^(1/3))."""
    return 0.25 / np.cbrt(np.asarray(n, dtype=np.float64))


def cluster_batch(n_clusters: int = 4096, n_lo: int = 16, n_hi: int = 4096,
                  seed: int = MASTER_SEED):
    """Independent Plummer clusters: list of Particles (cluster c seeded by (seed, c))."""
    sizes = cluster_sizes(n_clusters, n_lo, n_hi, seed)
    return [plummer(int(n), int(key(seed, 8, c))) for c, n in enumerate(sizes)]


@dataclass
class Request:
    """One request of the serving workload."""

    rid: int
    arrival: float     # seconds after the stream starts
    galaxy: int        # which of the 11 galaxies the subsystem comes from
    n: int
    kind: str          # "force" or "evolve"
    t_span: float      # N-body time to integrate (evolve only)


def request_stream(n_requests: int, rate_hz: float, seed: int = MASTER_SEED,
                   n_lo: int = 2 ** 8, n_hi: int = 2 ** 18, n_galaxies: int = 11,
                   t_span: float = 0.125):
    """Poisson arrivals of force / evolve requests on subsystems of uneven size."""
    c = np.arange(n_requests, dtype=np.uint64)
    gaps = -np.log(uniform_open0(key(seed, 9), c)) / rate_hz
    arrival = np.cumsum(gaps) - gaps[0]
    gal = np.floor(uniform(key(seed, 10), c) * n_galaxies).astype(np.int64)
    u = uniform(key(seed, 11), c)
    n = np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    kind = np.where(uniform(key(seed, 12), c) < 0.5, "force", "evolve")
    return [Request(int(i), float(arrival[i]), int(gal[i]), int(n[i]), str(kind[i]),
                    float(t_span) if kind[i] == "evolve" else 0.0) for i in range(n_requests)]


def request_particles(req: Request, seed: int = MASTER_SEED) -> Particles:
    """The subsystem a request carries: galaxy-shaped, seeded by (seed, galaxy, request id)."""
    return galaxy(req.n, int(key(seed, 13, req.galaxy, req.rid)))
