"""Seeded synthetic inputs: Plummer spheres, Salpeter masses, ensembles and request streams.

This module only draws random numbers and maps them onto the initial-condition
distributions of the paper's benchmark workload (Section 3: the Plummer model in
the standard units of Heggie & Mathieu 1986, M = G = -4E = 1). It holds none of
the force, predictor, corrector or tree arithmetic: both the FP64 oracle and the
CUDA path take its arrays as plain inputs.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014, "Fast splittable
pseudorandom number generators"), written here from its published definition
with numpy uint64 arithmetic so that the same seed gives the same bits on any
machine.  Each quantity uses its own stream (seed, stream id) so that adding a
draw to one quantity never shifts another.

Plummer sampling follows Aarseth, Henon & Wielen (1974): radius by inverse CDF of
the cumulative mass M(r) = r^3 (1 + r^2)^(-3/2), isotropic directions, speed
fraction q = v / v_esc by von Neumann rejection on g(q) = q^2 (1 - q^2)^(7/2).
Scaling to standard units uses the analytic Plummer energy E = -3 pi / 64
(G = M = a = 1), i.e. lengths x 3 pi / 16 and velocities x sqrt(16 / (3 pi)).
The cumulative mass fraction is capped at 0.999 (about 22.8 scale radii) so that
no particle lands absurdly far out.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASS_CAP = 0.999

# stream ids, one per drawn quantity
_S_RADIUS, _S_POS_DIR, _S_VEL_Q, _S_VEL_DIR, _S_MASS, _S_ENSEMBLE, _S_ARRIVAL = range(7)


def splitmix64(seed: int, stream: int, n: int) -> np.ndarray:
    """Return n successive splitmix64 outputs (uint64) for (seed, stream)."""
    base = (int(seed) * 0x2545F4914F6CDD1D + int(stream) * 0x9E3779B97F4A7C15 + 1) & 0xFFFFFFFFFFFFFFFF
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(base) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles strictly inside (0, 1): the top 53 bits plus one half ulp."""
    z = splitmix64(seed, stream, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def _isotropic(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    cos_t = 2.0 * u1 - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * u2
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def _plummer_q(seed: int, n: int) -> np.ndarray:
    """Speed fractions q in [0,1) with density proportional to q^2 (1-q^2)^(7/2)."""
    out = np.empty(n)
    filled = 0
    rnd = 0
    while filled < n:
        m = max(64, 2 * (n - filled) + 64)
        u = uniform(seed, _S_VEL_Q + 16 * rnd, 2 * m)
        q, y = u[0::2], u[1::2]
        ok = 0.1 * y < q * q * (1.0 - q * q) ** 3.5
        take = q[ok][: n - filled]
        out[filled:filled + take.size] = take
        filled += take.size
        rnd += 1
    return out


def plummer(n: int, seed: int = 0, masses: np.ndarray | None = None):
    """Seeded Plummer sphere in standard units; returns (x[n,3], v[n,3], m[n]) in FP64.

    masses: optional per-particle masses (normalised here to a total of 1);
    equal masses 1/n when omitted.  The centre of mass is moved to the origin
    at rest.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    u_r = uniform(seed, _S_RADIUS, n) * _MASS_CAP
    r = 1.0 / np.sqrt(u_r ** (-2.0 / 3.0) - 1.0)
    ud = uniform(seed, _S_POS_DIR, 2 * n)
    x = r[:, None] * _isotropic(ud[0::2], ud[1::2])
    q = _plummer_q(seed, n)
    v_esc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    uv = uniform(seed, _S_VEL_DIR, 2 * n)
    v = (q * v_esc)[:, None] * _isotropic(uv[0::2], uv[1::2])
    if masses is None:
        m = np.full(n, 1.0 / n)
    else:
        m = np.asarray(masses, dtype=np.float64).copy()
        m /= m.sum()
    x *= 3.0 * math.pi / 16.0
    v *= math.sqrt(16.0 / (3.0 * math.pi))
    x -= (m[:, None] * x).sum(0) / m.sum()
    v -= (m[:, None] * v).sum(0) / m.sum()
    return np.ascontiguousarray(x), np.ascontiguousarray(v), m


def salpeter_masses(n: int, seed: int = 0, slope: float = 2.35, ratio: float = 100.0) -> np.ndarray:
    """Masses with dN/dm ~ m^-slope on [1, ratio] by inverse CDF, normalised to a total of 1."""
    u = uniform(seed, _S_MASS, n)
    p = 1.0 - slope
    lo, hi = 1.0, float(ratio)
    m = (lo ** p + u * (hi ** p - lo ** p)) ** (1.0 / p)
    return m / m.sum()


def plummer_salpeter(n: int, seed: int = 0, slope: float = 2.35, ratio: float = 100.0):
    """Plummer positions/velocities with an independent Salpeter mass spectrum."""
    return plummer(n, seed, masses=salpeter_masses(n, seed, slope, ratio))


@dataclass
class EnsembleMember:
    seed: int
    n: int
    theta: float


def ensemble(count: int = 256, n_lo: int = 1024, n_hi: int = 32768, seed: int = 0,
             thetas=(0.3, 0.5, 0.7)) -> list[EnsembleMember]:
    """Independent clusters: N log-uniform in [n_lo, n_hi], theta drawn from `thetas`."""
    u = uniform(seed, _S_ENSEMBLE, 2 * count)
    out = []
    for k in range(count):
        n = int(round(math.exp(math.log(n_lo) + u[2 * k] * (math.log(n_hi) - math.log(n_lo)))))
        th = thetas[min(len(thetas) - 1, int(u[2 * k + 1] * len(thetas)))]
        out.append(EnsembleMember(seed=k, n=n, theta=th))
    return out


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    t_end: float
    seed: int


def request_stream(count: int, rate_per_s: float = 20.0, n_lo: int = 1 << 10, n_hi: int = 1 << 18,
                   t_ends=(0.125, 0.25, 0.5), seed: int = 0) -> list[Request]:
    """Poisson arrivals (exponential gaps) of cluster-simulation requests."""
    u = uniform(seed, _S_ARRIVAL, 3 * count)
    t = 0.0
    out = []
    for k in range(count):
        t += -math.log(u[3 * k]) / rate_per_s
        n = int(round(math.exp(math.log(n_lo) + u[3 * k + 1] * (math.log(n_hi) - math.log(n_lo)))))
        te = t_ends[min(len(t_ends) - 1, int(u[3 * k + 2] * len(t_ends)))]
        out.append(Request(rid=k, arrival_s=t, n=n, t_end=te, seed=1000 + k))
    return out
