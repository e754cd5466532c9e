"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

Holds none of the method's arithmetic: only random numbers and point sets.
The generator is counter-based so that any slice can be produced without
generating the prefix: value i of stream ``seed`` is the SplitMix64 output
function (Steele, Lea and Flood, OOPSLA 2014) applied to
``mix(seed) + (i + 1) * 0x9E3779B97F4A7C15`` (mod 2^64).  Doubles take the
top 53 bits; normals use the Box-Muller transform.

The point-set recipes follow the workloads of the paper (Sec. 5: locations
in the unit square [0, 1]^2, irregular, n from thousands to a million)
with the shapes used by the benchmark configurations: uniform points, and
a uniform/Gaussian-blob mixture.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uint64_stream(seed: int, n: int, offset: int = 0) -> np.ndarray:
    with np.errstate(over="ignore"):
        base = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix(base + ctr * _GAMMA)


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1)."""
    return (uint64_stream(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]                 # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n]


def locations_uniform(n: int, d: int = 2, seed: int = 1) -> np.ndarray:
    """n points i.i.d. uniform in [0, 1]^d, row-major (n, d)."""
    return uniform(seed, n * d).reshape(n, d)


def locations_blobs(n: int, d: int = 2, frac_blob: float = 0.3, nblobs: int = 8,
                    sd: float = 0.03, seed: int = 1) -> np.ndarray:
    """(1 - frac_blob) n uniform points plus frac_blob n points in ``nblobs``
    Gaussian blobs (centres uniform in [0.1, 0.9]^d, standard deviation
    ``sd``), clipped to [0, 1]^d.  Uniform points come first, then blobs
    in order."""
    nb = int(round(frac_blob * n))
    nu_ = n - nb
    pts = np.empty((n, d))
    pts[:nu_] = uniform(seed, nu_ * d).reshape(nu_, d)
    centres = 0.1 + 0.8 * uniform(seed + 0x1000, nblobs * d).reshape(nblobs, d)
    which = (uniform(seed + 0x2000, nb) * nblobs).astype(np.int64)
    off = normal(seed + 0x3000, nb * d).reshape(nb, d) * sd
    pts[nu_:] = np.clip(centres[which] + off, 0.0, 1.0)
    return pts


def locations_collinear(n: int, seed: int = 1, y: float = 0.5) -> np.ndarray:
    """n points on the horizontal line y = const, x uniform in [0, 1] and
    sorted (a degenerate 2-D geometry with an exact O(n) likelihood for
    the exponential kernel)."""
    x = np.sort(uniform(seed, n))
    return np.stack([x, np.full(n, y)], axis=1)


# --- workload recipes -------------------------------------------------------

SMALL = dict(n=2000, d=2, theta=(0.1, 0.5, 1.0, 0.01), leaf=32, eta=2.0,
             aca_eps=1e-8, theta0=(0.2, 1.0, 0.5, 0.05), seed=1000)
"""n = 2000 uniform points, Matern (ell, nu, sigma2, tau2) = (0.1, 0.5, 1, 0.01),
leaf 32, eta 2, ACA eps 1e-8; fit from (0.2, 1.0, 0.5, 0.05)."""

MEDIUM = dict(n=65536, d=2, theta=(0.05, 0.5, 1.0, 1e-3), nus=(0.5, 0.8, 1.5, 2.5),
              leaf=64, eta=2.0, aca_eps=1e-6, frac_blob=0.3, nblobs=8, sd=0.03,
              seed=1001, subset=16384)
"""n = 65536: 70 % uniform + 30 % in 8 blobs (sd 0.03); ell 0.05, sigma2 1,
tau2 1e-3, nu in {0.5, 0.8, 1.5, 2.5}; leaf 64, ACA eps 1e-6."""

LARGE = dict(n=2_000_000, d=2, theta=(0.02, 0.5, 1.0, 1e-3), nus=(0.5, 1.0),
             leaf=128, eta=2.0, aca_eps=1e-5, frac_blob=0.2, nblobs=8, sd=0.03,
             seed=1004)
"""n = 2,000,000: 80 % uniform + 20 % blobs; ell 0.02, sigma2 1, tau2 1e-3,
nu in {0.5, 1.0}; leaf 128, ACA eps 1e-5."""


def medium_locations(n: int | None = None) -> np.ndarray:
    c = MEDIUM
    return locations_blobs(n or c["n"], c["d"], c["frac_blob"], c["nblobs"], c["sd"], c["seed"])
