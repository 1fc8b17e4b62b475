"""Seeded synthetic inputs for local level-set grain growth.

This module is shared by the CUDA path, the FP64 oracle, the tests and the
benchmark.  It draws random numbers and nothing else: it holds none of the
method's arithmetic (no tessellation, no level-set function, no kernel).

Generator.  Every random number comes from the SplitMix64 generator
(G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used in counter mode::

    u64(seed, k) = mix(seed + (k + 1) * 0x9E3779B97F4A7C15)   (mod 2**64)
    mix(z):  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
             z = (z ^ (z >> 27)) * 0x94D049BB133111EB
             return z ^ (z >> 31)
    u01(seed, k) = (u64(seed, k) >> 11) * 2**-53          in [0, 1)

Counter k = (stream << 40) + index, one stream per quantity (STREAM_*).
The C library implements the same generator from the same definition
(``lsgg_generate_seeds``); a CPU test checks that both agree bit for bit.

Workload recipes (synthetic stand-ins for the paper's tessellation input,
Sec. 3.1, and its 3D benchmark, Sec. 4.2 / Sec. 6.3 "starting from a Voronoi
tessellation"):

* ``voronoi_seeds``     uniform seed points in the periodic box [0, N)^D.
* ``laguerre_weights``  lognormal radii (sigma) with a fraction of grains of
                        ``big_volume`` times the volume; weight = radius^2.
* ``random_quaternions`` uniform random rotations (K. Shoemake, "Uniform
                        random rotations", Graphics Gems III, 1992).
* ``jittered_hex_seeds`` 2D seeds on a jittered hexagonal lattice: most cells
                        get 5, 6 or 7 sides (von Neumann-Mullins tests).
* ``serving_requests``  an arrival stream of independent simulations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

STREAM_SEEDS = 0
STREAM_RADII = 1
STREAM_BIG = 2
STREAM_ORIENT = 3
STREAM_SERVE = 4
STREAM_JITTER = 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * M1
    z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def u64(seed: int, counters) -> np.ndarray:
    """SplitMix64 output number ``counters`` of the stream started at ``seed``."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (k + np.uint64(1)) * GOLDEN
        return _mix(z)


def u01(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) from counters (stream << 40) + index."""
    idx = np.asarray(index, dtype=np.uint64)
    k = (np.uint64(stream) << np.uint64(40)) + idx
    return (u64(seed, k) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def voronoi_seeds(seed: int, n_grains: int, shape_xyz) -> np.ndarray:
    """Seed points, shape (n_grains, 3) as (x, y, z), uniform in [0, N_a).

    Coordinate a of grain i uses counter 3*i + a of STREAM_SEEDS.  In 2D
    (shape z == 1) the z coordinate is 0.
    """
    nx, ny, nz = (int(v) for v in shape_xyz)
    idx = np.arange(3 * n_grains, dtype=np.uint64)
    u = u01(seed, STREAM_SEEDS, idx).reshape(n_grains, 3)
    s = u * np.array([nx, ny, nz], dtype=np.float64)
    if nz == 1:
        s[:, 2] = 0.0
    return s


def laguerre_weights(seed: int, n_grains: int, shape_xyz, sigma: float = 0.5,
                     big_fraction: float = 0.01, big_volume: float = 5.0) -> np.ndarray:
    """Power-diagram weights w_i = r_i^2 for a lognormal size distribution.

    r_i = c * exp(sigma * z_i), z_i standard normal by Box-Muller from two
    uniforms; grain i is 'big' when a third uniform is below big_fraction and
    then r_i is multiplied by big_volume^(1/D).  c scales the mean radius to
    half the mean seed spacing (N^D / n_grains)^(1/D).
    """
    nx, ny, nz = (int(v) for v in shape_xyz)
    dim = 2 if nz == 1 else 3
    i = np.arange(n_grains, dtype=np.uint64)
    u1 = u01(seed, STREAM_RADII, 2 * i)
    u2 = u01(seed, STREAM_RADII, 2 * i + np.uint64(1))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    r = np.exp(sigma * z)
    big = u01(seed, STREAM_BIG, i) < big_fraction
    r = np.where(big, r * big_volume ** (1.0 / dim), r)
    spacing = (nx * ny * nz / n_grains) ** (1.0 / dim)
    r = r * (0.5 * spacing / r.mean())
    return r * r


def random_quaternions(seed: int, n_grains: int) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z), Shoemake's method."""
    i = np.arange(n_grains, dtype=np.uint64)
    a = u01(seed, STREAM_ORIENT, 3 * i)
    b = u01(seed, STREAM_ORIENT, 3 * i + np.uint64(1))
    c = u01(seed, STREAM_ORIENT, 3 * i + np.uint64(2))
    s1, s2 = np.sqrt(1.0 - a), np.sqrt(a)
    t1, t2 = 2.0 * math.pi * b, 2.0 * math.pi * c
    q = np.stack([s2 * np.cos(t2), s1 * np.sin(t1), s1 * np.cos(t1), s2 * np.sin(t2)], axis=1)
    return q


def jittered_hex_seeds(seed: int, nx: int, ny: int, cols: int, rows: int,
                       jitter: float = 0.25) -> np.ndarray:
    """2D seeds on a hexagonal lattice of cols x rows points, each moved by a
    uniform offset of up to ``jitter`` lattice spacings per axis.  rows should
    be even so the lattice is periodic in y."""
    ax = nx / cols
    ay = ny / rows
    pts = []
    for r in range(rows):
        for c in range(cols):
            pts.append(((c + 0.5 * (r % 2)) * ax, (r + 0.5) * ay))
    p = np.array(pts, dtype=np.float64)
    n = p.shape[0]
    i = np.arange(2 * n, dtype=np.uint64)
    u = u01(seed, STREAM_JITTER, i).reshape(n, 2)
    p[:, 0] += (2.0 * u[:, 0] - 1.0) * jitter * ax
    p[:, 1] += (2.0 * u[:, 1] - 1.0) * jitter * ay
    p[:, 0] %= nx
    p[:, 1] %= ny
    return np.concatenate([p, np.zeros((n, 1))], axis=1)


@dataclass
class Request:
    """One served simulation: a cubic periodic domain of side n, n_grains
    Voronoi grains from ``seed``, advanced ``steps`` steps; arrives at
    ``arrival`` seconds after the start of the run."""
    index: int
    seed: int
    n: int
    n_grains: int
    steps: int
    arrival: float


def serving_requests(count: int, rate_per_s: float, base_seed: int = 1000,
                     sizes=tuple(range(32, 257, 16)), cells_per_grain: float = 3355.0,
                     grains_range=(20, 5000), steps_range=(10, 200)) -> list[Request]:
    """Poisson arrivals at ``rate_per_s``; per request the side n is uniform in
    ``sizes``, grains = round(n^3 / cells_per_grain) clamped to grains_range,
    steps uniform in steps_range (inclusive), seed = base_seed + index."""
    out = []
    t = 0.0
    for k in range(count):
        u = u01(base_seed, STREAM_SERVE, np.arange(4 * k, 4 * k + 4, dtype=np.uint64))
        t += -math.log1p(-float(u[0])) / rate_per_s
        n = sizes[min(int(u[1] * len(sizes)), len(sizes) - 1)]
        g = int(round(n ** 3 / cells_per_grain))
        g = max(grains_range[0], min(grains_range[1], g))
        lo, hi = steps_range
        steps = lo + min(int(u[2] * (hi - lo + 1)), hi - lo)
        out.append(Request(index=k, seed=base_seed + k, n=n, n_grains=g, steps=steps, arrival=t))
    return out
