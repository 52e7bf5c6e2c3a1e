"""Seeded synthetic inputs shared by the tests, the benchmark and the
serving loop.  This module holds no arithmetic of the method itself: it only
draws initial states and request streams from numpy generators.

State arrays are float64 of shape (7, nz, ny, nx), x fastest, field order
ln rho, u_x, u_y, u_z, A_x, A_y, A_z.
"""
from __future__ import annotations

import math

import numpy as np


def seed_field_state(nx: int, ny: int | None = None, nz: int | None = None,
                     seed: int = 0, amp: float = 1e-5) -> np.ndarray:
    """Initial condition of Sec. 4: uniform density (ln rho = 0), u = 0 and a
    weak delta-correlated Gaussian vector potential A ~ amp * N(0, 1)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    q = np.zeros((7, nz, ny, nx))
    q[4:7] = amp * rng.standard_normal((3, nz, ny, nx))
    return q


def uniform_state(nx: int, ny: int | None = None, nz: int | None = None,
                  seed: int = 0, lo: float = 0.0, hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    """All seven fields uniform in [lo, hi): the benchmark state of App. A."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    if np.dtype(dtype) == np.float64:
        return rng.uniform(lo, hi, size=(7, nz, ny, nx))
    q = rng.random(size=(7, nz, ny, nx), dtype=np.dtype(dtype))
    q *= np.asarray(hi - lo, dtype=dtype)
    q += np.asarray(lo, dtype=dtype)
    return q


def random_modes_state(nx: int, ny: int | None = None, nz: int | None = None,
                       seed: int = 0, amp: float = 0.1, kmax: int = 3,
                       nmodes: int = 6) -> np.ndarray:
    """Smooth random state: each field is a sum of nmodes plane waves with
    integer wave vectors |k_i| <= kmax, random amplitudes and phases."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * (2 * math.pi / nx)
    y = np.arange(ny) * (2 * math.pi / ny)
    z = np.arange(nz) * (2 * math.pi / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    q = np.zeros((7, nz, ny, nx))
    for f in range(7):
        for _ in range(nmodes):
            k = rng.integers(-kmax, kmax + 1, size=3)
            a = amp * rng.standard_normal() / math.sqrt(nmodes)
            ph = rng.uniform(0, 2 * math.pi)
            q[f] += a * np.cos(k[0] * X + k[1] * Y + k[2] * Z + ph)
    return q


def noise_state(nx: int, ny: int | None = None, nz: int | None = None,
                seed: int = 0, amp: float = 0.05) -> np.ndarray:
    """Delta-correlated Gaussian noise of amplitude amp in every field
    (grid-scale structure that exercises every stencil point)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((7, nz, ny, nx))


def serving_requests(n: int = 200, seed: int = 2025, rate: float = 1.0,
                     grids=(64, 96, 128, 192, 256), rem=(10.0, 250.0),
                     steps=(500, 5000)) -> list[dict]:
    """Poisson stream of dynamo-run requests: exponential inter-arrival
    times of mean 1/rate, grid uniform over `grids`, Re_M log-uniform over
    `rem`, helicity sigma in {0, 1}, a uniform integer step budget, and a
    per-request seed for the initial field and the forcing."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        out.append(dict(
            id=i,
            arrival=t,
            n=int(rng.choice(grids)),
            re_m=float(math.exp(rng.uniform(math.log(rem[0]), math.log(rem[1])))),
            sigma=float(rng.integers(0, 2)),
            steps=int(rng.integers(steps[0], steps[1] + 1)),
            seed=int(rng.integers(0, 2**62)),
        ))
    return out


def _splitmix64(key: int, ctr: np.ndarray) -> np.ndarray:
    """Output ctr of the SplitMix64 stream keyed by key (Steele, Lea & Flood
    2014), vectorised on uint64 with wrap-around arithmetic."""
    with np.errstate(over="ignore"):
        z = np.uint64(key & 0xFFFFFFFFFFFFFFFF) + (ctr + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_seed_field_state(nx: int, ny: int | None = None, nz: int | None = None,
                             seed: int = 0, amp: float = 1e-5) -> np.ndarray:
    """The initial state that mhd_set_seed_field generates on the device,
    built on the host from the same published generators: ln rho = 0, u = 0,
    A = amp * N(0,1) with normal n = c * npts + e by Box-Muller from SplitMix64
    outputs 2n, 2n + 1 of the stream keyed by seed."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    npts = nx * ny * nz
    g = _counter_normals(seed, np.arange(3 * npts, dtype=np.uint64))
    q = np.zeros((7, nz, ny, nx))
    q[4:7] = amp * g.reshape(3, nz, ny, nx)
    return q


def _counter_normals(seed: int, n: np.ndarray) -> np.ndarray:
    """Normal number n of the seed-field stream: Box-Muller of SplitMix64
    outputs 2n and 2n + 1 (53-bit uniforms, the first shifted off zero)."""
    n = n.astype(np.uint64)
    u1 = ((_splitmix64(seed, np.uint64(2) * n) >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (_splitmix64(seed, np.uint64(2) * n + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def counter_seed_field_at(nx: int, ny: int, nz: int, i, j, k, seed: int = 0, amp: float = 1e-5) -> np.ndarray:
    """A = (A_x, A_y, A_z) of the device seed field (counter_seed_field_state)
    at grid points (i, j, k), periodic indexes allowed: array (3, len(i)).
    Lets a test rebuild any neighbourhood of a grid too large for the host."""
    i, j, k = (np.asarray(v, dtype=np.int64) for v in (i, j, k))
    e = ((k % nz) * ny + (j % ny)) * nx + (i % nx)
    npts = nx * ny * nz
    return np.stack([amp * _counter_normals(seed, c * npts + e) for c in range(3)])
