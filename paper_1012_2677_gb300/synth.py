"""Seeded synthetic input generators shared by the tests, the bench and the oracle runs.

This module holds none of the method's arithmetic (no potential, no forces, no
integration, no cell grid): only seeded random draws and the shapes of the
workloads (random directions, displacements, subsets, replica parameters).
Random numbers that the method itself needs are passed in from here as inputs.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def unit_vectors(n: int, seed: int) -> np.ndarray:
    """n random directions, uniform on the sphere, float64 (n, 3)."""
    u = rng(seed).normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def displacements(n: int, amplitude: float, seed: int) -> np.ndarray:
    """Uniform random displacements in [-amplitude, amplitude]^3, float64 (n, 3)."""
    return rng(seed).uniform(-amplitude, amplitude, size=(n, 3))


def uniform_positions(n: int, L: float, seed: int) -> np.ndarray:
    """n positions uniform in the periodic box [0, L)^3."""
    x = rng(seed).uniform(0.0, L, size=(n, 3))
    return np.where(x >= L, 0.0, x)


def gaussian(shape, seed: int) -> np.ndarray:
    return rng(seed).normal(size=shape)


def subset(n_total: int, n_keep: int, seed: int) -> np.ndarray:
    """Sorted random subset of range(n_total) of size n_keep (thinning a filled lattice)."""
    return np.sort(rng(seed).choice(n_total, size=n_keep, replace=False))


def replica_table(R: int, seed: int, n_range=(500, 50000), rho_range=(0.3, 0.9), T_range=(0.7, 1.5)):
    """Per-replica (N, rho, T) drawn uniformly: the batched-replica workload shape."""
    g = rng(seed)
    N = g.integers(n_range[0], n_range[1] + 1, size=R)
    rho = g.uniform(*rho_range, size=R)
    T = g.uniform(*T_range, size=R)
    return N.astype(np.int64), rho, T


def dyadic(x, bits: int = 40) -> np.ndarray:
    """Round values to multiples of 2^-bits, so that adding a power-of-two offset up to
    2^(52 - bits) is exact (inputs then survive any offset storage bit for bit)."""
    s = float(2 ** bits)
    return np.round(np.asarray(x, dtype=np.float64) * s) / s


def fcc_thinned(N: int, rho: float, seed: int):
    """Positions of N particles in a cubic box of side L = (N / rho)^(1/3): an FCC lattice of
    M = ceil((N / 4)^(1/3)) cells of side L / M with a seeded random N-subset of its 4 M^3 sites
    kept.  Returns (x[N, 3], L)."""
    L = (N / rho) ** (1.0 / 3.0)
    M = int(np.ceil((N / 4.0) ** (1.0 / 3.0)))
    a = L / M
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    g = np.arange(M)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 1, 3)
    sites = ((cells + basis[None]) * a).reshape(-1, 3)
    keep = subset(len(sites), N, seed)
    return sites[keep].copy(), L


def thermal_velocities(N: int, T: float, seed: int) -> np.ndarray:
    """Seeded Gaussian velocities with the mean removed and sum v^2 = 3 (N - 1) T."""
    v = gaussian((N, 3), seed)
    v -= v.mean(0)
    return v * np.sqrt(3.0 * (N - 1) * T / (v ** 2).sum())


def batch_workload(R: int, seed: int, n_range=(500, 50000)):
    """The batched-replica workload: R replicas with (N, rho, T) from replica_table, FCC-thinned
    positions and thermal velocities (replica seeds seed + r).  Returns (n[R], box[R], x[sum n, 3],
    v[sum n, 3], T[R])."""
    n, rho, T = replica_table(R, seed, n_range=n_range)
    xs, vs, box = [], [], []
    for r in range(R):
        x, L = fcc_thinned(int(n[r]), float(rho[r]), seed + r)
        xs.append(x)
        vs.append(thermal_velocities(int(n[r]), float(T[r]), seed + 7919 + r))
        box.append(L)
    return n, np.array(box), np.concatenate(xs), np.concatenate(vs), T
