"""Seeded synthetic inputs for the SPFC solver and its CPU oracle.

This module is the only code shared by the CUDA path's tests/bench and the
oracle. It holds none of the numerical method: it only turns a seed into
random numbers and lays them out as initial fields or run parameters.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a counter-based generator. Output
number ``i`` (0-based) of the stream with seed ``s`` is the SplitMix64
finaliser applied to ``s + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64)``, which
is exactly the i-th value the sequential generator returns after being seeded
with ``s``. A uniform double in [0, 1) is ``(x >> 11) * 2^-53``.

Field layout: row-major with x fastest, i.e. a numpy array of shape
``(Ny, Nx)`` in 2D and ``(Nz, Ny, Nx)`` in 3D; grid point with flat index
``j`` receives stream value ``j``.

The paper draws its initial data as ``0.05 * (2 r - 1)`` with ``r`` uniform in
[0, 1] (Sec. 5.2); the workloads here use ``mean + amp * U(-1, 1)`` with the
same construction ``U = 2 r - 1``.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Return stream values ``start .. start+count-1`` of seed ``seed`` (uint64)."""
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from stream values ``start ..`` of ``seed``."""
    x = splitmix64(seed, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def noisy_field(shape, mean: float, amp: float, seed: int) -> np.ndarray:
    """``mean + amp * U(-1, 1)`` per grid point, float64, x fastest."""
    shape = tuple(int(s) for s in shape)
    count = int(np.prod(shape))
    u = 2.0 * uniform01(seed, 0, count) - 1.0
    return (mean + amp * u).reshape(shape)


# --- workload recipes -------------------------------------------------------

def small_2d_case():
    """2D 64x64 on [0,32]^2, eps=0.1, beta=1, dt=0.01, phi0 = 0.2 + 0.05 U, seed 0."""
    n = 64
    return dict(d=2, n=n, L=32.0, eps=0.1, beta=1.0, dt=0.01,
                phi0=noisy_field((n, n), 0.2, 0.05, 0))


def crystal_2d_case(n: int = 512):
    """2D square-lattice crystallisation: N=512 on [0,256]^2, eps=0.25, beta=1,
    dt=0.05, phi0 = 0.2 + 0.02 U from seed 1 (h = 0.5; ``n`` may shrink it
    for tests with L = n/2)."""
    return dict(d=2, n=n, L=0.5 * n, eps=0.25, beta=1.0, dt=0.05,
                phi0=noisy_field((n, n), 0.2, 0.02, 1))


def cube_3d_case(n: int = 128):
    """3D SPFC: N=128 on [0,64]^3, eps=0.2, beta=1, dt=0.02,
    phi0 = 0.15 + 0.05 U from seed 2 (h = 0.5)."""
    return dict(d=3, n=n, L=0.5 * n, eps=0.2, beta=1.0, dt=0.02,
                phi0=noisy_field((n, n, n), 0.15, 0.05, 2))


ENSEMBLE_SIZES = (64, 128, 256, 512)


def ensemble_run(i: int, sizes=ENSEMBLE_SIZES, first_seed: int = 100):
    """Run ``i`` of the batched 2D ensemble.

    Seed ``first_seed + i``; grid ``sizes[i % len(sizes)]`` squared with
    L = N/2; the field uses stream values ``0 .. N^2-1`` (amp 0.05 around the
    drawn mean) and the next three values give eps ~ U[0.05, 0.35],
    beta ~ U[0.5, 1.5] and the mean ~ U[0.1, 0.3], in that order.
    """
    seed = first_seed + i
    n = int(sizes[i % len(sizes)])
    p = n * n
    e, b, m = uniform01(seed, p, 3)
    eps = 0.05 + 0.30 * e
    beta = 0.5 + 1.0 * b
    mean = 0.1 + 0.2 * m
    u = 2.0 * uniform01(seed, 0, p) - 1.0
    phi0 = (mean + 0.05 * u).reshape(n, n)
    return dict(d=2, n=n, L=0.5 * n, eps=float(eps), beta=float(beta),
                dt=0.02, mean=float(mean), seed=seed, phi0=phi0)


SURROGATE_TRAIN_SEED = 1000
SURROGATE_HELD_OUT_SEED = 9000


def surrogate_run(i: int, n: int = 256, held_out: bool = False):
    """Run ``i`` of the surrogate's training set (seeds 1000 + i) or of its
    held-out evaluation set (seeds 9000 + i): the ensemble recipe on one grid
    size (L = N/2, dt = 0.02)."""
    first = SURROGATE_HELD_OUT_SEED if held_out else SURROGATE_TRAIN_SEED
    return ensemble_run(i, sizes=(n,), first_seed=first)
