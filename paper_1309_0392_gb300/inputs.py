"""Seeded synthetic grids shaped like the paper's workloads.

This module holds no hierarchization arithmetic: it only samples functions on
grid coordinates and draws seeded random numbers (numpy PCG64), in flat
storage order (dimension 0 contiguous).  Both the GPU tests and the oracle
tests take their inputs from here, so parity never depends on the generator.

A grid of level vector ``levels`` has ``2**l_k + 1`` points in dimension k and
coordinates ``x_k = i_k / 2**l_k`` on [0, 1] (boundary included).
"""
from __future__ import annotations

import numpy as np


def shape_of(levels):
    """numpy shape (n_{d-1}, ..., n_0); dimension 0 is the last (contiguous) axis."""
    return tuple(2 ** int(l) + 1 for l in reversed(list(levels)))


def num_points(levels) -> int:
    return int(np.prod([2 ** int(l) + 1 for l in levels], dtype=np.int64))


def coords(levels):
    """List of 1-D coordinate arrays, one per dimension (dimension 0 first)."""
    return [np.arange(2 ** int(l) + 1, dtype=np.float64) / float(2 ** int(l)) for l in levels]


def _broadcast(levels, k, v):
    """View the dimension-k vector v so it broadcasts over shape_of(levels)."""
    d = len(levels)
    shp = [1] * d
    shp[d - 1 - k] = v.shape[0]
    return v.reshape(shp)


def uniform(levels, seed, lo=-1.0, hi=1.0, dtype=np.float64):
    """u = uniform[lo, hi) from PCG64(seed), flat order."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, num_points(levels)).astype(dtype, copy=False)


def cfg1a():
    """2-D grid, level (5,5): uniform[-1,1] from seed 0."""
    return (5, 5), uniform((5, 5), 0)


def cfg1b():
    """2-D grid, level (5,5): u(x, y) = x^2 + 3xy (x = dimension 0)."""
    levels = (5, 5)
    x, y = coords(levels)
    u = _broadcast(levels, 0, x) ** 2 + 3.0 * _broadcast(levels, 0, x) * _broadcast(levels, 1, y)
    return levels, np.ascontiguousarray(u, dtype=np.float64).reshape(-1)


def cfg2(levels=(9, 9, 9), seed=1):
    """3-D grid: sin(2 pi x) exp(-y) (1 + z^2) + 1e-3 N(0, 1)."""
    x, y, z = coords(levels)
    f = (_broadcast(levels, 0, np.sin(2 * np.pi * x)) * _broadcast(levels, 1, np.exp(-y))
         * _broadcast(levels, 2, 1.0 + z * z))
    rng = np.random.default_rng(seed)
    u = f.reshape(-1) + 1e-3 * rng.standard_normal(num_points(levels))
    return levels, u


def cfg3(levels=(6, 6, 5, 5, 5), seed=2):
    """5-D grid: prod_k (1 + 0.5 cos(pi x_k)) + 1e-4 N(0, 1); returned in
    float64 (callers cast to float32 for the FP32 form)."""
    f = np.ones(shape_of(levels), dtype=np.float64)
    for k, x in enumerate(coords(levels)):
        f = f * _broadcast(levels, k, 1.0 + 0.5 * np.cos(np.pi * x))
    rng = np.random.default_rng(seed)
    u = f.reshape(-1) + 1e-4 * rng.standard_normal(num_points(levels))
    return levels, u


def scheme_grid(levels, grid_index):
    """One combination grid of the batched workload: uniform[-1,1] from seed
    1000 + grid index."""
    return uniform(levels, 1000 + int(grid_index))


def cfg5(batch=16, levels=(8, 8, 8), seed=5):
    """Differentiation workload: `batch` grids, uniform[-1,1] from one seed,
    returned as an array [batch, N]."""
    rng = np.random.default_rng(seed)
    return levels, rng.uniform(-1.0, 1.0, (batch, num_points(levels)))


def sample(levels, fn):
    """Sample a separable-or-not function fn(*coordinate arrays) on the grid
    (arguments broadcast in dimension order 0..d-1)."""
    args = [_broadcast(levels, k, x) for k, x in enumerate(coords(levels))]
    return np.ascontiguousarray(np.broadcast_to(fn(*args), shape_of(levels)),
                                dtype=np.float64).reshape(-1)
