"""Seeded synthetic inputs for hypercube convolution.

This module is shared by the tests, the benchmark and the oracle checks.  It
generates inputs only and contains none of the convolution arithmetic.  All
draws use numpy's PCG64 (``numpy.random.default_rng(seed)``).

Layout: a hypercube over {0,1}^D is a flat array of 2^D values, row-major,
axis 1 the slowest (the first half of the array is x[0, ...]).

Workloads (sizes and distributions of the paper's use cases):

* ``uniform_int``   -- iid integers, inclusive range [lo, hi] (int64 exact mode).
* ``prob_exponential`` -- iid Exponential(1), divided by the sum: a probability
  mass function over {0,1}^D (the paper's motivating use, PMFs of sums of
  Bernoulli-axis random vectors).
* ``prob_separable`` -- a product PMF x[i] = prod_d a_d[i_d] with each
  (a_d[0], a_d[1]) ~ Dirichlet(1, 1); returns the per-axis factors too.
* ``uniform01``     -- iid U[0, 1).
* ``normal``        -- iid N(0, 1).
* ``paper_accuracy`` -- the Results-section accuracy input x.flat = [1, 2, ..., 2^D].
* ``batched_dims``  -- D for each instance of the batched workload, iid U{lo..hi}.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_int(D: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return rng(seed).integers(lo, hi + 1, size=1 << D, dtype=np.int64)


def uniform_int_pair(D: int, lo: int, hi: int, seed: int):
    g = rng(seed)
    x = g.integers(lo, hi + 1, size=1 << D, dtype=np.int64)
    y = g.integers(lo, hi + 1, size=1 << D, dtype=np.int64)
    return x, y


def prob_exponential_pair(D: int, seed: int):
    g = rng(seed)
    x = g.exponential(1.0, size=1 << D)
    y = g.exponential(1.0, size=1 << D)
    return x / x.sum(), y / y.sum()


def separable_factors(D: int, seed: int, kind: str = "dirichlet"):
    """Per-axis pairs a[d] = (a_d[0], a_d[1]) for d = 0..D-1 (axis 1 first)."""
    g = rng(seed)
    if kind == "dirichlet":
        u = g.random(D)
        return np.stack([u, 1.0 - u], axis=1)
    if kind == "int":
        return g.integers(-3, 4, size=(D, 2), dtype=np.int64)
    raise ValueError(kind)


def outer_product_cube(factors: np.ndarray) -> np.ndarray:
    """x[i] = prod_d factors[d][bit_d(i)], axis 1 (d = 0) most significant."""
    x = np.ones(1, dtype=factors.dtype)
    for d in range(factors.shape[0]):
        x = np.kron(x, factors[d])
    return x


def prob_separable_pair(D: int, seed: int):
    a = separable_factors(D, seed, "dirichlet")
    b = separable_factors(D, seed + 1, "dirichlet")
    return outer_product_cube(a), outer_product_cube(b), a, b


def uniform01_pair(D: int, seed: int, dtype=np.float32):
    g = rng(seed)
    return g.random(1 << D).astype(dtype), g.random(1 << D).astype(dtype)


def normal(shape_or_n, seed: int, dtype=np.float32) -> np.ndarray:
    return rng(seed).standard_normal(shape_or_n).astype(dtype)


def normal_pair(D: int, seed: int, dtype=np.float32):
    g = rng(seed)
    return (g.standard_normal(1 << D).astype(dtype), g.standard_normal(1 << D).astype(dtype))


def paper_accuracy(D: int, dtype=np.float64) -> np.ndarray:
    return np.arange(1, (1 << D) + 1).astype(dtype)


def batched_dims(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    return rng(seed).integers(lo, hi + 1, size=n).astype(np.int64)


def batched_uniform01(dims, seed: int, dtype=np.float32):
    """One (x, y) pair per instance, drawn in instance order from one stream."""
    g = rng(seed)
    out = []
    for D in dims:
        n = 1 << int(D)
        out.append((g.random(n).astype(dtype), g.random(n).astype(dtype)))
    return out


def dyadic(v: np.ndarray, bits: int) -> np.ndarray:
    """round(v * 2^bits) as int64: inputs that are exact in binary32/binary64
    once divided by 2^bits, so the int64 oracle gives the exact real result."""
    return np.rint(np.asarray(v, dtype=np.float64) * float(1 << bits)).astype(np.int64)
