"""Seeded synthetic inputs for the Legendre<->Chebyshev transforms.

This module holds only random-number recipes (no transform arithmetic).  It
is the one piece shared by the CPU oracle's users (tests, bench CPU leg) and
the GPU path's users, so that both see the same arrays.

The paper measures on random coefficient vectors that decay like j^{-r}
(Sec. 5, "Accuracy"): uniform draws scaled by a power of (j+1).  The
workloads below follow that recipe with seeded PCG64 generators
(numpy.random.default_rng), all in float64:

  uniform_vector      U[-1, 1], seed 0, n = 1024                 (plain FP64 check)
  decaying_vector     N(0,1) * (j+1)^-r                          (n = 1e6, r = 1, seed 1)
  sample_rows         rows 0, 1, n-2, n-1 plus distinct uniform rows (seed 10001)
  ragged_lengths      n_i = round(exp(U(ln 64, ln 65536))), seed 2
  ragged_batch        N(0,1) * (j+1)^-1/2 per member, seed 3
  cube                N(0,1) / ((i+1)(j+1)(k+1)), seed 4
  fit_pair            x, y ~ N(0,1) * (j+1)^-1, seeds 5 and 6
"""
from __future__ import annotations

import numpy as np


def uniform_vector(n: int = 1024, seed: int = 0) -> np.ndarray:
    """n i.i.d. U[-1, 1] float64 coefficients."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def decaying_vector(n: int, seed: int = 1, r: float = 1.0, batch: int | None = None) -> np.ndarray:
    """N(0,1) * (j+1)^-r, shape (n,) or (batch, n)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if batch is None else (batch, n)
    x = rng.standard_normal(shape)
    return x * (np.arange(1, n + 1, dtype=np.float64) ** (-r))


def sample_rows(n: int, count: int = 4096, seed: int = 10001) -> np.ndarray:
    """Sorted distinct output rows: 0, 1, n-2, n-1 and count-4 uniform others."""
    fixed = np.unique(np.array([0, 1, max(n - 2, 0), n - 1], np.int64))
    if n <= count:
        return np.arange(n, dtype=np.int64)
    rng = np.random.default_rng(seed)
    others = np.setdiff1d(np.arange(n, dtype=np.int64), fixed)
    pick = rng.choice(others, size=count - fixed.size, replace=False)
    return np.sort(np.concatenate([fixed, pick]).astype(np.int64))


def ragged_lengths(count: int = 4096, lo: int = 64, hi: int = 65536, seed: int = 2) -> np.ndarray:
    """Log-uniform lengths in [lo, hi]."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)
    return np.clip(n, lo, hi)


def ragged_batch(lengths, seed: int = 3, r: float = 0.5) -> np.ndarray:
    """Concatenation of members N(0,1) * (j+1)^-r, member i of length lengths[i]."""
    lengths = np.asarray(lengths, np.int64)
    rng = np.random.default_rng(seed)
    total = int(lengths.sum())
    x = rng.standard_normal(total)
    offs = np.concatenate([[0], np.cumsum(lengths)])
    for i in range(lengths.size):
        a, b = offs[i], offs[i + 1]
        x[a:b] *= np.arange(1, b - a + 1, dtype=np.float64) ** (-r)
    return x


def ragged_offsets(lengths) -> np.ndarray:
    """Exclusive prefix sum of lengths (int64, size count+1)."""
    return np.concatenate([[0], np.cumsum(np.asarray(lengths, np.int64))]).astype(np.int64)


def cube(n: int = 512, seed: int = 4) -> np.ndarray:
    """n^3 float64 array N(0,1) / ((i+1)(j+1)(k+1)), C order."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, n, n))
    w = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    x *= w[:, None, None]
    x *= w[None, :, None]
    x *= w[None, None, :]
    return x


def fit_pair(n: int = 65536, batch: int = 256, seeds=(5, 6)):
    """(x, y), each (batch, n) N(0,1) * (j+1)^-1."""
    return (decaying_vector(n, seeds[0], 1.0, batch), decaying_vector(n, seeds[1], 1.0, batch))
