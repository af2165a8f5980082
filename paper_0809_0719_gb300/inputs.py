"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds random-number recipes only (none of the method's arithmetic).
The paper's workload is white-noise sources (Sec. 5): f(k) with real and
imaginary parts i.i.d. standard normal.  Error samples follow eq. err, a seeded
random subset of the output grid.
"""
from __future__ import annotations

import numpy as np


def gaussian_sources(N: int, seed: int) -> np.ndarray:
    """(N, N) complex128 white noise; element [k1+N/2, k2+N/2] is f(k1, k2).

    Drawn as re = standard_normal((N, N)) then im = standard_normal((N, N)) from
    numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((N, N))
    im = rng.standard_normal((N, N))
    return re + 1j * im


def gaussian_batch(N: int, seeds) -> np.ndarray:
    """(R, N, N) complex128, one gaussian_sources() per seed."""
    return np.stack([gaussian_sources(N, int(s)) for s in seeds])


def sample_indices(N: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct flat grid indices (i1*N + i2) drawn without replacement."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N * N, size=min(count, N * N), replace=False)).astype(np.int64)
