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


ELLIPSE_16 = ("ellipse", (2.0, 1.0, 16.0, 1.0))  # c1, c2 = (2 + sin sin)/16, (2 + cos cos)/16
CIRCLE_20 = ("circle", (3.0, 1.0, 20.0, 1.0))    # c = (3 + sin sin)/20


def uneven_batch_specs(count: int = 96, seed: int = 4) -> list[dict]:
    """Plans of the uneven-batch workload, one dict {N, q, nrhs, phase, params} each.

    For plan i, N is drawn from (64, 128, 256, 512), then q from (5, 7, 9), then
    nrhs from 1..8, all with numpy.random.default_rng(seed) in that order; the
    phase alternates between the ellipse phase (even i) and the c(x)|k| phase
    (odd i)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        N = int(rng.choice([64, 128, 256, 512]))
        q = int(rng.choice([5, 7, 9]))
        nrhs = int(rng.integers(1, 9))
        phase, params = ELLIPSE_16 if i % 2 == 0 else CIRCLE_20
        specs.append({"N": N, "q": q, "nrhs": nrhs, "phase": phase, "params": params})
    return specs


def uneven_batch_sources(spec: dict, index: int) -> np.ndarray:
    """(nrhs, N, N) complex128 sources of plan `index`: gaussian_sources(N, 10000 + 100 index + r)."""
    return gaussian_batch(spec["N"], [10000 + 100 * index + r for r in range(spec["nrhs"])])
