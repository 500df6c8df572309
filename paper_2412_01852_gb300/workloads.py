"""Seeded synthetic inputs shaped like the paper's experiments.

This module only draws numbers: it holds none of the rotation arithmetic, and
it is the one module that both the CUDA path's callers and the CPU oracle's
tests take their inputs from.

Recipes (Section 8 experiments use random m = n matrices with k = 180; the
workloads below keep that shape family):

* ``matrix(m, n, seed)``      -- A with i.i.d. N(0,1) entries, column-major.
* ``rotations(n, k, seed)``   -- angles theta ~ U[0, 2*pi), C = cos(theta),
                                 S = sin(theta), each (n-1) x k column-major.
* ``batch_shapes(...)``       -- uneven instances: m log-uniform in [64, 4096],
                                 n log-uniform in [32, 2048], k uniform in [1, 96].
* ``serving_trace(...)``      -- Poisson arrivals of square problems with n drawn
                                 from {128, ..., 4096} with weights 1/n and k
                                 uniform in [2, 64].

Random draws use numpy's PCG64 generator seeded with the given integer; A and
the angles come from independent child streams so that the same seed gives the
same A whatever k is.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(seed, spawn_key=(stream,)))


def matrix(m: int, n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """m x n column-major matrix with i.i.d. N(0,1) entries."""
    g = _rng(seed, 0)
    # Draw as (n, m) in C order, which is (m, n) in Fortran order.
    a = g.standard_normal(size=(n, m))
    return np.asarray(a.T, dtype=dtype, order="F")


def angles(n: int, k: int, seed: int) -> np.ndarray:
    """(n-1) x k column-major angles, uniform in [0, 2*pi)."""
    g = _rng(seed, 1)
    t = g.uniform(0.0, TWO_PI, size=(k, max(n - 1, 0)))
    return np.asarray(t.T, order="F")


def rotations(n: int, k: int, seed: int, dtype=np.float64):
    """(C, S) = (cos theta, sin theta), each (n-1) x k column-major."""
    t = angles(n, k, seed)
    C = np.asarray(np.cos(t), dtype=dtype, order="F")
    S = np.asarray(np.sin(t), dtype=dtype, order="F")
    return C, S


def reflectors(n: int, k: int, seed: int):
    """(T, V) = (tau, nu) of 2x2 reflectors H = I - tau*v*v^T with v = (1, nu).

    nu = tan(phi) with phi uniform in [-pi/4, pi/4] and tau = 2 / (1 + nu^2),
    which makes every H orthogonal (up to the rounding of tau).
    """
    g = _rng(seed, 4)
    phi = g.uniform(-math.pi / 4, math.pi / 4, size=(k, max(n - 1, 0)))
    nu = np.tan(phi)
    tau = 2.0 / (1.0 + nu * nu)
    return np.asarray(tau.T, order="F"), np.asarray(nu.T, order="F")


def problem(m: int, n: int, k: int, seed: int, dtype=np.float64):
    """(A, C, S) for one instance."""
    A = matrix(m, n, seed, dtype)
    C, S = rotations(n, k, seed, dtype)
    return A, C, S


# Named workloads.  Sizes follow the paper's square m = n experiments.
WORKLOADS = {
    "plain-512": dict(m=512, n=512, k=16, seed=1),
    "plain-8192": dict(m=8192, n=8192, k=192, seed=2),
    # half-width instance of the same rows and sequences, used for profiler captures
    "plain-8192x4096": dict(m=8192, n=4096, k=192, seed=2),
    "precision-8192": dict(m=8192, n=8192, k=192, seed=2, nb=256, kb=64),
}


def batch_shapes(count: int = 512, seed: int = 4, m_range=(64, 4096), n_range=(32, 2048),
                 k_range=(1, 96)):
    """Uneven (m, n, k) triples: m, n log-uniform, k uniform (inclusive ranges)."""
    g = _rng(seed, 2)
    lm = g.uniform(math.log(m_range[0]), math.log(m_range[1]), size=count)
    ln = g.uniform(math.log(n_range[0]), math.log(n_range[1]), size=count)
    ks = g.integers(k_range[0], k_range[1] + 1, size=count)
    ms = np.floor(np.exp(lm)).astype(np.int64)
    ns = np.floor(np.exp(ln)).astype(np.int64)
    return [(int(a), int(b), int(c)) for a, b, c in zip(ms, ns, ks)]


SERVING_SIZES = (128, 256, 512, 1024, 2048, 4096)


@dataclass
class Request:
    arrival_s: float
    n: int
    k: int
    seed: int


def serving_trace(num: int, rate_per_s: float, seed: int = 5, sizes=SERVING_SIZES,
                  k_range=(2, 64)):
    """Poisson arrivals; n with probability proportional to 1/n; k uniform."""
    g = _rng(seed, 3)
    w = np.array([1.0 / s for s in sizes])
    w /= w.sum()
    gaps = g.exponential(1.0 / rate_per_s, size=num)
    t = np.cumsum(gaps)
    ns = g.choice(np.array(sizes), size=num, p=w)
    ks = g.integers(k_range[0], k_range[1] + 1, size=num)
    return [Request(float(t[i]), int(ns[i]), int(ks[i]), seed * 1000003 + i) for i in range(num)]


def rotation_rows(m: int, n: int, k: int) -> int:
    """Number of rotation-row updates (one rotation applied to one row)."""
    return int(m) * max(int(n) - 1, 0) * int(k)
