"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the solver: only the counter-based
SplitMix64 generator (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014; public-domain reference constants) and the
recipes that turn its output into right-hand sides, per-element viscosities
and the batched problem list.

Recipes
-------
* RHS entry ``i`` of right-hand side ``r`` of problem ``p`` under ``seed``:
  ``2*u - 1`` with ``u = (mix64(s + (i+1)*GAMMA) >> 11) * 2**-53`` and
  ``s = stream_seed(seed, p, r)``: i.i.d. uniform on [-1, 1).
* Per-element viscosity ``nu_e = exp(g)``, ``g ~ N(0, 1)`` by Box-Muller from
  two uniforms of the stream ``stream_seed(seed, 1_000_003, 0)`` (lognormal(0,1)).
* Batched problem ``p``: side length ``16*round(exp(ln 64 + u*ln 8)/16)``
  (log-uniform in [64, 512], rounded to a multiple of 16) and
  ``dt = exp(ln 1e-6 + u'*ln 1e5)`` (log-uniform in [1e-6, 1e-1]).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (uint64 in, uint64 out, wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_seed(seed: int, p: int = 0, r: int = 0) -> np.uint64:
    """Start state of the stream for (seed, problem p, right-hand side r)."""
    s = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    key = np.uint64(((p & 0xFFFFFFFF) << 32) | (r & 0xFFFFFFFF))
    return mix64(s ^ key)


def uniform01(seed: int, count: int, p: int = 0, r: int = 0) -> np.ndarray:
    """``count`` doubles uniform on [0, 1) with 53 random bits each."""
    s = stream_seed(seed, p, r)
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = mix64(s + i * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rhs(seed: int, count: int, p: int = 0, r: int = 0) -> np.ndarray:
    """Right-hand side, i.i.d. uniform on [-1, 1), float64."""
    return 2.0 * uniform01(seed, count, p, r) - 1.0


def nu_elements(seed: int, n_elem: int) -> np.ndarray:
    """Per-element viscosity lognormal(0, 1), Box-Muller on the host."""
    u = uniform01(seed, 2 * n_elem, p=1_000_003, r=0)
    u1 = 1.0 - u[0::2]  # (0, 1]: log is finite
    u2 = u[1::2]
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return np.exp(g)


def batched_problems(seed: int, nprob: int = 64):
    """List of (n, dt) for the batched workload: n log-uniform in [64, 512]
    rounded to a multiple of 16, dt log-uniform in [1e-6, 1e-1]."""
    u = uniform01(seed, 2 * nprob, p=2_000_003, r=0)
    out = []
    for p in range(nprob):
        side = math.exp(math.log(64.0) + u[2 * p] * math.log(8.0))
        n = int(16 * round(side / 16.0))
        n = min(512, max(64, n))
        dt = math.exp(math.log(1e-6) + u[2 * p + 1] * math.log(1e5))
        out.append((n, dt))
    return out
