"""Seeded synthetic workloads (parameters only; no simulation arithmetic).

The method's inputs are lattice parameters: dimension, linear size L, inverse
temperature beta, a 64-bit seed and a start state.  This module turns the
benchmark workloads into concrete parameter lists from fixed numpy seeds.  It
is the one module that both the engine's tests/benchmarks and the oracle-side
checks read, and it holds none of the Ising arithmetic.

The temperatures bracket the exact critical points: 2D beta_c = ln(1+sqrt2)/2
= 0.4406868 (Onsager) and the 3D cubic estimate 0.2216544.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HOT, COLD_UP, COLD_DOWN = 0, 1, 2
INT8, BITPACK, AUTO = 0, 1, 2

BETA_C_2D = 0.4406868
BETA_C_3D = 0.2216544
BASE_SEED = 20031109


@dataclass
class LatticeSpec:
    dims: int
    L: int
    beta: float
    seed: int
    start: int = HOT
    sweeps: int = 1
    measure_every: int = 1
    layout: int = INT8

    @property
    def sites(self) -> int:
        return self.L ** self.dims


def critical_2d_small() -> LatticeSpec:
    """2D L=64 at beta_c, hot start, 1000 sweeps, E/M every sweep."""
    return LatticeSpec(2, 64, BETA_C_2D, BASE_SEED, HOT, 1000, 1, INT8)


def beta_scan_2d(L: int = 8192, sweeps: int = 2000, layout: int = INT8) -> list:
    """16 betas evenly spaced in [0.30, 0.60], cold start, seeds BASE_SEED + j."""
    return [LatticeSpec(2, L, round(0.30 + 0.02 * j, 10), BASE_SEED + j, COLD_UP,
                        sweeps, 1, layout) for j in range(16)]


def critical_3d(L: int = 256, sweeps: int = 1000, layout: int = INT8) -> LatticeSpec:
    """3D L=256 near beta_c, hot start, 1000 sweeps, E/M every 10 sweeps."""
    return LatticeSpec(3, L, BETA_C_3D, BASE_SEED, HOT, sweeps, 10, layout)


def _even_round(x: float) -> int:
    return max(2, int(2 * round(x / 2.0)))


def batched_mix(n: int = 2048, sweeps: int = 500, seed: int = 0) -> list:
    """Independent lattices: 70% 2D with L log-uniform in [16, 1024] and beta
    uniform in [0.2, 0.6]; 30% 3D with L log-uniform in [8, 128] and beta
    uniform in [0.15, 0.30]; L rounded to the nearest even integer; hot start;
    seeds 1000 + j; E/M recorded every 10 sweeps."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        if rng.uniform() < 0.7:
            L = _even_round(math.exp(rng.uniform(math.log(16), math.log(1024))))
            beta = float(rng.uniform(0.2, 0.6))
            dims = 2
        else:
            L = _even_round(math.exp(rng.uniform(math.log(8), math.log(128))))
            beta = float(rng.uniform(0.15, 0.30))
            dims = 3
        out.append(LatticeSpec(dims, L, beta, 1000 + j, HOT, sweeps, 10, AUTO))
    return out


@dataclass
class Job:
    job_id: int
    arrival_s: float
    spec: LatticeSpec


def poisson_jobs(n: int = 2000, rate_per_s: float = 200.0, seed: int = 1,
                 l2d=(32, 4096), l3d=(16, 256), sweeps=(100, 20000),
                 measure_every: int = 10) -> list:
    """Poisson job stream: dims uniform in {2, 3}; L log-uniform (2D 32-4096,
    3D 16-256) rounded to even; beta uniform within +-0.05 of the critical
    point; sweeps log-uniform in [100, 20000]; measure every 10 sweeps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for j in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        dims = 2 if rng.uniform() < 0.5 else 3
        lo, hi = l2d if dims == 2 else l3d
        L = _even_round(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        bc = BETA_C_2D if dims == 2 else BETA_C_3D
        beta = float(rng.uniform(bc - 0.05, bc + 0.05))
        nsw = int(round(math.exp(rng.uniform(math.log(sweeps[0]), math.log(sweeps[1])))))
        out.append(Job(j, t, LatticeSpec(dims, L, beta, 5000 + j, HOT, nsw,
                                         measure_every, AUTO)))
    return out


def demon_field(n: int, qmax: int = 3, beta: float = 0.5, seed: int = BASE_SEED) -> np.ndarray:
    """Initial demons for the deterministic (demon) dynamics: n values in
    0..qmax drawn independently with weights exp(-4 beta q), i.e. demons at
    inverse temperature beta (a demon of level q holds energy 4q).  uint8."""
    rng = np.random.default_rng(seed)
    w = np.exp(-4.0 * beta * np.arange(qmax + 1))
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    out = np.empty(n, dtype=np.uint8)
    chunk = 1 << 24
    for i in range(0, n, chunk):
        m = min(chunk, n - i)
        out[i:i + m] = np.searchsorted(cdf, rng.random(m), side="right")
    return out
