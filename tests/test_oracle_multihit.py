"""Pins of the oracle's multi-hit Metropolis rule (CPU only).

Multi-hit: each visited site takes several successive Metropolis trials with
its neighbours fixed (trial m draws Philox(seed; h>>2, t, c + 2m, 0)[h&3]).
Pins: one hit is the Metropolis pass itself; the exact multi-hit transition
matrices on 2x2 and 2x2x2 (each site a two-state chain taken `hits` steps)
keep Boltzmann stationary; the oracle's empirical transition frequencies
match them; a dE = 0 site flips iff the number of hits is odd; zero
temperature never raises E; equilibrium against enumeration.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact


def test_one_hit_is_metropolis(orc):
    for dims, L in ((2, 10), (3, 6)):
        thr = orc.thresholds(dims, 0.37)
        s = orc.init(dims, L, 4, oracle.HOT)
        a, b = s.copy(), s.copy()
        for t in range(5):
            for c in (0, 1):
                orc.half_sweep(dims, L, a, 4, thr, t, c)
                orc.half_sweep_multihit(dims, L, b, 4, thr, t, c, 1)
        assert np.array_equal(a, b)
        s1, E1, M1 = orc.run(dims, L, 0.37, 4, 5)
        s2, E2, M2 = orc.run_multihit(dims, L, 0.37, 4, 5, hits=1)
        assert np.array_equal(s1, s2) and np.array_equal(E1, E2) and np.array_equal(M1, M2)


def test_more_hits_change_the_chain(orc):
    s3, _, _ = orc.run_multihit(2, 16, 0.4, 9, 6, hits=3)
    s1, _, _ = orc.run(2, 16, 0.4, 9, 6)
    assert not np.array_equal(s1, s3)


@pytest.mark.parametrize("dims,L,beta,hits", [(2, 2, 0.3, 2), (2, 2, 0.9, 3), (3, 2, 0.2216544, 4)])
def test_multihit_matrices_preserve_boltzmann(orc, dims, L, beta, hits):
    thr = orc.thresholds(dims, beta)
    pi = exact.boltzmann_vector(dims, L, beta)
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thr, colour, hits=hits)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
        # each trial's accept probability is below exp(-beta dE) by < 2^-32;
        # hits trials per site, N/2 sites: relative error < hits N/2 / thr_min
        rtol = 1.05 * hits * (L ** dims / 2) / float(min(v for v in thr[:dims] if v > 0)) + 1e-12
        F = pi[:, None] * P
        assert np.allclose(F, F.T, rtol=rtol, atol=1e-15)
        assert np.allclose(pi @ P, pi, rtol=rtol, atol=1e-15)


@pytest.mark.parametrize("dims,L,beta,hits,n_draws", [(2, 2, 0.35, 2, 3000), (3, 2, 0.2, 3, 400)])
def test_multihit_transition_frequencies(orc, dims, L, beta, hits, n_draws):
    thr = orc.thresholds(dims, beta)
    n = L ** dims
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thr, colour, hits=hits)
        C = np.zeros_like(P)
        for a in range(2 ** n):
            s0 = exact.state_spins(a, n).astype(np.int8)
            for t in range(n_draws):
                s = s0.copy()
                orc.half_sweep_multihit(dims, L, s, 55, thr, t, colour, hits)
                C[a, exact.spins_state(s)] += 1
        assert np.all(C[P == 0] == 0)
        freq = C / n_draws
        sig = np.sqrt(P * (1 - P) / n_draws) + 1e-12
        assert np.all(np.abs(freq - P) <= 5 * sig + 1.0 / n_draws)


def test_level_sites_flip_on_odd_hits(orc):
    """A site with dE = 0 (as many agreeing as disagreeing neighbours) flips
    on every trial, so it ends flipped iff the number of hits is odd."""
    L = 4
    # black sites of a 2D stripe pattern: rows alternate +1/-1, so every site
    # has two agreeing (x) and two disagreeing (y) neighbours: k = 0
    y = np.arange(L * L) // L
    s0 = np.where(y % 2 == 0, 1, -1).astype(np.int8)
    thr = orc.thresholds(2, 0.5)
    black = ((np.arange(L * L) % L) + y) % 2 == 0
    for hits in (1, 2, 3, 4):
        s = s0.copy()
        orc.half_sweep_multihit(2, L, s, 1, thr, 0, 0, hits)
        assert np.array_equal(s[black], s0[black] * (-1) ** hits)
        assert np.array_equal(s[~black], s0[~black])


def test_zero_temperature_never_raises_energy(orc):
    s = orc.init(2, 24, 2, oracle.HOT)
    thr = orc.thresholds(2, math.inf)
    e_prev = orc.energy(2, 24, s)
    for t in range(20):
        for c in (0, 1):
            orc.half_sweep_multihit(2, 24, s, 2, thr, t, c, 3)
        e = orc.energy(2, 24, s)
        assert e <= e_prev
        e_prev = e


@pytest.mark.parametrize("dims,L,beta,hits", [(2, 4, exact.BETA_C_2D, 3), (3, 2, 0.2216544, 2)])
def test_multihit_vs_enumeration(orc, dims, L, beta, hits):
    hist = orc.enumerate_states(dims, L)
    want = exact.boltzmann_averages(hist, dims, L, beta)
    _, E, M = orc.run_multihit(dims, L, beta, 4444, 150_000, hits=hits)
    E = E[1000:].astype(np.float64)
    M = M[1000:].astype(np.float64)
    for series, key in ((E, "E"), (M * M, "M2")):
        err = exact.blocking_error(series)
        assert abs(series.mean() - want[key]) <= 5 * err, (key, series.mean(), want[key], err)
