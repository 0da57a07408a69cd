"""Pins of the oracle's heat-bath rule (CPU only).

The heat-bath rule is the other local update of Sec. 2.2's Monte Carlo: each
visited spin is drawn from its conditional Boltzmann distribution given its
neighbours, so it flips with probability 1 / (1 + exp(beta dE)), dE = 2k.
The integer form compares the site's draw with
thb[d] = floor(2^32 / (1 + exp(4 beta (dims - d)))), d the number of
disagreeing neighbours.  Pins: mpmath at 50 digits, the complement identity
p(d) + p(2 dims - d) = 1, zero- and infinite-temperature limits, the exact
transition matrix and its Boltzmann stationarity, and exact enumeration.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact

Z5 = 5.0
TWO32 = 2 ** 32


@pytest.mark.parametrize("dims,beta", [
    (2, 0.4406868), (3, 0.2216544), (2, 0.30), (2, 0.60), (3, 0.15), (3, 0.7),
    (2, 1e-3), (3, 2.5),
])
def test_heatbath_thresholds_match_mpmath(orc, dims, beta):
    assert orc.thresholds_heatbath(dims, beta).tolist() == \
        exact.exact_thresholds_heatbath(dims, beta)


def test_heatbath_thresholds_random_betas(orc):
    rng = np.random.default_rng(11)
    for beta in rng.uniform(0.01, 1.5, size=150):
        for dims in (2, 3):
            assert orc.thresholds_heatbath(dims, beta).tolist() == \
                exact.exact_thresholds_heatbath(dims, beta)


def test_heatbath_complement_identity(orc):
    """1/(1+e^x) + 1/(1+e^-x) = 1, so for d != dims the two floors of a and
    2^32 - a (a not an integer) add up to 2^32 - 1; thb[dims] = 2^31."""
    rng = np.random.default_rng(3)
    for beta in rng.uniform(0.05, 1.0, size=40):
        for dims in (2, 3):
            thb = orc.thresholds_heatbath(dims, beta).astype(np.int64)
            assert thb[dims] == 2 ** 31
            for d in range(dims):
                assert thb[d] + thb[2 * dims - d] == TWO32 - 1
            assert np.all(np.diff(thb[:2 * dims + 1]) > 0)  # more disagreement, likelier flip
            assert np.all(thb[2 * dims + 1:] == 0)


def test_heatbath_thresholds_limits(orc):
    # beta -> 0+: every flip probability tends to 1/2
    thb = orc.thresholds_heatbath(2, 1e-30).tolist()
    assert thb[:5] == [2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31, 2 ** 31, 2 ** 31]
    # beta = inf: downhill always (up to the 2^-32 quantum), level 1/2, uphill never
    thb = orc.thresholds_heatbath(3, math.inf).tolist()
    assert thb == [0, 0, 0, 2 ** 31, TWO32 - 1, TWO32 - 1, TWO32 - 1]
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(ValueError):
            orc.thresholds_heatbath(2, bad)
    with pytest.raises(ValueError):
        orc.thresholds_heatbath(1, 0.3)


def test_heatbath_published_config_values(orc):
    """At the critical-point betas of the 2D and 3D workloads."""
    assert orc.thresholds_heatbath(2, 0.4406868).tolist() == \
        exact.exact_thresholds_heatbath(2, 0.4406868)
    thb = orc.thresholds_heatbath(2, 0.4406868)
    # d = 0 (all four neighbours agree): 2^32 / (1 + e^{8 beta_c}) = 2^32 / (1 + (1 + sqrt 2)^4)
    want = TWO32 / (1.0 + (1.0 + math.sqrt(2.0)) ** 4)
    assert abs(int(thb[0]) - want) < 64  # beta_c rounded to 7 digits


@pytest.mark.parametrize("dims,L,beta", [(2, 2, 0.3), (2, 2, 0.9), (3, 2, 0.2216544)])
def test_heatbath_matrices_preserve_boltzmann(orc, dims, L, beta):
    thb = orc.thresholds_heatbath(dims, beta)
    pi = exact.boltzmann_vector(dims, L, beta)
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thb, colour, heatbath=True)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
        # each flip probability is below its exact value by < 2^-32, a
        # relative error < 1/thb; at most N/2 sites change in a pass and the
        # non-flip factors 1 - p are perturbed by < 2^-32 / (1 - p) each
        lo = float(min(thb[:2 * dims + 1]))
        rtol = 1.05 * (L ** dims) / lo + 1e-12
        F = pi[:, None] * P
        assert np.allclose(F, F.T, rtol=rtol, atol=1e-15)
        assert np.allclose(pi @ P, pi, rtol=rtol, atol=1e-15)


@pytest.mark.parametrize("dims,L,beta,n_draws", [(2, 2, 0.35, 3000), (3, 2, 0.2, 400)])
def test_heatbath_transition_frequencies(orc, dims, L, beta, n_draws):
    thb = orc.thresholds_heatbath(dims, beta)
    n = L ** dims
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thb, colour, heatbath=True)
        C = np.zeros_like(P)
        for a in range(2 ** n):
            s0 = exact.state_spins(a, n).astype(np.int8)
            for t in range(n_draws):
                s = s0.copy()
                orc.half_sweep(dims, L, s, 123, thb, t, colour, rule=oracle.HEATBATH_RULE)
                C[a, exact.spins_state(s)] += 1
        assert np.all(C[P == 0] == 0)
        freq = C / n_draws
        sig = np.sqrt(P * (1 - P) / n_draws) + 1e-12
        assert np.all(np.abs(freq - P) <= 5 * sig + 1.0 / n_draws)


@pytest.mark.parametrize("dims,L", [(2, 2), (2, 6), (2, 10), (3, 2), (3, 4)])
def test_heatbath_vectorised_restatement(orc, dims, L):
    """Simultaneous update of one colour from the pre-pass state, every site
    drawing Philox(seed; hh>>2, t, c, 0)[hh & 3] and flipping iff u < thb[d]."""
    seed, beta = 91, 0.35
    thb = orc.thresholds_heatbath(dims, beta)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    s = orc.init(dims, L, seed, oracle.HOT)
    n = L ** dims
    idx = np.arange(n)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    colour = (x + y + (z if dims == 3 else 0)) % 2
    for t, c in ((0, 0), (0, 1), (5, 0), (5, 1)):
        a = s.reshape((L,) * dims).astype(np.int64)
        h = sum(np.roll(a, sh, axis=ax) for ax in range(dims) for sh in (1, -1)).reshape(-1)
        d = (2 * dims - s.astype(np.int64) * h) // 2
        want = s.copy()
        for i in np.nonzero(colour == c)[0]:
            hh = i >> 1
            u = orc.philox4x32_10([hh >> 2, t, c, 0], key)[hh & 3]
            if u < thb[d[i]]:
                want[i] = -want[i]
        orc.half_sweep(dims, L, s, seed, thb, t, c, rule=oracle.HEATBATH_RULE)
        assert np.array_equal(s, want)


def test_heatbath_zero_temperature_never_raises_energy(orc):
    s = orc.init(2, 32, 8, oracle.HOT)
    thb = orc.thresholds_heatbath(2, math.inf)
    e_prev = orc.energy(2, 32, s)
    for t in range(30):
        for c in (0, 1):
            orc.half_sweep(2, 32, s, 8, thb, t, c, rule=oracle.HEATBATH_RULE)
        e = orc.energy(2, 32, s)
        assert e <= e_prev
        e_prev = e


def test_heatbath_run_matches_passes(orc):
    """run(heatbath=True) is black-then-white heat-bath passes with the
    records of E and M taken from the state."""
    dims, L, beta, seed = 2, 12, 0.41, 5
    s_run, E, M = orc.run(dims, L, beta, seed, 7, measure_every=1, heatbath=True)
    thb = orc.thresholds_heatbath(dims, beta)
    s = orc.init(dims, L, seed, oracle.HOT)
    for t in range(7):
        orc.half_sweep(dims, L, s, seed, thb, t, 0, rule=oracle.HEATBATH_RULE)
        orc.half_sweep(dims, L, s, seed, thb, t, 1, rule=oracle.HEATBATH_RULE)
        assert E[t] == orc.energy(dims, L, s) and M[t] == orc.magnetization(dims, L, s)
    assert np.array_equal(s, s_run)
    s_m, _, _ = orc.run(dims, L, beta, seed, 7, measure_every=1)
    assert not np.array_equal(s_m, s_run)  # a different chain from Metropolis


def _check(series, want, what):
    mean = float(np.mean(series))
    err = exact.blocking_error(series)
    assert abs(mean - want) <= Z5 * err, \
        f"{what}: got {mean:.6f} +- {err:.2e}, exact {want:.6f}"


@pytest.mark.parametrize("dims,L,beta,nsweeps", [
    (2, 4, exact.BETA_C_2D, 200_000),
    (2, 4, 0.6, 100_000),
    (3, 2, 0.2216544, 100_000),
])
def test_heatbath_vs_enumeration(orc, dims, L, beta, nsweeps):
    """The heat-bath chain reaches Eq. 1's averages."""
    hist = orc.enumerate_states(dims, L)
    want = exact.boltzmann_averages(hist, dims, L, beta)
    _, E, M = orc.run(dims, L, beta, 4343, nsweeps, measure_every=1, heatbath=True)
    E = E[1000:].astype(np.float64)
    M = M[1000:].astype(np.float64)
    _check(E, want["E"], "E")
    _check(M * M, want["M2"], "M^2")
