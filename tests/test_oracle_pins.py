"""Pins of the CPU oracle against things other than itself (CPU only).

Each test names what fixes the expected value: a library routine (Triton's
Philox, mpmath), brute force on tiny lattices, an exact closed form (Kaufman,
Onsager), exact enumeration (Eq. 1), or an exact transition matrix.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from oracle import exact

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# Philox4x32-10 vs Triton's library implementation (interpreted on the CPU)
# ---------------------------------------------------------------------------
def test_philox_matches_triton_library(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
    ctr[0] = [0, 0, 0, 0]
    ctr[1] = [2 ** 32 - 1] * 4
    ctr[2] = [7, 3, 1, 0]  # shape of a sweep counter (group, sweep, colour, tag)
    seeds = [0, 1, 20031109, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF]
    env = dict(os.environ, TRITON_INTERPRET="1")
    req = json.dumps({"seeds": seeds, "ctr": ctr.tolist()})
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox_ref.py"), req],
                          capture_output=True, text=True, env=env, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for si, seed in enumerate(seeds):
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for j in range(ctr.shape[0]):
            got = orc.philox4x32_10(ctr[j].astype(np.uint32), key)
            assert got.tolist() == ref[si][j], (seed, ctr[j])


def test_philox_output_statistics(orc):
    """Bit balance of 4096 outputs: every bit is set ~half the time."""
    key = np.array([20031109, 0], dtype=np.uint32)
    words = np.array([orc.philox4x32_10([j, 5, 1, 0], key) for j in range(1024)],
                     dtype=np.uint64).reshape(-1)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint64)) & 1).astype(np.float64)
    frac = bits.mean(axis=0)
    # 4096 samples per bit: sigma = 0.5/64; 5 sigma
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / 64)


# ---------------------------------------------------------------------------
# Thresholds vs mpmath at 50 digits
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,beta", [
    (2, 0.4406868), (3, 0.2216544), (2, 0.30), (2, 0.60), (3, 0.15), (3, 0.30),
    (2, 1e-3), (3, 2.5), (2, 0.1), (3, 0.7),
])
def test_thresholds_match_mpmath(orc, dims, beta):
    got = orc.thresholds(dims, beta)
    want = exact.exact_thresholds(dims, beta)
    assert got[:dims].tolist() == want
    assert got[dims:].tolist() == [0] * (3 - dims)


def test_thresholds_random_betas(orc):
    rng = np.random.default_rng(7)
    for beta in rng.uniform(0.01, 1.5, size=200):
        for dims in (2, 3):
            assert orc.thresholds(dims, beta)[:dims].tolist() == \
                exact.exact_thresholds(dims, beta)


def test_thresholds_published_config_values(orc):
    # exp(-2 beta k) 2^32 at the critical-point betas of the workloads
    assert orc.thresholds(2, 0.4406868).tolist()[:2] == [736899868, 126432026]
    assert orc.thresholds(3, 0.2216544).tolist() == [1769728846, 729211650, 300469550]


def test_thresholds_edges(orc):
    # beta -> 0+: the accept probability tends to 1, floor is 2^32 - 1
    assert orc.thresholds(2, 1e-30).tolist()[:2] == [0xFFFFFFFF, 0xFFFFFFFF]
    # beta = +inf (zero temperature): no uphill move is ever accepted
    assert orc.thresholds(3, math.inf).tolist() == [0, 0, 0]
    # large finite beta underflows to 0 as well
    assert orc.thresholds(2, 50.0).tolist() == [0, 0, 0]
    for bad in (0.0, -0.1, float("nan")):
        with pytest.raises(ValueError):
            orc.thresholds(2, bad)
    with pytest.raises(ValueError):
        orc.thresholds(4, 0.3)


# ---------------------------------------------------------------------------
# E, M and the local dE = 2k against brute force on tiny lattices
# ---------------------------------------------------------------------------
def _energy_by_rolls(dims, L, s):
    a = s.reshape((L,) * dims).astype(np.int64)  # axes (z,) y, x
    e = 0
    for ax in range(dims):
        e -= int((a * np.roll(a, -1, axis=ax)).sum())
    return e


@pytest.mark.parametrize("dims,L", [(2, 2), (2, 3), (2, 4), (3, 2)])
def test_energy_magnetisation_all_states(orc, dims, L):
    n = L ** dims
    for state in range(2 ** n):
        s = np.array([1 if (state >> j) & 1 else -1 for j in range(n)], dtype=np.int8)
        assert orc.energy(dims, L, s) == _energy_by_rolls(dims, L, s)
        assert orc.magnetization(dims, L, s) == int(s.astype(np.int64).sum())


@pytest.mark.parametrize("dims,L", [(2, 6), (2, 10), (3, 3), (3, 4), (3, 6)])
def test_energy_random_states_and_local_rule(orc, dims, L):
    rng = np.random.default_rng(L * 10 + dims)
    n = L ** dims
    for _ in range(20):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=n)
        e0 = orc.energy(dims, L, s)
        assert e0 == _energy_by_rolls(dims, L, s)
        a = s.reshape((L,) * dims).astype(np.int64)
        h = sum(np.roll(a, sh, axis=ax) for ax in range(dims) for sh in (1, -1))
        for i in rng.integers(0, n, size=10):
            s2 = s.copy()
            s2[i] = -s2[i]
            # flipping site i changes E by 2 * s_i * h_i
            assert orc.energy(dims, L, s2) - e0 == 2 * int(s[i]) * int(h.reshape(-1)[i])


# ---------------------------------------------------------------------------
# Exact enumeration vs Kaufman's closed form; enumeration invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L", [2, 4])
def test_enumeration_matches_kaufman(orc, L):
    hist = orc.enumerate_states(2, L)
    assert hist.sum() == 2 ** (L * L)
    for beta in (0.1, 0.3, exact.BETA_C_2D, 0.6, 1.0):
        avg = exact.boltzmann_averages(hist, 2, L, beta)
        assert avg["logZ"] == pytest.approx(float(exact.kaufman_log_z(beta, L, L)), rel=1e-12)
        assert avg["E"] == pytest.approx(exact.kaufman_mean_energy(beta, L), rel=1e-9)


def test_enumeration_invariants_3d(orc):
    for L in (2, 3):
        n = L ** 3
        hist = orc.enumerate_states(3, L)
        assert hist.sum() == 2 ** n
        # spin-flip symmetry g(E, M) = g(E, -M)
        assert np.array_equal(hist, hist[:, ::-1])
        # two ground states (all up, all down) at E = -3N
        assert hist[0, 0] == 1 and hist[0, 2 * n] == 1
        assert hist[0].sum() == 2
    # 3x3x3: 81 distinct bonds, E has the parity of the bond count
    hist = orc.enumerate_states(3, 3)
    e_idx = np.nonzero(hist.sum(axis=1))[0] - 81
    assert np.all((e_idx - 81) % 2 == 0)


# ---------------------------------------------------------------------------
# The checkerboard chain with integer thresholds: exact stationarity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,L,beta", [(2, 2, 0.3), (2, 2, 0.9), (3, 2, 0.2216544)])
def test_half_sweep_matrices_preserve_boltzmann(orc, dims, L, beta):
    thr = orc.thresholds(dims, beta)
    pi = exact.boltzmann_vector(dims, L, beta)
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thr, colour)
        assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
        # detailed balance per colour pass, up to the quantisation of the
        # accept probability: thr/2^32 is below exp(-2 beta k) by less than
        # 2^-32, a relative error below 1/thr per flipped site, and at most
        # N/2 sites flip in one pass (non-flipping factors cancel exactly)
        rtol = 1.05 * (L ** dims / 2) / float(min(v for v in thr[:dims] if v > 0)) + 1e-12
        F = pi[:, None] * P
        assert np.allclose(F, F.T, rtol=rtol, atol=1e-15)
        assert np.allclose(pi @ P, pi, rtol=rtol, atol=1e-15)


def _empirical_half_sweep(orc, dims, L, seed, thr, colour, n_draws):
    n = L ** dims
    counts = np.zeros((2 ** n, 2 ** n))
    for a in range(2 ** n):
        s0 = exact.state_spins(a, n).astype(np.int8)
        for t in range(n_draws):
            s = s0.copy()
            orc.half_sweep(dims, L, s, seed, thr, t, colour)
            counts[a, exact.spins_state(s)] += 1
    return counts


@pytest.mark.parametrize("dims,L,beta,n_draws", [(2, 2, 0.35, 3000), (3, 2, 0.2, 400)])
def test_oracle_transition_frequencies(orc, dims, L, beta, n_draws):
    """The oracle's colour pass, sampled over independent sweep counters t,
    reproduces the exact transition matrix (binomial 5-sigma per entry)."""
    thr = orc.thresholds(dims, beta)
    for colour in (0, 1):
        P = exact.half_sweep_matrix(dims, L, thr, colour)
        C = _empirical_half_sweep(orc, dims, L, 99, thr, colour, n_draws)
        assert np.all(C[P == 0] == 0)  # nothing impossible ever happens
        freq = C / n_draws
        sig = np.sqrt(P * (1 - P) / n_draws) + 1e-12
        assert np.all(np.abs(freq - P) <= 5 * sig + 1.0 / n_draws)


# ---------------------------------------------------------------------------
# Special cases with a unique answer
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,L", [(2, 8), (3, 4)])
def test_neel_state_zero_temperature(orc, dims, L):
    """From the antiferromagnetic (Neel) state at beta = inf, the black pass
    flips every black site (k = -2d <= 0), then every white site has
    k = +2d and stays: all spins end at -1 if black (+1) goes first."""
    n = L ** dims
    idx = np.arange(n)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    par = (x + y + (z if dims == 3 else 0)) % 2
    s = np.where(par == 0, 1, -1).astype(np.int8)
    thr = orc.thresholds(dims, math.inf)
    orc.sweep(dims, L, s, 1, thr, 0)
    assert np.all(s == -1)
    assert orc.energy(dims, L, s) == -dims * n


def test_zero_temperature_never_raises_energy(orc):
    s = orc.init(2, 32, 5, oracle.HOT)
    thr = orc.thresholds(2, math.inf)
    e_prev = orc.energy(2, 32, s)
    for t in range(30):
        orc.sweep(2, 32, s, 5, thr, t)
        e = orc.energy(2, 32, s)
        assert e <= e_prev
        e_prev = e


def test_high_temperature_limit(orc):
    """beta -> 0+: thresholds are 2^32 - 1, so every site flips unless its
    draw is exactly 2^32 - 1; after one sweep the state is the negation."""
    s = orc.init(2, 16, 3, oracle.HOT)
    s0 = s.copy()
    thr = orc.thresholds(2, 1e-30)
    orc.sweep(2, 16, s, 3, thr, 0)
    assert np.array_equal(s, -s0)


# ---------------------------------------------------------------------------
# Initial state
# ---------------------------------------------------------------------------
def test_init_states(orc):
    for dims, L in ((2, 256), (3, 32)):
        s = orc.init(dims, L, 20031109, oracle.HOT)
        n = L ** dims
        assert set(np.unique(s).tolist()) == {-1, 1}
        assert abs(int(s.astype(np.int64).sum())) < 5 * math.sqrt(n)
        assert np.all(orc.init(dims, L, 1, oracle.COLD_UP) == 1)
        assert np.all(orc.init(dims, L, 1, oracle.COLD_DOWN) == -1)
        assert not np.array_equal(s, orc.init(dims, L, 20031110, oracle.HOT))


def test_init_uses_documented_counter(orc):
    """Site i is +1 iff word i&3 of Philox(seed; i>>2, 0, 0, 1) is below 2^31."""
    seed = 0xDEADBEEF12345678
    s = orc.init(2, 8, seed, oracle.HOT)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i in range(64):
        u = orc.philox4x32_10([i >> 2, 0, 0, 1], key)[i & 3]
        assert s[i] == (1 if u < 2 ** 31 else -1)


# ---------------------------------------------------------------------------
# Colour pass: loop order does not matter (vectorised restatement)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,L", [(2, 2), (2, 6), (2, 10), (3, 2), (3, 4)])
def test_half_sweep_vectorised_restatement(orc, dims, L):
    """All sites of one colour see only the other colour, so the pass equals a
    simultaneous update of that colour computed from the pre-pass state."""
    seed, beta = 77, 0.35
    thr = orc.thresholds(dims, beta)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    s = orc.init(dims, L, seed, oracle.HOT)
    n = L ** dims
    idx = np.arange(n)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    colour = (x + y + (z if dims == 3 else 0)) % 2
    for t, c in ((0, 0), (0, 1), (3, 0)):
        a = s.reshape((L,) * dims).astype(np.int64)
        h = sum(np.roll(a, sh, axis=ax) for ax in range(dims) for sh in (1, -1)).reshape(-1)
        k = s.astype(np.int64) * h
        want = s.copy()
        for i in np.nonzero(colour == c)[0]:
            hh = i >> 1
            if k[i] <= 0:
                flip = True
            else:
                u = orc.philox4x32_10([hh >> 2, t, c, 0], key)[hh & 3]
                flip = u < thr[k[i] // 2 - 1]
            if flip:
                want[i] = -want[i]
        orc.half_sweep(dims, L, s, seed, thr, t, c)
        assert np.array_equal(s, want)


def test_run_records_and_resume(orc):
    """run(): records after sweep t iff (t+1) % every == 0; splitting a run in
    two with the right t0 reproduces it exactly (counter-based draws)."""
    s_a, E_a, M_a = orc.run(2, 16, 0.4, 9, 30, measure_every=3)
    assert len(E_a) == 10
    s_b, E_b1, M_b1 = orc.run(2, 16, 0.4, 9, 13, measure_every=3)
    s_b, E_b2, M_b2 = orc.run(2, 16, 0.4, 9, 17, measure_every=3, s=s_b, t0=13)
    assert np.array_equal(s_a, s_b)
    assert np.array_equal(E_a, np.concatenate([E_b1, E_b2]))
    assert np.array_equal(M_a, np.concatenate([M_b1, M_b2]))
    assert E_a[-1] == orc.energy(2, 16, s_a) and M_a[-1] == orc.magnetization(2, 16, s_a)


@pytest.mark.parametrize("dims,L,rule", [(2, 10, 0), (2, 12, 1), (3, 6, 0), (3, 4, 1)])
def test_site_update_is_the_pass_decision(orc, dims, L, rule):
    """site_update (used to check huge lattices one sampled site at a time)
    gives, site by site, the spins the colour pass writes."""
    seed, beta, t = 13, 0.37, 4
    thr = orc.thresholds_heatbath(dims, beta) if rule else orc.thresholds(dims, beta)
    s = orc.init(dims, L, seed, oracle.HOT)
    n = L ** dims
    idx = np.arange(n)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    colour = (x + y + (z if dims == 3 else 0)) % 2
    for c in (0, 1):
        sites = np.nonzero(colour == c)[0]
        got = orc.site_update(dims, L, s, seed, thr, t, sites, rule=rule)
        orc.half_sweep(dims, L, s, seed, thr, t, c, rule=rule)
        assert np.array_equal(got, s[sites])
