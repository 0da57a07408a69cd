"""Pins of the oracle's demon dynamics (CPU only).

Creutz's deterministic checkerboard dynamics, which Sec. 2.2 cites: every site
carries a demon of energy 4q (q = 0..qmax); a site flips iff its demon can pay
or absorb the cost within its range; after each sweep the demons move one half
row on within their colour.  Pins: exact conservation of E + 4 sum q, each
colour pass is an involution (so the dynamics runs backwards exactly), a hand-
worked sweep, the demon move's own structure, and -- the physics -- the demons
thermalise to a Boltzmann distribution with one temperature for every level,
at which the spins' energy equals Onsager's closed form.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact


def _random_state(dims, L, qmax, seed):
    rng = np.random.default_rng(seed)
    n = L ** dims
    s = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    q = rng.integers(0, qmax + 1, size=n).astype(np.uint8)
    return s, q


def _total(dims, L, s, q):
    return oracle.energy(dims, L, s) + 4 * int(q.astype(np.int64).sum())


@pytest.mark.parametrize("dims,L,qmax", [(2, 2, 1), (2, 6, 3), (2, 10, 7), (3, 2, 3), (3, 4, 3),
                                         (3, 6, 15)])
def test_energy_plus_demons_is_conserved(orc, dims, L, qmax):
    s, q = _random_state(dims, L, qmax, 5 + L)
    total = _total(dims, L, s, q)
    for t in range(40):
        for c in (0, 1):
            orc.demon_half_sweep(dims, L, s, q, qmax, c)
            assert _total(dims, L, s, q) == total
            assert q.max() <= qmax
        orc.demon_shift(dims, L, q, 1)
        assert _total(dims, L, s, q) == total


@pytest.mark.parametrize("dims,L", [(2, 8), (3, 4)])
def test_passes_are_involutions_and_the_dynamics_reverses(orc, dims, L):
    qmax = 3
    s0, q0 = _random_state(dims, L, qmax, 17)
    for c in (0, 1):  # a pass undoes itself: the other colour is unchanged
        s, q = s0.copy(), q0.copy()
        orc.demon_half_sweep(dims, L, s, q, qmax, c)
        orc.demon_half_sweep(dims, L, s, q, qmax, c)
        assert np.array_equal(s, s0) and np.array_equal(q, q0)
    s, q = s0.copy(), q0.copy()
    n = 25
    for _ in range(n):
        orc.demon_sweep(dims, L, s, q, qmax)
    assert not np.array_equal(s, s0)
    for _ in range(n):  # inverse sweep: demons back, white pass, black pass
        orc.demon_shift(dims, L, q, -1)
        orc.demon_half_sweep(dims, L, s, q, qmax, 1)
        orc.demon_half_sweep(dims, L, s, q, qmax, 0)
    assert np.array_equal(s, s0) and np.array_equal(q, q0)


def test_worked_sweep_2d_L4(orc):
    """Cold start, every demon q = 2 = dims, qmax = 3, by hand: each black site
    has d = 0 (cost 4*2), its demon pays it (q -> 0) and it flips; then every
    white site has d = 4 (cost -8), its demon would need q = 4 > qmax, so none
    flips.  E goes from -32 (all bonds agree) to +32 (all disagree)."""
    L, n = 4, 16
    s = np.ones(n, dtype=np.int8)
    q = np.full(n, 2, dtype=np.uint8)
    orc.demon_half_sweep(2, L, s, q, 3, 0)
    orc.demon_half_sweep(2, L, s, q, 3, 1)
    idx = np.arange(n)
    black = ((idx % L) + (idx // L)) % 2 == 0
    assert np.all(s[black] == -1) and np.all(s[~black] == 1)
    assert np.all(q[black] == 0) and np.all(q[~black] == 2)
    assert orc.energy(2, L, s) == 32
    # with demons q = 0 the cold state is frozen: no site can pay for a flip
    s = np.ones(n, dtype=np.int8)
    q = np.zeros(n, dtype=np.uint8)
    for _ in range(5):
        orc.demon_sweep(2, L, s, q, 3)
    assert np.all(s == 1) and np.all(q == 0)


@pytest.mark.parametrize("dims,L", [(2, 6), (3, 4)])
def test_demon_move(orc, dims, L):
    """One half row on within the colour: the demon of (x, y, z) = (0, 0, 0)
    (colour 0, half row 0, half column 0) goes to the colour-0 site of half row
    1, half column 0, i.e. (1, 1, 0); L^(dims-1) moves bring every demon back;
    a move back undoes a move on."""
    n = L ** dims
    q = np.zeros(n, dtype=np.uint8)
    q[0] = 9
    orc.demon_shift(dims, L, q, 1)
    assert q[1 + L] == 9 and q.sum() == 9
    rng = np.random.default_rng(2)
    q0 = rng.integers(0, 50, size=n).astype(np.uint8)
    q = q0.copy()
    orc.demon_shift(dims, L, q, 1)
    assert not np.array_equal(q, q0)
    orc.demon_shift(dims, L, q, -1)
    assert np.array_equal(q, q0)
    for _ in range(L ** (dims - 1)):
        orc.demon_shift(dims, L, q, 1)
    assert np.array_equal(q, q0)
    # colours are kept
    idx = np.arange(n)
    colour = (idx % L + (idx // L) % L + (idx // (L * L) if dims == 3 else 0)) % 2
    q = colour.astype(np.uint8) + 1
    orc.demon_shift(dims, L, q, 1)
    assert np.array_equal(q, colour.astype(np.uint8) + 1)


def test_run_records(orc):
    dims, L, qmax = 2, 12, 3
    s, q = _random_state(dims, L, qmax, 3)
    s2, q2, E, M = orc.run_demon(dims, L, s, q, qmax, 9, measure_every=3, t0=1)
    # records after sweeps t = 1..9 with (t + 1) % 3 == 0: t = 2, 5, 8
    assert len(E) == 3
    ss, qq = s.copy(), q.copy()
    for k in range(9):
        orc.demon_sweep(dims, L, ss, qq, qmax)
        if (1 + k + 1) % 3 == 0:
            i = [2, 5, 8].index(1 + k)
            assert E[i] == orc.energy(dims, L, ss) and M[i] == orc.magnetization(dims, L, ss)
    assert np.array_equal(ss, s2) and np.array_equal(qq, q2)


def _thermalised(orc, L, qmax, beta0, hot, seed, burn=3000, keep=2000):
    """Cold or hot spins, demons drawn from exp(-4 beta0 q) on 0..qmax."""
    n = L * L
    rng = np.random.default_rng(seed)
    w = np.exp(-4 * beta0 * np.arange(qmax + 1))
    q = rng.choice(qmax + 1, size=n, p=w / w.sum()).astype(np.uint8)
    s = (np.where(rng.random(n) < 0.5, 1, -1) if hot else np.ones(n)).astype(np.int8)
    s, q, _, _ = orc.run_demon(2, L, s, q, qmax, burn)
    hist = np.zeros(qmax + 1)
    energies = []
    for _ in range(keep):
        orc.demon_sweep(2, L, s, q, qmax)
        hist += np.bincount(q, minlength=qmax + 1)
        energies.append(orc.energy(2, L, s) / n)
    return hist, np.array(energies)


@pytest.mark.parametrize("qmax,beta0,hot", [(3, 0.5, False), (15, 0.3, True)])
def test_demons_thermalise_and_spins_follow_onsager(orc, qmax, beta0, hot):
    """Microcanonical = canonical for a large lattice: every demon level gives
    the same beta, p(q+1)/p(q) = exp(-4 beta), and at that beta the spins'
    mean energy per site is Onsager's u(beta).  Betas are read from the best-
    populated levels; the bands are 5 sigma of the counting and blocking
    errors plus the finite-size shift of u at L = 128 away from beta_c (<1e-3)."""
    L = 128
    hist, u = _thermalised(orc, L, qmax, beta0, hot, seed=11)
    levels = [k for k in range(qmax) if hist[k + 1] > 1e5]
    betas = np.array([-math.log(hist[k + 1] / hist[k]) / 4 for k in levels])
    # counts are correlated in time; 2000 sweeps of 16384 demons, effective
    # samples taken as 1/20 of the raw counts
    sig = np.array([math.sqrt(20 / hist[k] + 20 / hist[k + 1]) / 4 for k in levels])
    b = float(np.sum(betas / sig ** 2) / np.sum(1 / sig ** 2))
    assert np.all(np.abs(betas - b) <= 5 * sig + 1e-4), (betas, sig)
    assert abs(b - exact.BETA_C_2D) > 0.08  # away from the critical point
    b_err = float(1 / math.sqrt(np.sum(1 / sig ** 2)))
    du = abs(exact.onsager_energy_per_site(b + 1e-4) - exact.onsager_energy_per_site(b)) / 1e-4
    want = exact.onsager_energy_per_site(b)
    err = exact.blocking_error(u)
    assert abs(u.mean() - want) <= 5 * (err + du * b_err) + 1e-3, (u.mean(), want, b)
