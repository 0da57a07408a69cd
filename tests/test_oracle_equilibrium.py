"""Equilibrium pins of the oracle's Markov chain (CPU only).

Long oracle runs are compared with exact values: enumeration (Eq. 1) on 4x4,
2x2x2 and 3x3x3 lattices, Kaufman's finite-torus <E>, and Onsager's
infinite-lattice energy and spontaneous magnetisation.  Error bars come from
blocking analysis; the acceptance bands are 5 sigma.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact

Z5 = 5.0


def _check(series, want, what, extra=0.0):
    mean = float(np.mean(series))
    err = exact.blocking_error(series)
    assert abs(mean - want) <= Z5 * err + extra, \
        f"{what}: got {mean:.6f} +- {err:.2e}, exact {want:.6f}"


@pytest.mark.parametrize("dims,L,beta,nsweeps", [
    (2, 4, 0.2, 200_000),
    (2, 4, exact.BETA_C_2D, 400_000),
    (2, 4, 0.6, 200_000),
    (3, 2, 0.15, 200_000),
    (3, 2, 0.2216544, 200_000),
    (3, 2, 0.3, 200_000),
])
def test_checkerboard_vs_enumeration(orc, dims, L, beta, nsweeps):
    hist = orc.enumerate_states(dims, L)
    want = exact.boltzmann_averages(hist, dims, L, beta)
    _, E, M = orc.run(dims, L, beta, 4242, nsweeps, measure_every=1)
    E = E[1000:].astype(np.float64)
    M = M[1000:].astype(np.float64)
    _check(E, want["E"], "E")
    _check(M * M, want["M2"], "M^2")
    _check(np.abs(M), want["absM"], "|M|")


@pytest.mark.parametrize("beta", [0.15, 0.2216544, 0.3])
def test_sequential_3x3x3_vs_enumeration(orc, beta):
    """Odd L has no checkerboard; the sequential single-site chain uses the
    same acceptance rule and thresholds and must reach Eq. 1's averages."""
    hist = orc.enumerate_states(3, 3)
    want = exact.boltzmann_averages(hist, 3, 3, beta)
    _, E, M = orc.run(3, 3, beta, 777, 150_000, measure_every=1, sequential=True)
    E = E[1000:].astype(np.float64)
    M = M[1000:].astype(np.float64)
    _check(E, want["E"], "E")
    _check(M * M, want["M2"], "M^2")


@pytest.mark.parametrize("L,beta,nsweeps", [(16, 0.40, 150_000), (32, 0.4406868, 120_000)])
def test_kaufman_finite_torus_energy(orc, L, beta, nsweeps):
    want = exact.kaufman_mean_energy(beta, L)
    _, E, _ = orc.run(2, L, beta, 31337, nsweeps, measure_every=1)
    _check(E[2000:].astype(np.float64), want, f"<E> L={L}")


@pytest.mark.parametrize("beta,start", [(0.30, oracle.HOT), (0.50, oracle.COLD_UP),
                                        (0.60, oracle.COLD_UP)])
def test_onsager_energy_and_magnetisation(orc, beta, start):
    """L = 128 is many correlation lengths at these betas, so the infinite-
    lattice values apply up to exponentially small corrections."""
    L, nsweeps, burn = 128, 3000, 300
    n = L * L
    _, E, M = orc.run(2, L, beta, 1000 + int(beta * 100), nsweeps, measure_every=1,
                      start=start)
    u = E[burn:].astype(np.float64) / n
    _check(u, exact.onsager_energy_per_site(beta), f"u({beta})", extra=2e-4)
    if beta > exact.BETA_C_2D:
        m = np.abs(M[burn:].astype(np.float64)) / n
        _check(m, exact.onsager_magnetization(beta), f"m({beta})", extra=1e-3)


def test_critical_energy_approaches_minus_sqrt2():
    """Onsager: u(beta_c) = -sqrt 2.  Kaufman's exact finite-torus energy per
    site approaches it with a 1/L correction: L * (u_L + sqrt 2) settles to a
    constant as L doubles (this ties the finite-L formula, which pins the
    oracle above, to the infinite-lattice closed form)."""
    d = {L: abs(exact.kaufman_mean_energy(exact.BETA_C_2D, L) / L ** 2 + math.sqrt(2.0))
         for L in (16, 32, 64, 128)}
    assert d[16] > d[32] > d[64] > d[128] > 0
    scaled = [L * d[L] for L in (32, 64, 128)]
    assert abs(scaled[2] - scaled[1]) < 0.02 * scaled[2]
    assert d[128] < 6e-3


def _onsager_integral_minus_beta_f(beta, n=256):
    """-beta f from Onsager's double integral (periodic trapezoid rule, which
    converges exponentially for the smooth integrand away from beta_c):
    ln 2 / 2 + (1 / 8 pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)]."""
    t = 2 * np.pi * np.arange(n) / n
    c = np.cos(t)
    arg = np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (c[:, None] + c[None, :])
    return math.log(2.0) / 2 + np.log(arg).mean() / 2


@pytest.mark.parametrize("beta", [0.30, 0.50, 0.60])
def test_onsager_energy_against_the_free_energy_integral(beta):
    """The elliptic-integral form of u(beta) that the equilibrium pins use
    equals -d(-beta f)/d beta of Onsager's double integral (an independent
    form), and the printed values u(0.30) = -0.704499, u(0.50) = -1.745565."""
    h = 1e-5
    u_int = -(_onsager_integral_minus_beta_f(beta + h) -
              _onsager_integral_minus_beta_f(beta - h)) / (2 * h)
    assert abs(u_int - exact.onsager_energy_per_site(beta)) < 1e-7
    if beta in (0.30, 0.50):
        assert abs(exact.onsager_energy_per_site(beta) - {0.30: -0.704499, 0.50: -1.745565}[beta]) < 1e-6


def test_kaufman_large_torus_tends_to_onsager():
    """Away from beta_c the finite torus converges exponentially fast: at
    L = 64 Kaufman's exact <E>/N equals Onsager's u(beta) to 1e-9."""
    for beta in (0.30, 0.60):
        assert abs(exact.kaufman_mean_energy(beta, 64) / 64 ** 2 -
                   exact.onsager_energy_per_site(beta)) < 1e-9


@pytest.mark.parametrize("beta", [0.06, 0.08])
def test_cubic_energy_high_temperature_series(orc, beta):
    """3D has no closed form, but its high-temperature series fixes the
    leading terms: with t = tanh(beta), ln Z / N = ln 2 + 3 ln cosh(beta)
    + 3 t^4 + O(t^6) on the simple cubic lattice (three elementary squares per
    site; no closed graph has fewer bonds), so the energy per site is
    u = -3 t - 12 t^3 (1 - t^2) + O(t^5).  The t^3 term is 5x the acceptance
    band here, so a dropped or misplaced z coupling fails; the band adds
    200 t^5 for the next term (6 a_6 t^5 with a_6, the six-bond closed graphs
    per site, well below 33)."""
    L, nsweeps, burn = 16, 60_000, 500
    t = math.tanh(beta)
    want = -3.0 * t - 12.0 * t ** 3 * (1.0 - t * t)
    _, E, _ = orc.run(3, L, beta, 555 + int(1000 * beta), nsweeps, measure_every=1)
    u = E[burn:].astype(np.float64) / L ** 3
    _check(u, want, f"u_3D({beta})", extra=200.0 * t ** 5)
    # the t^3 term is resolved: the first-order value alone is rejected
    err = exact.blocking_error(u)
    assert abs(float(np.mean(u)) - (-3.0 * t)) > Z5 * err + 200.0 * t ** 5
