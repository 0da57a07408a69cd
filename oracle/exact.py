"""Exact results that pin the oracle: closed forms, enumeration, transition
matrices and error bars.

TEST INFRASTRUCTURE (same rule as the rest of ``oracle/``).

- Eq. 1 (expected value over all states with Boltzmann weights, Sec. 2.2):
  ``boltzmann_averages`` sums over the exact density of states g(E, M) that
  ``oracle.enumerate_states`` counts.
- Onsager's infinite-lattice results for the 2D square lattice (J = 1):
  beta_c = ln(1 + sqrt 2) / 2, the energy per site u(beta) (elliptic-integral
  form) with u(beta_c) = -sqrt 2, and the spontaneous magnetisation
  m(beta) = (1 - sinh(2 beta)^-4)^(1/8) for beta > beta_c (Yang).
- Kaufman's exact partition function of the finite m x n torus, which gives
  the exact finite-size <E> by differentiation.
- Exact half-sweep transition matrices of the checkerboard chain on 2 x 2 and
  2 x 2 x 2 lattices, built from the integer acceptance rule.
- Blocking (binning) error bars for correlated Monte Carlo series.
"""
from __future__ import annotations

import math

import mpmath
import numpy as np
from scipy.special import ellipk

BETA_C_2D = math.log(1.0 + math.sqrt(2.0)) / 2.0


# --------------------------------------------------------------------------
# Onsager (2D square lattice, infinite volume)
# --------------------------------------------------------------------------
def onsager_energy_per_site(beta: float) -> float:
    """u(beta) = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(kappa)],
    kappa = 2 sinh(2b) / cosh^2(2b); the limit -sqrt(2) at beta_c."""
    if abs(beta - BETA_C_2D) < 1e-12:
        return -math.sqrt(2.0)
    t = 2.0 * beta
    kappa = 2.0 * math.sinh(t) / math.cosh(t) ** 2
    kk = float(ellipk(kappa * kappa))  # scipy takes the parameter m = kappa^2
    return -(1.0 / math.tanh(t)) * (1.0 + (2.0 / math.pi)
                                   * (2.0 * math.tanh(t) ** 2 - 1.0) * kk)


def onsager_magnetization(beta: float) -> float:
    """Spontaneous magnetisation per site; 0 at and above the critical point."""
    if beta <= BETA_C_2D:
        return 0.0
    return (1.0 - math.sinh(2.0 * beta) ** -4) ** 0.125


# --------------------------------------------------------------------------
# Kaufman: exact Z of the 2D Ising model on an m x n torus (2mn bonds)
# --------------------------------------------------------------------------
def kaufman_log_z(K, m: int, n: int):
    """ln Z for couplings K = beta*J on an m-column, n-row periodic lattice.

    Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4) with
    Z1 = prod_r 2cosh(m g_{2r+1}/2), Z2 = prod_r 2sinh(m g_{2r+1}/2),
    Z3 = prod_r 2cosh(m g_{2r}/2),   Z4 = prod_r 2sinh(m g_{2r}/2), r < n,
    cosh g_l = cosh 2K coth 2K - cos(pi l / n) for l >= 1 and
    g_0 = 2K + ln tanh K (negative in the high-temperature phase).
    """
    K = mpmath.mpf(K)
    c2 = mpmath.cosh(2 * K) * mpmath.coth(2 * K)

    def gamma(l):
        if l == 0:
            return 2 * K + mpmath.log(mpmath.tanh(K))
        return mpmath.acosh(c2 - mpmath.cos(mpmath.pi * l / n))

    z1 = z2 = z3 = z4 = mpmath.mpf(1)
    for r in range(n):
        go, ge = gamma(2 * r + 1), gamma(2 * r)
        z1 *= 2 * mpmath.cosh(m * go / 2)
        z2 *= 2 * mpmath.sinh(m * go / 2)
        z3 *= 2 * mpmath.cosh(m * ge / 2)
        z4 *= 2 * mpmath.sinh(m * ge / 2)
    pref = (2 * mpmath.sinh(2 * K)) ** (mpmath.mpf(m * n) / 2) / 2
    return mpmath.log(pref * (z1 + z2 + z3 + z4))


def kaufman_mean_energy(beta: float, L: int, dps: int = 40) -> float:
    """Exact <E> (whole lattice, E = -sum_bonds s s) on the L x L torus."""
    with mpmath.workdps(dps):
        d = mpmath.diff(lambda k: kaufman_log_z(k, L, L), mpmath.mpf(beta))
        return float(-d)


# --------------------------------------------------------------------------
# Eq. 1 over the exact density of states
# --------------------------------------------------------------------------
def boltzmann_averages(hist: np.ndarray, dims: int, L: int, beta: float) -> dict:
    """<E>, <E^2>, <M^2>, <|M|>, ln Z from g(E, M) (``enumerate_states``)."""
    n = L ** dims
    e_vals = np.arange(-dims * n, dims * n + 1, dtype=np.float64)
    m_vals = np.arange(-n, n + 1, dtype=np.float64)
    g = hist.astype(np.float64)
    ee, mm = np.meshgrid(e_vals, m_vals, indexing="ij")
    mask = g > 0
    logw = np.full(g.shape, -np.inf)
    logw[mask] = np.log(g[mask]) - beta * ee[mask]
    lmax = logw[mask].max()
    w = np.where(mask, np.exp(logw - lmax), 0.0)
    z = w.sum()
    p = w / z
    return {
        "E": float((p * ee).sum()),
        "E2": float((p * ee * ee).sum()),
        "M2": float((p * mm * mm).sum()),
        "absM": float((p * np.abs(mm)).sum()),
        "logZ": float(lmax + math.log(z)),
    }


# --------------------------------------------------------------------------
# Exact checkerboard transition matrices on tiny lattices (all 2^N states)
# --------------------------------------------------------------------------
def _coords(dims: int, L: int):
    n = L ** dims
    out = []
    for i in range(n):
        x, y, z = i % L, (i // L) % L, i // (L * L)
        out.append((x, y, z if dims == 3 else 0))
    return out


def _neighbours(dims: int, L: int):
    nb = []
    for (x, y, z) in _coords(dims, L):
        lst = [((x + 1) % L, y, z), ((x - 1) % L, y, z),
               (x, (y + 1) % L, z), (x, (y - 1) % L, z)]
        if dims == 3:
            lst += [(x, y, (z + 1) % L), (x, y, (z - 1) % L)]
        nb.append([a + L * b + L * L * c for (a, b, c) in lst])
    return nb


def state_spins(state: int, n: int) -> np.ndarray:
    """Bit j of ``state`` set <=> spin j is +1."""
    return np.array([1 if (state >> j) & 1 else -1 for j in range(n)], dtype=np.int64)


def spins_state(s) -> int:
    return int(sum(1 << j for j, v in enumerate(s) if v > 0))


def state_energy(s, nb_fwd) -> int:
    return -int(sum(s[i] * sum(s[j] for j in nb_fwd[i]) for i in range(len(s))))


def half_sweep_matrix(dims: int, L: int, thr, colour: int,
                      heatbath: bool = False, hits: int = 1) -> np.ndarray:
    """P[a, b] = probability that one colour pass maps state a to state b.

    Each site of the colour flips independently (its neighbours all have the
    other colour).  Metropolis: with probability 1 if k <= 0 and
    thr[k/2 - 1] / 2^32 if k > 0, k = s_i * (sum of its 2*dims neighbours).
    Heat bath: with probability thr[d] / 2^32, d = (2*dims - k)/2 the number
    of disagreeing neighbours.  Metropolis with ``hits`` trials per visit: the
    site's own two-state chain (flip with the Metropolis probability of its
    current state; the flipped state's move back has k <= 0 or k > 0 as its
    own k says) taken ``hits`` steps by a matrix power.
    """
    n = L ** dims
    coords = _coords(dims, L)
    nb = _neighbours(dims, L)
    sites = [i for i, (x, y, z) in enumerate(coords) if (x + y + z) % 2 == colour]
    P = np.zeros((2 ** n, 2 ** n))
    for a in range(2 ** n):
        s = state_spins(a, n)
        probs = []
        for i in sites:
            k = int(s[i] * sum(s[j] for j in nb[i]))
            if heatbath:
                probs.append(float(thr[(2 * dims - k) // 2]) / 2.0 ** 32)
            elif hits == 1:
                probs.append(1.0 if k <= 0 else float(thr[k // 2 - 1]) / 2.0 ** 32)
            else:
                def acc(kk):
                    return 1.0 if kk <= 0 else float(thr[kk // 2 - 1]) / 2.0 ** 32
                T = np.array([[1 - acc(k), acc(k)], [acc(-k), 1 - acc(-k)]])
                probs.append(float(np.linalg.matrix_power(T, hits)[0, 1]))
        for mask in range(2 ** len(sites)):
            b, pr = a, 1.0
            for bit, i in enumerate(sites):
                if (mask >> bit) & 1:
                    b ^= 1 << i
                    pr *= probs[bit]
                else:
                    pr *= 1.0 - probs[bit]
            P[a, b] += pr
    return P


def boltzmann_vector(dims: int, L: int, beta: float) -> np.ndarray:
    n = L ** dims
    coords = _coords(dims, L)
    fwd = []
    for (x, y, z) in coords:
        lst = [((x + 1) % L) + L * y + L * L * z, x + L * ((y + 1) % L) + L * L * z]
        if dims == 3:
            lst.append(x + L * y + L * L * ((z + 1) % L))
        fwd.append(lst)
    e = np.array([state_energy(state_spins(a, n), fwd) for a in range(2 ** n)],
                 dtype=np.float64)
    w = np.exp(-beta * (e - e.min()))
    return w / w.sum()


# --------------------------------------------------------------------------
# Error bars for correlated series
# --------------------------------------------------------------------------
def blocking_error(x, min_blocks: int = 32) -> float:
    """Standard error of the mean by repeated pairwise blocking (Flyvbjerg-
    Petersen); returns the largest estimate over levels with >= min_blocks
    blocks, which is conservative once the blocks exceed the correlation time.
    """
    x = np.asarray(x, dtype=np.float64)
    best = 0.0
    while len(x) >= min_blocks:
        n = len(x)
        var = x.var(ddof=1) if n > 1 else 0.0
        best = max(best, math.sqrt(var / n))
        if n % 2:
            x = x[:-1]
        x = 0.5 * (x[0::2] + x[1::2])
    return best


# --------------------------------------------------------------------------
# Thresholds at 50 significant digits
# --------------------------------------------------------------------------
def exact_thresholds(dims: int, beta: float, dps: int = 50) -> list:
    """floor(exp(-2 beta k) 2^32) for k = 2, .., 2*dims, with beta taken as the
    exact binary value of the double and the exponential evaluated by mpmath."""
    out = []
    with mpmath.workdps(dps):
        b = mpmath.mpf(beta)  # exact conversion of the IEEE double
        for k in range(2, 2 * dims + 1, 2):
            out.append(int(mpmath.floor(mpmath.exp(-2 * b * k) * mpmath.mpf(2) ** 32)))
    return out


def exact_thresholds_heatbath(dims: int, beta: float, dps: int = 50) -> list:
    """floor(2^32 / (1 + exp(2 beta k))) for d = 0, .., 2*dims disagreeing
    neighbours, k = 2(dims - d) the energy-change numerator (dE = 2k), padded
    with zeros to 7 entries; beta is the exact binary value of the double."""
    out = []
    with mpmath.workdps(dps):
        b = mpmath.mpf(beta)
        for d in range(2 * dims + 1):
            k = 2 * (dims - d)
            out.append(int(mpmath.floor(mpmath.mpf(2) ** 32 / (1 + mpmath.exp(2 * b * k)))))
    return out + [0] * (7 - len(out))
