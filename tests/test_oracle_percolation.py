"""Pins of the percolation oracle (CPU only), Sec. 2.3.

The porosity field, the invasion cluster, its spanning and its growth time
are checked against things other than the oracle: the documented Philox
counter (itself pinned to Triton's library Philox), the binomial law of the
pore count, scipy's connected-component labelling (ndimage.label) for the
cluster, scipy's breadth-first shortest paths (csgraph) for the number of
growth passes, and the paper's printed porosity threshold 0.592746 for the
spanning probability (tests/golden/paper_values.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle

ndimage = pytest.importorskip("scipy.ndimage")
csgraph = pytest.importorskip("scipy.sparse.csgraph")
sparse = pytest.importorskip("scipy.sparse")

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(key):
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line.startswith(key):
                return float(line.split("=")[1])
    raise KeyError(key)


def test_threshold_is_the_exact_floor(orc):
    assert orc.perc_threshold(0.0) == 0
    assert orc.perc_threshold(0.5) == 2 ** 31
    assert orc.perc_threshold(1.0) == 2 ** 32 - 1
    assert orc.perc_threshold(0.592746) == math.floor(0.592746 * 2 ** 32)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(ValueError):
            orc.perc_threshold(bad)


def test_pores_follow_the_documented_counter(orc):
    seed, P = 0xABCDEF0123456789, 0.6
    pore = orc.perc_pores(2, 37, seed, P)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    thr = orc.perc_threshold(P)
    for i in list(range(40)) + [37 * 37 - 1]:
        u = orc.philox4x32_10([i >> 2, 0, 0, 3], key)[i & 3]
        assert pore[i] == (1 if u <= thr else 0)


@pytest.mark.parametrize("dims,L,P", [(2, 300, 0.3), (2, 300, 0.592746), (3, 40, 0.3116),
                                      (3, 40, 0.8)])
def test_pore_fraction_is_binomial(orc, dims, L, P):
    pore = orc.perc_pores(dims, L, 99, P)
    n = pore.size
    assert abs(pore.sum() - n * P) <= 5 * math.sqrt(n * P * (1 - P))


def test_porosity_limits(orc):
    assert orc.perc_pores(2, 50, 1, 1.0).all()
    assert orc.perc_pores(3, 12, 1, 0.0).sum() == 0  # u = 0 exactly: never in 1728 draws


def _structure(dims):
    return ndimage.generate_binary_structure(dims, 1)  # nearest neighbours only


def _scipy_cluster(dims, L, pore, source, site):
    lab, _ = ndimage.label(pore.reshape((L,) * dims), structure=_structure(dims))
    lab = lab.reshape(-1)
    face = L ** (dims - 1)
    if source == oracle.PERC_POINT:
        keep = {lab[site]} - {0}
    else:
        keep = set(np.unique(lab[:face])) - {0}
    return np.isin(lab, list(keep)).astype(np.uint8) if keep else np.zeros_like(pore)


def _scipy_steps(dims, L, pore, source, site):
    """Largest breadth-first distance from the invasion sites through pores."""
    n = pore.size
    idx = np.arange(n)
    coords = np.unravel_index(idx, (L,) * dims)  # axis 0 is the slowest (y in 2D, z in 3D)
    rows, cols = [], []
    for ax in range(dims):
        ok = coords[ax] < L - 1
        stride = L ** (dims - 1 - ax)
        a = idx[ok]
        b = a + stride
        both = (pore[a] == 1) & (pore[b] == 1)
        rows += [a[both], b[both]]
        cols += [b[both], a[both]]
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    g = sparse.csr_matrix((np.ones(r.size), (r, c)), shape=(n, n))
    face = L ** (dims - 1)
    src = [site] if source == oracle.PERC_POINT else list(np.nonzero(pore[:face])[0])
    src = [s for s in src if pore[s]]
    if not src:
        return 0
    d = csgraph.shortest_path(g, unweighted=True, indices=src, directed=False)
    d = np.min(np.atleast_2d(d), axis=0)
    return int(np.max(d[np.isfinite(d)]))


@pytest.mark.parametrize("dims,L,P", [(2, 1, 1.0), (2, 2, 0.5), (2, 17, 0.55), (2, 64, 0.592746),
                                      (2, 64, 0.7), (3, 9, 0.3116), (3, 16, 0.4)])
@pytest.mark.parametrize("source", [0, 1])
def test_cluster_and_steps_against_scipy(orc, dims, L, P, source):
    for seed in range(3):
        pore = orc.perc_pores(dims, L, 500 + seed, P)
        site = (L ** dims) // 2 + (L // 2 if dims == 2 else 0)
        site = min(site, L ** dims - 1)
        cluster, size, spans, steps = orc.perc_invade(dims, L, pore, source, site)
        want = _scipy_cluster(dims, L, pore, source, site)
        assert np.array_equal(cluster, want)
        assert size == int(want.sum())
        face = L ** (dims - 1)
        assert spans == bool(cluster[:face].any() and cluster[-face:].any())
        assert steps == _scipy_steps(dims, L, pore, source, site)


def test_point_on_solid_and_hand_cases(orc):
    # a solid invasion point gives an empty cluster
    pore = np.ones(16, dtype=np.uint8)
    pore[5] = 0
    c, size, spans, steps = orc.perc_invade(2, 4, pore, oracle.PERC_POINT, 5)
    assert size == 0 and not spans and steps == 0 and c.sum() == 0
    # a straight pore column in a solid 5x5 medium: spans in 4 passes from the face
    pore = np.zeros(25, dtype=np.uint8)
    pore[2::5] = 1
    c, size, spans, steps = orc.perc_invade(2, 5, pore, oracle.PERC_FACE)
    assert size == 5 and spans and steps == 4
    # cut it once: no span, and the face cluster stops above the cut
    pore[12] = 0
    c, size, spans, steps = orc.perc_invade(2, 5, pore, oracle.PERC_FACE)
    assert size == 2 and not spans and steps == 1


def test_spanning_probability_crosses_one_half_at_the_papers_threshold(orc):
    """Face invasion of 2D L = 256 media: the porosity at which half of them
    span (a logistic fit of 5 x 1000 media around it) equals the paper's
    0.592746 within 5 standard errors of the fit plus 5e-4 for the finite
    size (the spanning probability of a square at p_c tends to 1/2)."""
    pc = golden("percolation_threshold_2d")
    L, N = 256, 1000
    Ps = pc + np.array([-0.012, -0.006, 0.0, 0.006, 0.012])
    R = []
    for j, P in enumerate(Ps):
        span = 0
        for k in range(N):
            pore = orc.perc_pores(2, L, 7_000_000 + j * N + k, P)
            span += orc.perc_invade(2, L, pore)[2]
        R.append(span / N)
    R = np.array(R)
    assert np.all(np.diff(R) > 0)
    logit = np.log(R / (1 - R))
    W = np.diag(N * R * (1 - R))
    A = np.vstack([Ps - pc, np.ones_like(Ps)]).T
    cov = np.linalg.inv(A.T @ W @ A)
    a, b = cov @ A.T @ W @ logit
    p_half = pc - b / a
    g = np.array([b / a ** 2, -1 / a])
    sd = float(np.sqrt(g @ cov @ g))
    assert abs(p_half - pc) <= 5 * sd + 5e-4, (p_half, sd)
    # far from the threshold the answer is nearly certain
    assert sum(orc.perc_invade(2, L, orc.perc_pores(2, L, s, 0.50))[2] for s in range(50)) == 0
    assert sum(orc.perc_invade(2, L, orc.perc_pores(2, L, s, 0.70))[2] for s in range(50)) == 50
