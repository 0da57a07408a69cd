"""Parity of the GPU percolation engine with the oracle (bit-exact), Sec. 2.3.

Porosity fields, invasion clusters, sizes, spanning and the number of growth
passes must equal the oracle's for every medium: ragged and tiny L (rows that
start inside a Philox group, a last word with padding bits), both sources, 2D
and 3D, the single-medium path and the one-CTA-per-medium batch, and the
full-size 2D L = 4096 medium near the threshold (thousands of passes).
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

POINT, FACE = 0, 1


@pytest.fixture(scope="module")
def perc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, percolation
    _build.build()
    return percolation


def centre(dims, L):
    return (L // 2) + L * (L // 2) + (L * L * (L // 2) if dims == 3 else 0)


def check_medium(perc, dims, L, seed, P, sources=(POINT, FACE)):
    m = perc.Medium(dims, L, seed)
    m.generate(P)
    pore_o = oracle.perc_pores(dims, L, seed, P)
    assert np.array_equal(m.pores(), pore_o), f"pores {dims}D L={L} P={P}"
    for source in sources:
        site = centre(dims, L)
        r = m.invade(source, site)
        c_o, size, spans, steps = oracle.perc_invade(dims, L, pore_o, source, site)
        assert np.array_equal(m.cluster(), c_o), f"cluster {dims}D L={L} P={P} src={source}"
        assert (r.size, bool(r.spans), r.steps) == (size, spans, steps), (dims, L, P, source)
    m.close()


@pytest.mark.parametrize("L", [1, 2, 3, 5, 31, 32, 33, 64, 100, 257])
@pytest.mark.parametrize("P", [0.0, 0.3, 0.592746, 1.0])
def test_medium_2d(perc, L, P):
    check_medium(perc, 2, L, 1000 + L, P)


@pytest.mark.parametrize("L", [1, 3, 8, 17, 32])
@pytest.mark.parametrize("P", [0.2, 0.3116, 0.6])
def test_medium_3d(perc, L, P):
    check_medium(perc, 3, L, 2000 + L, P)


def test_medium_repeat_and_regenerate(perc):
    """Invading twice gives the same answer; a new porosity replaces the field."""
    m = perc.Medium(2, 96, 5)
    m.generate(0.55)
    a = m.invade(FACE)
    b = m.invade(FACE)
    assert (a.size, a.spans, a.steps) == (b.size, b.spans, b.steps)
    m.generate(0.75)
    pore = oracle.perc_pores(2, 96, 5, 0.75)
    assert np.array_equal(m.pores(), pore)
    _, size, spans, steps = oracle.perc_invade(2, 96, pore, FACE)
    r = m.invade(FACE)
    assert (r.size, bool(r.spans), r.steps) == (size, spans, steps)
    m.close()


@pytest.mark.parametrize("dims,L,P", [(2, 16, 0.6), (2, 33, 0.592746), (2, 128, 0.592746),
                                      (2, 512, 0.6), (3, 8, 0.3116), (3, 17, 0.35),
                                      (3, 64, 0.3116)])
@pytest.mark.parametrize("source", [POINT, FACE])
def test_batch(perc, dims, L, P, source):
    import torch
    n = 24 if L <= 128 else 6
    seeds = [7_000 + 13 * k for k in range(n)]
    site = centre(dims, L)
    clusters = torch.zeros(n * L ** dims, dtype=torch.uint8, device="cuda")
    res = perc.batch(dims, L, P, seeds, source, site, clusters.data_ptr())
    got = clusters.cpu().numpy().reshape(n, -1)
    for k, seed in enumerate(seeds):
        pore = oracle.perc_pores(dims, L, seed, P)
        c_o, size, spans, steps = oracle.perc_invade(dims, L, pore, source, site)
        assert np.array_equal(got[k], c_o), (dims, L, k)
        assert (res[k].size, bool(res[k].spans), res[k].steps) == (size, spans, steps), k


def test_batch_spanning_fraction_at_threshold(perc):
    """2000 media of 2D L = 256 at the paper's 0.592746: every result equals
    the oracle on a sample, and the spanning fraction is near 1/2."""
    L, P, n = 256, 0.592746, 2000
    seeds = [90_000 + k for k in range(n)]
    res = perc.batch(2, L, P, seeds, FACE, 0)
    for k in range(0, n, 97):
        _, size, spans, steps = oracle.perc_invade(2, L, oracle.perc_pores(2, L, seeds[k], P))
        assert (res[k].size, bool(res[k].spans), res[k].steps) == (size, spans, steps)
    frac = sum(r.spans for r in res) / n
    assert abs(frac - 0.5) < 5 * (0.25 / n) ** 0.5 + 0.03


def test_medium_L4096_near_threshold(perc):
    L, P, seed = 4096, 0.6, 31337
    check_medium(perc, 2, L, seed, P, sources=(FACE,))


def test_refusals(perc):
    from paper_cs_0312006_gb300.engine import IsingError
    m = perc.Medium(2, 16, 1)
    with pytest.raises(IsingError):
        m.generate(-0.5)
    with pytest.raises(IsingError):
        m.invade(POINT, 16 * 16)
    with pytest.raises(IsingError):
        m.invade(7, 0)
    m.close()
    with pytest.raises(IsingError):
        perc.batch(3, 65, 0.3, [1])


def test_bench_configurations(perc):
    """The bench's two percolation workloads in the launch configuration it
    times: the L = 16384 medium at P = 0.6 in full (porosity field, cluster,
    size, spanning and all 34,572 passes), and its batch of 8192 media of
    L = 128 at 0.592746 (seeds 20031109 + k) checked medium by medium on a
    sample."""
    L, P, seed = 16384, 0.6, 20031109
    check_medium(perc, 2, L, seed, P, sources=(FACE,))
    n, Lb, Pb = 8192, 128, 0.592746
    seeds = [seed + k for k in range(n)]
    res = perc.batch(2, Lb, Pb, seeds, FACE, 0)
    for k in range(0, n, 257):
        _, size, spans, steps = oracle.perc_invade(2, Lb, oracle.perc_pores(2, Lb, seeds[k], Pb))
        assert (res[k].size, bool(res[k].spans), res[k].steps) == (size, spans, steps), k


@pytest.mark.parametrize("mode", [1, 2])
def test_pass_modes_agree(perc, mode):
    """The graph-replayed passes (the default) and the persistent cooperative
    launch give the oracle's results."""
    for dims, L, P in ((2, 257, 0.6), (2, 1024, 0.592746), (3, 40, 0.3116)):
        m = perc.Medium(dims, L, 77 + L)
        m.set_passes(mode)
        m.generate(P)
        pore = oracle.perc_pores(dims, L, 77 + L, P)
        for source in (POINT, FACE):
            site = centre(dims, L)
            r = m.invade(source, site)
            c_o, size, spans, steps = oracle.perc_invade(dims, L, pore, source, site)
            assert np.array_equal(m.cluster(), c_o), (dims, L, source, mode)
            assert (r.size, bool(r.spans), r.steps) == (size, spans, steps)
        m.close()


def test_persistent_barrier_timeout_is_reported(perc):
    """With the test hook on, one CTA of the persistent launch leaves before
    the first grid barrier: the others' bounded waits run out, perc_invade
    returns ISING_ETIMEOUT, nothing hangs, and the next invasion is right."""
    from paper_cs_0312006_gb300 import engine
    m = perc.Medium(2, 2048, 5)
    m.set_passes(perc.PASSES_PERSISTENT)
    m.generate(0.6)
    engine.test_inject_timeout(True)
    try:
        with pytest.raises(engine.IsingError) as ei:
            m.invade(FACE)
        assert ei.value.code == engine.ETIMEOUT
    finally:
        engine.test_inject_timeout(False)
    r = m.invade(FACE)
    _, size, spans, steps = oracle.perc_invade(2, 2048, oracle.perc_pores(2, 2048, 5, 0.6))
    assert (r.size, bool(r.spans), r.steps) == (size, spans, steps)
    m.close()


def test_spanning_threshold_at_L512(perc):
    """Sec. 5's 2D threshold from the GPU batch: 5 x 4096 media of L = 512
    around 0.592746; the fitted porosity where half of them span equals the
    paper's value within 5 standard errors plus 5e-4 for the finite size, and
    the transition is steeper than at L = 64 (its width falls with L)."""
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "paper_values.txt")) as f:
        pc = next(float(ln.split("#")[0].split("=")[1]) for ln in f
                  if ln.startswith("percolation_threshold_2d"))
    n = 4096

    def fractions(L, Ps, base):
        return [sum(r.spans for r in perc.batch(2, L, P, [base + 10_000 * j + k for k in range(n)]))
                / n for j, P in enumerate(Ps)]

    Ps = [pc + d for d in (-0.008, -0.004, 0.0, 0.004, 0.008)]
    f512 = fractions(512, Ps, 5_000_000)
    assert all(b > a for a, b in zip(f512, f512[1:]))
    p_half, sd = perc.spanning_threshold(Ps, f512, n)
    assert abs(p_half - pc) <= 5 * sd + 5e-4, (p_half, sd)
    f64 = fractions(64, [Ps[0], Ps[-1]], 6_000_000)
    assert f512[-1] - f512[0] > f64[1] - f64[0]
