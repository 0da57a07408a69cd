"""Single lattices far larger than L2: 2D L = 32768 (1.07e9 sites) and
L = 65536 (2^32 sites, the engine's maximum).

L = 32768 is compared with the oracle in full for its first two sweeps.  At
L = 65536 a full oracle sweep takes minutes, so the check is one sweep taken
site by site on a random sample (the oracle's own per-site decision, applied
to the GPU's state before the sweep) plus a from-scratch recount of E and M
of the whole lattice, which the fused reductions must equal exactly.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle

import _oracle_jobs as jobs

pytestmark = pytest.mark.gpu

HOT, COLD_UP = 0, 1
INT8, BITPACK = 0, 1
KERNEL_AUTO, KERNEL_STRIP, KERNEL_TMA = 0, 1, 2


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


@pytest.fixture(scope="module")
def pool():
    with cf.ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn")) as ex:
        yield ex


def test_L32768_first_two_sweeps(eng, pool):
    L, beta, seed = 32768, 0.4406868, 20031109
    fut = pool.submit(jobs.run, 2, L, beta, seed, HOT, 2, 1)
    got = []
    for layout, kernel in ((INT8, KERNEL_AUTO), (INT8, KERNEL_TMA), (BITPACK, KERNEL_AUTO)):
        lat = eng.Lattice(2, L, beta, seed, layout=layout, kernel=kernel)
        lat.sweep(2, 1)
        E, M = lat.observables()
        got.append(((layout, kernel), lat.get_spins(), E, M))
        lat.close()
    s_o, E_o, M_o = fut.result()
    for what, s, E, M in got:
        assert np.array_equal(E, E_o) and np.array_equal(M, M_o), what
        diff = np.count_nonzero(s != s_o)
        assert diff == 0, f"{what}: {diff} spins differ"


@pytest.mark.parametrize("layout,rule", [(INT8, 0), (BITPACK, 0), (INT8, 1)])
def test_L65536_sampled_sweep_and_recount(eng, layout, rule):
    L, beta, seed, t = 65536, 0.4406868, 7, 3
    n = L * L
    thr = oracle.thresholds_heatbath(2, beta) if rule else oracle.thresholds(2, beta)
    rng = np.random.default_rng(layout + 2 * rule)
    lat = eng.Lattice(2, L, beta, seed, layout=layout, rule=rule)
    s0 = lat.get_spins()
    # the hot start, sampled: site i is +1 iff word i&3 of Philox(seed; i>>2, 0, 0, 1) < 2^31
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i in list(rng.integers(0, n, size=256)) + [0, n - 1]:
        u = oracle.philox4x32_10([int(i) >> 2, 0, 0, 1], key)[int(i) & 3]
        assert s0[i] == (1 if u < 2 ** 31 else -1), i
    del s0
    lat.sweep(t, 1)
    lat.observables()
    s3 = lat.get_spins()
    lat.sweep(1, 1)
    E, M = lat.observables()
    s4 = lat.get_spins()
    lat.close()
    sites = np.concatenate([rng.integers(0, n, size=20000), [0, 1, L - 1, L, n - L, n - 1]])
    colour = ((sites % L) + (sites // L)) % 2
    black, white = sites[colour == 0], sites[colour == 1]
    # black pass of sweep t reads the state after sweep t-1
    want_b = oracle.site_update(2, L, s3, seed, thr, t, black, rule=rule)
    assert np.array_equal(s4[black], want_b)
    # white pass reads the black sites as the black pass left them
    mid = s4.copy()
    mid[white] = s3[white]
    del s3
    want_w = oracle.site_update(2, L, mid, seed, thr, t, white, rule=rule)
    assert np.array_equal(s4[white], want_w)
    del mid
    assert (int(E[0]), int(M[0])) == (oracle.energy(2, L, s4), oracle.magnetization(2, L, s4))
