"""Parity of the heat-bath rule on the GPU with the oracle (bit-exact).

The heat-bath rule draws at every site and flips iff the draw is below
floor(2^32 / (1 + exp(4 beta (dims - d)))), d the number of disagreeing
neighbours; the draw is the same Philox word as the Metropolis rule's.  Every
kernel that runs a colour pass is covered: the int8 strip, general and staged
(TMA) passes, the bit-packed pass, the single-launch path for small lattices,
the persistent batched kernel (rules mixed in one batch) and its no-allocation
entry point.
"""
import concurrent.futures as cf
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle

import _oracle_jobs as jobs

pytestmark = pytest.mark.gpu

HOT, COLD_UP, COLD_DOWN = 0, 1, 2
INT8, BITPACK = 0, 1
RULE_METROPOLIS, RULE_HEATBATH = 0, 1


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
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        yield ex


def gpu_run(eng, dims, L, beta, seed, start, chunks, every=1, layout=INT8, kernel=0):
    lat = eng.Lattice(dims, L, beta, seed, layout=layout, start=start, kernel=kernel,
                      rule=RULE_HEATBATH)
    assert lat.info().rule == RULE_HEATBATH
    for c in chunks:
        lat.sweep(c, every)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    return s, E, M


def assert_same(gpu, want, what):
    s_g, E_g, M_g = gpu
    s_o, E_o, M_o = want
    assert len(E_g) == len(E_o), what
    bad = np.nonzero((E_g != E_o) | (M_g != M_o))[0]
    assert bad.size == 0, f"{what}: first E/M mismatch at record {bad[:1]}"
    diff = np.nonzero(s_g != s_o)[0]
    assert diff.size == 0, f"{what}: {diff.size} spins differ, first at {diff[:3]}"


@pytest.mark.parametrize("L", [2, 4, 6, 10, 30, 32, 34, 62, 64, 96, 160, 192, 258])
@pytest.mark.parametrize("beta", [0.25, 0.4406868, 0.7, math.inf])
def test_heatbath_2d(eng, L, beta):
    n = 12
    want = oracle.run(2, L, beta, 31 + L, n, start=HOT, heatbath=True)
    for layout in (INT8, BITPACK):
        # one call (single-launch path for small lattices) and one pass per call
        for chunks in ([n], [1] * n):
            g = gpu_run(eng, 2, L, beta, 31 + L, HOT, chunks, layout=layout)
            assert_same(g, want, f"2D L={L} beta={beta} layout={layout} chunks={len(chunks)}")


@pytest.mark.parametrize("L", [2, 4, 6, 10, 32, 34, 64])
@pytest.mark.parametrize("beta", [0.15, 0.2216544, 0.4])
def test_heatbath_3d(eng, L, beta):
    n = 6
    want = oracle.run(3, L, beta, 17 + L, n, start=HOT, heatbath=True)
    for layout in (INT8, BITPACK):
        for chunks in ([n], [1] * n):
            g = gpu_run(eng, 3, L, beta, 17 + L, HOT, chunks, layout=layout)
            assert_same(g, want, f"3D L={L} beta={beta} layout={layout}")


@pytest.mark.parametrize("dims,L", [(2, 32), (2, 96), (2, 1024), (3, 32), (3, 64)])
def test_heatbath_staged_and_strip_kernels(eng, dims, L):
    n = 6 if dims == 2 else 3
    beta = 0.4406868 if dims == 2 else 0.2216544
    want = oracle.run(dims, L, beta, 3 + L, n, start=COLD_UP, heatbath=True)
    for kernel in (1, 2):  # strip, staged
        g = gpu_run(eng, dims, L, beta, 3 + L, COLD_UP, [1] * n, layout=INT8, kernel=kernel)
        assert_same(g, want, f"{dims}D L={L} kernel={kernel}")


def test_heatbath_L8192_first_sweeps(eng, pool):
    """The full-size 2D lattice (67M sites) at three betas: the first 4 sweeps
    in every kernel and layout."""
    betas = [0.30, 0.4406868, 0.60]
    futs = [pool.submit(jobs.run, 2, 8192, b, 555 + j, COLD_UP, 4, 1, None, 0, True)
            for j, b in enumerate(betas)]
    for j, b in enumerate(betas):
        want = futs[j].result()
        for layout, kernel in ((INT8, 1), (INT8, 2), (BITPACK, 0)):
            g = gpu_run(eng, 2, 8192, b, 555 + j, COLD_UP, [4], layout=layout, kernel=kernel)
            assert_same(g, want, f"L=8192 beta={b} layout={layout} kernel={kernel}")


def test_rule_switch_mid_run(eng):
    """Metropolis for 7 sweeps, then heat bath for 9: the oracle's two runs
    chained through the state and the sweep counter."""
    dims, L, beta, seed = 2, 96, 0.42, 8
    s7, E1, M1 = oracle.run(dims, L, beta, seed, 7, start=HOT)
    s16, E2, M2 = oracle.run(dims, L, beta, seed, 9, s=s7, t0=7, heatbath=True)
    for layout in (INT8, BITPACK):
        lat = eng.Lattice(dims, L, beta, seed, layout=layout)
        lat.sweep(7, 1)
        lat.set_rule(RULE_HEATBATH)
        lat.sweep(9, 1)
        E, M = lat.observables()
        s = lat.get_spins()
        lat.close()
        assert_same((s, E, M), (s16, np.concatenate([E1, E2]), np.concatenate([M1, M2])),
                    f"rule switch layout={layout}")


def test_batch_mixed_rules(eng):
    """One batch, both rules, cluster and per-CTA jobs, two launches: each
    lattice equals its oracle run."""
    specs = []  # (dims, L, beta, rule, layout)
    for k, L in enumerate((6, 34, 64, 130, 256, 512, 1024)):
        for rule in (RULE_METROPOLIS, RULE_HEATBATH):
            specs.append((2, L, 0.38 + 0.01 * k, rule, (INT8, BITPACK)[(k + rule) % 2]))
    for L in (4, 32, 64):
        specs.append((3, L, 0.2216544, RULE_HEATBATH, INT8))
        specs.append((3, L, 0.2216544, RULE_METROPOLIS, BITPACK))
    sweeps, every = 6, 2
    lats = []
    for i, (dims, L, beta, rule, layout) in enumerate(specs):
        lats.append(eng.Lattice(dims, L, beta, 900 + i, layout=layout, rule=rule))
    b = eng.Batch(lats, sweeps=[sweeps] * len(lats), measure_every=[every] * len(lats),
                  cluster_size=2, big_sites=1 << 14)
    b.launch()
    b.launch()
    b.sync()
    for i, (dims, L, beta, rule, layout) in enumerate(specs):
        want = oracle.run(dims, L, beta, 900 + i, 2 * sweeps, measure_every=every, start=HOT,
                          heatbath=rule == RULE_HEATBATH)
        E, M = lats[i].observables()
        assert_same((lats[i].get_spins(), E, M), want, f"batch job {i} {specs[i]}")
    # the queues are per rule: changing a lattice's rule under a batch is refused
    lats[0].set_rule(RULE_HEATBATH)
    with pytest.raises(eng.IsingError):
        b.launch()
    b.close()
    for lat in lats:
        lat.close()


def test_batch_run_static_mixed_rules(eng):
    import torch
    specs = [(2, 64, 0.4, RULE_HEATBATH), (2, 64, 0.4, RULE_METROPOLIS),
             (2, 300, 0.45, RULE_HEATBATH), (3, 16, 0.22, RULE_HEATBATH)]
    lats = [eng.Lattice(d, L, b, 40 + i, layout=INT8 if i % 2 else BITPACK, rule=r)
            for i, (d, L, b, r) in enumerate(specs)]
    n = 5
    rec = torch.zeros(2 * n * len(lats), dtype=torch.int64, device="cuda")
    eng.batch_run_static(lats, [n] * len(lats), [1] * len(lats), rec.data_ptr(),
                         n * len(lats), cluster_size=2, big_sites=1 << 12)
    torch.cuda.synchronize()
    got = rec.cpu().numpy().reshape(len(lats), n, 2)
    for i, (d, L, b, r) in enumerate(specs):
        s_o, E_o, M_o = oracle.run(d, L, b, 40 + i, n, start=HOT, heatbath=r == RULE_HEATBATH)
        assert np.array_equal(got[i, :, 0], E_o) and np.array_equal(got[i, :, 1], M_o), i
        assert np.array_equal(lats[i].get_spins(), s_o), i
        lats[i].close()
