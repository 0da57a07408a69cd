"""Parity of the multi-hit Metropolis rule on the GPU with the oracle (bit-exact).

Each visit takes `hits` Metropolis trials with the neighbours fixed; trial m
draws with counter word 2 = c + 2m.  Covered: the int8 strip, general and
staged (TMA) passes and the bit-packed pass, 2D and 3D, ragged sizes, one hit
(= Metropolis), the full-size 2D L = 8192 lattice, a lattice in a batch (the
per-lattice path) and the refusals.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HOT, COLD_UP = 0, 1
INT8, BITPACK = 0, 1
RULE_METROPOLIS, RULE_MULTIHIT = 0, 3


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def gpu_run(eng, dims, L, beta, seed, start, chunks, hits, layout, kernel=0, every=1):
    lat = eng.Lattice(dims, L, beta, seed, layout=layout, start=start, kernel=kernel,
                      rule=RULE_MULTIHIT)
    lat.set_hits(hits)
    for c in chunks:
        lat.sweep(c, every)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    return s, E, M


def assert_same(got, want, what):
    s_g, E_g, M_g = got
    s_o, E_o, M_o = want
    assert len(E_g) == len(E_o), what
    assert np.array_equal(E_g, E_o) and np.array_equal(M_g, M_o), f"{what}: E/M differ"
    assert np.array_equal(s_g, s_o), f"{what}: {np.count_nonzero(s_g != s_o)} spins differ"


@pytest.mark.parametrize("L", [2, 4, 6, 10, 30, 32, 34, 64, 96, 160, 258])
@pytest.mark.parametrize("hits", [1, 2, 3])
def test_multihit_2d(eng, L, hits):
    beta, n = 0.42, 8
    want = oracle.run_multihit(2, L, beta, 60 + L, n, hits)
    for layout in (INT8, BITPACK):
        got = gpu_run(eng, 2, L, beta, 60 + L, HOT, [n], hits, layout)
        assert_same(got, want, f"2D L={L} hits={hits} layout={layout}")


@pytest.mark.parametrize("L", [2, 4, 6, 32, 34, 64])
def test_multihit_3d(eng, L):
    beta, n, hits = 0.2216544, 4, 3
    want = oracle.run_multihit(3, L, beta, 5 * L, n, hits, measure_every=2)
    for layout in (INT8, BITPACK):
        got = gpu_run(eng, 3, L, beta, 5 * L, HOT, [n], hits, layout, every=2)
        assert_same(got, want, f"3D L={L} layout={layout}")


@pytest.mark.parametrize("dims,L", [(2, 32), (2, 1024), (3, 32)])
def test_multihit_int8_kernels(eng, dims, L):
    beta = 0.4406868 if dims == 2 else 0.2216544
    want = oracle.run_multihit(dims, L, beta, 9, 4, 2, start=COLD_UP)
    for kernel in (1, 2):
        got = gpu_run(eng, dims, L, beta, 9, COLD_UP, [1, 3], 2, INT8, kernel=kernel)
        assert_same(got, want, f"{dims}D L={L} kernel={kernel}")


def test_multihit_L8192(eng):
    L, beta, hits, n = 8192, 0.44, 2, 3
    want = oracle.run_multihit(2, L, beta, 20031109, n, hits, start=COLD_UP)
    for layout in (INT8, BITPACK):
        got = gpu_run(eng, 2, L, beta, 20031109, COLD_UP, [n], hits, layout)
        assert_same(got, want, f"L=8192 layout={layout}")


def test_multihit_in_a_batch_and_refusals(eng):
    import torch
    lat = eng.Lattice(2, 64, 0.41, 3, layout=BITPACK, rule=RULE_MULTIHIT)
    lat.set_hits(3)
    other = eng.Lattice(2, 64, 0.41, 4, layout=INT8)
    b = eng.Batch([lat, other], sweeps=[5, 5], measure_every=[1, 1])
    b.launch()
    b.sync()
    E, M = lat.observables()
    assert_same((lat.get_spins(), E, M), oracle.run_multihit(2, 64, 0.41, 3, 5, 3), "batched")
    E2, _ = other.observables()
    s_o, E_o, _ = oracle.run(2, 64, 0.41, 4, 5)
    assert np.array_equal(E2, E_o) and np.array_equal(other.get_spins(), s_o)
    b.close()
    rec = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(eng.IsingError):
        eng.batch_run_static([lat], [1], [1], rec.data_ptr(), 32)
    for bad in (0, 65):
        with pytest.raises(eng.IsingError):
            lat.set_hits(bad)
    lat.close()
    other.close()
