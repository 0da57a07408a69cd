"""Parity of the demon dynamics on the GPU with the oracle (bit-exact).

Creutz's deterministic checkerboard dynamics (Sec. 2.2 cites it): no draws,
so the spins, the demons and the E/M records after every sweep are fixed by
the initial spins and demons alone.  Covered: the int8 strip kernel
(L/2 % 16 == 0), the int8 per-site kernel (any even L) and the bit-packed
kernel (qmax 3, two demon bit planes; padded rows) in 2D and 3D, runs long enough for the
demons to go all the way round (their storage offset wraps), calls split
into chunks, a switch from Metropolis to demon dynamics mid-run, the batched
form (demon lattices take the per-lattice path), the refusals, and the full-
size 2D L = 8192 lattice.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HOT, COLD_UP = 0, 1
INT8, BITPACK = 0, 1
RULE_METROPOLIS, RULE_DEMON = 0, 2


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def random_state(dims, L, qmax, seed, hot=True):
    rng = np.random.default_rng(seed)
    n = L ** dims
    s = (np.where(rng.random(n) < 0.5, 1, -1) if hot else np.ones(n)).astype(np.int8)
    q = rng.integers(0, qmax + 1, size=n).astype(np.uint8)
    return s, q


def gpu_demon(eng, dims, L, s, q, qmax, chunks, every=1, layout=INT8):
    lat = eng.Lattice(dims, L, 0.4, 1, layout=layout)
    lat.set_spins(s, 0)
    lat.set_demons(q, qmax=qmax)
    lat.set_rule(RULE_DEMON)
    assert lat.info().rule == RULE_DEMON
    for c in chunks:
        lat.sweep(c, every)
    E, M = lat.observables()
    out = (lat.get_spins(), lat.get_demons(), E, M)
    lat.close()
    return out


def assert_same(got, want, what):
    s_g, q_g, E_g, M_g = got
    s_o, q_o, E_o, M_o = want
    assert len(E_g) == len(E_o), what
    bad = np.nonzero((E_g != E_o) | (M_g != M_o))[0]
    assert bad.size == 0, f"{what}: first E/M mismatch at record {bad[:1]}"
    assert np.array_equal(s_g, s_o), f"{what}: {np.count_nonzero(s_g != s_o)} spins differ"
    assert np.array_equal(q_g, q_o), f"{what}: {np.count_nonzero(q_g != q_o)} demons differ"


@pytest.mark.parametrize("L", [2, 4, 6, 10, 30, 32, 34, 64, 96, 160, 258])
@pytest.mark.parametrize("qmax", [3, 15])
def test_demon_2d(eng, L, qmax):
    s, q = random_state(2, L, qmax, 100 + L + qmax)
    n = min(L + 5, 70)  # past one full round of the demons where affordable
    want = oracle.run_demon(2, L, s, q, qmax, n)
    got = gpu_demon(eng, 2, L, s, q, qmax, [n])
    assert_same(got, want, f"2D L={L} qmax={qmax}")
    got = gpu_demon(eng, 2, L, s, q, qmax, [1] * 3 + [n - 3])
    assert_same(got, want, f"2D L={L} qmax={qmax} chunked")
    if qmax == 3:
        got = gpu_demon(eng, 2, L, s, q, qmax, [2, n - 2], layout=BITPACK)
        assert_same(got, want, f"2D L={L} bit-packed")


@pytest.mark.parametrize("L", [2, 4, 6, 32, 34, 64])
def test_demon_3d(eng, L):
    qmax = 7
    s, q = random_state(3, L, qmax, 7 * L)
    n = L * L + 3 if L <= 6 else 12
    want = oracle.run_demon(3, L, s, q, qmax, n, measure_every=2)
    got = gpu_demon(eng, 3, L, s, q, qmax, [n], every=2)
    assert_same(got, want, f"3D L={L}")
    s, q = random_state(3, L, 3, 11 * L)
    want = oracle.run_demon(3, L, s, q, 3, n, measure_every=2)
    got = gpu_demon(eng, 3, L, s, q, 3, [n], every=2, layout=BITPACK)
    assert_same(got, want, f"3D L={L} bit-packed")


def test_demon_cold_start_and_uniform_demons(eng):
    """The hand-worked case of the oracle pins, on the GPU: cold spins, every
    demon q = 2, qmax = 3: the black sites flip and pay, the white ones cannot."""
    L = 64
    s = np.ones(L * L, dtype=np.int8)
    lat = eng.Lattice(2, L, 0.4, 1, layout=INT8, start=COLD_UP)
    lat.set_demons(None, fill=2, qmax=3)
    lat.set_rule(RULE_DEMON)
    lat.sweep(1, 1)
    E, M = lat.observables()
    got_s, got_q = lat.get_spins(), lat.get_demons()
    lat.close()
    want = oracle.run_demon(2, L, s, np.full(L * L, 2, dtype=np.uint8), 3, 1)
    assert_same((got_s, got_q, E, M), want, "cold, q = 2")
    assert E[0] == 2 * L * L


def test_metropolis_then_demons(eng):
    dims, L, beta, seed, qmax = 2, 96, 0.45, 12, 3
    s5, E1, M1 = oracle.run(dims, L, beta, seed, 5, start=HOT)
    rng = np.random.default_rng(0)
    q = rng.integers(0, qmax + 1, size=L * L).astype(np.uint8)
    s_o, q_o, E2, M2 = oracle.run_demon(dims, L, s5, q, qmax, 9, t0=5)
    lat = eng.Lattice(dims, L, beta, seed, layout=INT8)
    lat.sweep(5, 1)
    lat.set_demons(q, qmax=qmax)
    lat.set_rule(RULE_DEMON)
    lat.sweep(9, 1)
    E, M = lat.observables()
    got = (lat.get_spins(), lat.get_demons(), E, M)
    lat.close()
    assert_same(got, (s_o, q_o, np.concatenate([E1, E2]), np.concatenate([M1, M2])),
                "Metropolis then demons")


def test_demon_refusals(eng):
    lat = eng.Lattice(2, 32, 0.4, 1, layout=INT8)
    with pytest.raises(eng.IsingError):
        lat.set_rule(RULE_DEMON)  # no demons yet
    with pytest.raises(eng.IsingError):
        lat.set_demons(None, fill=4, qmax=3)
    with pytest.raises(eng.IsingError):
        lat.set_demons(np.full(32 * 32, 9, dtype=np.uint8), qmax=8)
    with pytest.raises(eng.IsingError):
        lat.set_demons(None, fill=0, qmax=64)
    with pytest.raises(eng.IsingError):
        lat.get_demons()
    lat.close()
    packed = eng.Lattice(2, 32, 0.4, 1, layout=BITPACK)
    with pytest.raises(eng.IsingError):
        packed.set_demons(None, fill=0, qmax=7)  # the packed layout holds qmax = 3
    packed.set_demons(None, fill=2, qmax=3)
    assert np.all(packed.get_demons() == 2)
    packed.close()


def test_demon_lattice_in_a_batch(eng):
    """A demon lattice in a batch goes through the per-lattice kernels and ends
    as it would alone; the no-allocation entry point refuses it."""
    import torch
    qmax = 3
    s, q = random_state(2, 64, qmax, 5)
    dem = eng.Lattice(2, 64, 0.4, 1, layout=INT8)
    dem.set_spins(s, 0)
    dem.set_demons(q, qmax=qmax)
    dem.set_rule(RULE_DEMON)
    met = eng.Lattice(2, 64, 0.4, 2, layout=INT8)
    b = eng.Batch([met, dem], sweeps=[6, 6], measure_every=[2, 2])
    b.launch()
    b.sync()
    E, M = dem.observables()
    assert_same((dem.get_spins(), dem.get_demons(), E, M),
                oracle.run_demon(2, 64, s, q, qmax, 6, measure_every=2), "batched demon")
    Em, Mm = met.observables()
    s_m, E_m, M_m = oracle.run(2, 64, 0.4, 2, 6, measure_every=2, start=HOT)
    assert np.array_equal(Em, E_m) and np.array_equal(met.get_spins(), s_m)
    b.close()
    rec = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(eng.IsingError):
        eng.batch_run_static([met, dem], [1, 1], [1, 1], rec.data_ptr(), 32)
    met.close()
    dem.close()


def test_demon_L8192(eng):
    L, qmax = 8192, 3
    rng = np.random.default_rng(8192)
    beta0 = 0.5
    w = np.exp(-4 * beta0 * np.arange(qmax + 1))
    q = rng.choice(qmax + 1, size=L * L, p=w / w.sum()).astype(np.uint8)
    s = np.ones(L * L, dtype=np.int8)
    n = 12
    want = oracle.run_demon(2, L, s, q, qmax, n)
    total = oracle.energy(2, L, s) + 4 * int(q.astype(np.int64).sum())
    for layout in (INT8, BITPACK):
        got = gpu_demon(eng, 2, L, s, q, qmax, [n], layout=layout)
        assert_same(got, want, f"2D L=8192 demons layout={layout}")
        assert int(got[2][-1]) + 4 * int(got[1].astype(np.int64).sum()) == total


@pytest.mark.parametrize("dims,L,n", [(2, 256, 261), (2, 512, 20), (3, 256, 3)])
def test_demon_packed_vector_rows(eng, dims, L, n):
    """Rows of whole 16-byte groups (L % 256 == 0) take the four-word path of
    the bit-packed demon pass; 2D L = 256 runs long enough to wrap the demons."""
    s, q = random_state(dims, L, 3, 3 * L + dims)
    want = oracle.run_demon(dims, L, s, q, 3, n, measure_every=1)
    got = gpu_demon(eng, dims, L, s, q, 3, [1, n - 1], layout=BITPACK)
    assert_same(got, want, f"{dims}D L={L} bit-packed vectors")


def test_demon_L32768_both_layouts(eng):
    """The out-of-L2 demon workload's size (2D L = 32768, 2^30 sites): two
    sweeps in full in both layouts, from cold spins and demons at beta 0.30."""
    from paper_cs_0312006_gb300 import workloads
    L, qmax, n = 32768, 3, 2
    q = workloads.demon_field(L * L, qmax, 0.30, 20031109)
    s = np.ones(L * L, dtype=np.int8)
    want = oracle.run_demon(2, L, s, q, qmax, n)
    for layout in (INT8, BITPACK):
        got = gpu_demon(eng, 2, L, s, q, qmax, [n], layout=layout)
        assert_same(got, want, f"2D L=32768 demons layout={layout}")
