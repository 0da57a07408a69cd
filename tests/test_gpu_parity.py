"""Parity of the CUDA engine with the CPU oracle, called through the C ABI.

Everything here is integer and keyed by (seed, sweep, colour, site), so the
bar is bit-exact: spins after the run and the int64 E and M after every
recorded sweep must equal the oracle's.  Sizes cover the general kernel
(ragged half rows, tiny L), the vector kernel (L % 32 == 0) and the full-size
workloads (2D L=8192 beta scan: first 20 sweeps; 2D L=512 scan: full 2000
sweeps; 3D L=256: first 20 sweeps in full and single-sweep transitions later).
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
INT8, BITPACK, AUTO = 0, 1, 2


def layouts_for(L):
    return [INT8, BITPACK]


@pytest.fixture(scope="module")
def pool():
    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        yield ex


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def gpu_run(eng, dims, L, beta, seed, start, nsweeps, every, chunks=None, layout=0, kernel=0):
    lat = eng.Lattice(dims, L, beta, seed, layout=layout, start=start, kernel=kernel)
    if chunks is None:
        chunks = [nsweeps]
    assert sum(chunks) == nsweeps
    for c in chunks:
        lat.sweep(c, every)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    return s, E, M


def assert_same(gpu, orc_res, what):
    s_g, E_g, M_g = gpu
    s_o, E_o, M_o = orc_res
    assert len(E_g) == len(E_o), what
    bad = np.nonzero((E_g != E_o) | (M_g != M_o))[0]
    assert bad.size == 0, f"{what}: first E/M mismatch at record {bad[:1]}"
    diff = np.nonzero(s_g != s_o)[0]
    assert diff.size == 0, f"{what}: {diff.size} spins differ, first at site {diff[:3]}"


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,L", [(2, 2), (2, 4), (2, 6), (2, 64), (2, 100), (2, 192), (3, 2),
                                    (3, 4), (3, 6), (3, 32), (3, 34), (3, 64)])
@pytest.mark.parametrize("start", [HOT, COLD_UP, COLD_DOWN])
def test_init_matches_oracle(eng, dims, L, start):
    want = oracle.init(dims, L, 20031109, start)
    for layout in layouts_for(L):
        lat = eng.Lattice(dims, L, 0.3, 20031109, layout=layout, start=start)
        got = lat.get_spins()
        lat.close()
        assert np.array_equal(got, want), f"layout {layout}"


SMALL_2D = [2, 4, 6, 10, 30, 32, 34, 62, 64, 96, 128, 160, 192, 258]
SMALL_3D = [2, 4, 6, 10, 32, 34, 64, 128]


@pytest.mark.parametrize("L", SMALL_2D)
@pytest.mark.parametrize("beta", [0.25, 0.4406868, 0.7])
def test_sweeps_match_oracle_2d(eng, L, beta):
    n = 25
    o = oracle.run(2, L, beta, 77 + L, n, measure_every=1, start=HOT)
    for layout in layouts_for(L):
        g = gpu_run(eng, 2, L, beta, 77 + L, HOT, n, 1, layout=layout)
        assert_same(g, o, f"2D L={L} beta={beta} layout={layout}")


@pytest.mark.parametrize("L", SMALL_3D)
@pytest.mark.parametrize("beta", [0.15, 0.2216544, 0.4])
def test_sweeps_match_oracle_3d(eng, L, beta):
    n = 12 if L < 128 else 4
    o = oracle.run(3, L, beta, 99 + L, n, measure_every=1, start=HOT)
    for layout in layouts_for(L):
        g = gpu_run(eng, 3, L, beta, 99 + L, HOT, n, 1, layout=layout)
        assert_same(g, o, f"3D L={L} beta={beta} layout={layout}")


@pytest.mark.parametrize("dims,L", [(2, 32), (2, 64), (2, 96), (2, 160), (2, 1024), (3, 32),
                                    (3, 64), (3, 96)])
def test_tma_staged_kernel_matches_oracle(eng, dims, L):
    """The int8 pass with its rows staged in shared memory by bulk copies."""
    n = 8 if dims == 2 else 4
    beta = 0.4406868 if dims == 2 else 0.2216544
    o = oracle.run(dims, L, beta, 5 + L, n, measure_every=1, start=HOT)
    g = gpu_run(eng, dims, L, beta, 5 + L, HOT, n, 1, layout=INT8, kernel=eng.KERNEL_TMA)
    assert_same(g, o, f"TMA {dims}D L={L}")


def test_auto_layout_choice_and_identity(eng):
    for L in (128, 96, 34):
        lat = eng.Lattice(2, L, 0.44, 3, layout=AUTO)
        assert lat.info().layout == BITPACK
        lat.close()
    for L in (96, 34, 130):  # padded rows, rows starting inside a Philox group
        runs = [gpu_run(eng, 2, L, 0.44, 3, HOT, 15, 1, layout=lay)
                for lay in (INT8, BITPACK, AUTO)]
        for r in runs[1:]:
            assert_same(r, runs[0], f"layout identity L={L}")


@pytest.mark.parametrize("layout", [INT8, BITPACK])
def test_critical_2d_L64_1000_sweeps(eng, layout):
    """2D L=64 at beta_c, hot start, seed 20031109: 1000 sweeps, E/M each sweep."""
    g = gpu_run(eng, 2, 64, 0.4406868, 20031109, HOT, 1000, 1, layout=layout)
    o = oracle.run(2, 64, 0.4406868, 20031109, 1000, measure_every=1, start=HOT)
    assert_same(g, o, "2D L=64 beta_c")


def test_measure_interval_and_chunked_calls(eng):
    g = gpu_run(eng, 2, 96, 0.42, 5, COLD_UP, 30, 3, chunks=[7, 13, 10])
    o = oracle.run(2, 96, 0.42, 5, 30, measure_every=3, start=COLD_UP)
    assert len(o[1]) == 10
    assert_same(g, o, "every=3 over three calls")


@pytest.mark.parametrize("layout", [INT8, BITPACK])
def test_checkpoint_and_resume(eng, layout):
    dims, L, beta, seed = 2, 128, 0.44, 31
    full = gpu_run(eng, dims, L, beta, seed, HOT, 30, 1)
    lat = eng.Lattice(dims, L, beta, seed, layout=layout)
    lat.sweep(17, 1)
    E1, M1 = lat.observables()
    mid = lat.get_spins()
    lat.close()
    # resume in the other layout: the state is layout-free
    lat2 = eng.Lattice(dims, L, beta, seed, layout=BITPACK if layout == INT8 else INT8)
    lat2.set_spins(mid, 17)
    assert lat2.info().sweeps_done == 17
    lat2.sweep(13, 1)
    E2, M2 = lat2.observables()
    s2 = lat2.get_spins()
    lat2.close()
    assert_same((s2, np.concatenate([E1, E2]), np.concatenate([M1, M2])), full, "resume")


@pytest.mark.parametrize("beta", [math.inf, 1e-30])
def test_temperature_limits(eng, beta):
    g = gpu_run(eng, 2, 64, beta, 3, HOT, 5, 1)
    o = oracle.run(2, 64, beta, 3, 5, measure_every=1, start=HOT)
    assert_same(g, o, f"beta={beta}")


def test_torch_side_stream(eng):
    import torch
    s = torch.cuda.Stream()
    lat = eng.Lattice(2, 256, 0.4, 8, stream=s)
    lat.sweep(10, 1)
    E, M = lat.observables()
    sp = lat.get_spins()
    dev = torch.empty(256 * 256, dtype=torch.int8, device="cuda")
    lat.export_device(dev.data_ptr())
    s.synchronize()
    lat.close()
    o = oracle.run(2, 256, 0.4, 8, 10, measure_every=1)
    assert_same((sp, E, M), o, "side stream")
    assert np.array_equal(dev.cpu().numpy(), o[0])


def test_errors_on_gpu(eng):
    lat = eng.Lattice(2, 32, 0.4, 1)
    s = lat.get_spins()
    lat.set_spins(s, 2 ** 32 - 1)
    with pytest.raises(eng.IsingError) as ei:
        lat.sweep(2, 1)
    assert ei.value.code == eng.ERANGE
    lat.sweep(1, 1)  # the last representable sweep index
    bad = s.copy()
    bad[5] = 0
    with pytest.raises(eng.IsingError) as ei:
        lat.set_spins(bad, 0)
    assert ei.value.code == eng.EINVAL
    with pytest.raises(eng.IsingError):
        lat.sweep(-1, 1)
    with pytest.raises(eng.IsingError):
        lat.sweep(1, 0)
    lat.close()


# ---------------------------------------------------------------------------
# Full-size workloads
# ---------------------------------------------------------------------------
SCAN_BETAS = [round(0.30 + 0.02 * j, 10) for j in range(16)]


def test_beta_scan_L512_full_runs(eng, pool):
    """2D L=512, 16 betas in [0.30, 0.60], cold start, 2000 sweeps each, both layouts."""
    futs = [pool.submit(jobs.run, 2, 512, b, 20031109 + j, COLD_UP, 2000, 1)
            for j, b in enumerate(SCAN_BETAS)]
    for j, b in enumerate(SCAN_BETAS):
        want = futs[j].result()
        for layout in (INT8, BITPACK):
            g = gpu_run(eng, 2, 512, b, 20031109 + j, COLD_UP, 2000, 1, layout=layout)
            assert_same(g, want, f"L=512 beta={b} layout={layout}")


def test_beta_scan_L8192_first_20_sweeps(eng, pool):
    """2D L=8192 (67M sites), 16 betas, cold start: the first 20 sweeps, both layouts."""
    futs = [pool.submit(jobs.run, 2, 8192, b, 20031109 + j, COLD_UP, 20, 1)
            for j, b in enumerate(SCAN_BETAS)]
    for j, b in enumerate(SCAN_BETAS):
        want = futs[j].result()
        for layout, kernel in ((INT8, 1), (INT8, 2), (BITPACK, 0)):
            g = gpu_run(eng, 2, 8192, b, 20031109 + j, COLD_UP, 20, 1, layout=layout,
                        kernel=kernel)
            assert_same(g, want, f"L=8192 beta={b} layout={layout} kernel={kernel}")


@pytest.mark.parametrize("layout", [INT8, BITPACK])
def test_3d_L256_near_critical(eng, pool, layout):
    """3D L=256 at beta=0.2216544, hot start: the first 20 sweeps against the
    oracle in full; then sweeps 20..999 with E/M every 10, and the final
    sweep checked as a single oracle transition from the GPU's state."""
    dims, L, beta, seed = 3, 256, 0.2216544, 20031109
    fut = pool.submit(jobs.run, dims, L, beta, seed, HOT, 20, 1)
    lat = eng.Lattice(dims, L, beta, seed, layout=layout)
    lat.sweep(20, 1)
    E, M = lat.observables()
    s20 = lat.get_spins()
    assert_same((s20, E, M), fut.result(), "3D L=256 first 20 sweeps")
    lat.sweep(979, 10)
    E_rec, M_rec = lat.observables()
    assert len(E_rec) == 97  # after sweeps t with t + 1 in {30, 40, ..., 990}
    s999 = lat.get_spins()
    lat.sweep(1, 10)
    E_last, M_last = lat.observables()
    s1000 = lat.get_spins()
    lat.close()
    # the fused reductions agree with a from-scratch recount of the GPU state
    e_chk = pool.submit(jobs.observables, dims, L, s1000)
    step = pool.submit(jobs.one_sweep, dims, L, beta, seed, s999, 999)
    s_o, e_o, m_o = step.result()
    assert np.array_equal(s_o, s1000), "sweep 999 transition"
    assert (E_last[0], M_last[0]) == (e_o, m_o) == e_chk.result()


def test_device_philox_matches_oracle(eng):
    """The device generator (every kernel's draws) against the oracle's Philox
    (itself pinned to Triton's library implementation)."""
    import torch
    rng = np.random.default_rng(4)
    for seed, (c1, c2, c3) in [(20031109, (0, 0, 0)), (0xFFFFFFFFFFFFFFFF, (7, 1, 0)),
                               (12345, (2 ** 32 - 1, 1, 2))]:
        n = 4096
        out = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
        eng.philox_fill(out.data_ptr(), n, c1, c2, c3, seed)
        got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for i in list(rng.integers(0, n, size=64)) + [0, n - 1]:
            assert got[i].tolist() == oracle.philox4x32_10([i, c1, c2, c3], key).tolist()


def test_observables_async_matches_the_oracle(eng):
    """ising_observables_async: the records land in pinned host memory once the
    stream passes the call, equal to the oracle's, and are cleared."""
    import torch
    lat = eng.Lattice(2, 96, 0.43, 17, layout=INT8)
    pairs = torch.zeros((8, 2), dtype=torch.int64).pin_memory().numpy()
    lat.sweep(5, 1)
    n = lat.observables_async(pairs)
    assert n == 5
    lat.synchronize()
    s_o, E_o, M_o = oracle.run(2, 96, 0.43, 17, 5, measure_every=1)
    assert np.array_equal(pairs[:5, 0], E_o) and np.array_equal(pairs[:5, 1], M_o)
    assert lat.observables_async(pairs) == 0  # cleared
    lat.sweep(3, 1)
    small = torch.zeros((2, 2), dtype=torch.int64).pin_memory().numpy()
    with pytest.raises(eng.IsingError):
        lat.observables_async(small)  # 3 pending, room for 2: nothing copied or cleared
    E, M = lat.observables()
    assert len(E) == 3
    lat.close()
