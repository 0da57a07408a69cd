"""Spins in and out of the device without waiting (ising_set_spins_async,
ising_get_spins_async), and the conversion kernels behind every spin
transfer and initial state: canonical int8 +-1 <-> the int8 and bit-packed
layouts, by whole 16-byte vectors / 32-bit words where the half rows allow it
and site by site elsewhere.  Checked against the oracle, which keeps the
canonical order itself."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

INT8, BITPACK = 0, 1
HOT, COLD_UP, COLD_DOWN = 0, 1, 2

# (dims, L): whole vectors and words (64, 128), int8 vectors but ragged packed
# words (96), ragged everywhere (34, 10), 3D with and without whole words
SHAPES = [(2, 64), (2, 128), (2, 96), (2, 34), (3, 32), (3, 10), (3, 64)]


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def pinned(a: np.ndarray):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t


@pytest.mark.parametrize("layout", [INT8, BITPACK])
@pytest.mark.parametrize("dims,L", SHAPES)
def test_initial_states_match_oracle(eng, dims, L, layout):
    for start in (HOT, COLD_UP, COLD_DOWN):
        lat = eng.Lattice(dims, L, 0.3, 20031109 + L, layout=layout, start=start)
        got = lat.get_spins()
        lat.close()
        assert np.array_equal(got, oracle.init(dims, L, 20031109 + L, start)), (dims, L, start)


@pytest.mark.parametrize("layout", [INT8, BITPACK])
@pytest.mark.parametrize("dims,L", SHAPES)
def test_async_load_sweep_and_read_match_oracle(eng, dims, L, layout):
    import torch
    rng = np.random.default_rng(dims * 1000 + L)
    n = L ** dims
    s0 = rng.choice(np.array([-1, 1], dtype=np.int8), size=n)
    src = pinned(s0)
    out = torch.empty(n, dtype=torch.int8).pin_memory()
    beta, seed, t0, sweeps = 0.41, 77 + L, 5, 4
    lat = eng.Lattice(dims, L, beta, seed, layout=layout)
    lat.set_spins_async(src.data_ptr(), t0)
    lat.sweep(sweeps, 1)
    lat.get_spins_async(out.data_ptr())
    lat.synchronize()
    E, M = lat.observables()
    assert lat.info().sweeps_done == t0 + sweeps
    lat.close()
    s_o, E_o, M_o = oracle.run(dims, L, beta, seed, sweeps, measure_every=1, s=s0, t0=t0)
    assert np.array_equal(out.numpy(), s_o), (dims, L, layout)
    assert np.array_equal(E, E_o) and np.array_equal(M, M_o), (dims, L, layout)


@pytest.mark.parametrize("layout", [INT8, BITPACK])
def test_device_memory_both_ways(eng, layout):
    import torch
    dims, L = 2, 256
    rng = np.random.default_rng(3)
    s0 = rng.choice(np.array([-1, 1], dtype=np.int8), size=L * L)
    dev_in = torch.from_numpy(s0).cuda()
    dev_out = torch.zeros(L * L, dtype=torch.int8, device="cuda")
    lat = eng.Lattice(dims, L, 0.44, 9, layout=layout)
    lat.set_spins_async(dev_in.data_ptr(), 0)
    lat.get_spins_async(dev_out.data_ptr())
    lat.synchronize()
    assert np.array_equal(dev_out.cpu().numpy(), s0)
    # the synchronous read into pinned memory (written by the kernel) and into
    # pageable memory (through a device buffer) agree
    pin = torch.empty(L * L, dtype=torch.int8).pin_memory()
    lat.get_spins(pin.numpy())
    assert np.array_equal(pin.numpy(), s0)
    assert np.array_equal(lat.get_spins(), s0)
    lat.close()


@pytest.mark.parametrize("layout", [INT8, BITPACK])
@pytest.mark.parametrize("L", [64, 34])
def test_invalid_values_reported_once(eng, L, layout):
    lat = eng.Lattice(2, L, 0.4, 1, layout=layout)
    good = oracle.init(2, L, 1, HOT)
    bad = good.copy()
    bad[3] = 0
    bad[L + 1] = 5
    src = pinned(bad)
    lat.set_spins_async(src.data_ptr(), 0)
    with pytest.raises(eng.IsingError) as ei:
        lat.synchronize()
    assert ei.value.code == eng.EINVAL
    lat.synchronize()  # reported once, then cleared
    # a valid load afterwards restores a defined state
    src_ok = pinned(good)
    lat.set_spins_async(src_ok.data_ptr(), 0)
    lat.sweep(3, 1)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    s_o, E_o, M_o = oracle.run(2, L, 0.4, 1, 3, measure_every=1, s=good)
    assert np.array_equal(s, s_o) and np.array_equal(E, E_o) and np.array_equal(M, M_o)


def test_pageable_memory_refused(eng):
    lat = eng.Lattice(2, 64, 0.4, 1)
    host = np.ones(64 * 64, dtype=np.int8)
    with pytest.raises(eng.IsingError) as ei:
        lat.set_spins_async(host.ctypes.data, 0)
    assert ei.value.code == eng.EINVAL
    with pytest.raises(eng.IsingError) as ei:
        lat.get_spins_async(host.ctypes.data)
    assert ei.value.code == eng.EINVAL
    with pytest.raises(eng.IsingError) as ei:
        lat.set_spins_async(pinned(host).data_ptr(), 2 ** 32 + 1)
    assert ei.value.code == eng.ERANGE
    assert lat.info().sweeps_done == 0
    lat.close()
