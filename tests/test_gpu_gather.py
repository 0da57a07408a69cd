"""ising_observables_gather on the GPU: one queued kernel reads and clears
the pending (E, M) records of many lattices into pinned host memory.  Every
lattice's records must equal those of a twin lattice read with
ising_observables (and the oracle's, for the lattices it can run here), the
slots must be clear afterwards, and bad buffers, small capacities and mixed
streams must be refused with nothing queued."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HOT = 0
INT8, BITPACK = 0, 1


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


# (dims, L, beta, seed, layout, sweeps, measure_every): the single-launch small
# path, the staged int8 kernel, the bit-packed pass, 3D, a lattice with no
# records pending (every > sweeps)
CASES = [(2, 64, 0.44, 11, INT8, 7, 1), (2, 8192, 0.40, 12, INT8, 3, 1),
         (2, 256, 0.30, 13, BITPACK, 6, 2), (3, 32, 0.22, 14, INT8, 5, 1),
         (2, 128, 0.50, 15, INT8, 3, 10)]


def make(eng, c):
    dims, L, beta, seed, layout, _, _ = c
    return eng.Lattice(dims, L, beta, seed, layout=layout)


def test_gather_equals_per_lattice_reads(eng):
    import torch
    lats = [make(eng, c) for c in CASES]
    twins = [make(eng, c) for c in CASES]
    pairs = torch.zeros((64, 2), dtype=torch.int64).pin_memory().numpy()
    for rnd in range(2):  # twice: the first read must have cleared the slots
        for lat, twin, c in zip(lats, twins, CASES):
            lat.sweep(c[5], c[6])
            twin.sweep(c[5], c[6])
        counts = eng.observables_gather(lats, pairs)
        torch.cuda.synchronize()
        off = 0
        for k, (twin, c) in enumerate(zip(twins, CASES)):
            E, M = twin.observables()
            assert counts[k] == len(E), (rnd, c)
            assert np.array_equal(pairs[off:off + counts[k], 0], E), (rnd, c)
            assert np.array_equal(pairs[off:off + counts[k], 1], M), (rnd, c)
            off += counts[k]
        assert counts[-1] == 0  # every 10th sweep: none yet
    # nothing pending now
    again = eng.observables_gather(lats, pairs)
    assert not again.any()
    # a handle listed twice: its records at the first entry, none at the second
    lats[0].sweep(2, 1)
    counts = eng.observables_gather([lats[0], lats[1], lats[0]], pairs)
    torch.cuda.synchronize()
    assert list(counts) == [2, 0, 0]
    twins[0].sweep(2, 1)
    E, M = twins[0].observables()
    assert np.array_equal(pairs[:2, 0], E) and np.array_equal(pairs[:2, 1], M)
    # the small 2D lattice against the oracle: 14 sweeps, E/M after each
    lat = eng.Lattice(2, 64, 0.44, 11, layout=INT8)
    lat.sweep(14, 1)
    counts = eng.observables_gather([lat], pairs)
    torch.cuda.synchronize()
    _, E_o, M_o = oracle.run(2, 64, 0.44, 11, 14, start=HOT)
    assert counts[0] == 14
    assert np.array_equal(pairs[:14, 0], E_o) and np.array_equal(pairs[:14, 1], M_o)
    for x in lats + twins + [lat]:
        x.close()


def test_gather_refusals(eng):
    import torch
    a = eng.Lattice(2, 64, 0.4, 1)
    b = eng.Lattice(2, 64, 0.4, 2)
    a.sweep(3, 1)
    b.sweep(3, 1)
    pinned = torch.zeros((8, 2), dtype=torch.int64).pin_memory().numpy()
    pageable = np.zeros((8, 2), dtype=np.int64)
    with pytest.raises(eng.IsingError) as ei:
        eng.observables_gather([a, b], pageable)
    assert ei.value.code == eng.EINVAL
    with pytest.raises(eng.IsingError) as ei:
        eng.observables_gather([a, b], pinned[:5])  # 6 records pending
    assert ei.value.code == eng.ERANGE
    side = torch.cuda.Stream()
    c = eng.Lattice(2, 64, 0.4, 3, stream=side)
    with pytest.raises(eng.IsingError) as ei:
        eng.observables_gather([a, c], pinned)
    assert ei.value.code == eng.EINVAL
    # nothing was cleared by the refused calls
    counts = eng.observables_gather([a, b], pinned)
    torch.cuda.synchronize()
    assert list(counts) == [3, 3]
    for x in (a, b, c):
        x.close()


def test_gather_signal_flag(eng):
    """ising_observables_gather_signal: once the host sees the value in the
    pinned flag word, the records are in place -- read here before any
    synchronisation -- and equal the twins' per-lattice reads."""
    import time
    import torch
    lats = [make(eng, c) for c in CASES[:4]]
    twins = [make(eng, c) for c in CASES[:4]]
    pairs = torch.zeros((64, 2), dtype=torch.int64).pin_memory().numpy()
    flag = torch.zeros(2, dtype=torch.int64).pin_memory().numpy()
    for k in (1, 2, 3):
        for lat, twin, c in zip(lats, twins, CASES):
            lat.sweep(c[5], c[6])
            twin.sweep(c[5], c[6])
        counts = eng.observables_gather(lats, pairs, flag=flag[1:], value=k)
        t0 = time.monotonic()
        while flag[1] != k:
            assert time.monotonic() - t0 < 30.0, "the flag never arrived"
        got = pairs[:int(counts.sum())].copy()  # before any synchronisation
        off = 0
        for c_k, twin in zip(counts, twins):
            E, M = twin.observables()
            assert c_k == len(E)
            assert np.array_equal(got[off:off + c_k, 0], E)
            assert np.array_equal(got[off:off + c_k, 1], M)
            off += int(c_k)
    # nothing pending: the flag still arrives
    counts = eng.observables_gather(lats, pairs, flag=flag[1:], value=99)
    torch.cuda.synchronize()
    assert flag[1] == 99 and not counts.any()
    assert flag[0] == 0  # the neighbouring word is untouched
    with pytest.raises(eng.IsingError) as ei:
        eng.observables_gather(lats, pairs, flag=np.zeros(1, dtype=np.int64), value=1)
    assert ei.value.code == eng.EINVAL
    for x in lats + twins:
        x.close()
