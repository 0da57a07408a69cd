"""The batched launch that allocates nothing (ising_batch_run_static).

Callers that must not allocate device memory while running (real-time loops,
fixed memory pools) advance their lattices with this entry point; its work
queue lives in a fixed device array inside the library.  Through the C ABI it
must give exactly what the allocating batched entry point gives -- spins and
every E/M record bit-identical -- on two calls in a row (the second call
reuses the array the first one left behind).  Kept in a file that is
collected last, and independent of every other test's state.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

INT8, BITPACK = 0, 1

SPECS = [  # dims, L, beta, seed, layout, sweeps per call, measure interval
    (2, 64, 0.44, 11, INT8, 7, 1),
    (2, 96, 0.40, 12, BITPACK, 5, 2),
    (2, 34, 0.30, 13, INT8, 9, 3),
    (2, 200, 0.50, 14, BITPACK, 6, 1),
    (2, 512, 0.44, 15, INT8, 4, 4),
    (3, 16, 0.22, 16, INT8, 8, 1),
    (3, 10, 0.20, 17, BITPACK, 6, 5),
    (3, 32, 0.25, 18, BITPACK, 3, 1),
    (2, 1024, 0.44, 19, BITPACK, 3, 1),
]


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def records_in(t, n, every):
    return (t + n) // every - t // every


def make(eng):
    return [eng.Lattice(d, L, b, sd, layout=lay) for (d, L, b, sd, lay, _, _) in SPECS]


@pytest.mark.parametrize("cluster_size,big_sites", [(4, 1 << 12), (1, 0)])
def test_static_batch_equals_allocating_batch(eng, cluster_size, big_sites):
    import torch
    sweeps = [sp[5] for sp in SPECS]
    every = [sp[6] for sp in SPECS]

    # the allocating entry point: two launches of one batch
    ref = make(eng)
    batch = eng.Batch(ref, sweeps, every, cluster_size=cluster_size, big_sites=big_sites)
    batch.launch()
    batch.launch()
    batch.sync()
    want = [lat.observables() for lat in ref]
    want_spins = [lat.get_spins() for lat in ref]
    batch.close()

    # the entry point that allocates nothing: two calls in a row
    got_E = [[] for _ in SPECS]
    got_M = [[] for _ in SPECS]
    lats = make(eng)
    t = [0] * len(SPECS)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        counts = [records_in(t[i], sweeps[i], every[i]) for i in range(len(SPECS))]
        cap = sum(counts)
        # the caller owns the record buffer (filled with garbage: the call zeroes it)
        rec = torch.full((cap + 3, 2), -7, dtype=torch.int64, device="cuda")
        eng.batch_run_static(lats, sweeps, every, rec.data_ptr(), cap + 3,
                             cluster_size=cluster_size, big_sites=big_sites, stream=stream)
        stream.synchronize()
        host = rec.cpu().numpy()
        off = 0
        for i, c in enumerate(counts):
            got_E[i].append(host[off:off + c, 0])
            got_M[i].append(host[off:off + c, 1])
            off += c
        assert (host[cap:] == -7).all()  # nothing written past this call's records
        t = [t[i] + sweeps[i] for i in range(len(SPECS))]
    for i, lat in enumerate(lats):
        assert lat.info().sweeps_done == 2 * sweeps[i]
        assert np.array_equal(lat.get_spins(), want_spins[i]), SPECS[i]
        assert np.array_equal(np.concatenate(got_E[i]), want[i][0]), SPECS[i]
        assert np.array_equal(np.concatenate(got_M[i]), want[i][1]), SPECS[i]
        # the handle's own record buffer is untouched
        assert lat.info().pending_records == 0
    for lat in lats + ref:
        lat.close()


def test_static_batch_rejects_too_many_or_too_little_room(eng):
    import torch
    lat = eng.Lattice(2, 32, 0.4, 1)
    rec = torch.zeros((8, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(eng.IsingError) as ei:  # more lattices than the fixed table holds
        eng.batch_run_static([lat] * 2049, 1, 1, rec.data_ptr(), 8)
    assert ei.value.code == eng.ERANGE
    with pytest.raises(eng.IsingError) as ei:  # 10 records do not fit in 8 pairs
        eng.batch_run_static([lat], 10, 1, rec.data_ptr(), 8)
    assert ei.value.code == eng.ERANGE
    assert lat.info().sweeps_done == 0  # nothing was issued
    lat.close()


def test_static_batch_refuses_lattices_on_another_stream(eng):
    """The call is ordered against a handle's own work by stream order alone,
    so lattices must already be on the call's stream: a lattice on a side
    stream is refused with nothing issued, and the same call on that stream
    gives the allocating batch's result."""
    import torch
    side = torch.cuda.Stream()
    spec = SPECS[0]
    lat = eng.Lattice(*spec[:5])
    lat.set_stream(side)
    rec = torch.zeros((spec[5] + 1, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(eng.IsingError) as ei:
        eng.batch_run_static([lat], spec[5], spec[6], rec.data_ptr(), spec[5] + 1,
                             stream=torch.cuda.default_stream())
    assert ei.value.code == eng.EINVAL
    assert lat.info().sweeps_done == 0
    with torch.cuda.stream(side):
        rec.zero_()
    eng.batch_run_static([lat], spec[5], spec[6], rec.data_ptr(), spec[5] + 1, stream=side)
    side.synchronize()
    got = rec.cpu().numpy()[:spec[5]]
    ref = eng.Lattice(*spec[:5])
    batch = eng.Batch([ref], [spec[5]], [spec[6]])
    batch.launch()
    batch.sync()
    E, M = ref.observables()
    batch.close()
    assert np.array_equal(got[:, 0], E) and np.array_equal(got[:, 1], M)
    assert np.array_equal(lat.get_spins(), ref.get_spins())
    lat.close()
    ref.close()
