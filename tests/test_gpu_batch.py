"""The batched persistent launch gives every lattice exactly the result it
gets alone (same arithmetic, same counter-based draws), for any mix of
dims, sizes, layouts, sweep counts and measurement intervals, for every
launch option, and across repeated (graph-replayed) launches."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

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


def mix_specs(seed=0, n=48):
    rng = np.random.default_rng(seed)
    sizes2 = [2, 4, 6, 10, 16, 30, 34, 64, 96, 128, 200, 256, 384, 512, 640]
    sizes3 = [2, 4, 6, 8, 10, 16, 32, 34, 64]
    specs = []
    for j in range(n):
        dims = 2 if j % 3 else 3
        L = int(rng.choice(sizes2 if dims == 2 else sizes3))
        beta = float(rng.uniform(0.2, 0.6) if dims == 2 else rng.uniform(0.15, 0.3))
        layout = BITPACK if j % 2 == 0 else INT8
        sweeps = int(rng.integers(3, 25))
        every = int(rng.choice([1, 3, 10]))
        specs.append((dims, L, beta, 1000 + j, layout, sweeps, every))
    return specs


def run_alone(eng, spec, launches=1):
    dims, L, beta, seed, layout, sweeps, every = spec
    lat = eng.Lattice(dims, L, beta, seed, layout=layout)
    for _ in range(launches):
        lat.sweep(sweeps, every)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    return s, E, M


def run_batch(eng, specs, launches=1, **opts):
    lats = [eng.Lattice(d, L, b, sd, layout=lay) for (d, L, b, sd, lay, _, _) in specs]
    batch = eng.Batch(lats, [sp[5] for sp in specs], [sp[6] for sp in specs], **opts)
    for _ in range(launches):
        batch.launch()
    batch.sync()
    out = []
    for lat in lats:
        E, M = lat.observables()
        out.append((lat.get_spins(), E, M))
    batch.close()
    for lat in lats:
        lat.close()
    return out


def same(a, b):
    return (np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            and np.array_equal(a[2], b[2]))


def test_batch_equals_alone(eng):
    specs = mix_specs(0)
    got = run_batch(eng, specs, launches=2, cluster_size=4, big_sites=4096)
    for spec, g in zip(specs, got):
        assert same(g, run_alone(eng, spec, launches=2)), spec


def test_batch_against_oracle(eng):
    specs = [(2, 34, 0.44, 7, INT8, 9, 1), (3, 6, 0.22, 8, INT8, 9, 3),
             (2, 128, 0.5, 9, BITPACK, 9, 1), (2, 200, 0.3, 10, INT8, 9, 2),
             (2, 70, 0.4, 11, BITPACK, 9, 1), (3, 10, 0.2, 12, BITPACK, 9, 2)]
    got = run_batch(eng, specs, launches=1, cluster_size=2, big_sites=2000)
    for (d, L, b, sd, _, sw, ev), g in zip(specs, got):
        o = oracle.run(d, L, b, sd, sw, measure_every=ev)
        assert same(g, o), (d, L)


@pytest.mark.parametrize("opts", [
    dict(cluster_size=1),
    dict(cluster_size=2, big_sites=1 << 12, block_threads=128),
    dict(cluster_size=8, big_sites=1 << 14, block_threads=256),
    dict(cluster_size=4, big_sites=1 << 10, use_graph=False),
])
def test_batch_options_do_not_change_results(eng, opts):
    specs = mix_specs(1, n=24)
    ref = run_batch(eng, specs, launches=1)
    got = run_batch(eng, specs, launches=1, **opts)
    for spec, a, b in zip(specs, ref, got):
        assert same(a, b), (spec, opts)


def test_batch_replays_continue(eng):
    specs = [(2, 96, 0.4, 5, INT8, 7, 1), (3, 16, 0.2, 6, INT8, 7, 2),
             (2, 256, 0.44, 7, BITPACK, 7, 7)]
    got = run_batch(eng, specs, launches=3, cluster_size=2, big_sites=10000)
    for (d, L, b, sd, lay, sw, ev), g in zip(specs, got):
        alone = run_alone(eng, (d, L, b, sd, lay, 3 * sw, ev))
        assert same(g, alone)


def test_batch_then_direct_use(eng):
    """After sync the lattices can be swept directly and batched again."""
    lat = eng.Lattice(2, 64, 0.44, 3)
    ref = eng.Lattice(2, 64, 0.44, 3)
    b = eng.Batch([lat], [5], [1])
    b.launch()
    b.sync()
    lat.sweep(4, 1)
    b.launch()
    b.sync()
    ref.sweep(14, 1)
    assert np.array_equal(lat.get_spins(), ref.get_spins())
    E1, M1 = lat.observables()
    E2, M2 = ref.observables()
    assert np.array_equal(E1, E2) and np.array_equal(M1, M2)
    b.close()
    lat.close()
    ref.close()


def test_batch_rejects_bad_arguments(eng):
    lat = eng.Lattice(2, 32, 0.4, 1)
    with pytest.raises(eng.IsingError):
        eng.Batch([lat, lat], [1, 1])
    with pytest.raises(eng.IsingError):
        eng.Batch([lat], [1], block_threads=1000)
    with pytest.raises(eng.IsingError):
        eng.Batch([lat], [1], cluster_size=9)
    with pytest.raises(eng.IsingError):
        eng.Batch([lat], [1], measure_every=[0])
    lat.close()


def test_batch_run_one_call_against_oracle(eng):
    """ising_batch_run (create + launch + sync + destroy in one call): every
    lattice's spins and E/M records equal the oracle's own run."""
    specs = [(2, 64, 0.4406868, 20031109, INT8, 12, 1),
             (2, 128, 0.35, 7, BITPACK, 9, 1),
             (3, 16, 0.2216544, 5, INT8, 10, 1),
             (2, 34, 0.55, 3, INT8, 11, 1),
             (3, 8, 0.3, 9, BITPACK, 7, 1)]
    lats = [eng.Lattice(d, L, b, sd, layout=lay) for (d, L, b, sd, lay, _, _) in specs]
    eng.batch_run(lats, [sp[5] for sp in specs], 1)
    for lat, (d, L, b, sd, lay, n, every) in zip(lats, specs):
        E, M = lat.observables()
        s = lat.get_spins()
        lat.close()
        s_o, E_o, M_o = oracle.run(d, L, b, sd, n, measure_every=every)
        assert np.array_equal(E, E_o) and np.array_equal(M, M_o), (d, L)
        assert np.array_equal(s, s_o), (d, L)


def test_batch_run_refusals(eng):
    lat = eng.Lattice(2, 32, 0.4, 1)
    for args in (([lat], [1], 0), ([lat, lat], [1, 1], 1), ([lat], [-1], 1)):
        with pytest.raises(eng.IsingError) as ei:
            eng.batch_run(*args)
        assert ei.value.code == eng.EINVAL
    assert lat.info().sweeps_done == 0
    lat.close()


def test_batch_update_between_launches_equals_alone(eng):
    """One batch reused for changing lattice sets (ising_batch_update), the
    second launch queued behind the first with no synchronisation: every
    lattice ends as if its sweeps had run alone."""
    specs = mix_specs(5, n=24)
    lats = [eng.Lattice(d, L, b, sd, layout=lay) for (d, L, b, sd, lay, _, _) in specs]
    first, second = list(range(0, 16)), list(range(8, 24))  # overlapping sets
    batch = eng.Batch([lats[i] for i in first], [specs[i][5] for i in first],
                      [specs[i][6] for i in first], cluster_size=2, big_sites=4096,
                      use_graph=False)
    batch.launch()
    batch.update([lats[i] for i in second], [specs[i][5] for i in second],
                 [specs[i][6] for i in second])
    batch.launch()
    batch.sync()
    batch.close()
    for i, (spec, lat) in enumerate(zip(specs, lats)):
        launches = (i in first) + (i in second)
        E, M = lat.observables()
        got = (lat.get_spins(), E, M)
        lat.close()
        assert same(got, run_alone(eng, spec, launches=launches)), (i, spec)
