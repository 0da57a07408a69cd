"""The int8 pass configurations the autotuner chooses from (register strips,
or tiles staged by bulk copies with 1, 2 or 4 rows per tile and 2, 3 or as
many CTAs per SM as fit): every candidate gives bit-identical spins and E/M,
the winner is what ISING_KERNEL_AUTO then runs, and the result equals the
oracle's."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    yield engine
    engine.clear_int8_configs()


@pytest.mark.parametrize("dims,L", [(2, 512), (3, 64)])
def test_tuned_int8_configuration_runs_and_matches_oracle(eng, dims, L):
    from paper_cs_0312006_gb300 import autotune
    entry = autotune.tune_int8(dims, L, sweeps=3, use_cache=False)
    kinds = {r["config"]["kernel"] for r in entry["results"]}
    assert kinds == {eng.KERNEL_STRIP, eng.KERNEL_TMA}  # both kernels were measured
    assert len(entry["results"]) >= 4
    beta = 0.4 if dims == 2 else 0.22
    lat = eng.Lattice(dims, L, beta, 7)
    assert lat.int8_config() == entry["config"]
    lat.sweep(4, 1)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    s_o, E_o, M_o = oracle.run(dims, L, beta, 7, 4, measure_every=1)
    assert np.array_equal(s, s_o) and np.array_equal(E, E_o) and np.array_equal(M, M_o)
    eng.clear_int8_configs()


def test_configuration_ranges_and_fallback(eng):
    eng.clear_int8_configs()
    eng.set_int8_config(2, 256, 1024, eng.KERNEL_TMA, tile_rows=1, ctas_per_sm=2)
    a = eng.Lattice(2, 512, 0.4, 1)
    assert a.int8_config() == {"kernel": eng.KERNEL_TMA, "tile_rows": 1, "ctas_per_sm": 2}
    b = eng.Lattice(2, 2048, 0.4, 1)  # outside the range: the built-in choice (strip)
    assert b.int8_config()["kernel"] == eng.KERNEL_STRIP
    # half rows of 1025 bytes are not whole 16-byte vectors: the general kernels run
    eng.set_int8_config(2, 2050, 2050, eng.KERNEL_TMA, tile_rows=2)
    e = eng.Lattice(2, 2050, 0.4, 1)
    assert e.int8_config()["kernel"] == eng.KERNEL_STRIP
    c = eng.Lattice(2, 512, 0.4, 1, layout=eng.BITPACK)
    assert c.int8_config()["kernel"] == -1
    for lat in (a, b, c, e):
        lat.close()
    eng.clear_int8_configs()
    d = eng.Lattice(2, 512, 0.4, 1)
    assert d.int8_config()["kernel"] == eng.KERNEL_STRIP  # built-in choice again
    d.close()
