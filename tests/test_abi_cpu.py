"""The C-ABI library without a GPU: it builds, loads, exports every function
that include/*.h declares (ising.h, percolation.h), validates arguments on the host, and its
host-side threshold builder agrees with the oracle and with mpmath."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    return engine.load_library()


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b((?:ising|perc)_\w+)\s*\(", text,
                            flags=re.M)
    return sorted(set(names))


def test_header_symbols_exported(lib):
    names = _declared_functions()
    assert "ising_create" in names and "ising_sweep" in names
    assert "ising_observables" in names and "ising_destroy" in names
    assert "perc_create" in names and "perc_invade" in names and "perc_batch" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version_and_strerror(lib):
    assert b"sm_103a" in lib.ising_version()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.ising_strerror(code)
    assert lib.ising_strerror(-99) == b"unknown status"


@pytest.mark.parametrize("dims,L,beta,layout", [
    (1, 64, 0.4, 0), (4, 64, 0.4, 0), (2, 63, 0.4, 0), (2, 0, 0.4, 0), (2, 1, 0.4, 0),
    (2, -4, 0.4, 0), (2, 64, 0.0, 0), (2, 64, -0.3, 0), (2, 64, float("nan"), 0),
    (2, 64, 0.4, 7), (3, 1 << 12, 0.2, 0),
])
def test_create_rejects_invalid_arguments_on_host(lib, dims, L, beta, layout):
    h = ctypes.c_void_p(1234)
    rc = lib.ising_create(ctypes.byref(h), dims, L, beta, 1, layout)
    assert rc == -1  # ISING_EINVAL, decided before any CUDA call
    assert not h.value


def test_null_handles(lib):
    assert lib.ising_sweep(None, 1, 1) == -1
    assert lib.ising_init(None, 0) == -1
    assert lib.ising_synchronize(None) == -1
    lib.ising_destroy(None)  # NULL-safe


def test_engine_thresholds_match_oracle_and_mpmath(lib, orc):
    from oracle import exact
    from paper_cs_0312006_gb300.engine import compute_thresholds
    rng = np.random.default_rng(3)
    betas = [0.4406868, 0.2216544, 1e-30, 1e-9, 50.0, math.inf] + \
        list(rng.uniform(0.01, 2.0, size=300))
    for beta in betas:
        for dims in (2, 3):
            eng = compute_thresholds(dims, beta)
            assert eng.tolist() == orc.thresholds(dims, beta).tolist()
            if math.isfinite(beta) and beta < 10:
                assert eng[:dims].tolist() == exact.exact_thresholds(dims, beta)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(Exception):
            compute_thresholds(2, bad)


def test_engine_heatbath_thresholds_match_oracle_and_mpmath(lib, orc):
    from oracle import exact
    from paper_cs_0312006_gb300.engine import compute_thresholds_heatbath
    rng = np.random.default_rng(4)
    betas = [0.4406868, 0.2216544, 1e-30, 1e-12, 1e-9, 3.0, 50.0, math.inf] + \
        list(rng.uniform(0.01, 2.0, size=300))
    for beta in betas:
        for dims in (2, 3):
            eng = compute_thresholds_heatbath(dims, beta)
            assert eng.tolist() == orc.thresholds_heatbath(dims, beta).tolist(), (dims, beta)
            if math.isfinite(beta) and beta < 10:
                assert eng.tolist() == exact.exact_thresholds_heatbath(dims, beta)
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(Exception):
            compute_thresholds_heatbath(3, bad)


def test_set_rule_rejects_null_and_unknown(lib):
    assert lib.ising_set_rule(None, 0) == -1
    assert lib.ising_compute_thresholds_heatbath(4, ctypes.c_double(0.3), None) == -1


def test_percolation_rejects_bad_arguments_on_the_host(lib):
    from paper_cs_0312006_gb300 import percolation
    lib = percolation._lib()
    h = ctypes.c_void_p()
    assert lib.perc_create(ctypes.byref(h), 4, 16, 1) == -1
    assert lib.perc_create(ctypes.byref(h), 2, 0, 1) == -1
    assert lib.perc_create(ctypes.byref(h), 3, 2000, 1) == -1  # more than 2^32 sites
    assert lib.perc_generate(None, 0.5) == -1
    assert lib.perc_invade(None, 1, 0, None) == -1
    seeds = (ctypes.c_uint64 * 1)(1)
    res = (percolation.PercResult * 1)()
    assert lib.perc_batch(2, 1024, 0.5, seeds, 1, 1, 0, res, None, None) == -1  # too large
    assert lib.perc_batch(2, 64, 1.5, seeds, 1, 1, 0, res, None, None) == -1
    assert lib.perc_batch(2, 64, 0.5, seeds, 0, 1, 0, res, None, None) == -1
    lib.perc_destroy(None)


def test_observables_gather_rejects_bad_arguments_on_the_host(lib):
    counts = (ctypes.c_int64 * 2)()
    pairs = (ctypes.c_int64 * 8)()
    none2 = (ctypes.c_void_p * 2)(None, None)
    assert lib.ising_observables_gather(None, 1, pairs, 4, counts) == -1
    assert lib.ising_observables_gather(none2, 0, pairs, 4, counts) == -1
    assert lib.ising_observables_gather(none2, 2, pairs, 4, counts) == -1  # NULL lattices
    assert lib.ising_observables_gather(none2, 2, pairs, 4, None) == -1


def test_observables_gather_signal_rejects_bad_arguments_on_the_host(lib):
    counts = (ctypes.c_int64 * 2)()
    pairs = (ctypes.c_int64 * 8)()
    flag = (ctypes.c_int64 * 1)()
    none2 = (ctypes.c_void_p * 2)(None, None)
    assert lib.ising_observables_gather_signal(None, 1, pairs, 4, counts, flag, 1) == -1
    assert lib.ising_observables_gather_signal(none2, 0, pairs, 4, counts, flag, 1) == -1
    assert lib.ising_observables_gather_signal(none2, 2, pairs, 4, counts, flag, 1) == -1


def test_int8_configuration_arguments_checked_on_host():
    from paper_cs_0312006_gb300 import engine
    engine.load_library()
    bad = [(4, 64, 64, dict(kernel=2)), (2, 64, 32, dict(kernel=2)), (2, 64, 64, dict(kernel=5)),
           (2, 64, 64, dict(kernel=2, tile_rows=3)), (2, 64, 64, dict(kernel=2, ctas_per_sm=9)),
           (2, 1, 64, dict(kernel=1))]
    for dims, lo, hi, cfg in bad:
        with pytest.raises(engine.IsingError) as ei:
            engine.set_int8_config(dims, lo, hi, **cfg)
        assert ei.value.code == engine.EINVAL
    engine.set_int8_config(3, 16, 256, kernel=2, tile_rows=4, ctas_per_sm=2)
    engine.clear_int8_configs()


def test_package_exports_the_public_python_api():
    """Every name of the package's public API resolves (the README's calls)."""
    import paper_cs_0312006_gb300 as ising
    from paper_cs_0312006_gb300 import percolation
    for name in ising.__all__:
        assert hasattr(ising, name), name
    for name in ("Lattice", "Batch", "batch_run", "batch_run_static", "observables_gather"):
        assert callable(getattr(ising, name))
    assert callable(percolation.batch) and hasattr(percolation, "FACE")
