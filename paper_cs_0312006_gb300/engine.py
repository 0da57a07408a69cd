"""Thin Python binding of the C ABI in ``include/ising.h`` (argument marshalling
only; every step of the simulation runs in the CUDA kernels of the shared
library).

There is no CPU path: if the compiled library is missing or cannot be loaded,
``load_library()`` raises ``ImportError``.  PyTorch is used only to hand the
engine a CUDA stream (``Lattice.set_stream``) and to receive device exports
into a tensor (``Lattice.export_device``).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

INT8, BITPACK, AUTO = 0, 1, 2
HOT, COLD_UP, COLD_DOWN = 0, 1, 2
KERNEL_AUTO, KERNEL_STRIP, KERNEL_TMA = 0, 1, 2
RULE_METROPOLIS, RULE_HEATBATH, RULE_DEMON, RULE_MULTIHIT = 0, 1, 2, 3

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUDGET, ERANGE = 0, -1, -2, -3, -4, -5, -6

_lock = threading.Lock()
_lib = None


class IsingError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load_library().ising_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})")


class BatchOpts(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("cluster_size", ctypes.c_int),
                ("big_sites", ctypes.c_int64), ("use_graph", ctypes.c_int),
                ("huge_sites", ctypes.c_int64)]


class Int8Config(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int)]


class IsingInfo(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("L", ctypes.c_int), ("layout", ctypes.c_int),
                ("rule", ctypes.c_int), ("beta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("sweeps_done", ctypes.c_uint64),
                ("sites", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("pending_records", ctypes.c_int64)]


def library_path() -> str:
    return _build.LIB_PATH


def load_library():
    """Load the compiled engine (built by ``__graft_entry__.build()`` or
    ``python -m paper_cs_0312006_gb300._build``).  Raises ImportError if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"CUDA engine library not built: {path} is missing; "
                              "run paper_cs_0312006_gb300._build.build() first")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        sig = {
            "ising_create": ([ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_uint64, ctypes.c_int], ctypes.c_int),
            "ising_init": ([P, ctypes.c_int], ctypes.c_int),
            "ising_sweep": ([P, ctypes.c_int64, ctypes.c_int], ctypes.c_int),
            "ising_observables": ([P, i64p, i64p, ctypes.c_int64, i64p], ctypes.c_int),
            "ising_observables_async": ([P, P, ctypes.c_int64, i64p], ctypes.c_int),
            "ising_observables_gather": ([ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_int64,
                                          i64p], ctypes.c_int),
            "ising_observables_gather_signal": ([ctypes.POINTER(P), ctypes.c_int, P,
                                                 ctypes.c_int64, i64p, P, ctypes.c_int64],
                                                ctypes.c_int),
            "ising_get_spins": ([P, P], ctypes.c_int),
            "ising_set_spins": ([P, P, ctypes.c_uint64], ctypes.c_int),
            "ising_set_spins_async": ([P, P, ctypes.c_uint64], ctypes.c_int),
            "ising_get_spins_async": ([P, P], ctypes.c_int),
            "ising_export_device": ([P, P], ctypes.c_int),
            "ising_set_stream": ([P, P], ctypes.c_int),
            "ising_thresholds": ([P, u32p], ctypes.c_int),
            "ising_compute_thresholds": ([ctypes.c_int, ctypes.c_double, u32p], ctypes.c_int),
            "ising_compute_thresholds_heatbath": ([ctypes.c_int, ctypes.c_double, u32p],
                                                  ctypes.c_int),
            "ising_set_rule": ([P, ctypes.c_int], ctypes.c_int),
            "ising_set_demons": ([P, P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ising_set_hits": ([P, ctypes.c_int], ctypes.c_int),
            "ising_get_demons": ([P, P], ctypes.c_int),
            "ising_get_info": ([P, ctypes.POINTER(IsingInfo)], ctypes.c_int),
            "ising_synchronize": ([P], ctypes.c_int),
            "ising_set_kernel": ([P, ctypes.c_int], ctypes.c_int),
            "ising_get_kernel": ([P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "ising_set_int8_config": ([ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Int8Config)], ctypes.c_int),
            "ising_clear_int8_configs": ([], ctypes.c_int),
            "ising_get_int8_config": ([P, ctypes.POINTER(Int8Config)], ctypes.c_int),
            "ising_test_inject_timeout": ([ctypes.c_int], ctypes.c_int),
            "ising_philox_fill": ([P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint64, P], ctypes.c_int),
            "ising_philox_probe": ([P, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_uint64, P], ctypes.c_int),
            "ising_destroy": ([P], None),
            "ising_release_cached_memory": ([], ctypes.c_int),
            "ising_batch_create": ([ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int, i64p,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(BatchOpts), P],
                                   ctypes.c_int),
            "ising_batch_launch": ([P], ctypes.c_int),
            "ising_batch_update": ([P, ctypes.POINTER(P), ctypes.c_int, i64p,
                                    ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
            "ising_batch_sync": ([P], ctypes.c_int),
            "ising_batch_info": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                                 ctypes.c_int),
            "ising_batch_destroy": ([P], None),
            "ising_batch_run": ([ctypes.POINTER(P), ctypes.c_int, i64p, ctypes.c_int, P],
                                ctypes.c_int),
            "ising_batch_run_static": ([ctypes.POINTER(P), ctypes.c_int, i64p,
                                        ctypes.POINTER(ctypes.c_int), P, ctypes.c_int64,
                                        ctypes.POINTER(BatchOpts), P], ctypes.c_int),
            "ising_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "ising_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise IsingError(rc, what)


def philox_fill(dev_ptr: int, n: int, c1: int, c2: int, c3: int, seed: int, stream=None) -> None:
    """``ising_philox_fill``: 4n uint32 of Philox4x32-10 at ``dev_ptr``."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(load_library().ising_philox_fill(ctypes.c_void_p(dev_ptr), n, c1, c2, c3,
                                            ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                            ctypes.c_void_p(int(raw) if raw else 0)),
           "ising_philox_fill")


def philox_probe(dev_ptr: int, blocks: int, threads: int, iters: int, variant: int = 0,
                 chains: int = 8, seed: int = 0, stream=None) -> None:
    """``ising_philox_probe``: blocks x threads threads each fold iters x chains
    Philox4x32-10 calls into one uint32 at ``dev_ptr``."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(load_library().ising_philox_probe(ctypes.c_void_p(dev_ptr), blocks, threads, iters,
                                             variant, chains,
                                             ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF),
                                             ctypes.c_void_p(int(raw) if raw else 0)),
           "ising_philox_probe")


def set_int8_config(dims: int, L_min: int, L_max: int, kernel: int, tile_rows: int = 0,
                    ctas_per_sm: int = 0) -> None:
    """``ising_set_int8_config``: the int8 pass configuration that
    ISING_KERNEL_AUTO runs for lattices of ``dims`` with L_min <= L <= L_max."""
    cfg = Int8Config(kernel, tile_rows, ctas_per_sm)
    _check(load_library().ising_set_int8_config(dims, L_min, L_max, ctypes.byref(cfg)),
           "ising_set_int8_config")


def clear_int8_configs() -> None:
    _check(load_library().ising_clear_int8_configs(), "ising_clear_int8_configs")


def test_inject_timeout(on: bool) -> None:
    """Test hook: make every staged (TMA) pass's bounded wait run out."""
    _check(load_library().ising_test_inject_timeout(1 if on else 0), "ising_test_inject_timeout")


def compute_thresholds(dims: int, beta: float) -> np.ndarray:
    """``ising_compute_thresholds``: the engine's host-side threshold table."""
    out = np.zeros(3, dtype=np.uint32)
    _check(load_library().ising_compute_thresholds(
        dims, float(beta), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
        f"ising_compute_thresholds(dims={dims}, beta={beta})")
    return out


def compute_thresholds_heatbath(dims: int, beta: float) -> np.ndarray:
    """``ising_compute_thresholds_heatbath``: the engine's heat-bath table (7 entries)."""
    out = np.zeros(7, dtype=np.uint32)
    _check(load_library().ising_compute_thresholds_heatbath(
        dims, float(beta), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
        f"ising_compute_thresholds_heatbath(dims={dims}, beta={beta})")
    return out


class Lattice:
    """One lattice on the current CUDA device (``ising_create``)."""

    def __init__(self, dims: int, L: int, beta: float, seed: int, layout: int = INT8,
                 start: int = HOT, stream=None, kernel: int = KERNEL_AUTO,
                 rule: int = RULE_METROPOLIS):
        lib = load_library()
        self._lib = lib
        self._h = ctypes.c_void_p()
        _check(lib.ising_create(ctypes.byref(self._h), dims, L, float(beta),
                                ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), layout),
               f"ising_create(dims={dims}, L={L}, beta={beta})")
        if stream is not None:
            self.set_stream(stream)
        if kernel != KERNEL_AUTO:
            self.set_kernel(kernel)
        if rule != RULE_METROPOLIS:
            self.set_rule(rule)
        if start != HOT:
            self.init(start)

    # -- lifetime ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ising_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ------------------------------------------------------------
    def init(self, start: int = HOT) -> None:
        _check(self._lib.ising_init(self._h, start), "ising_init")

    def sweep(self, n: int, measure_every: int = 1) -> None:
        _check(self._lib.ising_sweep(self._h, int(n), int(measure_every)), "ising_sweep")

    def observables(self):
        """Pending (E, M) records as two int64 numpy arrays (clears them)."""
        cnt = ctypes.c_int64(0)
        _check(self._lib.ising_observables(self._h, None, None, 0, ctypes.byref(cnt)),
               "ising_observables")
        n = cnt.value
        E = np.zeros(max(n, 1), dtype=np.int64)
        M = np.zeros(max(n, 1), dtype=np.int64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        _check(self._lib.ising_observables(self._h, E.ctypes.data_as(i64p),
                                           M.ctypes.data_as(i64p), len(E), ctypes.byref(cnt)),
               "ising_observables")
        return E[:n].copy(), M[:n].copy()

    def observables_async(self, pairs: np.ndarray) -> int:
        """Enqueue the pending records' copy into ``pairs`` (a pinned int64
        array of shape (cap, 2) or a view of one) and clear them; returns their
        number at once.  The values are valid after the stream passes this
        point (e.g. an event recorded next)."""
        assert pairs.dtype == np.int64 and pairs.flags.c_contiguous
        cnt = ctypes.c_int64(0)
        _check(self._lib.ising_observables_async(self._h, pairs.ctypes.data, pairs.size // 2,
                                                 ctypes.byref(cnt)),
               "ising_observables_async")
        return cnt.value

    def get_spins(self, out: np.ndarray | None = None) -> np.ndarray:
        info = self.info()
        if out is None:
            out = np.empty(info.sites, dtype=np.int8)
        assert out.dtype == np.int8 and out.size == info.sites and out.flags.c_contiguous
        _check(self._lib.ising_get_spins(self._h, out.ctypes.data), "ising_get_spins")
        return out

    def set_spins(self, spins: np.ndarray, t: int = 0) -> None:
        s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        _check(self._lib.ising_set_spins(self._h, s.ctypes.data, int(t)), "ising_set_spins")

    def set_spins_async(self, spins_ptr: int, t: int = 0) -> None:
        """``ising_set_spins_async``: load L^dims canonical int8 spins from
        device memory or pinned host memory at ``spins_ptr`` (e.g.
        ``tensor.data_ptr()`` of a pinned CPU or a CUDA int8 tensor) in stream
        order; invalid values are reported by the next synchronising call."""
        _check(self._lib.ising_set_spins_async(self._h, ctypes.c_void_p(spins_ptr), int(t)),
               "ising_set_spins_async")

    def get_spins_async(self, out_ptr: int) -> None:
        """``ising_get_spins_async``: write canonical int8 spins to device
        memory or pinned host memory at ``out_ptr`` in stream order."""
        _check(self._lib.ising_get_spins_async(self._h, ctypes.c_void_p(out_ptr)),
               "ising_get_spins_async")

    def export_device(self, out_ptr: int) -> None:
        """Write canonical int8 spins to device memory at ``out_ptr``
        (e.g. ``tensor.data_ptr()`` of an int8 CUDA tensor), on the handle's stream."""
        _check(self._lib.ising_export_device(self._h, ctypes.c_void_p(out_ptr)),
               "ising_export_device")

    def set_stream(self, stream) -> None:
        """Accepts a raw cudaStream_t (int) or an object with ``.cuda_stream``."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(self._lib.ising_set_stream(self._h, ctypes.c_void_p(int(raw) if raw else 0)),
               "ising_set_stream")

    def thresholds(self) -> np.ndarray:
        out = np.zeros(3, dtype=np.uint32)
        _check(self._lib.ising_thresholds(self._h,
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
               "ising_thresholds")
        return out

    def info(self) -> IsingInfo:
        inf = IsingInfo()
        _check(self._lib.ising_get_info(self._h, ctypes.byref(inf)), "ising_get_info")
        return inf

    def synchronize(self) -> None:
        _check(self._lib.ising_synchronize(self._h), "ising_synchronize")

    def set_kernel(self, kernel: int) -> None:
        """int8 pass kernel: KERNEL_AUTO, KERNEL_STRIP or KERNEL_TMA."""
        _check(self._lib.ising_set_kernel(self._h, int(kernel)), "ising_set_kernel")

    def int8_config(self) -> dict:
        """``ising_get_int8_config``: the int8 pass this lattice runs now."""
        c = Int8Config()
        _check(self._lib.ising_get_int8_config(self._h, ctypes.byref(c)), "ising_get_int8_config")
        return {"kernel": c.kernel, "tile_rows": c.tile_rows, "ctas_per_sm": c.ctas_per_sm}

    def kernel(self) -> int:
        """The int8 pass kernel the sweeps run (KERNEL_STRIP / KERNEL_TMA; -1 if packed)."""
        k = ctypes.c_int(0)
        _check(self._lib.ising_get_kernel(self._h, ctypes.byref(k)), "ising_get_kernel")
        return k.value

    def set_rule(self, rule: int) -> None:
        """Local update rule of later sweeps: RULE_METROPOLIS, RULE_HEATBATH or
        RULE_DEMON (after set_demons)."""
        _check(self._lib.ising_set_rule(self._h, int(rule)), "ising_set_rule")

    def set_hits(self, hits: int) -> None:
        """Trials per visit of RULE_MULTIHIT."""
        _check(self._lib.ising_set_hits(self._h, int(hits)), "ising_set_hits")

    def set_demons(self, q: np.ndarray | None = None, fill: int = 0, qmax: int = 3) -> None:
        """Demons of the deterministic dynamics: canonical uint8 array ``q``
        (values <= qmax), or every demon = ``fill``."""
        if q is None:
            _check(self._lib.ising_set_demons(self._h, None, int(fill), int(qmax)),
                   "ising_set_demons")
            return
        qq = np.ascontiguousarray(q, dtype=np.uint8).reshape(-1)
        assert qq.size == self.info().sites
        _check(self._lib.ising_set_demons(self._h, qq.ctypes.data, 0, int(qmax)),
               "ising_set_demons")

    def get_demons(self) -> np.ndarray:
        out = np.empty(self.info().sites, dtype=np.uint8)
        _check(self._lib.ising_get_demons(self._h, out.ctypes.data), "ising_get_demons")
        return out

    @property
    def handle(self) -> int:
        return int(self._h.value or 0)


class Batch:
    """Many lattices advanced by one persistent launch (``ising_batch_*``).

    ``sweeps`` and ``measure_every`` are per lattice (sequences) or scalars.
    While a launch is in flight the lattices must not be used directly; call
    ``sync()`` first.
    """

    def __init__(self, lattices, sweeps, measure_every=1, block_threads=0, cluster_size=0,
                 big_sites=0, use_graph=True, huge_sites=0, stream=None):
        lib = load_library()
        self._lib = lib
        self.lattices = list(lattices)
        n = len(self.lattices)
        sw = np.asarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (n,)),
                        dtype=np.int64).copy()
        ev = np.asarray(np.broadcast_to(np.asarray(measure_every, dtype=np.int32), (n,)),
                        dtype=np.int32).copy()
        handles = (ctypes.c_void_p * n)(*[lat.handle for lat in self.lattices])
        opts = BatchOpts(block_threads, cluster_size, big_sites, 0 if use_graph else -1,
                         huge_sites)
        raw = getattr(stream, "cuda_stream", stream)
        self._h = ctypes.c_void_p()
        _check(lib.ising_batch_create(ctypes.byref(self._h), handles, n,
                                      sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      ctypes.byref(opts), ctypes.c_void_p(int(raw) if raw else 0)),
               "ising_batch_create")

    def update(self, lattices, sweeps, measure_every=1) -> None:
        """``ising_batch_update``: replace the batch's lattices and sweep counts
        (the next launch advances these), keeping its device tables."""
        self.lattices = list(lattices)
        n = len(self.lattices)
        sw = np.asarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (n,)),
                        dtype=np.int64).copy()
        ev = np.asarray(np.broadcast_to(np.asarray(measure_every, dtype=np.int32), (n,)),
                        dtype=np.int32).copy()
        handles = (ctypes.c_void_p * n)(*[lat.handle for lat in self.lattices])
        _check(self._lib.ising_batch_update(self._h, handles, n,
                                            sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                            ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "ising_batch_update")

    def launch(self) -> None:
        _check(self._lib.ising_batch_launch(self._h), "ising_batch_launch")

    def sync(self) -> None:
        _check(self._lib.ising_batch_sync(self._h), "ising_batch_sync")

    def info(self) -> dict:
        g, nb, ns, nh = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self._lib.ising_batch_info(self._h, ctypes.byref(g), ctypes.byref(nb),
                                          ctypes.byref(ns), ctypes.byref(nh)), "ising_batch_info")
        return {"grid": g.value, "n_big": nb.value, "n_small": ns.value, "n_huge": nh.value}

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ising_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_run(lattices, sweeps, measure_every: int = 1, stream=None) -> None:
    """``ising_batch_run``: advance every lattice by its sweeps in one
    persistent launch on ``stream`` and wait; records go to the handles."""
    lib = load_library()
    n = len(lattices)
    sw = np.asarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (n,)),
                    dtype=np.int64).copy()
    handles = (ctypes.c_void_p * n)(*[lat.handle for lat in lattices])
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib.ising_batch_run(handles, n, sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               int(measure_every), ctypes.c_void_p(int(raw) if raw else 0)),
           "ising_batch_run")


def batch_run_static(lattices, sweeps, measure_every, records_ptr: int, records_cap: int,
                     block_threads=0, cluster_size=0, big_sites=0, stream=None) -> None:
    """``ising_batch_run_static``: one persistent launch over ``lattices`` that
    allocates nothing; E/M records go to the caller's device buffer at
    ``records_ptr`` ((E, M) int64 pairs, ``records_cap`` pairs, lattice by
    lattice in order)."""
    lib = load_library()
    n = len(lattices)
    sw = np.asarray(np.broadcast_to(np.asarray(sweeps, dtype=np.int64), (n,)),
                    dtype=np.int64).copy()
    ev = np.asarray(np.broadcast_to(np.asarray(measure_every, dtype=np.int32), (n,)),
                    dtype=np.int32).copy()
    handles = (ctypes.c_void_p * n)(*[lat.handle for lat in lattices])
    opts = BatchOpts(block_threads, cluster_size, big_sites, 0, 0)
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib.ising_batch_run_static(handles, n,
                                      sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      ctypes.c_void_p(records_ptr), int(records_cap),
                                      ctypes.byref(opts),
                                      ctypes.c_void_p(int(raw) if raw else 0)),
           "ising_batch_run_static")


def observables_gather(lattices, pairs: np.ndarray, counts: np.ndarray | None = None,
                       flag: np.ndarray | None = None, value: int = 0) -> np.ndarray:
    """``ising_observables_gather``: enqueue, with one kernel on the lattices'
    common stream, the copy of every lattice's pending (E, M) records into
    ``pairs`` (a pinned int64 array of shape (cap, 2), written by the device
    directly) and clear them.  Returns the per-lattice record counts at once;
    lattice i's records start at row counts[:i].sum().  The values are valid
    once the stream passes this point (e.g. an event recorded next), or, with
    ``flag`` (a one-element view of a pinned int64 array), once the device has
    stored ``value`` there (``ising_observables_gather_signal``)."""
    lib = load_library()
    assert pairs.dtype == np.int64 and pairs.flags.c_contiguous
    n = len(lattices)
    if counts is None:
        counts = np.zeros(n, dtype=np.int64)
    assert counts.dtype == np.int64 and counts.size >= n and counts.flags.c_contiguous
    handles = (ctypes.c_void_p * n)(*[lat.handle for lat in lattices])
    cnt = counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if flag is None:
        _check(lib.ising_observables_gather(handles, n, ctypes.c_void_p(pairs.ctypes.data),
                                            pairs.size // 2, cnt),
               "ising_observables_gather")
    else:
        assert flag.dtype == np.int64 and flag.size >= 1
        _check(lib.ising_observables_gather_signal(handles, n,
                                                   ctypes.c_void_p(pairs.ctypes.data),
                                                   pairs.size // 2, cnt,
                                                   ctypes.c_void_p(flag.ctypes.data),
                                                   int(value)),
               "ising_observables_gather_signal")
    return counts
