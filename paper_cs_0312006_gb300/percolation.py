"""Python binding of the percolation engine (C ABI of include/percolation.h).

Argument marshalling only: the porosity field, the invasion passes and the
measurements all run in the library's kernels (csrc/percolation.cu).  The one
piece of host arithmetic is spanning_threshold, a fit over the spanning
fractions those kernels report.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from .engine import IsingError, load_library

POINT, FACE = 0, 1
PASSES_AUTO, PASSES_GRAPH, PASSES_PERSISTENT = 0, 1, 2


class PercResult(ctypes.Structure):
    _fields_ = [("size", ctypes.c_int64), ("spans", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("steps", ctypes.c_int64)]


_bound = False


def _lib():
    global _bound
    lib = load_library()
    if not _bound:
        P = ctypes.c_void_p
        sig = {
            "perc_create": ([ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_uint64],
                            ctypes.c_int),
            "perc_generate": ([P, ctypes.c_double], ctypes.c_int),
            "perc_invade": ([P, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(PercResult)],
                            ctypes.c_int),
            "perc_get_pores": ([P, P], ctypes.c_int),
            "perc_get_cluster": ([P, P], ctypes.c_int),
            "perc_set_stream": ([P, P], ctypes.c_int),
            "perc_set_passes": ([P, ctypes.c_int], ctypes.c_int),
            "perc_destroy": ([P], None),
            "perc_batch": ([ctypes.c_int, ctypes.c_int, ctypes.c_double,
                            ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int,
                            ctypes.c_int64, ctypes.POINTER(PercResult), P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _bound = True
    return lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise IsingError(rc, what)


class Medium:
    """One porous medium of L^dims sites on the current CUDA device."""

    def __init__(self, dims: int, L: int, seed: int, stream=None):
        self._lib = _lib()
        self.dims, self.L = dims, L
        self._h = ctypes.c_void_p()
        _check(self._lib.perc_create(ctypes.byref(self._h), dims, L,
                                     ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)),
               f"perc_create(dims={dims}, L={L})")
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            _check(self._lib.perc_set_stream(self._h, ctypes.c_void_p(int(raw) if raw else 0)),
                   "perc_set_stream")

    def generate(self, porosity: float) -> None:
        _check(self._lib.perc_generate(self._h, float(porosity)), "perc_generate")

    def invade(self, source: int = FACE, site: int = 0) -> PercResult:
        out = PercResult()
        _check(self._lib.perc_invade(self._h, int(source), int(site), ctypes.byref(out)),
               "perc_invade")
        return out

    def set_passes(self, mode: int) -> None:
        """PASSES_AUTO, PASSES_GRAPH or PASSES_PERSISTENT (same results)."""
        _check(self._lib.perc_set_passes(self._h, int(mode)), "perc_set_passes")

    def pores(self) -> np.ndarray:
        out = np.empty(self.L ** self.dims, dtype=np.uint8)
        _check(self._lib.perc_get_pores(self._h, out.ctypes.data), "perc_get_pores")
        return out

    def cluster(self) -> np.ndarray:
        out = np.empty(self.L ** self.dims, dtype=np.uint8)
        _check(self._lib.perc_get_cluster(self._h, out.ctypes.data), "perc_get_cluster")
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            self._lib.perc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch(dims: int, L: int, porosity: float, seeds, source: int = FACE, site: int = 0,
          clusters_ptr: int = 0, stream=None):
    """``perc_batch``: one launch over len(seeds) media; returns a list of
    PercResult (size, spans, steps)."""
    lib = _lib()
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    res = (PercResult * len(s))()
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib.perc_batch(dims, L, float(porosity),
                          s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), len(s), int(source),
                          int(site), res, ctypes.c_void_p(clusters_ptr or None),
                          ctypes.c_void_p(int(raw) if raw else 0)),
           "perc_batch")
    return list(res)


def spanning_threshold(porosities, fractions, n: int):
    """Finite-size estimate of the porosity threshold from spanning fractions
    (host statistics on results the kernels produced; Sec. 2.3 asks whether a
    spanning cluster forms, Sec. 5 prints the 2D threshold).

    Weighted least squares of logit(f) = a (P - P0) + b over the points with
    0 < f < 1, each weighted by its binomial information n f (1 - f); P0 is
    the mean porosity.  Returns (p_half, sd): the porosity where half the
    media span, P0 - b / a, and its standard error by the delta method.
    Raises ValueError with fewer than two usable points."""
    P = np.asarray(porosities, dtype=np.float64)
    f = np.asarray(fractions, dtype=np.float64)
    keep = (f > 0.0) & (f < 1.0)
    if np.count_nonzero(keep) < 2:
        raise ValueError("need two spanning fractions strictly between 0 and 1")
    P, f = P[keep], f[keep]
    P0 = float(P.mean())
    y = np.log(f / (1.0 - f))
    w = n * f * (1.0 - f)
    A = np.vstack([P - P0, np.ones_like(P)]).T
    cov = np.linalg.inv(A.T @ (w[:, None] * A))
    a, b = cov @ (A.T @ (w * y))
    grad = np.array([b / a ** 2, -1.0 / a])
    return P0 - b / a, math.sqrt(float(grad @ cov @ grad))
