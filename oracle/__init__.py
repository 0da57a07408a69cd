"""CPU oracle for the checkerboard-Metropolis Ising model.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA engine in ``paper_cs_0312006_gb300`` and neither imports the other.

The arithmetic lives in plain single-threaded C (``ising_oracle.c`` for the
Ising model, Sec. 2.2; ``percolation_oracle.c`` for the percolation model,
Sec. 2.3); this module compiles them with gcc on first use and marshals numpy
arrays through ctypes.  The
exact closed forms and enumeration-based averages used to pin the oracle are in
``oracle.exact``.

Every function follows Tomov et al. (2003), Sec. 2.2 (Ising model) and Eq. 1;
the readings taken where the paper is silent are stated in ``ising_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ising_oracle.c")
_SOURCES = [_SRC, os.path.join(_HERE, "percolation_oracle.c")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None

HOT, COLD_UP, COLD_DOWN = 0, 1, 2
CHECKERBOARD, SEQUENTIAL, HEATBATH = 0, 1, 2
METROPOLIS_RULE, HEATBATH_RULE = 0, 1


def build(force: bool = False) -> str:
    """Compile ``ising_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc -O2)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SOURCES)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, *_SOURCES, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i8p = ctypes.POINTER(ctypes.c_int8)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_thresholds.argtypes = [ctypes.c_int, ctypes.c_double, u32p]
        lib.orc_thresholds.restype = ctypes.c_int
        lib.orc_energy.argtypes = [ctypes.c_int, ctypes.c_int, i8p]
        lib.orc_energy.restype = ctypes.c_int64
        lib.orc_magnetization.argtypes = [ctypes.c_int, ctypes.c_int, i8p]
        lib.orc_magnetization.restype = ctypes.c_int64
        lib.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_int, i8p]
        lib.orc_init.restype = ctypes.c_int
        lib.orc_half_sweep.argtypes = [ctypes.c_int, ctypes.c_int, i8p,
                                       ctypes.c_uint64, u32p, ctypes.c_uint32,
                                       ctypes.c_int]
        lib.orc_half_sweep.restype = ctypes.c_int
        lib.orc_half_sweep_rule.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64,
                                            u32p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int]
        lib.orc_half_sweep_rule.restype = ctypes.c_int
        lib.orc_site_update.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64, u32p,
                                        ctypes.c_uint32, ctypes.c_int64, ctypes.c_int]
        lib.orc_site_update.restype = ctypes.c_int
        lib.orc_half_sweep_multihit.argtypes = [ctypes.c_int, ctypes.c_int, i8p,
                                                ctypes.c_uint64, u32p, ctypes.c_uint32,
                                                ctypes.c_int, ctypes.c_int]
        lib.orc_half_sweep_multihit.restype = ctypes.c_int
        lib.orc_run_multihit.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint64, i8p, ctypes.c_uint32, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int, i64p, i64p, ctypes.c_int64]
        lib.orc_run_multihit.restype = ctypes.c_int64
        lib.orc_thresholds_heatbath.argtypes = [ctypes.c_int, ctypes.c_double, u32p]
        lib.orc_thresholds_heatbath.restype = ctypes.c_int
        lib.orc_sweep.argtypes = [ctypes.c_int, ctypes.c_int, i8p, ctypes.c_uint64,
                                  u32p, ctypes.c_uint32]
        lib.orc_sweep.restype = ctypes.c_int
        lib.orc_sweep_sequential.argtypes = lib.orc_sweep.argtypes
        lib.orc_sweep_sequential.restype = ctypes.c_int
        lib.orc_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                ctypes.c_uint64, i8p, ctypes.c_uint32,
                                ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                i64p, i64p, ctypes.c_int64]
        lib.orc_run.restype = ctypes.c_int64
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_demon_half_sweep.argtypes = [ctypes.c_int, ctypes.c_int, i8p, u8p, ctypes.c_int,
                                             ctypes.c_int]
        lib.orc_demon_half_sweep.restype = ctypes.c_int
        lib.orc_demon_shift.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int]
        lib.orc_demon_shift.restype = ctypes.c_int
        lib.orc_demon_sweep.argtypes = [ctypes.c_int, ctypes.c_int, i8p, u8p, ctypes.c_int]
        lib.orc_demon_sweep.restype = ctypes.c_int
        lib.orc_demon_run.argtypes = [ctypes.c_int, ctypes.c_int, i8p, u8p, ctypes.c_int,
                                      ctypes.c_uint32, ctypes.c_int64, ctypes.c_int, i64p, i64p,
                                      ctypes.c_int64]
        lib.orc_demon_run.restype = ctypes.c_int64
        lib.orc_perc_threshold.argtypes = [ctypes.c_double, u32p]
        lib.orc_perc_threshold.restype = ctypes.c_int
        lib.orc_perc_pores.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_uint32, u8p]
        lib.orc_perc_pores.restype = ctypes.c_int
        lib.orc_perc_invade.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                        ctypes.c_int64, u8p, i64p,
                                        ctypes.POINTER(ctypes.c_int), i64p]
        lib.orc_perc_invade.restype = ctypes.c_int
        lib.orc_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, i64p]
        lib.orc_enumerate.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def n_sites(dims: int, L: int) -> int:
    return L ** dims


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key (uint32 words)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                              _ptr(out, ctypes.c_uint32))
    return out


def thresholds(dims: int, beta: float) -> np.ndarray:
    """thr[j] = floor(exp(-2*beta*k) * 2^32) for k = 2(j+1), j < dims (rest 0)."""
    thr = np.zeros(3, dtype=np.uint32)
    rc = _load().orc_thresholds(dims, float(beta), _ptr(thr, ctypes.c_uint32))
    if rc != 0:
        raise ValueError(f"orc_thresholds(dims={dims}, beta={beta!r}) -> {rc}")
    return thr


def thresholds_heatbath(dims: int, beta: float) -> np.ndarray:
    """Heat-bath flip thresholds thb[d] = floor(2^32 / (1 + exp(4 beta (dims - d))))
    for d = 0..2*dims disagreeing neighbours (7 entries, unused ones 0)."""
    thb = np.zeros(7, dtype=np.uint32)
    rc = _load().orc_thresholds_heatbath(dims, float(beta), _ptr(thb, ctypes.c_uint32))
    if rc != 0:
        raise ValueError(f"orc_thresholds_heatbath(dims={dims}, beta={beta!r}) -> {rc}")
    return thb


def init(dims: int, L: int, seed: int, start: int = HOT) -> np.ndarray:
    """Initial state in canonical order (x fastest), int8 +-1."""
    s = np.zeros(n_sites(dims, L), dtype=np.int8)
    rc = _load().orc_init(dims, L, seed, start, _ptr(s, ctypes.c_int8))
    if rc != 0:
        raise ValueError(f"orc_init -> {rc}")
    return s


def energy(dims: int, L: int, s: np.ndarray) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_energy(dims, L, _ptr(s, ctypes.c_int8)))


def magnetization(dims: int, L: int, s: np.ndarray) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_magnetization(dims, L, _ptr(s, ctypes.c_int8)))


def half_sweep(dims: int, L: int, s: np.ndarray, seed: int, thr: np.ndarray,
               t: int, c: int, rule: int = METROPOLIS_RULE) -> None:
    """One colour pass, in place on the canonical int8 array ``s`` (``thr``:
    Metropolis thresholds, or heat-bath thresholds with rule=HEATBATH_RULE)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    src = np.asarray(thr, dtype=np.uint32).ravel()
    tab = np.zeros(7, dtype=np.uint32)
    tab[:min(7, src.size)] = src[:7]
    rc = _load().orc_half_sweep_rule(dims, L, _ptr(s, ctypes.c_int8), seed,
                                     _ptr(tab, ctypes.c_uint32), t, c, rule)
    if rc != 0:
        raise ValueError(f"orc_half_sweep -> {rc}")


def half_sweep_multihit(dims: int, L: int, s: np.ndarray, seed: int, thr: np.ndarray,
                        t: int, c: int, hits: int) -> None:
    """One multi-hit Metropolis colour pass in place (hits trials per site)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    thr = np.ascontiguousarray(np.asarray(thr, dtype=np.uint32)[:3])
    rc = _load().orc_half_sweep_multihit(dims, L, _ptr(s, ctypes.c_int8), seed,
                                         _ptr(thr, ctypes.c_uint32), t, c, hits)
    if rc != 0:
        raise ValueError(f"orc_half_sweep_multihit -> {rc}")


def run_multihit(dims: int, L: int, beta: float, seed: int, nsweeps: int, hits: int,
                 measure_every: int = 1, start: int = HOT, s: np.ndarray | None = None,
                 t0: int = 0):
    """Multi-hit checkerboard Metropolis sweeps numbered t0, t0+1, ...;
    returns (s, E, M) as run() does."""
    if s is None:
        s = init(dims, L, seed, start)
    else:
        s = np.ascontiguousarray(s, dtype=np.int8).copy()
    cap = nsweeps // measure_every + 2
    E = np.zeros(cap, dtype=np.int64)
    M = np.zeros(cap, dtype=np.int64)
    n = _load().orc_run_multihit(dims, L, float(beta), seed, _ptr(s, ctypes.c_int8), t0,
                                 nsweeps, measure_every, hits, _ptr(E, ctypes.c_int64),
                                 _ptr(M, ctypes.c_int64), cap)
    if n < 0:
        raise ValueError(f"orc_run_multihit -> {n}")
    return s, E[:n].copy(), M[:n].copy()


def site_update(dims: int, L: int, s: np.ndarray, seed: int, thr: np.ndarray, t: int,
                sites, rule: int = METROPOLIS_RULE) -> np.ndarray:
    """The spins that the canonical sites ``sites`` hold after their colour's
    pass of sweep t, each decided from the state ``s`` that pass starts from
    (the colour pass's own decision, one site at a time)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    src = np.asarray(thr, dtype=np.uint32).ravel()
    tab = np.zeros(7, dtype=np.uint32)
    tab[:min(7, src.size)] = src[:7]
    lib = _load()
    sp = _ptr(s, ctypes.c_int8)
    tp = _ptr(tab, ctypes.c_uint32)
    return np.array([lib.orc_site_update(dims, L, sp, seed, tp, t, int(i), rule)
                     for i in np.asarray(sites).ravel()], dtype=np.int8)


def sweep(dims: int, L: int, s: np.ndarray, seed: int, thr: np.ndarray,
          t: int, sequential: bool = False) -> None:
    """One sweep in place (black pass then white pass, or sequential order)."""
    assert s.dtype == np.int8 and s.flags.c_contiguous
    thr = np.ascontiguousarray(thr, dtype=np.uint32)
    fn = _load().orc_sweep_sequential if sequential else _load().orc_sweep
    rc = fn(dims, L, _ptr(s, ctypes.c_int8), seed, _ptr(thr, ctypes.c_uint32), t)
    if rc != 0:
        raise ValueError(f"oracle sweep -> {rc}")


def run(dims: int, L: int, beta: float, seed: int, nsweeps: int,
        measure_every: int = 1, start: int = HOT, s: np.ndarray | None = None,
        t0: int = 0, sequential: bool = False, heatbath: bool = False):
    """Run ``nsweeps`` sweeps numbered t0, t0+1, ... (checkerboard Metropolis,
    sequential Metropolis, or checkerboard heat bath).

    Returns (s, E, M): the final canonical state and the int64 energy and
    magnetisation recorded after every sweep t with (t+1) % measure_every == 0.
    """
    if s is None:
        s = init(dims, L, seed, start)
    else:
        s = np.ascontiguousarray(s, dtype=np.int8).copy()
    cap = nsweeps // measure_every + 2
    E = np.zeros(cap, dtype=np.int64)
    M = np.zeros(cap, dtype=np.int64)
    n = _load().orc_run(dims, L, float(beta), seed, _ptr(s, ctypes.c_int8), t0,
                        nsweeps, measure_every,
                        HEATBATH if heatbath else (SEQUENTIAL if sequential else CHECKERBOARD),
                        _ptr(E, ctypes.c_int64),
                        _ptr(M, ctypes.c_int64), cap)
    if n < 0:
        raise ValueError(f"orc_run -> {n}")
    return s, E[:n].copy(), M[:n].copy()


def _demon_args(s, q):
    assert s.dtype == np.int8 and s.flags.c_contiguous
    assert q.dtype == np.uint8 and q.flags.c_contiguous and q.size == s.size
    return _ptr(s, ctypes.c_int8), _ptr(q, ctypes.c_uint8)


def demon_half_sweep(dims: int, L: int, s: np.ndarray, q: np.ndarray, qmax: int, c: int) -> None:
    """One colour pass of Creutz's demon dynamics, in place on spins s and demons q."""
    sp, qp = _demon_args(s, q)
    rc = _load().orc_demon_half_sweep(dims, L, sp, qp, qmax, c)
    if rc != 0:
        raise ValueError(f"orc_demon_half_sweep -> {rc}")


def demon_shift(dims: int, L: int, q: np.ndarray, step: int = 1) -> None:
    """Move every demon one half row on (step=1) or back (step=-1), in place."""
    assert q.dtype == np.uint8 and q.flags.c_contiguous
    rc = _load().orc_demon_shift(dims, L, _ptr(q, ctypes.c_uint8), step)
    if rc != 0:
        raise ValueError(f"orc_demon_shift -> {rc}")


def demon_sweep(dims: int, L: int, s: np.ndarray, q: np.ndarray, qmax: int) -> None:
    sp, qp = _demon_args(s, q)
    rc = _load().orc_demon_sweep(dims, L, sp, qp, qmax)
    if rc != 0:
        raise ValueError(f"orc_demon_sweep -> {rc}")


def run_demon(dims: int, L: int, s: np.ndarray, q: np.ndarray, qmax: int, nsweeps: int,
              measure_every: int = 1, t0: int = 0):
    """Demon sweeps numbered t0, t0+1, ... from (s, q) (copied).  Returns
    (s, q, E, M) with E, M recorded after sweep t iff (t+1) % measure_every == 0."""
    s = np.ascontiguousarray(s, dtype=np.int8).copy()
    q = np.ascontiguousarray(q, dtype=np.uint8).copy()
    cap = nsweeps // measure_every + 2
    E = np.zeros(cap, dtype=np.int64)
    M = np.zeros(cap, dtype=np.int64)
    sp, qp = _demon_args(s, q)
    n = _load().orc_demon_run(dims, L, sp, qp, qmax, t0, nsweeps, measure_every,
                              _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64), cap)
    if n < 0:
        raise ValueError(f"orc_demon_run -> {n}")
    return s, q, E[:n].copy(), M[:n].copy()


# --------------------------------------------------------------------------
# Percolation (Sec. 2.3)
# --------------------------------------------------------------------------
PERC_POINT, PERC_FACE = 0, 1


def perc_threshold(P: float) -> int:
    """floor(P * 2^32) capped at 2^32 - 1: a site is a pore iff its draw u <= this."""
    thr = ctypes.c_uint32(0)
    if _load().orc_perc_threshold(float(P), ctypes.byref(thr)) != 0:
        raise ValueError(f"porosity {P!r} not in [0, 1]")
    return int(thr.value)


def perc_pores(dims: int, L: int, seed: int, P: float) -> np.ndarray:
    """Porosity field: uint8 1 (pore) / 0 (solid) per site, canonical order."""
    n = L ** dims
    pore = np.zeros(n, dtype=np.uint8)
    rc = _load().orc_perc_pores(dims, L, seed, perc_threshold(P), _ptr(pore, ctypes.c_uint8))
    if rc != 0:
        raise ValueError(f"orc_perc_pores -> {rc}")
    return pore


def perc_invade(dims: int, L: int, pore: np.ndarray, source: int = PERC_FACE, site: int = 0):
    """Invade ``pore`` from one site or the first face; returns
    (cluster uint8 array, size, spans, steps)."""
    pore = np.ascontiguousarray(pore, dtype=np.uint8)
    cluster = np.zeros(pore.size, dtype=np.uint8)
    size = ctypes.c_int64(0)
    spans = ctypes.c_int(0)
    steps = ctypes.c_int64(0)
    rc = _load().orc_perc_invade(dims, L, _ptr(pore, ctypes.c_uint8), source, int(site),
                                 _ptr(cluster, ctypes.c_uint8), ctypes.byref(size),
                                 ctypes.byref(spans), ctypes.byref(steps))
    if rc != 0:
        raise ValueError(f"orc_perc_invade -> {rc}")
    return cluster, int(size.value), bool(spans.value), int(steps.value)


def enumerate_states(dims: int, L: int) -> np.ndarray:
    """g(E, M): number of states with energy E and magnetisation M.

    Returned as an int64 array of shape (2*dims*N + 1, 2N + 1) indexed by
    (E + dims*N, M + N).
    """
    n = n_sites(dims, L)
    hist = np.zeros((2 * dims * n + 1, 2 * n + 1), dtype=np.int64)
    rc = _load().orc_enumerate(dims, L, _ptr(hist, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"orc_enumerate -> {rc}")
    return hist
