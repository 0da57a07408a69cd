"""Autotuner for the batched launch and the int8 per-lattice pass.

Searches the launch shape of the persistent batched kernel -- threads per CTA,
CTAs per cluster for large lattices, the size threshold of the cluster queue,
and the spin layout policy -- on a scaled-down sample of the workload, and
keeps the fastest; and, per lattice shape, the int8 colour pass (register
strips, or tiles staged by bulk copies with their rows per tile -- one or two
rows per thread at a time -- and resident CTAs per SM), registered with the
engine so that ISING_KERNEL_AUTO runs the winner.  Every candidate must produce bit-identical spins and E/M
for every lattice (the draws are keyed by site, sweep and colour, so the
launch shape never changes a result); a candidate that does not is an error,
not a slower choice.  The winner is cached as JSON per device name and
workload signature.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import batched

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_cs_0312006_gb300", "autotune.json")

CANDIDATES = [
    dict(block_threads=bt, cluster_size=cs, big_sites=bs)
    for bt in (128, 256)
    for cs in (1, 2, 4, 8)
    for bs in ((1 << 16, 1 << 18, 1 << 20) if cs > 1 else (1 << 30,))
]
LAYOUTS = ("auto", "int8")


def signature(specs) -> str:
    h = hashlib.sha1()
    for sp in specs:
        h.update(f"{sp.dims},{sp.L},{sp.sweeps},{sp.measure_every};".encode())
    return h.hexdigest()[:16]


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _fingerprint(lats):
    out = []
    for lat in lats:
        E, M = lat.observables()
        s = lat.get_spins()
        out.append((hashlib.sha1(s.tobytes()).hexdigest(), E.tobytes(), M.tobytes()))
        lat.close()
    return out


def tune(specs, sample_sweeps: int = 40, sample_lattices: int = 512, seed: int = 0,
         use_cache: bool = True, verbose: bool = False) -> dict:
    """Pick launch options for ``specs``; returns {"opts": ..., "layout": ...,
    "results": [...]}."""
    key = f"{_device_name()}|{signature(specs)}"
    if use_cache and os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                cache = json.load(f)
            if key in cache:
                return cache[key]
        except (OSError, ValueError):
            pass
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(specs), size=min(sample_lattices, len(specs)), replace=False)
    sample = batched.scaled([specs[i] for i in sorted(idx)], sample_sweeps)
    results = []
    reference = None
    for layout in LAYOUTS:
        for opts in CANDIDATES:
            batched.run_batched(sample, opts, 1, layout)[1]  # warm-up (graph capture)
            dt, lats = batched.run_batched(sample, opts, 1, layout)
            fp = _fingerprint(lats)
            if reference is None:
                reference = fp
            elif fp != reference:
                raise RuntimeError(f"autotune: candidate {opts} / {layout} changed a result")
            results.append({"opts": opts, "layout": layout, "seconds": dt})
            if verbose:
                print(f"{layout:5s} {opts} {dt * 1e3:.2f} ms")
    best = min(results, key=lambda r: r["seconds"])
    entry = {"opts": best["opts"], "layout": best["layout"], "results": results,
             "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            cache = {}
            if os.path.exists(CACHE):
                with open(CACHE) as f:
                    cache = json.load(f)
            cache[key] = entry
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except (OSError, ValueError):
            pass
    return entry


# ---------------------------------------------------------------------------
# The int8 per-lattice pass: which kernel (register strips or tiles staged by
# bulk copies), and for the staged kernel its rows per tile (1: each thread
# one row at a time; 2 and 4: two rows at a time, eight Philox calls in
# flight) and its resident CTAs per SM.
# ---------------------------------------------------------------------------
def int8_candidates(dims: int, L: int) -> list:
    """The strip kernel, and the staged kernel over rows per tile (short rows
    need tall tiles to give every thread work) and resident CTAs per SM."""
    W = L // 2
    rows = [r for r in (1, 2, 4, 8, 16, 32, 64) if r * W <= 32768 and L % r == 0]
    if dims == 3:
        rows = [r for r in rows if r * W >= 1024] or rows[-1:]
    else:
        rows = rows[:3]
    return [dict(kernel=1, tile_rows=0, ctas_per_sm=0)] + [
        dict(kernel=2, tile_rows=r, ctas_per_sm=c) for r in rows for c in (0, 3)]


L2_BYTES = 129 * 2 ** 20


def _int8_run(engine, dims, L, sweeps, seed=20031109, repeats=2):
    """Time `sweeps` sweeps of each of n cold lattices in turn (n chosen so
    that their spins exceed L2, as in a real run) with the registered
    configuration, best of `repeats`; returns (seconds per lattice-sweep,
    fingerprint, resolved config)."""
    import torch
    n = max(1, min(8, -(-3 * L2_BYTES // (L ** dims))))
    lats = [engine.Lattice(dims, L, 0.4 if dims == 2 else 0.22, seed + j, layout=engine.INT8,
                           start=engine.COLD_UP) for j in range(n)]
    resolved = lats[0].int8_config()
    for lat in lats:
        lat.sweep(1, 1)  # warm-up
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(sweeps):
            for lat in lats:
                lat.sweep(1, 1)
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b) / 1e3 / (sweeps * n))
    E, M = lats[0].observables()
    s = lats[0].get_spins()
    for lat in lats:
        lat.close()
    fp = (hashlib.sha1(s.tobytes()).hexdigest(), E.tobytes(), M.tobytes())
    return best, fp, resolved


def tune_int8(dims: int, L: int, L_range=None, sweeps: int = 5, use_cache: bool = True,
              register: bool = True) -> dict:
    """Measure every int8 pass configuration on a (dims, L) lattice, check
    that all give bit-identical spins and E/M, and register the fastest for
    lattices with L in ``L_range`` (default: L alone) so that
    ISING_KERNEL_AUTO runs it.  Returns {"config": ..., "results": [...]}."""
    from . import engine
    lo, hi = L_range or (L, L)
    key = f"int8|{_device_name()}|{dims}|{L}"
    entry = None
    if use_cache and os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                entry = json.load(f).get(key)
        except (OSError, ValueError):
            entry = None
    if entry is None:
        results, reference, seen = [], None, set()
        for cand in int8_candidates(dims, L):
            engine.clear_int8_configs()
            engine.set_int8_config(dims, L, L, **cand)
            dt, fp, resolved = _int8_run(engine, dims, L, sweeps)
            shape = tuple(sorted(resolved.items()))
            if resolved["kernel"] != cand["kernel"] or shape in seen:
                continue  # the staged kernel cannot take this shape, or a duplicate
            seen.add(shape)
            if reference is None:
                reference = fp
            elif fp != reference:
                raise RuntimeError(f"autotune: int8 configuration {cand} changed a result")
            results.append({"config": resolved, "seconds": dt,
                            "site_updates_per_s": L ** dims / dt})
        # the two leaders timed again, longer, before choosing
        results.sort(key=lambda r: r["seconds"])
        for r in results[:2]:
            engine.clear_int8_configs()
            engine.set_int8_config(dims, L, L, **r["config"])
            dt, _, _ = _int8_run(engine, dims, L, 3 * sweeps)  # results checked above
            r["seconds"] = min(r["seconds"], dt)
            r["site_updates_per_s"] = L ** dims / r["seconds"]
        engine.clear_int8_configs()
        best = min(results, key=lambda r: r["seconds"])
        entry = {"config": best["config"], "results": results,
                 "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
        if use_cache:
            try:
                os.makedirs(os.path.dirname(CACHE), exist_ok=True)
                cache = {}
                if os.path.exists(CACHE):
                    with open(CACHE) as f:
                        cache = json.load(f)
                cache[key] = entry
                with open(CACHE, "w") as f:
                    json.dump(cache, f, indent=1)
            except (OSError, ValueError):
                pass
    if register:
        engine.set_int8_config(dims, lo, hi, **entry["config"])
    return entry
