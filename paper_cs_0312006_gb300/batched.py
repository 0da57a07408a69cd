"""Batched workload driver: many independent lattices advanced by one
persistent CUDA-graph launch (``Batch``) versus the plain form, one
``ising_sweep`` call per lattice issued back to back on one stream.

Both forms run identical arithmetic, so every lattice must end bit-identical;
``compare_forms`` checks that for every lattice and reports aggregate site
updates per second of each form.
"""
from __future__ import annotations

import time

import numpy as np

from . import engine
from .workloads import AUTO, INT8, LatticeSpec


def layout_for(sp, layout_policy: str) -> int:
    """``layout_policy``: "auto" (the engine's choice, bit-packed), "int8",
    "bitpack", or "mixed": bit-packed where a half row fills whole words and
    starts on a Philox group (L/2 >= 32 and L % 8 == 0), int8 otherwise
    (short or unaligned rows waste bits and draw nine groups per word)."""
    if layout_policy == "int8":
        return INT8
    if layout_policy == "bitpack":
        return engine.BITPACK
    if layout_policy == "mixed":
        return engine.BITPACK if sp.L // 2 >= 32 and sp.L % 8 == 0 else INT8
    return AUTO


def make_lattices(specs, layout_policy: str = "auto", stream=None):
    """Create one handle per spec (hot start) in the layout the policy gives
    (see layout_for)."""
    lats = []
    for sp in specs:
        lay = layout_for(sp, layout_policy)
        lats.append(engine.Lattice(sp.dims, sp.L, sp.beta, sp.seed, layout=lay, start=sp.start,
                                   stream=stream))
    return lats


def total_updates(specs) -> int:
    return int(sum(sp.sites * sp.sweeps for sp in specs))


def run_batched(specs, opts: dict | None = None, launches: int = 1, layout_policy="auto",
                stream=None, warm=True):
    """Returns (seconds, lattices) for ``launches`` launches of one Batch."""
    import torch
    stream = stream or torch.cuda.current_stream()
    lats = make_lattices(specs, layout_policy, stream)
    batch = engine.Batch(lats, [sp.sweeps for sp in specs], [sp.measure_every for sp in specs],
                         stream=stream, **(opts or {}))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(launches):
        batch.launch()
    batch.sync()
    dt = time.perf_counter() - t0
    batch.close()
    return dt, lats


def run_plain(specs, launches: int = 1, layout_policy="auto", stream=None):
    """One ising_sweep(sweeps, measure_every) per lattice, back to back."""
    import torch
    stream = stream or torch.cuda.current_stream()
    lats = make_lattices(specs, layout_policy, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(launches):
        for sp, lat in zip(specs, lats):
            lat.sweep(sp.sweeps, sp.measure_every)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, lats


def run_plain_streams(specs, n_streams: int = 8, layout_policy="auto"):
    """The plain form spread over ``n_streams`` CUDA streams (lattice j on
    stream j mod n_streams), so that small lattices' launches can overlap."""
    import torch
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    lats = []
    for j, sp in enumerate(specs):
        lats += make_lattices([sp], layout_policy, streams[j % n_streams])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sp, lat in zip(specs, lats):
        lat.sweep(sp.sweeps, sp.measure_every)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, lats


def lattice_result(lat):
    E, M = lat.observables()
    return lat.get_spins(), E, M


def same_result(a, b) -> bool:
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def compare_forms(specs, opts=None, layout_policy="auto"):
    """Run both forms on the same specs; returns a dict with both rates and
    the number of lattices whose spins and E/M records differ (must be 0)."""
    upd = total_updates(specs)
    tb, lats_b = run_batched(specs, opts, 1, layout_policy)
    tp, lats_p = run_plain(specs, 1, layout_policy)
    ts, lats_s = run_plain_streams(specs, 8, layout_policy)
    mismatches = 0
    for a, b, c in zip(lats_b, lats_p, lats_s):
        ra = lattice_result(a)
        if not (same_result(ra, lattice_result(b)) and same_result(ra, lattice_result(c))):
            mismatches += 1
        a.close()
        b.close()
        c.close()
    return {"lattices": len(specs), "site_updates": upd,
            "batched_s": tb, "batched_updates_per_s": upd / tb,
            "plain_s": tp, "plain_updates_per_s": upd / tp,
            "plain_8_streams_s": ts, "plain_8_streams_updates_per_s": upd / ts,
            "batched_over_plain": tp / tb, "batched_over_plain_8_streams": ts / tb,
            "mismatches": mismatches}


def scaled(specs, sweeps: int):
    return [LatticeSpec(sp.dims, sp.L, sp.beta, sp.seed, sp.start, sweeps,
                        min(sp.measure_every, sweeps), sp.layout) for sp in specs]
