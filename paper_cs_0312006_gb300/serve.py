"""Serving: a continuous-batching loop for simulation jobs.

Jobs (dims, L, beta, seed, sweeps, measurement interval) arrive over time.
The server keeps every admitted job's spins, sweep counter and E/M records on
the device and runs rounds: each round, every resident job advances by a
quantum of sweeps inside one persistent batched launch (``Batch``), so the
work of all resident jobs overlaps on the GPU.  Between rounds, jobs whose
arrival time has passed are admitted in arrival order while both a slot and
device memory (an HBM budget, counted from each lattice's spin and record
buffers) are free; finished jobs are read back (E/M history and final spins)
and their memory is released.

Quanta share GPU time, not site updates: a round targets round_s seconds, and
each job's quantum of sweeps is what its execution class completes in that
time -- a lattice below the cluster threshold runs on one CTA, a larger one on
a thread-block cluster, and the largest (at least huge_sites) through the
full-GPU per-lattice kernels, one after another (so they split their share
of the round).  Short jobs therefore finish within a round or two while
20,000-sweep 4096^2 jobs progress at the GPU's full rate.  Because draws are
keyed by (seed, sweep, colour, site), a job's result does not depend on which
round or mix it ran in.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import engine
from .workloads import Job


@dataclass
class JobResult:
    job_id: int
    arrival_s: float
    admit_s: float
    done_s: float
    sweeps: int
    sites: int
    E: np.ndarray
    M: np.ndarray
    spins: np.ndarray | None

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


@dataclass
class _Resident:
    job: Job
    lat: engine.Lattice
    bytes: int
    remaining: int
    admit_s: float
    E: list = field(default_factory=list)
    M: list = field(default_factory=list)


def job_bytes(spec) -> int:
    """Device bytes a job holds: two colour arrays and its E/M records."""
    if spec.layout in (engine.BITPACK, engine.AUTO):
        rows = spec.L ** (spec.dims - 1)
        per_colour = rows * ((spec.L // 2 + 31) // 32) * 4 + 16  # padded rows of words
    else:
        per_colour = ((spec.sites // 2 + 15) // 16) * 16 + 16
    records = 16 * (spec.sweeps // spec.measure_every + 64)
    return 2 * per_colour + records


class Server:
    # execution-class throughputs (site updates/s) used to size quanta: the
    # whole GPU, one 8-CTA cluster, one CTA
    RATE_FULL = 6e11
    RATE_CLUSTER = 2.5e10
    RATE_CTA = 1.0e9

    def __init__(self, hbm_budget_bytes: int = 120 * 10 ** 9, max_resident: int = 4096,
                 round_s: float = 0.05, min_quantum: int = 1, keep_spins: bool = True,
                 batch_opts: dict | None = None, stream=None, clock=time.perf_counter,
                 lattice_factory=None, batch_factory=None, gather_records=None):
        self.budget = int(hbm_budget_bytes)
        self.max_resident = max_resident
        self.round_s = float(round_s)
        self.min_quantum = min_quantum
        self.keep_spins = keep_spins
        self.batch_opts = dict(batch_opts or {})
        self.big_sites = self.batch_opts.get("big_sites") or (1 << 18)
        self.huge_sites = self.batch_opts.get("huge_sites") or (1 << 22)
        self.stream = stream
        self.clock = clock
        # the engine by default; tests of the scheduling logic pass stand-ins
        self.lattice_factory = lattice_factory or engine.Lattice
        self.batch_factory = batch_factory or engine.Batch
        # records through one gather per round (engine lattices on one stream)
        self.gather_records = (self.lattice_factory is engine.Lattice
                               if gather_records is None else bool(gather_records))
        self.pending: list[Job] = []
        self.resident: list[_Resident] = []
        self.results: dict[int, JobResult] = {}
        self.bytes_in_use = 0
        self.peak_bytes = 0
        self.rounds = 0
        self.updates_done = 0
        self.t0 = None
        self._pinned = None  # host buffer of the records' gather (grown on demand)
        self._pinned_grow = False

    # -- requests ---------------------------------------------------------
    def submit(self, job: Job) -> None:
        if job_bytes(job.spec) > self.budget:
            raise ValueError(f"job {job.job_id} needs {job_bytes(job.spec)} B > budget")
        self.pending.append(job)

    def now(self) -> float:
        return self.clock() - self.t0

    # -- one scheduling step ------------------------------------------------
    def _admit(self) -> None:
        now = self.now()
        keep = []
        blocked = False
        for job in self.pending:
            need = job_bytes(job.spec)
            if (not blocked and job.arrival_s <= now and len(self.resident) < self.max_resident
                    and self.bytes_in_use + need <= self.budget):
                sp = job.spec
                lat = self.lattice_factory(sp.dims, sp.L, sp.beta, sp.seed, layout=sp.layout,
                                           start=sp.start, stream=self.stream)
                self.resident.append(_Resident(job, lat, need, sp.sweeps, now))
                self.bytes_in_use += need
                self.peak_bytes = max(self.peak_bytes, self.bytes_in_use)
            else:
                if job.arrival_s <= now:
                    blocked = True  # keep arrival order: no overtaking
                keep.append(job)
        self.pending = keep

    def _rate(self, sites: int, n_huge: int) -> float:
        if self.huge_sites > 0 and sites >= self.huge_sites:
            return self.RATE_FULL / max(n_huge, 1)
        if sites >= self.big_sites:
            return self.RATE_CLUSTER
        return self.RATE_CTA

    def _quanta(self) -> list:
        n_huge = sum(1 for r in self.resident
                     if self.huge_sites > 0 and r.job.spec.sites >= self.huge_sites)
        q = []
        for r in self.resident:
            sites = r.job.spec.sites
            sweeps = max(self.min_quantum,
                         int(self.round_s * self._rate(sites, n_huge) // sites))
            every = r.job.spec.measure_every
            if sweeps > every:  # whole measurement intervals keep rounds aligned
                sweeps -= sweeps % every
            q.append(min(r.remaining, sweeps))
        return q

    def _round(self) -> None:
        quanta = self._quanta()
        lats = [r.lat for r in self.resident]
        batch = self.batch_factory(lats, quanta,
                                   [r.job.spec.measure_every for r in self.resident],
                                   use_graph=False, stream=self.stream, **self.batch_opts)
        batch.launch()
        batch.sync()
        batch.close()
        self.rounds += 1
        records = self._read_records(lats)
        still = []
        for r, q, (E, M) in zip(self.resident, quanta, records):
            r.remaining -= q
            self.updates_done += q * r.job.spec.sites
            r.E.append(E)
            r.M.append(M)
            if r.remaining == 0:
                spins = r.lat.get_spins() if self.keep_spins else None
                done_s = self.now()
                self.results[r.job.job_id] = JobResult(
                    r.job.job_id, r.job.arrival_s, r.admit_s, done_s, r.job.spec.sweeps,
                    r.job.spec.sites, np.concatenate(r.E), np.concatenate(r.M), spins)
                r.lat.close()
                self.bytes_in_use -= r.bytes
            else:
                still.append(r)
        self.resident = still

    def _alloc_pinned(self, cap: int) -> np.ndarray:
        """A (cap, 2) int64 host buffer the device can write (pinned)."""
        import torch
        return torch.zeros((cap, 2), dtype=torch.int64).pin_memory().numpy()

    def _read_records(self, lats) -> list:
        """Every resident lattice's pending (E, M) records: engine lattices (one
        stream) through one ising_observables_gather into a pinned buffer and
        one synchronisation; stand-ins one by one."""
        if not self.gather_records or not lats:
            return [lat.observables() for lat in lats]
        while True:
            if self._pinned is None or self._pinned_grow:
                cap = max(1024, 2 * (0 if self._pinned is None else len(self._pinned)))
                self._pinned = self._alloc_pinned(cap)
                self._pinned_grow = False
            try:
                counts = engine.observables_gather(lats, self._pinned)
                break
            except engine.IsingError as e:
                if e.code != engine.ERANGE:
                    raise
                self._pinned_grow = True  # nothing was queued: retry with more room
        lats[0].synchronize()  # one wait (and the bounded-wait check) for all
        out, off = [], 0
        for c in counts:
            out.append((self._pinned[off:off + c, 0].copy(), self._pinned[off:off + c, 1].copy()))
            off += int(c)
        return out

    def run(self, jobs=None) -> dict:
        """Serve ``jobs`` (arriving at their ``arrival_s`` after start) until all
        are done; returns summary statistics."""
        for j in jobs or []:
            self.submit(j)
        self.pending.sort(key=lambda j: (j.arrival_s, j.job_id))
        self.t0 = self.clock()
        while self.pending or self.resident:
            self._admit()
            if self.resident:
                self._round()
            else:
                nxt = self.pending[0].arrival_s
                wait = nxt - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
        makespan = self.now()
        return self.summary(makespan)

    def summary(self, makespan: float, skip_first: int = 0) -> dict:
        res = sorted(self.results.values(), key=lambda r: r.job_id)
        lat = np.array([r.latency_s for r in res[skip_first:]]) if res else np.zeros(1)
        return {"jobs": len(res), "makespan_s": makespan,
                "site_updates": self.updates_done,
                "updates_per_s": self.updates_done / makespan if makespan > 0 else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "rounds": self.rounds, "peak_bytes": self.peak_bytes}


def run_plain_fifo(jobs, keep_spins: bool = False, clock=time.perf_counter):
    """The plain form: each job alone through ising_sweep, one after another in
    arrival order (a job starts when it has arrived and the previous one is
    done).  Returns (summary, results)."""
    import torch
    jobs = sorted(jobs, key=lambda j: (j.arrival_s, j.job_id))
    results = {}
    updates = 0
    t0 = clock()
    for job in jobs:
        now = clock() - t0
        if job.arrival_s > now:
            time.sleep(job.arrival_s - now)
        sp = job.spec
        start = clock() - t0
        lat = engine.Lattice(sp.dims, sp.L, sp.beta, sp.seed, layout=sp.layout, start=sp.start)
        lat.sweep(sp.sweeps, sp.measure_every)
        E, M = lat.observables()
        spins = lat.get_spins() if keep_spins else None
        lat.close()
        torch.cuda.synchronize()
        done = clock() - t0
        updates += sp.sites * sp.sweeps
        results[job.job_id] = JobResult(job.job_id, job.arrival_s, start, done, sp.sweeps,
                                        sp.sites, E, M, spins)
    makespan = clock() - t0
    return {"jobs": len(jobs), "makespan_s": makespan, "site_updates": updates,
            "updates_per_s": updates / makespan}, results


def run_alone(job: Job):
    """The same job through the plain API, for the alone-vs-mix identity."""
    sp = job.spec
    lat = engine.Lattice(sp.dims, sp.L, sp.beta, sp.seed, layout=sp.layout, start=sp.start)
    lat.sweep(sp.sweeps, sp.measure_every)
    E, M = lat.observables()
    s = lat.get_spins()
    lat.close()
    return s, E, M


def percentile_summary(results, skip_first: int) -> dict:
    res = sorted(results.values(), key=lambda r: r.job_id)[skip_first:]
    lat = np.array([r.latency_s for r in res])
    return {"p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "counted_jobs": len(res)}


def offered_load(jobs, rate_per_s: float) -> float:
    """Mean site updates per job times the arrival rate."""
    mean = float(np.mean([j.spec.sites * j.spec.sweeps for j in jobs]))
    return mean * rate_per_s


__all__ = ["Server", "JobResult", "job_bytes", "run_alone", "run_plain_fifo",
           "percentile_summary", "offered_load"]
