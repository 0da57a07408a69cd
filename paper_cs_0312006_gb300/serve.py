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

With engine lattices the rounds are pipelined: one long-lived batch is
updated in place each round (``ising_batch_update``), the huge jobs run
their per-lattice sweeps on a second stream so that they overlap the
persistent launch, each round's records are gathered into one half of a
pinned double buffer, and round k + 1 is queued before round k's records are
read and its finished jobs retired; lattice memory comes from the library's
stream-ordered pool, so admitting and retiring jobs never waits for the
device.  The class rates that size the quanta start from the constants below
and follow each round's measured GPU times.
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
    last_round: int = -1  # pipelined mode: the last round this job was queued in


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
    # pipelined mode: starting rates per slot (one CTA, one cluster), then
    # adapted to the measured time of each persistent launch
    RATE_CTA_SLOT = 1.5e9
    RATE_CLUSTER_SLOT = 1.0e10

    def __init__(self, hbm_budget_bytes: int = 120 * 10 ** 9, max_resident: int = 4096,
                 round_s: float = 0.05, min_quantum: int = 1, keep_spins: bool = True,
                 batch_opts: dict | None = None, stream=None, clock=time.perf_counter,
                 lattice_factory=None, batch_factory=None, gather_records=None,
                 pipelined=None, adapt_rates: bool = True):
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
        # class rates that size the quanta (pipelined mode: adapted to measured times)
        self.pipelined = (self.lattice_factory is engine.Lattice) if pipelined is None \
            else bool(pipelined)
        self.rate_full, self.rate_cluster, self.rate_cta = (self.RATE_FULL, self.RATE_CLUSTER,
                                                            self.RATE_CTA)
        if self.pipelined:  # per slot: the quanta share each class's slots
            self.rate_cluster, self.rate_cta = self.RATE_CLUSTER_SLOT, self.RATE_CTA_SLOT
        self.adapt_rates = adapt_rates
        # launch shape of the persistent kernel, for the processor-sharing quanta
        self.cluster_size = int(self.batch_opts.get("cluster_size") or 8)
        self.default_grid = 456
        self.round_log = []  # pipelined mode: (small jobs, huge jobs, GPU s of each part)
        self._admit_streams = None

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
                stream = self.stream
                if self._admit_streams is not None:  # pipelined: huge jobs on their own stream
                    huge = self.huge_sites > 0 and sp.sites >= self.huge_sites
                    stream = self._admit_streams[1 if huge else 0]
                lat = self.lattice_factory(sp.dims, sp.L, sp.beta, sp.seed, layout=sp.layout,
                                           start=sp.start, stream=stream)
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
            return self.rate_full / max(n_huge, 1)
        if sites >= self.big_sites:
            return self.rate_cluster
        return self.rate_cta

    def _quanta(self, resident=None) -> list:
        resident = self.resident if resident is None else resident
        n_huge = sum(1 for r in resident
                     if self.huge_sites > 0 and r.job.spec.sites >= self.huge_sites)
        q = []
        for r in resident:
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
        if self.pipelined:
            self._run_pipelined()
        else:
            while self.pending or self.resident:
                self._admit()
                if self.resident:
                    self._round()
                else:
                    self._idle()
        makespan = self.now()
        return self.summary(makespan)

    def _idle(self) -> None:
        if self.pending:
            wait = self.pending[0].arrival_s - self.now()
            if wait > 0:
                time.sleep(min(wait, 0.01))

    # -- pipelined rounds (engine lattices) ------------------------------------
    # Device operations behind small hooks (streams, events, the records
    # gather), so that the scheduling can be driven on the CPU by stand-ins.
    def _new_stream(self):
        import torch
        return torch.cuda.Stream()

    def _record(self, stream, timing: bool = False):
        import torch
        ev = torch.cuda.Event(enable_timing=timing)
        ev.record(stream)
        return ev

    def _gather(self, lats, slot: int):
        """Queue one gather of ``lats``' pending records into the pinned
        buffer of ``slot``; returns (buffer, counts).  The buffer doubles when
        the records do not fit (nothing is queued then)."""
        while True:
            buf = self._bufs.get(slot)
            if buf is None or self._grow.get(slot):
                cap = max(1024, 2 * (0 if buf is None else len(buf)))
                buf = self._alloc_pinned(cap)
                self._bufs[slot] = buf
                self._grow[slot] = False
            try:
                return buf, engine.observables_gather(lats, buf)
            except engine.IsingError as e:
                if e.code != engine.ERANGE:
                    raise
                self._grow[slot] = True

    def _is_huge(self, r) -> bool:
        return self.huge_sites > 0 and r.job.spec.sites >= self.huge_sites

    def _slots(self, batch):
        """Resident CTAs and clusters of the persistent launch."""
        grid = batch.info()["grid"] if batch is not None else 0
        if grid <= 0:
            grid = self.default_grid
        return grid, max(1, grid // self.cluster_size)

    def _shared_quanta(self, active, in_batch_huge: bool, batch):
        """Sweeps per job for one round, by processor sharing within each
        execution class: the class's time budget times its rate per slot times
        min(1, slots / jobs), over the job's sites.  Huge jobs run by the
        per-lattice kernels share the whole GPU; while there are at least as
        many of them as clusters they are cluster jobs instead."""
        n_cta, n_cl = self._slots(batch)
        huge = [r for r in active if self._is_huge(r)]
        cls = {}
        for r in active:
            if self._is_huge(r) and not in_batch_huge:
                cls[id(r)] = "huge"
            elif r.job.spec.sites >= self.big_sites:
                cls[id(r)] = "cluster"
            else:
                cls[id(r)] = "cta"
        count = {c: sum(1 for r in active if cls[id(r)] == c) for c in ("huge", "cluster", "cta")}
        both = count["cluster"] > 0 and count["cta"] > 0
        budget = self.round_s / 2 if both else self.round_s
        capacity = {"cluster": budget * self.rate_cluster * min(1.0, n_cl / max(1, count["cluster"])),
                    "cta": budget * self.rate_cta * min(1.0, n_cta / max(1, count["cta"])),
                    "huge": self.round_s * self.rate_full / max(1, len(huge))}
        q = []
        for r in active:
            sweeps = max(self.min_quantum, int(capacity[cls[id(r)]] // r.job.spec.sites))
            every = r.job.spec.measure_every
            if sweeps > every:  # whole measurement intervals keep rounds aligned
                sweeps -= sweeps % every
            q.append(min(r.remaining, sweeps))
        return q, cls

    def _run_pipelined(self) -> None:
        st = self._new_stream()
        self._admit_streams = (st, st)
        self._bufs, self._grow = {}, {}
        batch = None
        opts = dict(self.batch_opts)
        opts["huge_sites"] = -1  # the huge jobs' per-lattice sweeps are issued here
        opts.setdefault("cluster_size", self.cluster_size)
        opts.setdefault("big_sites", self.big_sites)
        inflight = None
        slot = 0
        while self.pending or self.resident or inflight is not None:
            self._admit()
            active = [r for r in self.resident if r.remaining > 0]
            issued = None
            if active:
                _, n_cl = self._slots(batch)
                in_batch_huge = sum(1 for r in active if self._is_huge(r)) >= n_cl
                quanta, cls = self._shared_quanta(active, in_batch_huge, batch)
                per_lattice = [(r, q) for r, q in zip(active, quanta) if cls[id(r)] == "huge"]
                in_batch = [(r, q) for r, q in zip(active, quanta) if cls[id(r)] != "huge"]
                ev = {"t0": self._record(st, timing=True)}
                for r, q in per_lattice:
                    r.lat.sweep(q, r.job.spec.measure_every)
                ev["t1"] = self._record(st, timing=True)
                if in_batch:
                    lats = [r.lat for r, _ in in_batch]
                    sweeps = [q for _, q in in_batch]
                    every = [r.job.spec.measure_every for r, _ in in_batch]
                    if batch is None:
                        batch = self.batch_factory(lats, sweeps, every, use_graph=False,
                                                   stream=st, **opts)
                    else:
                        batch.update(lats, sweeps, every)
                    batch.launch()
                ev["t2"] = self._record(st, timing=True)
                group = per_lattice + in_batch
                buf, counts = self._gather([r.lat for r, _ in group], slot)
                parts = [(group, buf, counts, self._record(st))]
                for r, q in zip(active, quanta):
                    r.remaining -= q
                    r.last_round = self.rounds
                    self.updates_done += q * r.job.spec.sites
                issued = {"parts": parts, "ev": ev, "index": self.rounds,
                          "n_small": len(in_batch), "n_huge": len(per_lattice),
                          "huge_work": sum(q * r.job.spec.sites for r, q in per_lattice),
                          "small_work": sum(q * r.job.spec.sites for r, q in in_batch)}
                self.rounds += 1
                slot ^= 1
            if inflight is not None:
                self._finish_round(inflight)
            inflight = issued
            if not active and inflight is None:
                self._idle()
        if batch is not None:
            batch.close()

    def _finish_round(self, rnd) -> None:
        """Wait for a queued round, hand its records to the jobs, retire the
        jobs it finished and adapt the class rates to its measured times."""
        for group, buf, counts, done in rnd["parts"]:
            done.synchronize()
            off = 0
            for (r, _), c in zip(group, counts):
                r.E.append(buf[off:off + c, 0].copy())
                r.M.append(buf[off:off + c, 1].copy())
                off += int(c)
        if rnd["parts"]:  # one bounded-wait / input check for the round
            first_group = rnd["parts"][0][0]
            first_group[0][0].lat.synchronize()
        ev = rnd["ev"]
        t_huge = ev["t0"].elapsed_time(ev["t1"]) / 1e3 if rnd["n_huge"] else 0.0
        t_small = ev["t1"].elapsed_time(ev["t2"]) / 1e3 if rnd["n_small"] else 0.0
        self.round_log.append((rnd["n_small"], rnd["n_huge"], t_small, t_huge))
        if self.adapt_rates and rnd["huge_work"] > 0 and t_huge > 0:
            self.rate_full = 0.5 * self.rate_full + 0.5 * rnd["huge_work"] / t_huge
        if self.adapt_rates and rnd["small_work"] > 0 and t_small > 0:
            # the persistent launch took t_small for work sized to round_s
            f = min(4.0, max(0.25, self.round_s / t_small)) ** 0.5
            f = min(f, 1.25)  # grow slowly: an underfilled round also runs short
            self.rate_cluster *= f
            self.rate_cta *= f
        still = []
        for r in self.resident:
            if r.remaining == 0 and r.last_round == rnd["index"]:
                spins = r.lat.get_spins() if self.keep_spins else None
                self.results[r.job.job_id] = JobResult(
                    r.job.job_id, r.job.arrival_s, r.admit_s, self.now(), r.job.spec.sweeps,
                    r.job.spec.sites, np.concatenate(r.E) if r.E else np.zeros(0, np.int64),
                    np.concatenate(r.M) if r.M else np.zeros(0, np.int64), spins)
                r.lat.close()
                self.bytes_in_use -= r.bytes
            else:
                still.append(r)
        self.resident = still

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
