"""Scheduling logic of the serving loop on the CPU, with stand-ins for the
lattice and batch objects (no GPU): admission by arrival time, slots and the
memory budget without overtaking, processor-sharing quanta, the bookkeeping
of records and latencies, and the workload generators."""
import numpy as np
import pytest

from paper_cs_0312006_gb300 import serve, workloads


class FakeLattice:
    live = 0

    def __init__(self, dims, L, beta, seed, layout=0, start=0, stream=None):
        self.dims, self.L, self.t, self.n_rec = dims, L, 0, 0
        self.E, self.M = [], []
        FakeLattice.live += 1
        self.closed = False

    def observables(self):
        E, M = np.array(self.E, dtype=np.int64), np.array(self.M, dtype=np.int64)
        self.E, self.M = [], []
        return E, M

    def get_spins(self):
        return np.full(self.L ** self.dims, 1, dtype=np.int8)

    def close(self):
        assert not self.closed
        self.closed = True
        FakeLattice.live -= 1


class FakeBatch:
    calls = []

    def __init__(self, lats, sweeps, every, use_graph=True, stream=None, **kw):
        self.lats, self.sweeps, self.every = lats, list(sweeps), list(every)
        FakeBatch.calls.append(list(sweeps))

    def launch(self):
        for lat, n, ev in zip(self.lats, self.sweeps, self.every):
            for _ in range(n):
                lat.t += 1
                if lat.t % ev == 0:  # record after sweep t-1 iff (t-1)+1 divisible
                    lat.E.append(lat.t)
                    lat.M.append(-lat.t)

    def sync(self):
        pass

    def close(self):
        pass


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.001  # each query advances the clock by 1 ms
        return self.t


def jobs_of(specs, gap=0.0):
    return [workloads.Job(i, i * gap, sp) for i, sp in enumerate(specs)]


def spec(L, sweeps, every=10, dims=2):
    return workloads.LatticeSpec(dims, L, 0.44, 7, 0, sweeps, every, 0)


def make_server(**kw):
    FakeBatch.calls.clear()
    return serve.Server(lattice_factory=FakeLattice, batch_factory=FakeBatch, clock=Clock(), **kw)


def test_all_jobs_complete_with_their_records():
    srv = make_server(round_s=1e-4)
    specs = [spec(32, 100), spec(64, 250, 5), spec(16, 30, 3)]
    summ = srv.run(jobs_of(specs))
    assert summ["jobs"] == 3 and FakeLattice.live == 0
    for j, sp in enumerate(specs):
        r = srv.results[j]
        want = [t for t in range(1, sp.sweeps + 1) if t % sp.measure_every == 0]
        assert r.E.tolist() == want and r.M.tolist() == [-t for t in want]
        assert r.sweeps == sp.sweeps and r.latency_s > 0
    assert summ["site_updates"] == sum(sp.sites * sp.sweeps for sp in specs)


def test_memory_budget_limits_residency_and_keeps_order():
    one = serve.job_bytes(spec(64, 100))
    srv = make_server(hbm_budget_bytes=2 * one + 10, round_s=1e-5)
    specs = [spec(64, 100) for _ in range(5)]
    srv.run(jobs_of(specs))
    assert srv.peak_bytes <= 2 * one + 10
    assert all(len(c) <= 2 for c in FakeBatch.calls)
    admits = [srv.results[j].admit_s for j in range(5)]
    assert admits == sorted(admits)  # first come, first admitted


def test_slots_limit_and_job_too_big():
    srv = make_server(max_resident=1, round_s=1.0)
    srv.run(jobs_of([spec(32, 10), spec(32, 10)]))
    assert all(len(c) == 1 for c in FakeBatch.calls)
    small = make_server(hbm_budget_bytes=1000)
    with pytest.raises(ValueError):
        small.submit(workloads.Job(0, 0.0, spec(256, 10)))


def test_time_sharing_quanta():
    srv = make_server(round_s=0.01)
    big = serve.Server.RATE_CLUSTER
    srv.big_sites = 64 * 64  # 64x64 runs on a cluster, 16x16 on one CTA
    srv.run(jobs_of([spec(64, 100000), spec(16, 100000), spec(2048, 100000)]))
    first = FakeBatch.calls[0]
    assert first[0] == int(0.01 * big // (64 * 64)) // 10 * 10
    assert first[1] == int(0.01 * serve.Server.RATE_CTA // 256) // 10 * 10
    huge = int(0.01 * serve.Server.RATE_FULL // (2048 * 2048))
    assert first[2] == (huge - huge % 10 if huge > 10 else huge)


def test_arrivals_respected():
    srv = make_server(round_s=1.0)
    jobs = [workloads.Job(0, 0.0, spec(16, 10)), workloads.Job(1, 0.5, spec(16, 10))]
    srv.run(jobs)
    assert srv.results[1].admit_s >= 0.5


def test_workload_generators():
    mix = workloads.batched_mix(2048)
    assert len(mix) == 2048
    d2 = [s for s in mix if s.dims == 2]
    assert 0.65 < len(d2) / 2048 < 0.75
    assert all(s.L % 2 == 0 for s in mix)
    assert min(s.L for s in d2) >= 16 and max(s.L for s in d2) <= 1024
    d3 = [s for s in mix if s.dims == 3]
    assert min(s.L for s in d3) >= 8 and max(s.L for s in d3) <= 128
    jobs = workloads.poisson_jobs(2000)
    gaps = np.diff([j.arrival_s for j in jobs])
    assert abs(gaps.mean() - 1 / 200) < 0.15 / 200
    assert all(100 <= j.spec.sweeps <= 20000 for j in jobs)
    scan = workloads.beta_scan_2d()
    assert [round(s.beta, 2) for s in scan] == [round(0.30 + 0.02 * j, 2) for j in range(16)]


class GatherLattice(FakeLattice):
    """A stand-in that also answers the gather path's calls."""
    syncs = 0

    @property
    def handle(self):
        return id(self)

    def synchronize(self):
        GatherLattice.syncs += 1


def fake_gather(lats, pairs, counts=None):
    """ising_observables_gather's contract on the host: ERANGE (nothing
    taken) when the buffer is too small, else every lattice's pending records
    in order, cleared."""
    from paper_cs_0312006_gb300 import engine
    total = sum(len(lat.E) for lat in lats)
    if total > len(pairs):
        raise engine.IsingError(engine.ERANGE, "ising_observables_gather")
    counts = np.zeros(len(lats), dtype=np.int64)
    off = 0
    for i, lat in enumerate(lats):
        E, M = lat.observables()
        counts[i] = len(E)
        pairs[off:off + len(E), 0] = E
        pairs[off:off + len(E), 1] = M
        off += len(E)
    return counts


def test_records_gather_grows_its_buffer_and_matches_per_lattice_reads(monkeypatch):
    """The gather path of a round: one read for all resident jobs into a host
    buffer that doubles on ERANGE (nothing lost), one synchronisation, and
    the same per-job records as the one-by-one path."""
    monkeypatch.setattr(serve.engine, "observables_gather", fake_gather)

    class HostServer(serve.Server):
        allocs = []

        def _alloc_pinned(self, cap):
            HostServer.allocs.append(cap)
            return np.zeros((cap, 2), dtype=np.int64)

    def jobs():
        out = []
        for k in range(40):
            spec = workloads.LatticeSpec(dims=2, L=64, beta=0.4, seed=k, sweeps=3000,
                                         measure_every=1, layout=0, start=0)
            out.append(workloads.Job(job_id=k, arrival_s=0.0, spec=spec))
        return out

    results = {}
    for gather in (False, True):
        GatherLattice.syncs = 0
        srv = HostServer(lattice_factory=GatherLattice, batch_factory=FakeBatch, clock=Clock(),
                         gather_records=gather, round_s=1.0, min_quantum=100)
        srv.run(jobs())
        results[gather] = srv.results
        if gather:
            assert HostServer.allocs[0] == 1024 and HostServer.allocs[-1] > 1024
            assert GatherLattice.syncs == srv.rounds
    for k, r in results[False].items():
        g = results[True][k]
        assert np.array_equal(r.E, g.E) and np.array_equal(r.M, g.M)
        assert len(g.E) == 3000


class SweepLattice(GatherLattice):
    """A stand-in that can also sweep alone (the pipelined loop's huge jobs)."""

    def sweep(self, n, every):
        for _ in range(n):
            self.t += 1
            if self.t % every == 0:
                self.E.append(self.t)
                self.M.append(-self.t)


class UpdatableBatch(FakeBatch):
    def info(self):
        return {"grid": 16}

    def update(self, lats, sweeps, every):
        self.lats, self.sweeps, self.every = lats, list(sweeps), list(every)
        FakeBatch.calls.append(list(sweeps))


class FakeEvent:
    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0  # ms


class PipelinedHostServer(serve.Server):
    """The pipelined loop with its device hooks on the host."""

    def _new_stream(self):
        return object()

    def _record(self, stream, timing=False):
        return FakeEvent()

    def _gather(self, lats, slot):
        buf = np.zeros((4096, 2), dtype=np.int64)
        return buf, fake_gather(lats, buf)


def test_pipelined_rounds_give_the_synchronous_results():
    """Rounds queued ahead of the record reads, a long-lived batch updated in
    place and huge jobs swept on their own stream: every job gets exactly the
    records of the one-round-at-a-time loop and is retired once."""
    def jobs():
        out = []
        for k in range(30):
            L = 64 if k % 3 else 512  # every third job is huge here
            sp = workloads.LatticeSpec(dims=2, L=L, beta=0.4, seed=k, sweeps=50 + 37 * k,
                                       measure_every=5, layout=0, start=0)
            out.append(workloads.Job(job_id=k, arrival_s=0.002 * k, spec=sp))
        return out

    results = {}
    for pipelined in (False, True):
        FakeLattice.live = 0
        cls = PipelinedHostServer if pipelined else serve.Server
        srv = cls(lattice_factory=SweepLattice, batch_factory=UpdatableBatch, clock=Clock(),
                  round_s=1e-3, pipelined=pipelined, gather_records=False,
                  batch_opts=dict(huge_sites=512 * 512))
        summ = srv.run(jobs())
        assert summ["jobs"] == 30 and FakeLattice.live == 0
        results[pipelined] = srv.results
    for k, r in results[False].items():
        p = results[True][k]
        assert np.array_equal(r.E, p.E) and np.array_equal(r.M, p.M), k
        assert len(p.E) == (50 + 37 * k) // 5
