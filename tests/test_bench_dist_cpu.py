"""The bench's multi-rank logic on the CPU with two gloo ranks: every rank
learns the slowest rank's time (the whole job's time), and the ranks' lattice
seeds do not collide (independent replicas, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, world)  # rank 1 is the slow one
    seeds = [bench.BASE_SEED + 16 * rank + j for j in range(16)]
    out.put((rank, t, seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(t for _, t, _ in got) == [2.5, 2.5]
    seeds = [s for _, _, ss in got for s in ss]
    assert len(set(seeds)) == len(seeds) == 32


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25



def test_measured_traffic_follows_the_kernel_sources():
    """A traffic figure is reported only for the sources it was captured on."""
    import bench
    for (workload, layout), t in bench.TRAFFIC.items():
        got = bench.measured_traffic(workload, layout, 10)
        if bench.kernel_sources_sha1(t["sources"]) == t["sha1"]:
            assert got == pytest.approx(10 * t["bytes_per_update"])
        else:
            assert got is None
        assert bench.measured_traffic(workload, layout, 10, rule="heatbath") is None
    assert bench.measured_traffic("cubic", "int8", 10) is None


def test_source_hash_ignores_comments_but_not_code():
    """A comment edit keeps a traffic capture valid; a code edit does not."""
    import bench
    src = "int f(int x) {  // doubles\n    /* the\n       product */ return 2 * x;\n}\n"
    same = "// header\nint f(int x) {   \n    return 2 * x;  // changed comment\n}\n\n"
    other = "int f(int x) {\n    return 3 * x;\n}\n"
    assert bench.code_only(src) == bench.code_only(same)
    assert bench.code_only(src) != bench.code_only(other)


@pytest.mark.parametrize("order", ["step", "wave"])
@pytest.mark.parametrize("n_lat,steps", [(1, 1), (16, 20), (16, 3), (3, 16)])
def test_e2e_issue_schedule_runs_every_sweep_once_in_order(order, n_lat, steps):
    """Every (lattice, sweep) pair is issued exactly once, each lattice's
    sweeps in increasing order, at most one sweep per lattice per wavefront;
    in wave order lattice j starts in wavefront j."""
    import bench
    waves = bench.issue_schedule(n_lat, steps, order)
    seen = [(j, k) for w in waves for (j, k) in w]
    assert sorted(seen) == [(j, k) for j in range(n_lat) for k in range(steps)]
    for w in waves:
        assert len({j for j, _ in w}) == len(w)
    for j in range(n_lat):
        ks = [k for w in waves for (jj, k) in w if jj == j]
        assert ks == list(range(steps))
        first = next(i for i, w in enumerate(waves) if any(jj == j for jj, _ in w))
        assert first == (j if order == "wave" else 0)
    assert len(waves) == steps + (n_lat - 1 if order == "wave" else 0)
