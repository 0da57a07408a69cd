"""Serving loop on the GPU: jobs that arrive while others run are admitted
between rounds (memory budget and slots permitting), their work shares each
round's batched launch, and every job's E/M history and final spins equal the
same job run alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0312006_gb300 import _build, engine
    _build.build()
    engine.load_library()
    return engine


def small_stream(n=40, seed=3):
    from paper_cs_0312006_gb300 import workloads
    return workloads.poisson_jobs(n, rate_per_s=4000.0, seed=seed, l2d=(16, 300), l3d=(8, 40),
                                  sweeps=(20, 300), measure_every=10)


@pytest.mark.parametrize("budget_mb,slots", [(120_000, 4096), (2, 6)])
def test_serving_results_equal_alone(eng, budget_mb, slots):
    from paper_cs_0312006_gb300 import serve
    jobs = small_stream()
    srv = serve.Server(hbm_budget_bytes=budget_mb * 10 ** 6, max_resident=slots,
                       round_s=0.002, batch_opts=dict(cluster_size=2, big_sites=20000,
                                                      huge_sites=60000))
    summ = srv.run(jobs)
    assert summ["jobs"] == len(jobs)
    assert summ["peak_bytes"] <= budget_mb * 10 ** 6
    assert summ["rounds"] > 1
    assert 0 < summ["p50_latency_s"] <= summ["p99_latency_s"]
    for job in jobs:
        r = srv.results[job.job_id]
        s, E, M = serve.run_alone(job)
        assert np.array_equal(r.spins, s), job.job_id
        assert np.array_equal(r.E, E) and np.array_equal(r.M, M), job.job_id
        assert len(E) == job.spec.sweeps // 10
