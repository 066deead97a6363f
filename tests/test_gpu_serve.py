"""Serving (continuous batching) and batched-vs-sequential solves.

A seeded Poisson stream of Exact-Cover-3 solves of uneven n, path and T is served: small states
join the running batch between rounds, large ones run on their own streams, admission obeys
an HBM budget.  Each served result equals the same job solved alone (within the complex64
tolerance) and, for small n, the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O

from _helpers import C64, TOL_STATE, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _oracle_state(job):
    from instances import generate_ec3, xx_pairs

    inst = generate_ec3(job.n, job.seed)
    pairs = xx_pairs(job.n, job.seed) if job.nonlinear else None
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = (O.nonlinear_path if job.nonlinear else O.linear_path)(job.T, job.s_kind)
    return O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(job.n), nthreads=8).psi


def test_served_results_equal_alone_and_oracle():
    import copy

    from paper_1311_3938_gb300 import workloads as W

    jobs = W.random_jobs(20, 500, n_range=(6, 15), T_range=(0.3, 2.0), rate=200.0, big_every=7, big_n=17,
                         path_mix=True)
    srv = W.Server(C64, batch_max_n=15, max_members=16, steps_per_round=8, big_chunk=32, keep_state=True)
    try:
        res = srv.serve(copy.deepcopy(jobs))
    finally:
        srv.close()
    assert res["completed"] == len(jobs)
    routes = {j.route for j in res["jobs"]}
    assert routes == {"batch", "stream"}
    assert res["p99_latency_s"] >= res["p50_latency_s"] > 0
    for served in res["jobs"]:
        alone = W.solve_single(copy.deepcopy(jobs[served.jid]), keep_state=True)
        assert served.steps == alone.steps
        assert rel_err(served.state, alone.state) < 2e-6, (served.jid, served.n)
        assert abs(served.P1 - alone.P1) < 1e-6
        if served.n <= 12:
            assert rel_err(served.state, _oracle_state(served)) < TOL_STATE[C64]


def test_shortest_first_policy_with_a_capped_large_job():
    """policy "shortest", one large job at a time with its launches capped at a few CTAs
    (aqc_set_grid_limit): every request completes, large jobs never overlap, each result equals
    the job solved alone (a large job's state bit for bit: the cap only lengthens its launches),
    and a time limit censors what is still running; the one-at-a-time baseline of the same stream
    gives the same results."""
    import copy

    from paper_1311_3938_gb300 import workloads as W

    jobs = W.random_jobs(14, 700, n_range=(8, 14), T_range=(0.3, 1.5), rate=100.0, big_every=5, big_n=18,
                         path_mix=True)
    srv = W.Server(C64, batch_max_n=14, max_members=16, steps_per_round=8, big_chunk=16, keep_state=True,
                   policy="shortest", max_large=1, large_grid=8)
    try:
        res = srv.serve(copy.deepcopy(jobs))
    finally:
        srv.close()
    assert res["completed"] == len(jobs) and not res["censored_jobs"]
    big = sorted((j for j in res["jobs"] if j.route == "stream"), key=lambda j: j.admitted)
    assert len(big) == 2
    assert big[0].finished <= big[1].admitted  # one large job at a time
    for served in res["jobs"]:
        alone = W.solve_single(copy.deepcopy(jobs[served.jid]), keep_state=True)
        assert served.steps == alone.steps
        if served.route == "stream":
            assert np.array_equal(served.state, alone.state)
        else:
            assert rel_err(served.state, alone.state) < 2e-6
    seq = copy.deepcopy(jobs)
    done, cens, wall = W.serve_one_at_a_time(seq, order="shortest")
    assert len(done) == len(jobs) and not cens
    by_id = {j.jid: j for j in res["jobs"]}
    for j in done:
        assert j.steps == by_id[j.jid].steps and abs(j.P1 - by_id[j.jid].P1) < 1e-6
    # a time limit ends the served run with work in flight, released and reported as censored
    srv = W.Server(C64, batch_max_n=14, max_members=16, steps_per_round=8, big_chunk=16, policy="shortest",
                   max_large=1, large_grid=8)
    try:
        res = srv.serve(copy.deepcopy(jobs), time_limit=0.05)
    finally:
        srv.close()
    assert res["completed"] + len(res["censored_jobs"]) + len(res["not_admitted"]) == len(jobs)


def test_admission_respects_hbm_budget():
    import copy

    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import workloads as W

    jobs = W.random_jobs(8, 900, n_range=(14, 16), T_range=(0.2, 0.5), rate=1000.0)
    one = max(N.aqc_workspace_bytes(j.n, C64) for j in jobs)
    srv = W.Server(C64, hbm_budget=2 * one + 1, batch_max_n=16, max_members=8, steps_per_round=4)
    try:
        res = srv.serve(copy.deepcopy(jobs))
    finally:
        srv.close()
    assert res["completed"] == len(jobs)
    assert res["hbm_peak_bytes"] <= 2 * one + 1


def test_batched_equals_sequential():
    import copy

    from paper_1311_3938_gb300 import workloads as W

    jobs = W.random_jobs(12, 1000, n_range=(8, 16), T_range=(0.5, 2.0), nonlinear=True)
    a = copy.deepcopy(jobs)
    b = copy.deepcopy(jobs)
    W.run_batched(a, keep_state=True, steps_per_round=8)
    W.run_sequential(b, keep_state=True)
    for x, y in zip(a, b):
        assert x.steps == y.steps
        assert rel_err(x.state, y.state) < 2e-6


def test_autotuner_picks_a_listed_shape(tmp_path, monkeypatch):
    from paper_1311_3938_gb300 import autotune as A
    from paper_1311_3938_gb300 import workloads as W

    monkeypatch.setenv("AQC_CACHE_DIR", str(tmp_path))
    jobs = W.random_jobs(6, 77, n_range=(10, 15), T_range=(5.0, 10.0))
    shapes = [(0, 256, 8), (12, 128, 8)]
    best, entry = A.autotune(jobs, shapes=shapes, rounds=2)
    assert list(best) in [list(s) for s in shapes]
    assert all(r["amp_steps_per_s"] > 0 for r in entry["results"])
    best2, _ = A.autotune(jobs, shapes=shapes)  # served from the cache
    assert best2 == best
