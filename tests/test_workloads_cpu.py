"""Host-side logic of the workload drivers (no GPU)."""
import math

import pytest


def test_random_jobs_seeded_and_poisson():
    from paper_1311_3938_gb300 import workloads as W

    a = W.random_jobs(50, 3, n_range=(10, 26), T_range=(10.0, 500.0), rate=4.0, big_every=10, big_n=30,
                      path_mix=True)
    b = W.random_jobs(50, 3, n_range=(10, 26), T_range=(10.0, 500.0), rate=4.0, big_every=10, big_n=30,
                      path_mix=True)
    assert [(j.n, j.T, j.arrival, j.nonlinear) for j in a] == [(j.n, j.T, j.arrival, j.nonlinear) for j in b]
    assert all(10 <= j.n <= 26 or j.n == 30 for j in a)
    assert sum(j.n == 30 for j in a) == 5
    assert all(10.0 <= j.T <= 500.0 for j in a)
    arr = [j.arrival for j in a]
    assert arr == sorted(arr) and arr[0] > 0
    gaps = [y - x for x, y in zip([0.0] + arr[:-1], arr)]
    assert 0.1 < sum(gaps) / len(gaps) < 0.5  # mean gap ~ 1/rate
    assert {j.nonlinear for j in a} == {True, False}


def _job(jid, n, arrival):
    from paper_1311_3938_gb300 import workloads as W

    return W.Job(jid=jid, n=n, seed=jid, nonlinear=False, T=10.0, arrival=arrival)


def _admit(pending, t, used, budget, members, max_members=4, batch_max_n=22):
    from paper_1311_3938_gb300 import workloads as W

    started = []

    def start(job, small):
        started.append((job.jid, small))
        if small:
            members.append(job.jid)

    used = W.admit_ready(pending, lambda: t, used, budget, lambda: len(members), max_members, batch_max_n, start)
    return used, started


def test_admission_fifo_by_hbm_budget():
    j = [_job(0, 20, 0.0), _job(1, 24, 0.1), _job(2, 12, 0.2), _job(3, 12, 5.0)]
    w = [x.workspace_bytes() for x in j]
    assert w[1] > w[0] > w[2] > 0
    pending = list(j)
    budget = w[0] + w[2] + w[2] // 2  # job 1 does not fit beside job 0; job 2 would
    members = []
    used, started = _admit(pending, 1.0, 0, budget, members)
    # job 0 admitted; job 1 waits for memory and blocks job 2 behind it; job 3 has not arrived
    assert started == [(0, True)] and used == w[0]
    assert [x.jid for x in pending] == [1, 2, 3]
    # job 0 retires: job 1 (a large state, its own stream) and then job 2 fit
    used, started = _admit(pending, 1.0, 0, w[1] + w[2], [])
    assert started == [(1, False), (2, True)] and used == w[1] + w[2]
    assert [x.jid for x in pending] == [3]
    used, started = _admit(pending, 4.9, used, 10 * w[1], [])
    assert started == [] and [x.jid for x in pending] == [3]  # not arrived yet
    used, started = _admit(pending, 5.0, used, 10 * w[1], [])
    assert started == [(3, True)] and pending == []


def test_admission_member_limit_blocks_the_queue():
    j = [_job(0, 12, 0.0), _job(1, 12, 0.0), _job(2, 12, 0.0), _job(3, 26, 0.0)]
    pending = list(j)
    members = []
    used, started = _admit(pending, 0.0, 0, 1 << 40, members, max_members=2)
    # two members fill the batch; the third small job waits and the large job behind it too
    assert started == [(0, True), (1, True)]
    assert [x.jid for x in pending] == [2, 3]
    members.pop()
    used, started = _admit(pending, 0.0, used, 1 << 40, members, max_members=2)
    assert started == [(2, True), (3, False)] and pending == []
    assert used == sum(x.workspace_bytes() for x in j)


def test_admission_shortest_first_with_one_large_job():
    """policy "shortest": arrived jobs by estimated work (T n 2^n); at most one large job runs;
    a job that does not fit the budget waits without blocking smaller ones."""
    from paper_1311_3938_gb300 import workloads as W

    j = [_job(0, 24, 0.0), _job(1, 14, 0.0), _job(2, 22, 0.0), _job(3, 12, 0.0), _job(4, 12, 9.0)]
    j[1].T, j[3].T = 50.0, 100.0  # 50 * 14 * 2^14 > 100 * 12 * 2^12
    assert W.work_estimate(j[3]) < W.work_estimate(j[1]) < W.work_estimate(j[2]) < W.work_estimate(j[0])
    pending = list(j)
    started, members, large = [], [], []

    def start(job, small):
        started.append(job.jid)
        (members if small else large).append(job.jid)

    used = W.admit_shortest_first(pending, lambda: 1.0, 0, 1 << 40, lambda: len(members), 8, 20,
                                  lambda: len(large), 1, start)
    # small jobs by work, then the smaller of the two large ones; job 0 waits; job 4 not arrived
    assert started == [3, 1, 2]
    assert [x.jid for x in pending] == [0, 4]
    assert used == sum(x.workspace_bytes() for x in (j[1], j[2], j[3]))
    large.clear()
    started.clear()
    # budget too small for job 0: it waits, job 4 (arrived now, small) does not wait behind it
    used = W.admit_shortest_first(pending, lambda: 10.0, 0, j[0].workspace_bytes() - 1, lambda: 0, 8, 20,
                                  lambda: len(large), 1, start)
    assert started == [4] and [x.jid for x in pending] == [0]


def test_server_rejects_an_unknown_policy():
    from paper_1311_3938_gb300 import workloads as W

    with pytest.raises(ValueError):
        W.serve_one_at_a_time([], order="random")
