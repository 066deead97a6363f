"""Host-side logic of the workload drivers (no GPU)."""
import math


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
