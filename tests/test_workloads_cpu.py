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
