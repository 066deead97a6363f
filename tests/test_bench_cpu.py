"""bench.py's accounting on the CPU: algorithmic bytes and flops per step, whole-job value,
layout count, the committed traffic profile's fields, and a short oracle sample."""
import json
import os

import pytest

import bench


def test_algorithmic_bytes_of_a_bench_step():
    n, amp, pec = 10, 8, 64
    N = 1 << n
    # 64 PEC steps at 7 vectors, 3 RK4 steps at 18, f_3 + predictor 8, init 1, energy 1
    assert bench.alg_bytes(n, amp, pec) == N * amp * (7 * 64 + 54 + 10)


def test_fp64_flops_of_a_pec_step():
    # 28 flips x 4 + diagonal 4 + 2 per class + corrector/predictor 32 + reductions 10
    assert bench.pec_flops_c128(28) == 112 + 4 + 2 + 32 + 10 == 160


def test_whole_job_value_is_weak_scaling():
    one = bench.whole_job_value(1e9, 5, 1, 1000.0)
    assert abs(one - 5.0) < 1e-12  # 5 GB in one second
    assert abs(bench.whole_job_value(1e9, 5, 4, 1000.0) - 4 * one) < 1e-12


@pytest.mark.parametrize("n,k", [(10, 1), (13, 1), (14, 2), (21, 2), (22, 3), (28, 3), (29, 3), (30, 4)])
def test_layout_count(n, k):
    assert bench.len_layouts(n, 13, 5) == k


def test_committed_traffic_profile_fields():
    p = os.path.join(bench.ROOT, "profiles", "pec_step_traffic.json")
    d = json.load(open(p))["c64"]
    assert len(d["kernel_hash"]) == 16 and d["launches"] == 3
    # 3k + 5 = 14 vectors of 2^28 complex64 amplitudes per PEC step, within a few percent
    assert abs(d["dram_bytes_per_pec_step"] / (14 * (1 << 28) * 8) - 1.0) < 0.05


def test_short_oracle_sample():
    gbs, cores, desc, secs = bench.cpu_sample(1.0)
    assert gbs > 0 and cores >= 1 and "oracle" in desc.lower()


def test_censored_quantiles():
    inf = float("inf")
    assert bench.quantile_censored([3.0, 1.0, 2.0], 0.5) == (2.0, False)
    assert bench.quantile_censored([3.0, 1.0, 2.0, inf], 0.5) == (2.0, False)
    assert bench.quantile_censored([3.0, 1.0, 2.0, inf], 0.99) == (None, True)
    assert bench.quantile_censored(list(range(1, 201)), 0.99) == (198, False)
    assert bench.quantile_censored([], 0.5) == (None, False)


def test_oracle_checks_in_spawned_workers_and_error_rows():
    """The host-side checker: two spawned workers solve small specs; the comparison rows of
    oracle_errors take the state of a finished job (here: the oracle's own, perturbed)."""
    import numpy as np

    from paper_1311_3938_gb300.workloads import Job

    checks = bench.OracleChecks(2)
    specs = {k: {"n": 6 + k, "seed": 1 + k, "nonlinear": bool(k % 2), "T": 2.0, "s_kind": k % 2} for k in range(3)}
    for k, sp in specs.items():
        checks.submit(("batch", k), sp)
    got = checks.results(timeout=120.0)
    assert set(got) == {("batch", k) for k in range(3)}
    jobs = []
    for k, sp in specs.items():
        _, N, P1, psi = got[("batch", k)]
        direct = bench.oracle_solve(sp)
        assert direct[1] == N and np.array_equal(direct[3], psi)
        j = Job(jid=k, n=sp["n"], seed=sp["seed"], nonlinear=sp["nonlinear"], T=sp["T"], s_kind=sp["s_kind"])
        j.state = (psi * (1 + 1e-7 * (k + 1))).astype(np.complex64)
        j.P1, j.steps = P1, N
        jobs.append(j)
    r = bench.oracle_errors(jobs, "batch", got)
    assert r["checked"] == 3 and r["eligible"] == 3 and r["step_grids_equal"]
    assert 2e-7 < r["max_state_err_vs_oracle"] < 1e-6
    assert r["max_P1_err_vs_oracle"] < 1e-12
