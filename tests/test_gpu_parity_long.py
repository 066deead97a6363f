"""Parity with the FP64 oracle on the step grids the workloads run (Sec. I.B integrator).

* long runtime: a full solve of more than 40 000 grid steps (EC3 n = 12, nonlinear path,
  smoothstep s(t), T = 250), where the rounding of the FP32 state has the whole run to
  accumulate;
* the n = 20 workload: full solves at T = 10 for both paths and both s(t);
* the n = 28 workload of the bench (EC3 seed 3, linear path, T = 100): the first 8 grid steps of
  its step grid (3 RK4, f_3 and the predictor, 5 PEC steps) at full size, i.e. three tile layouts,
  the TMA-fed partial passes, the clause byte cache and the fused PEC kernel as the bench runs them.

Each case is compared on the whole state vector, in both precisions (relative error <= 1e-10
for complex128, <= 1e-5 for complex64).  The complex64 long run and one n = 20 solve also run
with the compensated corrector (aqc_set_y_compensation), whose error must stay far below the
uncompensated one's.  The oracle solves run in worker threads (the C oracle
releases the GIL): the long single-threaded run beside a queue of multithreaded ones, all
started when the module's first test asks for them, so they overlap the GPU solves.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from instances import generate_ec3, xx_pairs
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, rel_err, tol_fidelity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LONG = dict(n=12, seed=11, T=250.0, nonlinear=True, s_kind=1)
N20 = [(nl, sk) for nl in (False, True) for sk in (0, 1)]
N28 = dict(n=28, seed=3, T=100.0, steps=8)


def _host_bytes_available():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def _problem(n, seed, T, nonlinear, s_kind):
    inst = generate_ec3(n, seed)
    pairs = xx_pairs(n, seed) if nonlinear else None
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = (O.nonlinear_path if nonlinear else O.linear_path)(T, s_kind)
    return inst, pairs, H, sched


def _oracle_solve(n, seed, T, nonlinear, s_kind, max_steps=-1, nthreads=1):
    inst, pairs, H, sched = _problem(n, seed, T, nonlinear, s_kind)
    N = O.step_count(H, sched)
    r = O.propagate(H, sched, N, O.uniform_state(n), max_steps=max_steps, nthreads=nthreads)
    return N, r


@pytest.fixture(scope="module")
def oracle_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cores = os.cpu_count() or 1
    big = _host_bytes_available() >= (72 << 30)  # ten 4 GiB oracle vectors + the GPU results
    # the long single-threaded run beside a queue of multithreaded ones, in the order the tests
    # ask for them
    side, main = ThreadPoolExecutor(max_workers=1), ThreadPoolExecutor(max_workers=1)
    futs = {"long": side.submit(_oracle_solve, **LONG, nthreads=1)}
    nt = max(1, cores - 1)
    for nl, sk in N20:
        futs[("n20", nl, sk)] = main.submit(_oracle_solve, 20, 2, 10.0, nl, sk, -1, nt)
    if big:
        futs["n28"] = main.submit(_oracle_solve, N28["n"], N28["seed"], N28["T"], False, 0, N28["steps"], nt)
    yield futs
    for ex in (side, main):
        ex.shutdown(wait=True, cancel_futures=True)


def _gpu_solve(n, seed, T, nonlinear, s_kind, prec, max_steps=-1, ycomp=False):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    pairs = xx_pairs(n, seed) if nonlinear else None
    ctx = Context(n, prec, extra_vector=ycomp)
    HB.load_ec3(ctx, inst, pairs=pairs)
    ctx.set_schedule(T, HB.nonlinear_schedule() if nonlinear else HB.linear_schedule(), s_kind)
    ctx.set_integrator(0, 0.0)
    if ycomp:
        ctx.set_y_compensation(True)
    ctx.set_initial_state("uniform")
    st = ctx.propagate(max_steps)
    psi = ctx.state()
    P1 = ctx.fidelity(inst.solution)
    ctx.close()
    return st, psi, P1, inst


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


@pytest.mark.parametrize("prec", [C128, C64])
def test_long_runtime_full_solve(prec, oracle_runs):
    """More than 40 000 steps of the fixed-step grid (step rule, kappa = 0.1): the state after
    the whole run, P_1 and ||psi||^2 against the oracle."""
    st, psi, P1, inst = _gpu_solve(**LONG, prec=prec)
    N, ref = oracle_runs["long"].result()
    assert N >= 40000 and st["n_steps"] == N and st["steps_done"] == N
    err = rel_err(psi, ref.psi)
    print(f"long runtime: precision {prec}, {N} steps, relative state error {err:.3e}")
    assert err < TOL_STATE[prec], (prec, N, err)
    assert abs(P1 - O.fidelity(ref.psi, inst.solution)) < (1e-10 if prec == C128 else tol_fidelity(prec, ref.psi))
    assert abs(st["norm2"] - O.norm2(ref.psi)) < (1e-10 if prec == C128 else 1e-5)


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("nonlinear,s_kind", N20)
def test_n20_full_solve(nonlinear, s_kind, prec, oracle_runs):
    """The n = 20 workload (EC3 seed 2, 2n random XX couplings on the nonlinear path), T = 10:
    every grid step of the solve, both s(t)."""
    st, psi, P1, inst = _gpu_solve(20, 2, 10.0, nonlinear, s_kind, prec)
    N, ref = oracle_runs[("n20", nonlinear, s_kind)].result()
    assert st["n_steps"] == N and st["steps_done"] == N
    err = rel_err(psi, ref.psi)
    print(f"n=20: precision {prec}, nonlinear {nonlinear}, s_kind {s_kind}, {N} steps, error {err:.3e}")
    assert err < TOL_STATE[prec], (prec, nonlinear, s_kind, err)
    assert abs(P1 - O.fidelity(ref.psi, inst.solution)) < (1e-10 if prec == C128 else tol_fidelity(prec, ref.psi))


@pytest.mark.parametrize("prec", [C128, C64])
def test_n28_first_steps_full_state(prec, oracle_runs):
    """The bench's n = 28 workload, first 8 grid steps, whole 2^28-amplitude state."""
    if "n28" not in oracle_runs:
        pytest.skip("fewer than 72 GiB of host memory available for the n = 28 oracle")
    st, psi, P1, inst = _gpu_solve(N28["n"], N28["seed"], N28["T"], False, 0, prec, max_steps=N28["steps"])
    N, ref = oracle_runs["n28"].result()
    assert st["steps_done"] == N28["steps"] and st["n_steps"] == N
    assert st["evaluations"] == ref.evaluations
    psi = psi.astype(np.complex128)
    err = rel_err(psi, ref.psi)
    del psi
    print(f"n=28: precision {prec}, first {N28['steps']} steps, relative state error {err:.3e}")
    assert err < TOL_STATE[prec], (prec, err)


def test_long_runtime_compensated_corrector(oracle_runs):
    """The 42 000-step run in complex64 with y compensation: the rounding of y no longer
    accumulates, so the state error falls well below the plain FP32 corrector's (5e-6)."""
    st, psi, P1, inst = _gpu_solve(**LONG, prec=C64, ycomp=True)
    N, ref = oracle_runs["long"].result()
    err = rel_err(psi, ref.psi)
    print(f"long runtime, compensated complex64: {N} steps, relative state error {err:.3e}")
    assert st["steps_done"] == N
    assert err < 1.5e-6, err


def test_n20_compensated_corrector(oracle_runs):
    """The n = 20 nonlinear smoothstep solve (three layout passes per step) with y compensation."""
    st, psi, P1, inst = _gpu_solve(20, 2, 10.0, True, 1, C64, ycomp=True)
    N, ref = oracle_runs[("n20", True, 1)].result()
    err = rel_err(psi, ref.psi)
    print(f"n=20 compensated complex64: {N} steps, relative state error {err:.3e}")
    assert err < TOL_STATE[C64], err
