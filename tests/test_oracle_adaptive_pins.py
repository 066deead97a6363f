"""Pins of the oracle's step-size control (or_propagate_adaptive), which the paper leaves open:
segments of constant step that land on T, a PEC step accepted if its Milne estimate is at most
tol ||y||, h halved after a rejection and doubled after a run of small estimates.

Pinned against: the fixed-grid integrator (itself pinned in test_oracle_pins.py) when nothing
is ever rejected; the exact exponential of a constant Hamiltonian (eigendecomposition); scipy's
DOP853 on the dense time-dependent H(t); and the segment bookkeeping (contiguous segments
covering [0, T], halving and doubling as logged).
"""
import math

import numpy as np
import pytest

from instances import generate_ec3, random_state, xx_pairs
from oracle import oracle as O

SEG_RUNNING, SEG_AT_T, SEG_REJECTED, SEG_GREW = O.SEG_RUNNING, O.SEG_AT_T, O.SEG_REJECTED, O.SEG_GREW


def _check_segments(res, T):
    """Segments are contiguous, cover [0, T], and each step change follows its segment's end."""
    segs = res.segments
    assert segs[0][0] == 0.0
    for (t0, h, steps, end), nxt in zip(segs, segs[1:]):
        assert end in (SEG_REJECTED, SEG_GREW)
        assert nxt[0] == pytest.approx(t0 + steps * h, rel=1e-13, abs=1e-13 * T)
        R = T - nxt[0]
        hp = h / 2 if end == SEG_REJECTED else 2 * h
        m = math.ceil(R / hp * (1 - 1e-12))
        assert nxt[1] == pytest.approx(R / m, rel=1e-14)
        assert nxt[1] <= hp * (1 + 1e-12)
    t0, h, steps, end = segs[-1]
    assert end == SEG_AT_T
    assert t0 + steps * h == pytest.approx(T, rel=1e-12)
    assert sum(s[2] for s in segs) == res.steps_done
    assert res.t_end == pytest.approx(T, rel=1e-12)


@pytest.mark.parametrize("s_kind", [0, 1])
def test_no_rejection_is_the_fixed_grid_bit_for_bit(s_kind):
    """tol = inf, no growth: one segment of the rule's grid, the same state as or_propagate."""
    inst = generate_ec3(9, 4)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(9, 4))
    sched = O.nonlinear_path(3.7, s_kind)
    N = O.step_count(H, sched)
    a = O.propagate_adaptive(H, sched, sched.T / N, math.inf, O.uniform_state(9), grow_after=0)
    b = O.propagate(H, sched, N, O.uniform_state(9))
    assert a.segments == [(0.0, sched.T / N, N, SEG_AT_T)]
    assert np.array_equal(a.psi, b.psi)
    assert (a.steps_done, a.evaluations, a.rejects) == (N, b.evaluations, 0)
    assert a.max_err_est == b.max_err_est


def _constant_problem(n=6, seed=2):
    """H = H_i + H_f + H_c, constant in time (all weights 1)."""
    inst = generate_ec3(n, seed)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(n, seed))
    sched = O.Schedule(1.0, 0, ((1.0, 0, 0, 0), (1.0, 0, 0, 0), (1.0, 0, 0, 0)))
    M = O.dense_matrix(H, [1.0, 1.0, 1.0, 0.0])
    return H, sched, M


def test_unstable_start_is_rejected_down_to_a_stable_step():
    """A first step 4x the step rule's (|h lambda| ~ 0.4, beyond the PEC scheme's stable range on
    the imaginary axis) is rejected and halved until accepted; the result matches the exact
    exponential, while the fixed grid at that step size does not."""
    H, sched, M = _constant_problem()
    T = 6.0
    sched.T = T
    lam, V = np.linalg.eigh(M)
    psi0 = random_state(6, 3)
    exact = V @ (np.exp(-1j * lam * T) * (V.conj().T @ psi0))
    N = O.step_count(H, sched)
    h0 = 4 * T / N
    res = O.propagate_adaptive(H, sched, h0, 1e-10, psi0, grow_after=0)
    _check_segments(res, T)
    assert res.rejects >= 1
    assert res.segments[0][3] == SEG_REJECTED
    assert res.segments[-1][1] < h0 / 2
    err = np.linalg.norm(res.psi - exact)
    assert err < 1e-7, err
    fixed = O.propagate(H, sched, int(round(T / h0)), psi0)
    assert np.linalg.norm(fixed.psi - exact) > 1e3 * err


def test_step_grows_after_small_estimates():
    """Started 64 times finer than needed, the step doubles repeatedly (after each run of
    `grow_after` small estimates), the run takes far fewer steps than the fine grid and still
    agrees with the exact exponential to the accumulated tolerance."""
    H, sched, M = _constant_problem(5, 7)
    T = 4.0
    sched.T = T
    lam, V = np.linalg.eigh(M)
    psi0 = O.uniform_state(5)
    exact = V @ (np.exp(-1j * lam * T) * (V.conj().T @ psi0))
    N = O.step_count(H, sched)
    h0 = T / (64 * N)
    res = O.propagate_adaptive(H, sched, h0, 1e-8, psi0, grow_after=4)
    _check_segments(res, T)
    grew = [s for s in res.segments if s[3] == SEG_GREW]
    assert len(grew) >= 4
    assert max(s[1] for s in res.segments) > 8 * h0
    assert res.steps_done < 64 * N / 4
    # the global error is at most the sum of the accepted local errors (each <= tol ||y||)
    assert np.linalg.norm(res.psi - exact) < 1e-8 * res.steps_done


def test_time_dependent_path_against_dop853_and_tolerance_scaling():
    """The interacting, time-dependent path (driver, clauses, XX couplings; smoothstep s(t)):
    the controlled run agrees with DOP853 on the dense H(t), and a 1000x tighter tolerance gives
    a much smaller error."""
    from scipy.integrate import solve_ivp

    n = 6
    inst = generate_ec3(n, 5)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(n, 5))
    sched = O.nonlinear_path(5.0, 1)
    psi0 = O.uniform_state(n)

    def rhs(t, y):
        return -1j * (O.dense_matrix(H, sched.weights(t)) @ y)

    ref = solve_ivp(rhs, (0.0, sched.T), psi0.astype(complex), method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1]
    N = O.step_count(H, sched)
    errs = []
    for tol in (1e-6, 1e-9):
        res = O.propagate_adaptive(H, sched, 4 * sched.T / N, tol, psi0, grow_after=8)
        _check_segments(res, sched.T)
        errs.append(np.linalg.norm(res.psi - ref))
    assert errs[1] < 1e-7
    assert errs[0] > 20 * errs[1]


def test_every_accepted_estimate_is_within_tolerance():
    """max over accepted steps of the Milne estimate <= tol ||y|| (||y|| ~ 1 here), while the
    first, rejected attempt was above it."""
    H, sched, M = _constant_problem()
    sched.T = 3.0
    N = O.step_count(H, sched)
    tol = 1e-8
    res = O.propagate_adaptive(H, sched, 4 * sched.T / N, tol, O.uniform_state(6), grow_after=0)
    nrm = math.sqrt(O.norm2(res.psi))
    assert res.rejects >= 1
    assert 0.0 < res.max_err_est <= tol * nrm * (1 + 1e-6)


def test_minimum_step_fails():
    """A tolerance below the rounding floor halves h until it falls below hmin: error."""
    H, sched, M = _constant_problem(5, 7)
    sched.T = 1.0
    with pytest.raises(RuntimeError):
        O.propagate_adaptive(H, sched, 0.05, 1e-30, O.uniform_state(5), hmin=0.05 / 64)
