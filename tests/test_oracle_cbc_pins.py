"""Pins of the oracle's clause-by-clause term H_d(s) (Eq. cbc, Eq. kpath).

The C oracle sums the definition over k with the Theta factors; the checks build H_d from
explicit partial sums H_j of clause diagonals, segment by segment, and test the properties the
paper states: H_d(0) = H_d(1) = 0 (H(0) = H^xy, H(1) = H_f), continuity at s = k/m, and on
s_k in [0, 1) the interpolation (1 - s_k) H_{k-1} + s_k H_k with H_0 = H_m = 0.
"""
import numpy as np
import pytest

from instances import generate_ec3
from oracle import oracle as O


def _diag_of(H, weights):
    n = H.n
    return np.array([O.hpsi(H, weights, np.eye(1, 1 << n, z, dtype=np.complex128)[0])[z].real for z in range(1 << n)])


def _partial_sum(n, clauses, j, m):
    d = np.zeros(1 << n)
    if 1 <= j <= m - 1:
        for c in clauses[:j]:
            d += O.clause_diagonal(n, c, O.PEN_INDICATOR)
    return d


@pytest.mark.parametrize("seed", [1, 4])
def test_segments_interpolate_partial_sums(seed):
    inst = generate_ec3(7, seed)
    n, cl = inst.n, list(inst.clauses)
    m = len(cl)
    H = O.Hamiltonian(n)
    O.add_clause_by_clause(H, cl, group=2)
    for k in range(1, m + 1):
        for sk in (0.0, 0.3, 0.9):
            s = (k - 1 + sk) / m
            got = _diag_of(H, [0.0, 0.0, 1.0, s])
            ref = (1 - sk) * _partial_sum(n, cl, k - 1, m) + sk * _partial_sum(n, cl, k, m)
            assert np.max(np.abs(got - ref)) < 1e-12, (k, sk)


def test_ends_vanish_and_continuity():
    inst = generate_ec3(8, 2)
    n, cl = inst.n, list(inst.clauses)
    m = len(cl)
    H = O.Hamiltonian(n)
    O.add_clause_by_clause(H, cl, group=2)
    assert np.max(np.abs(_diag_of(H, [0.0, 0.0, 1.0, 0.0]))) == 0.0
    assert np.max(np.abs(_diag_of(H, [0.0, 0.0, 1.0, 1.0]))) == 0.0
    for k in range(1, m):
        a = _diag_of(H, [0.0, 0.0, 1.0, k / m - 1e-12])
        b = _diag_of(H, [0.0, 0.0, 1.0, k / m])
        assert np.max(np.abs(a - b)) < 1e-9
    # the dense builder (segment formula) agrees with the C oracle (sum over k)
    for s in (0.05, 0.37, 0.5, 0.99):
        D = O.dense_matrix(H, [0.0, 0.0, 1.0, s])
        assert np.max(np.abs(np.diag(D).real - _diag_of(H, [0.0, 0.0, 1.0, s]))) < 1e-12


def test_cbc_path_from_xy_start_reaches_h_f():
    """Eq. cbc with the XY driver: H(0) = H^xy and H(1) = H_f exactly (the weights of the
    oracle's schedule and H_d vanish at the ends)."""
    inst = generate_ec3(7, 3)
    n, cl = inst.n, list(inst.clauses)
    H = O.xy_hamiltonian(inst, driver="xy")
    O.add_clause_by_clause(H, cl, group=2)
    sched = O.clause_by_clause_path(10.0)
    Hxy = O.Hamiltonian(n)
    O.add_xy_driver(Hxy, cl, 0)
    Hf = O.Hamiltonian(n)
    O.add_ec3_clauses(Hf, cl, 1)
    assert np.max(np.abs(O.dense_matrix(H, sched.weights(0.0)) - O.dense_matrix(Hxy, [1, 0, 0, 0]))) < 1e-12
    assert np.max(np.abs(O.dense_matrix(H, sched.weights(10.0)) - O.dense_matrix(Hf, [0, 1, 0, 0]))) < 1e-12


@pytest.mark.parametrize("m,N", [(11, 4620), (7, 2940), (13, 1001)])
def test_one_segment_on_step_grids(m, N):
    """On step grids whose points fall on segment ends up to rounding, every clause coefficient
    stays in [0, 1] and the coefficients match the segment formula (no segment counted twice)."""
    cl = [(0, 1, 2)] * m
    H = O.Hamiltonian(3)
    for j in range(m):
        H.add_clause(2, (0, 1, 2), O.PEN_INDICATOR, 1.0, step=j + 1)
    T = 6.0
    h = T / N
    for n in range(N + 1):
        for t in (n * h, n * h + 0.5 * h):
            s = t / T
            d = O.hpsi(H, [0.0, 0.0, 1.0, s], np.eye(1, 8, 0, dtype=np.complex128)[0])[0].real  # z = 0: pen 1 each
            # the segment of s from its integer part; sum of the coefficients of H_d on it
            k = min(int(np.floor(m * s)) + 1, m)
            sk = m * s - k + 1
            ref = 0.0
            if 0.0 <= s < 1.0:
                ref = (1 - sk) * (k - 1 if 1 <= k - 1 <= m - 1 else 0) + sk * (k if k <= m - 1 else 0)
            assert abs(d - ref) < 1e-9, (n, s * m, d, ref)


def test_cbc_path_matches_library_ode_solver():
    """The clause-by-clause XY path from the Dicke state against scipy's DOP853 on the dense
    H(t) of the segment formula, integrated segment by segment so that the library solver never
    steps across a kink at s = k/m.  The fixed-step PEC history spans the kinks, where dH/dt
    jumps, so its error falls at 2nd order rather than 4th."""
    from scipy.integrate import solve_ivp

    inst = generate_ec3(6, 3)
    n, cl = inst.n, list(inst.clauses)
    m = len(cl)
    H = O.xy_hamiltonian(inst, driver="xy")
    O.add_clause_by_clause(H, cl, group=2)
    T = 2.0
    sched = O.clause_by_clause_path(T)
    psi0 = O.dicke_state(n, bin(inst.solution).count("1"))
    y, t0 = psi0.copy(), 0.0
    for j in range(1, m + 1):
        t1 = T * j / m
        sol = solve_ivp(lambda t, v: -1j * (O.dense_matrix(H, sched.weights(t)) @ v), (t0, t1), y,
                        method="DOP853", rtol=1e-12, atol=1e-14)
        y, t0 = sol.y[:, -1], t1
    N = O.step_count(H, sched)
    errs = [np.linalg.norm(O.propagate(H, sched, j * N, psi0).psi - y) for j in (1, 2)]
    assert errs[0] < 1e-5
    assert 3.0 < errs[0] / errs[1] < 6.0
