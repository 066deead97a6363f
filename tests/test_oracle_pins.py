"""Pins of the FP64 CPU oracle against facts fixed by the paper or by mathematics.

Each test pins the oracle to something other than itself: the paper's printed example,
textbook Pauli matrices, dense linear algebra (numpy eigh / Kronecker products), closed forms
(Landau-Zener, product states, binomial spectra, free-fermion Ising chain), brute force, and
the convergence order of the scheme.
"""
import math
import os

import numpy as np
import pytest

from instances import generate_ec3, random_state, xx_pairs
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_pauli_ham(n, seed, nterms=12, nclauses=3):
    rng = np.random.default_rng(seed)
    H = O.Hamiltonian(n)
    for _ in range(nterms):
        g = int(rng.integers(0, 3))
        x = int(rng.integers(0, 1 << n))
        z = int(rng.integers(0, 1 << n))
        H.add_term(g, x, z, float(rng.normal()))
    if n >= 3:
        for _ in range(nclauses):
            bits = rng.choice(n, size=3, replace=False)
            H.add_clause(int(rng.integers(0, 3)), bits, int(rng.integers(0, 2)), float(rng.uniform(0.5, 2)))
    return H


# ---------------------------------------------------------------- conventions (paper-printed)
def test_golden_bit_order_and_clauses():
    """Sec. I.C / Fig. ec3: z = 1098 is printed as z_13..z_1 = 0010001001010, and the three
    printed clauses (Sec. III.A.1) are satisfied (exactly one upbit, Eq. sat) by it."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ec3_13bit_example.txt")) if l.strip() and l[0] != "#"]
    d = {r[0]: r[1:] for r in rows if r[0] != "clause"}
    clauses = [tuple(int(x) - 1 for x in r[1:]) for r in rows if r[0] == "clause"]
    n = int(d["n"][0])
    w = int(d["solution_decimal"][0])
    bits = d["solution_bits_msb_first"][0]
    # z = sum_i z_i 2^(i-1) with the string written z_n ... z_1
    assert sum(int(bits[n - i]) << (i - 1) for i in range(1, n + 1)) == w
    for c in clauses:
        # indicator and squared penalties (Eq. hci) are 0 at the solution, 1 at z = 0
        for pen in (O.PEN_INDICATOR, O.PEN_SQUARED):
            diag = O.clause_diagonal(n, c, pen)
            assert diag[w] == 0.0
            assert diag[0] == 1.0
    # sigma^x on qubit 1 flips the least-significant bit (Eq. ztensor ordering)
    H = O.Hamiltonian(n)
    H.add_term(0, 1, 0, 1.0)
    e = np.zeros(1 << n, complex)
    e[w] = 1
    out = O.hpsi(H, [1, 0, 0], e)
    assert abs(out[w ^ 1] - 1) < 1e-15 and np.count_nonzero(out) == 1


def test_single_qubit_paulis_textbook():
    """The dense builder reproduces the textbook 2x2 matrices, and qubit 1 is the low bit."""
    assert np.allclose(O.pauli_string_matrix(1, 1, 0), [[0, 1], [1, 0]])
    assert np.allclose(O.pauli_string_matrix(1, 0, 1), [[1, 0], [0, -1]])
    assert np.allclose(O.pauli_string_matrix(1, 1, 1), [[0, -1j], [1j, 0]])
    # sigma^x_1 on 2 qubits maps |z=0> to |z=1>; sigma^x_2 maps |0> to |2>
    M1 = O.pauli_string_matrix(2, 1, 0)
    M2 = O.pauli_string_matrix(2, 2, 0)
    assert M1[1, 0] == 1 and M2[2, 0] == 1
    # Y Z = i X on one qubit (Pauli algebra)
    Y = O.pauli_string_matrix(1, 1, 1)
    Z = O.pauli_string_matrix(1, 0, 1)
    X = O.pauli_string_matrix(1, 1, 0)
    assert np.allclose(Y @ Z, 1j * X)


# ---------------------------------------------------------------- SQH matvec
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7])
def test_hpsi_matches_dense(n):
    """Scatter-form SQH matvec (Sec. I.A) equals the dense Kronecker-product matrix."""
    for seed in range(3):
        H = _random_pauli_ham(n, 100 * n + seed)
        w = [0.3, -1.7, 0.9]
        psi = random_state(n, seed)
        got = O.hpsi(H, w, psi)
        ref = O.dense_matrix(H, w) @ psi
        assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("n", [3, 6, 9])
def test_hpsi_at_matches_dense_and_full(n):
    """Single-output evaluation equals the dense matrix row and the full scatter matvec."""
    H = _random_pauli_ham(n, 300 + n, nterms=20)
    w = [0.7, -0.2, 1.3]
    psi = random_state(n, 9)
    zs = np.arange(1 << n)
    got = O.hpsi_at(H, w, psi, zs)
    assert np.max(np.abs(got - O.dense_matrix(H, w) @ psi)) < 1e-13
    assert np.max(np.abs(got - O.hpsi(H, w, psi))) < 1e-13


def test_hpsi_threads_identical():
    H = _random_pauli_ham(9, 7, nterms=30, nclauses=8)
    psi = random_state(9, 3)
    a = O.hpsi(H, [1, 0.5, -2], psi, nthreads=1)
    b = O.hpsi(H, [1, 0.5, -2], psi, nthreads=4)
    assert np.array_equal(a, b)


def test_dense_hamiltonian_is_hermitian():
    H = _random_pauli_ham(5, 11)
    M = O.dense_matrix(H, [1.0, 2.0, 3.0])
    assert np.allclose(M, M.conj().T, atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_clause_form_equals_zz_form(seed):
    """Eq. final_ham: sum of squared clause penalties (Eq. hci) = the Z/ZZ form."""
    inst = generate_ec3(9, seed)
    Ha = O.Hamiltonian(9)
    O.add_ec3_clauses(Ha, inst.clauses, group=1, penalty=O.PEN_SQUARED)
    Hb = O.Hamiltonian(9)
    O.add_ec3_zz_form(Hb, 9, inst.clauses, group=1)
    psi = random_state(9, seed)
    a = O.hpsi(Ha, [0, 1, 0], psi)
    b = O.hpsi(Hb, [0, 1, 0], psi)
    assert np.max(np.abs(a - b)) < 1e-12


def test_x_driver_ground_state_and_spectrum():
    """Eq. Hix with weights 1/2: |S> has energy 0, spectrum {0..n} with binomial degeneracy."""
    n = 6
    H = O.x_driver(n)
    S = O.uniform_state(n)
    assert np.max(np.abs(O.hpsi(H, [1, 0, 0], S))) < 1e-15
    ev = np.linalg.eigvalsh(O.dense_matrix(H, [1, 0, 0]))
    ks, counts = np.unique(np.round(ev, 9), return_counts=True)
    assert list(ks) == list(range(n + 1))
    assert list(counts) == [math.comb(n, k) for k in range(n + 1)]


def test_paper_weighted_x_driver():
    """Eq. Hix with weights n_i/2: spectrum is all subset sums of the n_i."""
    inst = generate_ec3(6, 4)
    ni, _ = inst.clause_counts()
    H = O.x_driver(6, weights=[v / 2 for v in ni])
    ev = np.sort(np.linalg.eigvalsh(O.dense_matrix(H, [1, 0, 0])))
    sums = np.sort([sum(ni[i] for i in range(6) if (m >> i) & 1) for m in range(64)])
    assert np.allclose(ev, sums, atol=1e-12)


@pytest.mark.parametrize("n,seed", [(8, 1), (10, 1), (12, 5)])
def test_final_hamiltonian_ground_state_brute_force(n, seed):
    """H_f has a unique zero-energy basis state, the instance's solution w, and every other
    basis state costs at least Omega (Sec. II.B)."""
    inst = generate_ec3(n, seed)
    H = O.Hamiltonian(n)
    O.add_ec3_clauses(H, inst.clauses, group=1, penalty=O.PEN_INDICATOR)
    ones = np.ones(1 << n, complex)
    d = O.hpsi(H, [0, 1, 0], ones).real
    assert d[inst.solution] == 0.0
    others = np.delete(d, inst.solution)
    assert others.min() >= 1.0
    # brute force on the clause list directly
    z = np.arange(1 << n)
    sat = np.ones(1 << n, bool)
    for (a, b, c) in inst.clauses:
        sat &= (((z >> a) & 1) + ((z >> b) & 1) + ((z >> c) & 1)) == 1
    assert list(np.nonzero(sat)[0]) == [inst.solution]


def test_ising_chain_free_fermion_ground_energy():
    """Eq. ising (periodic transverse-field chain, Omega = 1): the ground energy from the
    oracle's terms matches the free-fermion closed form -sum_k sqrt(g^2 + J^2 - 2 g J cos k),
    k = pi (2j-1)/n, g = 1-s, J = s."""
    n = 8
    H = O.Hamiltonian(n)
    for i in range(n):
        H.add_term(0, 1 << i, 0, -1.0)
        H.add_term(1, 0, (1 << i) | (1 << ((i + 1) % n)), -1.0)
    for s in [0.0, 0.2, 0.5, 0.7, 1.0]:
        M = O.dense_matrix(H, [1 - s, s, 0])
        e0 = np.linalg.eigvalsh(M)[0]
        g, J = 1 - s, s
        ks = [math.pi * (2 * j - 1) / n for j in range(1, n + 1)]
        ref = -sum(math.sqrt(g * g + J * J - 2 * g * J * math.cos(k)) for k in ks)
        assert abs(e0 - ref) < 1e-10


# ---------------------------------------------------------------- integrator
def _expm_apply(M, psi, t):
    ev, V = np.linalg.eigh(M)
    return V @ (np.exp(-1j * ev * t) * (V.conj().T @ psi))


def _const_sched(T, w):
    return O.Schedule(T, O.S_LINEAR, ((w[0], 0, 0, 0), (w[1], 0, 0, 0), (w[2], 0, 0, 0)))


def test_rk4_startup_is_fourth_order_taylor():
    """For time-independent H, one classical RK4 step equals sum_{k<=4} (-i h H)^k / k!."""
    n = 4
    H = _random_pauli_ham(n, 5)
    w = [0.4, 0.3, -0.2]
    M = O.dense_matrix(H, w)
    psi0 = random_state(n, 8)
    h = 0.05
    res = O.propagate(H, _const_sched(h, w), 1, psi0)
    A = -1j * h * M
    ref = psi0.copy()
    term = psi0.copy()
    for k in range(1, 5):
        term = A @ term / k
        ref = ref + term
    assert np.max(np.abs(res.psi - ref)) < 1e-14
    assert res.evaluations == 4


@pytest.mark.parametrize("n", [3, 5])
def test_constant_hamiltonian_matches_exponential(n):
    """Frozen schedule: psi(T) = V exp(-i Lambda T) V^+ psi0 (exact diagonalisation)."""
    H = _random_pauli_ham(n, 21 + n)
    w = [0.5, 0.25, 0.3]
    M = O.dense_matrix(H, w)
    psi0 = random_state(n, n)
    T = 3.0
    lam = np.abs(np.linalg.eigvalsh(M)).max()
    N = int(math.ceil(T * lam / 0.01))
    res = O.propagate(H, _const_sched(T, w), N, psi0)
    ref = _expm_apply(M, psi0, T)
    assert np.linalg.norm(res.psi - ref) < 1e-8
    assert res.evaluations == 12 + 1 + (N - 3)
    assert abs(res.t_end - T) < 1e-12


def test_fourth_order_convergence():
    """Global error of the PEC scheme shrinks ~16x when h halves (fourth order, Sec. I.B)."""
    n = 4
    H = _random_pauli_ham(n, 77)
    w = [0.6, 0.4, 0.2]
    M = O.dense_matrix(H, w)
    psi0 = random_state(n, 1)
    T = 4.0
    ref = _expm_apply(M, psi0, T)
    errs = []
    lam = np.abs(np.linalg.eigvalsh(M)).max()
    N0 = int(math.ceil(T * lam / 0.05))
    for N in [N0, 2 * N0, 4 * N0]:
        errs.append(np.linalg.norm(O.propagate(H, _const_sched(T, w), N, psi0).psi - ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13 < r1 < 19 and 14 < r2 < 18, (errs, r1, r2)


def test_landau_zener():
    """H(t) = (v (t - T/2) / 2) sigma^z + (Delta / 2) sigma^x: starting in the instantaneous
    ground state, the diabatic probability -> exp(-pi Delta^2 / (2 v))."""
    v, Delta, T = 1.0, 0.5, 200.0
    H = O.Hamiltonian(1)
    H.add_term(0, 0, 1, 1.0)  # sigma^z, weight (v T / 2)(s - 1/2)
    H.add_term(1, 1, 0, 1.0)  # sigma^x, weight Delta / 2
    sched = O.Schedule(T, O.S_LINEAR, ((-v * T / 4, v * T / 2, 0, 0), (Delta / 2, 0, 0, 0), (0, 0, 0, 0)))
    M0 = O.dense_matrix(H, sched.weights(0.0))
    ev, V = np.linalg.eigh(M0)
    psi0 = V[:, 0].astype(complex)
    N = O.step_count(H, sched, kappa=0.05)
    res = O.propagate(H, sched, N, psi0)
    # diabatic state at the end: the basis state that was the ground state at the start (|0>)
    p_dia = abs(res.psi[0]) ** 2
    ref = math.exp(-math.pi * Delta ** 2 / (2 * v))
    assert abs(p_dia - ref) < 6e-3, (p_dia, ref)


def _single_qubit_reference(a0, a1, bz0, bz1, T, psi0, M=20000, smooth=False):
    """2x2 evolution under H(t) = (a0 + a1 s) X + (bz0 + bz1 s) Z, s = t/T or 3 tau^2 - 2 tau^3,
    by a product of exact 2x2 exponentials at midpoints (second order), refined by Richardson
    extrapolation."""
    def run(M):
        psi = np.array(psi0, complex)
        h = T / M
        for k in range(M):
            t = (k + 0.5) * h
            sv = t / T if not smooth else (t / T) ** 2 * (3 - 2 * t / T)
            ax = a0 + a1 * sv
            bz = bz0 + bz1 * sv
            r = math.hypot(ax, bz)
            # exp(-i h (ax X + bz Z)) = cos(hr) I - i sin(hr)/r (ax X + bz Z)
            c, s = math.cos(h * r), (math.sin(h * r) / r if r > 0 else h)
            U = np.array([[c - 1j * s * bz, -1j * s * ax], [-1j * s * ax, c + 1j * s * bz]])
            psi = U @ psi
        return psi

    a, b = run(M), run(2 * M)
    return (4 * b - a) / 3


@pytest.mark.parametrize("s_kind", [0, 1])
def test_product_state_time_dependent(s_kind):
    """Non-interacting H(s) = (1-s) sum c_i (1 - X_i) + s sum b_i Z_i factorises; the oracle's
    n-qubit solution equals the Kronecker product of single-qubit solutions (s = t/T and the
    smoothstep s(t))."""
    n = 5
    rng = np.random.default_rng(5)
    c = rng.uniform(0.3, 1.0, n)
    b = rng.uniform(-1.0, 1.0, n)
    T = 6.0
    H = O.Hamiltonian(n)
    O.add_x_driver(H, 0, list(c))
    for i in range(n):
        H.add_term(1, 0, 1 << i, b[i])
    sched = O.linear_path(T, s_kind)
    psi0 = O.uniform_state(n)
    N = O.step_count(H, sched, kappa=0.02)
    got = O.propagate(H, sched, N, psi0).psi
    # per qubit: H_q(t) = (1 - t/T) c (1 - X) + (t/T) b Z ; the identity part gives a phase
    full = np.ones(1, complex)
    phase = 0.0
    for q in range(n):
        # (1-s) c (I - X) + s b Z = (1-s) c I + [-(1-s) c] X + [s b] Z
        phase += c[q] * T / 2  # integral of (1 - s(t)) c over [0, T] (both s(t) average 1/2)
        psi_q = _single_qubit_reference(-c[q], c[q], 0.0, b[q], T, np.array([1, 1]) / math.sqrt(2),
                                        smooth=(s_kind == 1))
        full = np.kron(psi_q, full)  # qubit q is bit q: later qubits are more significant
    ref = full * np.exp(-1j * phase)
    assert np.linalg.norm(got - ref) < 1e-8


def test_adiabatic_limit_and_energy_bound():
    """Sec. II.B: P_1(T) -> 1 and E(T) -> 0 as T grows; always E(T) >= Omega (1 - P_1)."""
    inst = generate_ec3(8, 3)
    H = O.ec3_hamiltonian(inst)
    psi0 = O.uniform_state(8)
    fids, ens = [], []
    for T in [5.0, 20.0, 80.0, 320.0]:
        sched = O.linear_path(T)
        res = O.propagate(H, sched, O.step_count(H, sched), psi0)
        P1 = O.fidelity(res.psi, inst.solution)
        E = O.energy(H, res.psi, group=1)
        assert E >= (1 - P1) * O.norm2(res.psi) - 1e-9
        fids.append(P1)
        ens.append(E)
    assert fids[0] < fids[1] < fids[2] < fids[3] and fids[3] > 0.99
    assert ens[0] > ens[1] > ens[2] > ens[3] and ens[3] < 1e-2


def test_norm_drift_fourth_order():
    """The scheme does not preserve the norm exactly; the drift is O(h^4)."""
    inst = generate_ec3(6, 2)
    H = O.ec3_hamiltonian(inst)
    psi0 = O.uniform_state(6)
    sched = O.linear_path(10.0)
    N = O.step_count(H, sched)
    d1 = abs(O.norm2(O.propagate(H, sched, N, psi0).psi) - 1)
    d2 = abs(O.norm2(O.propagate(H, sched, 2 * N, psi0).psi) - 1)
    assert d1 < 1e-4
    assert d2 < d1 / 8


def test_step_count_rule():
    """N = ceil(T * Lambda / kappa), Lambda = max_s sum_g |w_g(s)| ||H_g||_1."""
    inst = generate_ec3(10, 1)
    H = O.ec3_hamiltonian(inst)
    # ||H_i||_1 = n/2 (identity) + n * 1/2 = n ; ||H_f||_1 = m (indicator penalties)
    assert O.step_count(H, O.linear_path(20.0)) == math.ceil(20.0 * max(10, inst.m) / O.KAPPA)
    pairs = xx_pairs(10, 1)
    Hc = O.ec3_hamiltonian(inst, pairs=pairs)
    J = sum(abs(p[2]) for p in pairs)
    lam = max(abs(1 - s) * 10 + s * inst.m + s * (1 - s) * J for s in np.linspace(0, 1, 1025))
    assert O.step_count(Hc, O.nonlinear_path(10.0)) == math.ceil(10.0 * lam / O.KAPPA)


def test_c_schedule_weights_closed_form():
    """The C oracle's w_g(s(t)) for both s(t) against the closed forms."""
    import ctypes as C

    lib = O._load()
    for kind in (0, 1):
        sc = O.nonlinear_path(8.0, kind, alpha=2.0)._ctypes()
        for t in (0.0, 1.0, 2.5, 4.0, 6.5, 8.0):
            w = (C.c_double * 4)()
            lib.or_weights(C.byref(sc), t, w)
            tau = t / 8.0
            s = tau if kind == 0 else 3 * tau * tau - 2 * tau ** 3
            assert abs(w[0] - (1 - s)) < 1e-15 and abs(w[1] - s) < 1e-15 and abs(w[2] - 2 * s * (1 - s)) < 1e-15
            assert abs(w[3] - s) < 1e-15


def test_smoothstep_schedule_weights():
    sc = O.linear_path(10.0, O.S_SMOOTHSTEP)
    for t, s in [(0.0, 0.0), (5.0, 0.5), (10.0, 1.0), (2.5, 3 * 0.0625 - 2 * 0.015625)]:
        w = sc.weights(t)
        assert abs(w[0] - (1 - s)) < 1e-15 and abs(w[1] - s) < 1e-15


@pytest.mark.parametrize("s_kind", [0, 1])
def test_diagonal_hamiltonian_phases(s_kind):
    """A diagonal H(t) = A(s) c 1 + B(s) H_f (clause penalties, no driver) turns each amplitude
    by exp(-i (c int A dt + d_z int B dt)); int A dt = int B dt = T/2 for both s(t) (the
    smoothstep is symmetric about t = T/2).  The oracle reaches that closed form at 4th order."""
    inst = generate_ec3(6, 5)
    n, T, c = inst.n, 4.0, 1.5
    H = O.Hamiltonian(n)
    O.add_ec3_clauses(H, inst.clauses, 1)
    H.add_term(0, 0, 0, c)
    d = np.zeros(1 << n)
    for z in range(1 << n):  # penalty [k != 1] counted by hand over the clauses
        d[z] = sum(1.0 for cl in inst.clauses if sum((z >> b) & 1 for b in cl) != 1)
    psi0 = random_state(n, 3)
    exact = psi0 * np.exp(-1j * (c * T / 2 + d * T / 2))
    sched = O.linear_path(T, s_kind)
    N = O.step_count(H, sched)
    errs = [np.linalg.norm(O.propagate(H, sched, k * N, psi0).psi - exact) for k in (1, 2)]  # unit-norm psi0
    assert errs[0] < 5e-5
    assert 10.0 < errs[0] / errs[1] < 24.0  # 4th order: halving h divides the error by ~16


def test_interacting_path_matches_library_ode_solver():
    """EC3 n = 6 with the X driver and XX couplings on the nonlinear path (all three groups time
    dependent): the oracle's PEC solution against scipy's DOP853 (an 8th-order Runge-Kutta
    method, tight tolerances) on the dense H(t), at the step rule's h and at h/2 (4th order)."""
    from scipy.integrate import solve_ivp

    inst = generate_ec3(6, 2)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(6, 2))
    T = 3.0
    sched = O.nonlinear_path(T)
    M = [O.dense_matrix(H, [1.0 * (g == k) for k in range(3)] + [0.0]) for g in range(3)]

    def rhs(t, y):
        w = sched.weights(t)
        return -1j * ((w[0] * M[0] + w[1] * M[1] + w[2] * M[2]) @ y)

    psi0 = O.uniform_state(6)
    ref = solve_ivp(rhs, (0.0, T), psi0, method="DOP853", rtol=1e-12, atol=1e-14).y[:, -1]
    N = O.step_count(H, sched)
    errs = [np.linalg.norm(O.propagate(H, sched, k * N, psi0).psi - ref) for k in (1, 2)]
    assert errs[0] < 1e-6
    assert 10.0 < errs[0] / errs[1] < 24.0
