"""Pins of the oracle's XY / XYZ algorithms (Sec. III.A.2-3) against mathematics.

* Eq. Hixyz and Eq. Hixy on basis states: sigma_i . sigma_j |z> = zeta |z> + 2 [z_i != z_j] |z'>
  (zeta = +1 for equal bits, -1 otherwise; z' swaps bits i and j), so
      H^xyz |z> = sum_{i<j, z_i != z_j} n_ij (|z> - |z'>)
      H^xy  |z> = 3 m |z> - sum_{i<j, z_i != z_j} n_ij |z'>
  by brute force over all basis states (a wrong Y sign or a dropped term breaks it).
* The Dicke state of every weight is a zero-energy (ground) state of H^xyz (Eq. initstate):
  the symmetric states are pair triplets, where sigma_i . sigma_j = 1.
* Hamming weight is a constant of motion (Eq. Sigmaz): the XY and XYZ paths keep amplitudes
  outside the start sector exactly zero.
* The XYZ algorithm started in the Dicke state of the solution's weight reaches the solution
  at large T, with the energy bound of Sec. II.B.
* The XY algorithm's start, the ground state of H^xy in the solution's sector
  (xy_sector_ground_state): against the sector block written from the hopping picture
  (sigma+ sigma- moves), the closed form of the complete clause graph (total spin: the Dicke
  state is the ground state, energy in closed form), and the Kronecker-product matrix.
"""
import math

import numpy as np
import pytest

from instances import generate_ec3
from oracle import oracle as O


def _basis(n, z):
    v = np.zeros(1 << n, dtype=np.complex128)
    v[z] = 1.0
    return v


def _swap(z, i, j):
    return z ^ ((1 << i) | (1 << j))


@pytest.mark.parametrize("seed", [1, 2])
def test_drivers_on_basis_states(seed):
    inst = generate_ec3(7, seed)
    n, m = inst.n, inst.m
    nij = {}
    for c in inst.clauses:  # counted here by hand, independently of the oracle's helper
        for a in c:
            for b in c:
                if a < b:
                    nij[(a, b)] = nij.get((a, b), 0) + 1
    Hxyz = O.Hamiltonian(n)
    O.add_xyz_driver(Hxyz, inst.clauses, 0)
    Hxy = O.Hamiltonian(n)
    O.add_xy_driver(Hxy, inst.clauses, 0)
    for z in range(1 << n):
        e_xyz = np.zeros(1 << n, dtype=np.complex128)
        e_xy = np.zeros(1 << n, dtype=np.complex128)
        e_xy[z] += 3 * m
        for (i, j), v in nij.items():
            if ((z >> i) & 1) != ((z >> j) & 1):
                e_xyz[z] += v
                e_xyz[_swap(z, i, j)] -= v
                e_xy[_swap(z, i, j)] -= v
        got_xyz = O.hpsi(Hxyz, [1.0, 0.0, 0.0], _basis(n, z))
        got_xy = O.hpsi(Hxy, [1.0, 0.0, 0.0], _basis(n, z))
        assert np.max(np.abs(got_xyz - e_xyz)) < 1e-13
        assert np.max(np.abs(got_xy - e_xy)) < 1e-13


def test_dicke_states_are_xyz_ground_states():
    inst = generate_ec3(8, 3)
    n = inst.n
    H = O.Hamiltonian(n)
    O.add_xyz_driver(H, inst.clauses, 0)
    for k in range(n + 1):
        d = O.dicke_state(n, k)
        assert abs(np.vdot(d, d).real - 1.0) < 1e-14
        w = np.array([bin(z).count("1") for z in range(1 << n)])
        assert np.all(d[w != k] == 0) and np.all(d[w == k].real > 0)
        assert np.max(np.abs(O.hpsi(H, [1.0, 0.0, 0.0], d))) < 1e-12
    # and zero is the bottom of the spectrum: 1 - sigma_i . sigma_j >= 0
    ev = np.linalg.eigvalsh(O.dense_matrix(H, [1.0, 0.0, 0.0]))
    assert abs(ev[0]) < 1e-10


@pytest.mark.parametrize("driver", ["xy", "xyz"])
def test_paths_conserve_hamming_weight(driver):
    inst = generate_ec3(8, 4)
    n = inst.n
    k = bin(inst.solution).count("1")
    keep = list(inst.clauses[:-1])
    H = O.xy_hamiltonian(inst, driver=driver, catalyst=keep)
    sched = O.nonlinear_path(3.0, alpha=8.0)
    res = O.propagate(H, sched, O.step_count(H, sched), O.dicke_state(n, k))
    w = np.array([bin(z).count("1") for z in range(1 << n)])
    assert np.all(res.psi[w != k] == 0)
    assert abs(np.vdot(res.psi, res.psi).real - 1.0) < 1e-5


def test_xyz_algorithm_adiabatic_limit():
    inst = generate_ec3(7, 5)
    n = inst.n
    k = bin(inst.solution).count("1")
    H = O.xy_hamiltonian(inst, driver="xyz")
    P1 = []
    for T in (5.0, 80.0):
        sched = O.linear_path(T)
        res = O.propagate(H, sched, O.step_count(H, sched), O.dicke_state(n, k))
        p1 = O.fidelity(res.psi, inst.solution)
        E = O.energy(H, res.psi, 1)
        assert E >= (1.0 - p1) - 1e-9  # Sec. II.B: every excited state costs at least Omega
        P1.append(p1)
    assert P1[1] > 0.9 and P1[1] > P1[0]


def test_xy_catalyst_path_matches_library_ode_solver():
    """The XY algorithm with the catalyst (Eq. nlpath, alpha = 8) from the Dicke state: the
    oracle's PEC solution against scipy's DOP853 on the dense H(t) (Y products make it
    complex), at the step rule's h and at h/2 (4th order)."""
    from scipy.integrate import solve_ivp

    inst = generate_ec3(6, 3)
    n = inst.n
    k = bin(inst.solution).count("1")
    H = O.xy_hamiltonian(inst, driver="xy", catalyst=list(inst.clauses[:-1]))
    T = 2.0
    sched = O.nonlinear_path(T, alpha=8.0)
    M = [O.dense_matrix(H, [1.0 * (g == j) for j in range(3)] + [0.0]) for g in range(3)]

    def rhs(t, y):
        w = sched.weights(t)
        return -1j * ((w[0] * M[0] + w[1] * M[1] + w[2] * M[2]) @ y)

    psi0 = O.dicke_state(n, k)
    ref = solve_ivp(rhs, (0.0, T), psi0, method="DOP853", rtol=1e-12, atol=1e-14).y[:, -1]
    N = O.step_count(H, sched)
    errs = [np.linalg.norm(O.propagate(H, sched, j * N, psi0).psi - ref) for j in (1, 2)]
    assert errs[0] < 2e-6
    assert 10.0 < errs[0] / errs[1] < 24.0


# ---- the XY algorithm's start: ground state of H^xy in one Hamming-weight sector (Sec. III.A.3)


def _hopping_block(n, clauses, k):
    """The sector block of Eq. Hixy written from the hopping picture, without Pauli products:
    (X_i X_j + Y_i Y_j)/2 = sigma+_i sigma-_j + sigma-_i sigma+_j moves a one-bit between i and
    j, so <z'|H^xy|z> = -n_ij when z' is z with differing bits i, j swapped, and 3 m on the
    diagonal."""
    idx = [z for z in range(1 << n) if bin(z).count("1") == k]
    pos = {z: a for a, z in enumerate(idx)}
    nij = {}
    for c in clauses:
        for a in c:
            for b in c:
                if a < b:
                    nij[(a, b)] = nij.get((a, b), 0) + 1
    B = np.zeros((len(idx), len(idx)))
    for a, z in enumerate(idx):
        B[a, a] = 3.0 * len(clauses)
        for (i, j), v in nij.items():
            if ((z >> i) & 1) != ((z >> j) & 1):
                B[pos[_swap(z, i, j)], a] -= v
    return np.array(idx), B


@pytest.mark.parametrize("n,seed", [(8, 1), (10, 2), (11, 4)])
def test_xy_ground_state_against_the_hopping_block(n, seed):
    """Energy and vector against the eigenpair of the hopping-picture block; the state lies in
    the sector, has unit norm and (Perron-Frobenius: the block's off-diagonal entries are <= 0
    on a connected clause graph) strictly positive amplitudes there."""
    inst = generate_ec3(n, seed)
    k = bin(inst.solution).count("1")
    E, psi = O.xy_sector_ground_state(n, inst.clauses, k)
    idx, B = _hopping_block(n, inst.clauses, k)
    lam, V = np.linalg.eigh(B)
    assert lam[1] - lam[0] > 1e-3  # unique ground state
    v = V[:, 0] * np.sign(V[:, 0].sum())
    assert abs(E - lam[0]) < 1e-11 * max(1.0, abs(lam[0]))
    assert np.max(np.abs(psi[idx] - v)) < 1e-10
    out = np.ones(1 << n, dtype=bool)
    out[idx] = False
    assert np.all(psi[out] == 0)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
    assert np.all(psi[idx].real > 0) and np.max(np.abs(psi[idx].imag)) < 1e-13


@pytest.mark.parametrize("n", [4, 5, 6])
def test_xy_ground_state_on_the_complete_graph_is_dicke(n):
    """All C(n,3) triples as clauses: every pair has n_ij = n - 2, and with S = sum sigma / 2,
    sum_{i<j} (X_i X_j + Y_i Y_j) = 2 (S^2 - S_z^2) - n.  The ground state of each sector is then
    the Dicke state (total spin n/2), at energy 3 m - (n - 2)/2 [2 (n/2 (n/2 + 1) - (n/2 - k)^2) - n]."""
    import itertools

    clauses = [tuple(c) for c in itertools.combinations(range(n), 3)]
    m = len(clauses)
    for k in range(n + 1):
        E, psi = O.xy_sector_ground_state(n, clauses, k)
        want = 3.0 * m - (n - 2) / 2.0 * (2.0 * (n / 2 * (n / 2 + 1) - (n / 2 - k) ** 2) - n)
        assert abs(E - want) < 1e-11 * max(1.0, abs(want)), (n, k, E, want)
        assert np.max(np.abs(psi - O.dicke_state(n, k))) < 1e-12


def test_xy_ground_state_against_the_kronecker_matrix():
    """The dense 2^n matrix of Eq. Hixy built from Kronecker products (dense_matrix, its own
    pins in test_oracle_pins.py): its lowest eigenvalue in the sector equals the energy, and
    the state is an eigenvector of it to rounding."""
    inst = generate_ec3(9, 6)
    n, k = inst.n, bin(inst.solution).count("1")
    E, psi = O.xy_sector_ground_state(n, inst.clauses, k)
    H = O.Hamiltonian(n)
    O.add_xy_driver(H, inst.clauses, 0)
    D = O.dense_matrix(H, [1.0, 0.0, 0.0, 0.0])
    idx = [z for z in range(1 << n) if bin(z).count("1") == k]
    ev = np.linalg.eigvalsh(D[np.ix_(idx, idx)])
    assert abs(ev[0] - E) < 1e-11 * max(1.0, abs(E))
    assert np.linalg.norm(D @ psi - E * psi) < 1e-10
    # below the Dicke state's energy (it is not an eigenstate of H^xy on this graph)
    d = O.dicke_state(n, k)
    assert E < np.vdot(d, D @ d).real - 1e-6
