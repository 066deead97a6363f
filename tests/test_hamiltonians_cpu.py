"""Host-side term builders of the package (no GPU): the XY/XYZ drivers and the catalyst
clause choice, checked against the oracle's independent builders and by brute force."""
import numpy as np
import pytest

from instances import generate_ec3
from oracle import oracle as O


def _oracle_from_terms(n, x, z, c, group=0):
    H = O.Hamiltonian(n)
    for a, b, v in zip(x, z, c):
        H.add_term(group, int(a), int(b), float(v))
    return H


@pytest.mark.parametrize("driver", ["xy", "xyz"])
@pytest.mark.parametrize("seed", [1, 7])
def test_driver_terms_match_oracle(driver, seed):
    from paper_1311_3938_gb300 import hamiltonians as HB

    inst = generate_ec3(7, seed)
    x, z, c = (HB.xy_driver_terms if driver == "xy" else HB.xyz_driver_terms)(inst.clauses)
    got = O.dense_matrix(_oracle_from_terms(inst.n, x, z, c), [1.0, 0.0, 0.0])
    ref = O.dense_matrix(O.xy_hamiltonian(inst, driver=driver), [1.0, 0.0, 0.0])
    assert np.max(np.abs(got - ref)) < 1e-12


def _components(n, clauses):
    adj = {b: set() for c in clauses for b in c}
    for c in clauses:
        for a in c:
            adj[a].update(c)
    seen, comps = set(), 0
    for s in adj:
        if s in seen:
            continue
        comps += 1
        stack = [s]
        while stack:
            u = stack.pop()
            if u in seen:
                continue
            seen.add(u)
            stack.extend(adj[u] - seen)
    return comps, set(adj)


@pytest.mark.parametrize("n,seed", [(8, 3), (10, 1), (13, 3), (16, 5)])
def test_removable_clauses_keep_the_graph_connected(n, seed):
    from paper_1311_3938_gb300 import hamiltonians as HB

    inst = generate_ec3(n, seed)
    cl = list(inst.clauses)
    comps0, bits0 = _components(n, cl)
    got = set(HB.removable_clauses(n, cl))
    for k in range(len(cl)):
        rest = cl[:k] + cl[k + 1:]
        comps, bits = _components(n, rest)
        keeps = comps <= comps0 and bits == bits0 if comps0 == 1 else True
        assert (k in got) == keeps, (k, comps, bits0 - bits)


@pytest.mark.parametrize("weighted", [False, True])
def test_x_driver_and_couplings_match_oracle(weighted):
    """x_driver_terms (uniform 1/2 or the paper's n_i/2) and xx_terms against the oracle's
    builders, as dense matrices."""
    from instances import xx_pairs
    from paper_1311_3938_gb300 import hamiltonians as HB

    n = 7
    inst = generate_ec3(n, 4)
    w = None
    if weighted:
        w = np.zeros(n)
        for c in inst.clauses:
            for b in c:
                w[b] += 0.5
    x, z, c = HB.x_driver_terms(n, w)
    H = O.Hamiltonian(n)
    O.add_x_driver(H, 0, weights=w)
    assert np.max(np.abs(O.dense_matrix(_oracle_from_terms(n, x, z, c), [1.0, 0.0, 0.0])
                         - O.dense_matrix(H, [1.0, 0.0, 0.0]))) < 1e-12
    pairs = xx_pairs(n, 4)
    x, z, c = HB.xx_terms(pairs)
    Hc = O.Hamiltonian(n)
    O.add_xx_terms(Hc, pairs, 2)
    assert np.max(np.abs(O.dense_matrix(_oracle_from_terms(n, x, z, c, 2), [0.0, 0.0, 1.0])
                         - O.dense_matrix(Hc, [0.0, 0.0, 1.0]))) < 1e-12


def test_zz_form_terms_match_clause_penalties():
    """ec3_zz_terms (Eq. final_ham) equals the squared clause penalties (1 - k)^2 of Eq. hci on
    every basis state."""
    from paper_1311_3938_gb300 import hamiltonians as HB

    inst = generate_ec3(8, 6)
    x, z, c = HB.ec3_zz_terms(inst.n, inst.clauses)
    assert not np.any(x)
    got = O.dense_matrix(_oracle_from_terms(inst.n, x, z, c, 1), [0.0, 1.0, 0.0])
    H = O.Hamiltonian(inst.n)
    O.add_ec3_clauses(H, inst.clauses, 1, penalty=O.PEN_SQUARED)
    assert np.max(np.abs(got - O.dense_matrix(H, [0.0, 1.0, 0.0]))) < 1e-12


@pytest.mark.parametrize("alpha", [1.0, 8.0])
def test_schedule_polynomials_match_oracle_paths(alpha):
    """The package's schedule coefficients give the oracle paths' weights at every s."""
    from paper_1311_3938_gb300 import hamiltonians as HB

    T = 10.0
    cases = [(HB.linear_schedule(), O.linear_path(T)), (HB.nonlinear_schedule(alpha), O.nonlinear_path(T, alpha=alpha)),
             (HB.clause_by_clause_schedule(), O.clause_by_clause_path(T))]
    for poly, path in cases:
        for t in np.linspace(0.0, T, 11):
            s = t / T
            want = path.weights(t)
            for g in range(3):
                got = sum(poly[g][k] * s ** k for k in range(4))
                assert abs(got - want[g]) < 1e-14, (g, t)
