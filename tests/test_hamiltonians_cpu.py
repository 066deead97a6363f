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
