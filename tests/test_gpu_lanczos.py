"""Lanczos spectrum of H(t) on the CUDA path (aqc_lanczos) against dense diagonalisation of
the oracle's Kronecker-product matrix: full space from a random start (X algorithm) and one
Hamming-weight sector from the Dicke start (XY algorithm, Eq. Sigmaz)."""
import numpy as np
import pytest

from instances import generate_ec3, random_state
from oracle import oracle as O

from _helpers import C64, C128

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _distinct(ev, tol=1e-7):
    out = []
    for v in np.sort(ev):
        if not out or v - out[-1] > tol:
            out.append(v)
    return np.array(out)


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("s", [0.15, 0.5, 0.85])
def test_x_algorithm_spectrum(prec, s):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, T = 10, 10.0
    inst = generate_ec3(n, 1)
    ctx = Context(n, prec)
    HB.load_ec3(ctx, inst)
    ctx.set_schedule(T, HB.linear_schedule())
    start = torch.from_numpy(random_state(n, 17)).cuda()
    eig, conv, iters = ctx.lanczos(s * T, start, max_iter=160, n_eig=3, tol=1e-12)
    ctx.close()
    H = O.ec3_hamiltonian(inst)
    ref = _distinct(np.linalg.eigvalsh(O.dense_matrix(H, O.linear_path(T).weights(s * T))))[:3]
    tol = 1e-9 if prec == C128 else 2e-4
    assert np.max(np.abs(np.array(eig) - ref)) < tol * max(1.0, np.abs(ref).max()), (eig, ref, iters)


@pytest.mark.parametrize("prec", [C128, C64])
def test_xy_sector_spectrum_and_gap(prec):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, T, s = 10, 10.0, 0.4
    inst = generate_ec3(n, 2)
    ctx = Context(n, prec)
    sched, k = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=8.0)
    ctx.set_schedule(T, sched)
    ctx.set_initial_state(("dicke", k))
    start = ctx.state(device=True)
    eig, conv, iters = ctx.lanczos(s * T, start, max_iter=120, n_eig=2, tol=1e-12)
    ctx.close()
    cl = list(inst.clauses)
    rem = HB.removable_clauses(n, cl)
    r = rem[-1] if rem else len(cl) - 1
    H = O.xy_hamiltonian(inst, driver="xy", catalyst=cl[:r] + cl[r + 1:])
    D = O.dense_matrix(H, O.nonlinear_path(T, alpha=8.0).weights(s * T))
    idx = [z for z in range(1 << n) if bin(z).count("1") == k]
    ref = _distinct(np.linalg.eigvalsh(D[np.ix_(idx, idx)]))[:2]
    tol = 1e-9 if prec == C128 else 2e-4
    assert np.max(np.abs(np.array(eig) - ref)) < tol * max(1.0, np.abs(ref).max()), (eig, ref, iters)
    assert eig[1] - eig[0] > 0
