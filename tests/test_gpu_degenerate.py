"""Degenerate Hamiltonians through the CUDA path: H = 0 leaves psi(0) unchanged bit for bit;
an identity prefactor alone and a diagonal alone (clauses, no driver) evolve every amplitude by
its own phase, as in the oracle (same step grid), on one tile layout (n = 3) and on several
(n = 16)."""
import numpy as np
import pytest

from instances import generate_ec3, random_state
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, load_both, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _run(n, prec, terms, clauses, T, psi0):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    ctx = Context(n, prec)
    H = O.Hamiltonian(n)
    load_both(ctx, H, terms, clauses)
    sched = O.linear_path(T)
    N = O.step_count(H, sched)
    ctx.set_schedule(T, HB.linear_schedule())
    ctx.set_integrator(N, 0.0)
    ctx.set_initial_state(psi0.astype(np.complex128 if prec == C128 else np.complex64))
    st = ctx.propagate(-1)
    got = ctx.state()
    ctx.close()
    ref = O.propagate(H, sched, N, psi0.astype(np.complex128))
    return got, ref, st, N


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n", [3, 16])
def test_zero_hamiltonian_keeps_the_state(prec, n):
    psi0 = random_state(n, 7)
    got, ref, st, N = _run(n, prec, [], [], 5.0, psi0)
    assert N == 4 and st["steps_done"] == 4
    want = psi0.astype(np.complex128 if prec == C128 else np.complex64)
    assert np.array_equal(got, want)
    assert np.array_equal(ref.psi, psi0.astype(np.complex128))


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n", [3, 16])
def test_identity_and_diagonal_only(prec, n):
    psi0 = random_state(n, 11)
    # identity prefactor in group A (weight 1 - s): a global phase
    got, ref, _, _ = _run(n, prec, [(0, 0, 0, 1.5)], [], 4.0, psi0)
    assert rel_err(got, ref.psi) < TOL_STATE[prec]
    # clause penalties only (group B, weight s): one phase per amplitude
    inst = generate_ec3(n if n >= 6 else 6, 5)
    cl = [(1, tuple(b % n for b in c), O.PEN_INDICATOR, 1.0) for c in inst.clauses if len({b % n for b in c}) == 3]
    got, ref, _, _ = _run(n, prec, [], cl, 4.0, psi0)
    assert rel_err(got, ref.psi) < TOL_STATE[prec]
