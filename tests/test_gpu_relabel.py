"""Qubit relabelling (aqc_set_relabel) is transparent: every entry point gives the same
results, in qubit order, with and without it, on an XY instance whose pair products span
layouts (so the library does reorder the index bits)."""
import numpy as np
import pytest

from instances import generate_ec3, random_state
from oracle import oracle as O

from _helpers import C64, C128, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _ctx(n, prec, inst, relabel):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    ctx = Context(n, prec)
    ctx.set_relabel(relabel)
    sched, k = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=8.0)
    ctx.set_schedule(10.0, sched)
    ctx.set_integrator(0, 0.0)
    return ctx, k


@pytest.mark.parametrize("prec", [C128, C64])
def test_relabelled_results_match(prec):
    n = 22
    inst = generate_ec3(n, 3)
    a, k = _ctx(n, prec, inst, True)
    b, _ = _ctx(n, prec, inst, False)
    tol = 1e-12 if prec == C128 else 2e-6
    psi = torch.from_numpy(random_state(n, 5)).cuda()
    ha, hb = a.hpsi(3.1, psi).cpu().numpy(), b.hpsi(3.1, psi).cpu().numpy()
    assert rel_err(ha, hb) < tol
    for c in (a, b):
        c.set_initial_state(("dicke", k))
        c.propagate(12)
    assert rel_err(a.state(), b.state()) < tol
    assert rel_err(a.state(device=True).cpu().numpy(), b.state()) < tol
    assert abs(a.fidelity(inst.solution) - b.fidelity(inst.solution)) < tol * 1e-2 + 1e-15
    assert abs(a.energy() - b.energy()) < tol * 10
    ea, _, _ = a.lanczos(4.0, psi, max_iter=60, n_eig=2, tol=1e-12)
    eb, _, _ = b.lanczos(4.0, psi, max_iter=60, n_eig=2, tol=1e-12)
    assert np.max(np.abs(np.array(ea) - np.array(eb))) < (1e-9 if prec == C128 else 1e-3)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_state_round_trips_are_exact(prec):
    n = 21
    inst = generate_ec3(n, 4)
    a, _ = _ctx(n, prec, inst, True)
    v = random_state(n, 9).astype(np.complex128 if prec == C128 else np.complex64)
    a.set_initial_state(v)  # host copy
    assert np.array_equal(a.state(), v)
    a.set_initial_state(torch.from_numpy(v).cuda())  # device copy
    assert np.array_equal(a.state(device=True).cpu().numpy(), v)
    a.set_initial_state(123457)
    s = a.state()
    assert s[123457] == 1 and np.count_nonzero(s) == 1
    a.close()


def test_reorder_of_a_live_state():
    """Loading more products after the state is set (the order may change at the next table
    build) gives the same propagation as loading them first."""
    n = 21
    inst = generate_ec3(n, 4)
    extra = [(2, (1 << 3) | (1 << 17), 0, 0.4), (2, (1 << 9) | (1 << 20), 0, -0.3)]
    a, k = _ctx(n, C128, inst, True)
    a.set_initial_state(("dicke", k))
    for (g, x, z, c) in extra:
        a.load_terms(g, [x], [z], [c])
    a.propagate(8)
    b, _ = _ctx(n, C128, inst, False)
    for (g, x, z, c) in extra:
        b.load_terms(g, [x], [z], [c])
    b.set_initial_state(("dicke", k))
    b.propagate(8)
    assert rel_err(a.state(), b.state()) < 1e-12
    a.close()
    b.close()
