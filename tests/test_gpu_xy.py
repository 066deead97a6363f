"""XY and XYZ algorithms (Sec. III.A.2-3) on the CUDA path, against the oracle.

Dicke initial states (Eq. initstate), the drivers of Eq. Hixy / Eq. Hixyz (Y products go through
the general-product loop, pairs across layouts through the remote-product gather), the catalyst
alpha s(1-s) H_{m-1} of Eq. nlpath, and Hamming-weight conservation (Eq. Sigmaz).
"""
import numpy as np
import pytest

from instances import generate_ec3
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, rel_err, tol_fidelity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


@pytest.mark.parametrize("prec", [C128, C64])
def test_dicke_initial_states(prec):
    from paper_1311_3938_gb300.engine import Context

    n = 12
    with Context(n, prec) as ctx:
        ctx.load_terms(0, [1], [0], [1.0])
        ctx.set_schedule(1.0, ((1, 0, 0, 0), (0, 0, 0, 0), (0, 0, 0, 0)))
        for k in (0, 1, 5, 6, n):
            ctx.set_initial_state(("dicke", k))
            got = ctx.state()
            assert rel_err(got, O.dicke_state(n, k)) < (1e-15 if prec == C128 else 1e-7)
        from paper_1311_3938_gb300 import _native as N

        with pytest.raises(N.AqcError):
            ctx.set_initial_state(("dicke", n + 1))


def _run_xy(n, seed, prec, driver, alpha, T, steps=None):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    ctx = Context(n, prec)
    sched_poly, k = HB.load_xy(ctx, inst, driver=driver, catalyst_alpha=alpha)
    ctx.set_schedule(T, sched_poly)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state(("dicke", k))
    st = ctx.propagate(-1 if steps is None else steps)
    psi = ctx.state()
    ctx.close()
    cl = list(inst.clauses)
    keep = None
    if alpha:
        rem = HB.removable_clauses(n, cl)
        r = rem[-1] if rem else len(cl) - 1
        keep = cl[:r] + cl[r + 1:]
    H = O.xy_hamiltonian(inst, driver=driver, catalyst=keep)
    sched = O.nonlinear_path(T, alpha=alpha) if alpha else O.linear_path(T)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.dicke_state(n, k),
                      max_steps=-1 if steps is None else steps, nthreads=16)
    return inst, k, st, psi, ref


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("driver,alpha", [("xy", 0.0), ("xyz", 0.0), ("xy", 8.0)])
def test_xy_algorithms_full_solve(prec, driver, alpha):
    """n = 12: full solves of the XY and XYZ algorithms (and XY with the alpha = 8 catalyst of
    the paper's 13-qubit example) from the Dicke state of the solution's weight."""
    inst, k, st, psi, ref = _run_xy(12, 11, prec, driver, alpha, 4.0)
    assert st["steps_done"] == ref.steps_done
    assert rel_err(psi, ref.psi) < TOL_STATE[prec]
    # Hamming weight is conserved exactly: amplitudes outside the sector stay zero
    w = np.array([bin(z).count("1") for z in range(1 << 12)])
    assert np.all(psi[w != k] == 0)
    assert abs(abs(psi[inst.solution]) ** 2 - abs(ref.psi[inst.solution]) ** 2) < (
        1e-12 if prec == C128 else tol_fidelity(prec, ref.psi))


@pytest.mark.parametrize("prec", [C128, C64])
def test_xy_n21_first_steps(prec):
    """n = 21 (two layouts; pairs across layouts go through the remote-product gather): the
    first 10 steps of the XY algorithm with catalyst against the oracle."""
    inst, k, st, psi, ref = _run_xy(21, 4, prec, "xy", 8.0, 10.0, steps=10)
    assert rel_err(psi, ref.psi) < TOL_STATE[prec] * 0.1


@pytest.mark.parametrize("prec", [C128, C64])
def test_clause_by_clause_path_full_solve(prec):
    """Eq. cbc / Eq. kpath on the XY algorithm at n = 12: the step grid crosses every segment
    boundary; full solve against the oracle, and H(t) psi at points inside segments."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, T = 12, 6.0
    inst = generate_ec3(n, 13)
    cl = list(inst.clauses)
    ctx = Context(n, prec)
    sched_poly, k = HB.load_xy(ctx, inst, driver="xy", clause_by_clause=True)
    ctx.set_schedule(T, sched_poly)
    H = O.xy_hamiltonian(inst, driver="xy")
    O.add_clause_by_clause(H, cl, group=2)
    sched = O.clause_by_clause_path(T)
    psi = O.dicke_state(n, k) * (1.0 + 0.5j)
    dpsi = torch.from_numpy(psi).cuda()
    m = len(cl)
    for t in (0.0, T * 0.37 / m, T * (2.5 / m), T * (m - 0.5) / m, T):
        got = ctx.hpsi(t, dpsi).cpu().numpy()
        ref = O.hpsi(H, sched.weights(t), dpsi.cpu().numpy().astype(np.complex128))
        assert rel_err(got, ref) < (1e-13 if prec == C128 else 2e-6), t
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state(("dicke", k))
    ctx.propagate(-1)
    got = ctx.state()
    ctx.close()
    ref = O.propagate(H, sched, O.step_count(H, sched), O.dicke_state(n, k), nthreads=16)
    assert rel_err(got, ref.psi) < TOL_STATE[prec]
