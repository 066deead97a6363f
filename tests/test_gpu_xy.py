"""XY and XYZ algorithms (Sec. III.A.2-3) on the CUDA path, against the oracle.

Dicke initial states (Eq. initstate, the XYZ start), the XY start (the ground state of H^xy in
the solution's Hamming-weight sector, aqc_lanczos_ground, against the oracle's dense sector
diagonalisation), the drivers of Eq. Hixy / Eq. Hixyz (Y products go through the general-product
loop, pairs across layouts through the remote-product gather), the catalyst alpha s(1-s) H_{m-1}
of Eq. nlpath, and Hamming-weight conservation (Eq. Sigmaz).
"""
import numpy as np
import pytest

from instances import generate_ec3
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, rel_err, tol_fidelity

# the XY start vector against the oracle's sector ground state (relative, up to a global phase)
TOL_GROUND = {C128: 1e-10, C64: 1e-5}


def _phase_err(a, b):
    """min over phases phi of ||a e^{i phi} - b|| / ||b||."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    ph = ov / abs(ov) if abs(ov) > 0 else 1.0
    return rel_err(a * ph, b)

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


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n,seed,alpha", [(10, 2, 0.0), (12, 11, 8.0), (12, 13, 0.0)])
def test_xy_start_is_the_sector_ground_state(prec, n, seed, alpha):
    """set_xy_ground_start (Lanczos from the Dicke state, FP64 reductions) against the oracle's
    dense diagonalisation of the sector block of H^xy: vector up to a global phase, energy, and
    the reported residual; the vector stays in the sector."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    k = bin(inst.solution).count("1")
    E_ref, psi_ref = O.xy_sector_ground_state(n, inst.clauses, k)
    with Context(n, prec) as ctx:
        sched_poly, kk = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=alpha)
        assert kk == k
        ctx.set_schedule(5.0, sched_poly)
        E, resid, iters = HB.set_xy_ground_start(ctx, k)
        psi = ctx.state()
        e_at0 = ctx.energy_at(0.0)
    err = _phase_err(psi, psi_ref)
    print(f"XY start: n={n} precision {prec}: {iters} Lanczos steps, residual {resid:.2e}, "
          f"state error {err:.2e}, energy error {abs(E - E_ref):.2e}")
    assert err < TOL_GROUND[prec], err
    scale = max(1.0, abs(E_ref))
    assert abs(E - E_ref) < (1e-11 if prec == C128 else 1e-5) * scale
    assert abs(e_at0 - E_ref) < (1e-11 if prec == C128 else 1e-5) * scale
    assert resid < (1e-9 if prec == C128 else 1e-4) * scale
    w = np.array([bin(z).count("1") for z in range(1 << n)])
    assert np.all(psi[w != k] == 0)


def _run_xy(n, seed, prec, driver, alpha, T, steps=None, ground=True):
    """GPU and oracle solves of the XY (start: sector ground state of H^xy, each side its own)
    or XYZ (start: the Dicke state) algorithm; ground=False starts XY from the Dicke state."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    ctx = Context(n, prec)
    sched_poly, k = HB.load_xy(ctx, inst, driver=driver, catalyst_alpha=alpha)
    ctx.set_schedule(T, sched_poly)
    ctx.set_integrator(0, 0.0)
    xy_ground = driver == "xy" and ground
    if xy_ground:
        HB.set_xy_ground_start(ctx, k)
        psi0 = O.xy_sector_ground_state(n, inst.clauses, k)[1]
        start_err = _phase_err(ctx.state(), psi0)
        assert start_err < TOL_GROUND[prec]
    else:
        ctx.set_initial_state(("dicke", k))
        psi0 = O.dicke_state(n, k)
        start_err = 0.0
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
    ref = O.propagate(H, sched, O.step_count(H, sched), psi0, max_steps=-1 if steps is None else steps, nthreads=16)
    return inst, k, st, psi, ref, start_err


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("driver,alpha", [("xy", 0.0), ("xyz", 0.0), ("xy", 8.0)])
def test_xy_algorithms_full_solve(prec, driver, alpha):
    """n = 12: full solves of the XY algorithm from the ground state of H^xy in the solution's
    sector (and with the alpha = 8 catalyst of the paper's 13-qubit example) and of the XYZ
    algorithm from the Dicke state.  The evolution is unitary, so the start vectors' difference
    (bounded by TOL_GROUND) carries over unchanged; the bar adds it to the state bar."""
    inst, k, st, psi, ref, e0 = _run_xy(12, 11, prec, driver, alpha, 4.0)
    assert st["steps_done"] == ref.steps_done
    # the GPU start carries the phase <Dicke|x> > 0, the oracle's a positive amplitude sum:
    # both are the positive Perron vector, so no phase is removed here
    assert rel_err(psi, ref.psi) < TOL_STATE[prec] + e0
    # Hamming weight is conserved exactly: amplitudes outside the sector stay zero
    w = np.array([bin(z).count("1") for z in range(1 << 12)])
    assert np.all(psi[w != k] == 0)
    # |P_1 - P_1(oracle)| <= (2 + d) d for unit states at distance d (tol_fidelity's bound)
    bar = (1e-12 if prec == C128 else tol_fidelity(prec, ref.psi)) + (2.0 + e0) * e0
    assert abs(abs(psi[inst.solution]) ** 2 - abs(ref.psi[inst.solution]) ** 2) < bar


@pytest.mark.parametrize("prec", [C128, C64])
def test_xy_n21_first_steps(prec):
    """n = 21 (two layouts; pairs across layouts go through the remote-product gather): the
    first 10 steps of the XY path with catalyst against the oracle, from the Dicke state (an
    in-sector start that the oracle can form at this size; the step arithmetic is the same)."""
    inst, k, st, psi, ref, _ = _run_xy(21, 4, prec, "xy", 8.0, 10.0, steps=10, ground=False)
    assert rel_err(psi, ref.psi) < TOL_STATE[prec] * 0.1


@pytest.mark.parametrize("prec", [C128, C64])
def test_clause_by_clause_path_full_solve(prec):
    """Eq. cbc / Eq. kpath on the XY algorithm at n = 12: the step grid crosses every segment
    boundary; full solve against the oracle from the sector ground state of H^xy, and H(t) psi
    at points inside segments."""
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
    HB.set_xy_ground_start(ctx, k)
    psi0 = O.xy_sector_ground_state(n, cl, k)[1]
    e0 = _phase_err(ctx.state(), psi0)
    assert e0 < TOL_GROUND[prec]
    ctx.propagate(-1)
    got = ctx.state()
    ctx.close()
    ref = O.propagate(H, sched, O.step_count(H, sched), psi0, nthreads=16)
    assert rel_err(got, ref.psi) < TOL_STATE[prec] + e0
