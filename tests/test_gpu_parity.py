"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: relative state error <= 1e-10 for complex128 and <= 1e-5 for complex64 (the FP32
state path with FP64 reductions); observables compared at matching accuracy.
"""
import math

import numpy as np
import pytest

from instances import generate_ec3, random_state, xx_pairs
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, load_both, random_clauses, random_terms, rel_err, tol_fidelity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _ctx(n, prec):
    from paper_1311_3938_gb300.engine import Context

    return Context(n, prec)


def _setup_ec3(n, prec, seed, T, nonlinear=False, s_kind=0, penalty=0):
    from paper_1311_3938_gb300 import hamiltonians as HB

    inst = generate_ec3(n, seed)
    pairs = xx_pairs(n, seed) if nonlinear else None
    ctx = _ctx(n, prec)
    HB.load_ec3(ctx, inst, pairs=pairs, penalty=penalty)
    ctx.set_schedule(T, HB.nonlinear_schedule() if nonlinear else HB.linear_schedule(), s_kind)
    H = O.ec3_hamiltonian(inst, penalty=penalty, pairs=pairs)
    sched = (O.nonlinear_path if nonlinear else O.linear_path)(T, s_kind)
    return inst, ctx, H, sched


# ------------------------------------------------------------------ matvec
@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 13, 14, 16, 19])
def test_hpsi_random_pauli_products(n, prec):
    """SQH matvec (Sec. I.A) with X/Y/Z strings, identities and clauses of both penalty kinds
    in all three groups, at sizes spanning one tile, several tiles and several layouts."""
    for seed in range(2):
        ctx = _ctx(n, prec)
        H = O.Hamiltonian(n)
        load_both(ctx, H, random_terms(n, 1000 * n + seed, nterms=24), random_clauses(n, 1000 * n + seed))
        T = 5.0
        ctx.set_schedule(T, ((0.3, 0.2, -0.1, 0.05), (1.1, -0.4, 0.0, 0.2), (-0.7, 0.0, 0.5, 0.0)), 1)
        sched = O.Schedule(T, 1, ((0.3, 0.2, -0.1, 0.05), (1.1, -0.4, 0.0, 0.2), (-0.7, 0.0, 0.5, 0.0)))
        psi = random_state(n, seed)
        for t in (0.0, 1.7, T):
            got = ctx.hpsi(t, torch.from_numpy(psi).cuda()).cpu().numpy()
            ref = O.hpsi(H, sched.weights(t), psi, nthreads=8)
            tol = 1e-13 if prec == C128 else 3e-6
            assert rel_err(got, ref) < tol, (n, prec, t, rel_err(got, ref))
        ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_hpsi_basis_vectors_dense(prec):
    """H|z> for every basis state at n = 6 equals the dense Kronecker matrix's column z."""
    n = 6
    ctx = _ctx(n, prec)
    H = O.Hamiltonian(n)
    load_both(ctx, H, random_terms(n, 5, nterms=20), random_clauses(n, 5))
    ctx.set_schedule(1.0, ((1, 0, 0, 0), (1, 0, 0, 0), (1, 0, 0, 0)))
    M = O.dense_matrix(H, [1, 1, 1])
    tol = 1e-13 if prec == C128 else 3e-6
    for z in range(1 << n):
        e = np.zeros(1 << n, complex)
        e[z] = 1
        got = ctx.hpsi(0.0, torch.from_numpy(e).cuda()).cpu().numpy()
        assert np.max(np.abs(got - M[:, z])) < tol * max(1.0, np.abs(M[:, z]).max())
    ctx.close()


# ------------------------------------------------------------------ integrator
@pytest.mark.parametrize("prec", [C128, C64])
def test_ec3_n10_linear_T20_full_solve(prec):
    """The small Exact-Cover-3 workload: n = 10, linear path, T = 20, uniform start."""
    inst, ctx, H, sched = _setup_ec3(10, prec, 1, 20.0)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    st = ctx.propagate(-1)
    N = O.step_count(H, sched)
    assert st["n_steps"] == N and st["steps_done"] == N
    assert abs(st["t"] - 20.0) < 1e-12
    ref = O.propagate(H, sched, N, O.uniform_state(10))
    got = ctx.state()
    assert rel_err(got, ref.psi) < TOL_STATE[prec], rel_err(got, ref.psi)
    assert st["evaluations"] == ref.evaluations
    fid = ctx.fidelity(inst.solution)
    assert abs(fid - O.fidelity(ref.psi, inst.solution)) < (1e-12 if prec == C128 else tol_fidelity(prec, ref.psi))
    e = ctx.energy(1)
    assert abs(e - O.energy(H, ref.psi, 1)) < (1e-11 if prec == C128 else 1e-5)
    assert abs(st["norm2"] - O.norm2(ref.psi)) < (1e-12 if prec == C128 else 1e-6)
    if prec == C128:
        assert abs(st["max_err_est"] - ref.max_err_est) <= 1e-6 * ref.max_err_est + 1e-15
    else:
        # in FP32 the Milne estimate (19/270)||y - p|| has a rounding floor ~ 2^-24 ||y||
        assert ref.max_err_est * 0.5 <= st["max_err_est"] <= ref.max_err_est + 1e-8
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("s_kind", [0, 1])
def test_ec3_n12_nonlinear_path(prec, s_kind):
    """Nonlinear path (1-s) H_i + s H_f + s(1-s) H_c with random XX couplings, both s(t)."""
    inst, ctx, H, sched = _setup_ec3(12, prec, 5, 6.0, nonlinear=True, s_kind=s_kind)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    st = ctx.propagate(-1)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(12), nthreads=8)
    assert st["n_steps"] == O.step_count(H, sched)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[prec]
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_multilayout_random_terms_full_solve(prec):
    """n = 16 (more bits than one tile: two or more layouts plus products no layout holds),
    random X/Y/Z products and clauses, squared penalties, random initial state."""
    n = 16
    ctx = _ctx(n, prec)
    H = O.Hamiltonian(n)
    terms = [(g, x, z, 0.3 * c) for (g, x, z, c) in random_terms(n, 77, nterms=20)]
    load_both(ctx, H, terms, random_clauses(n, 77, m=5))
    sched = O.Schedule(1.0, 0, ((1, -1, 0, 0), (0, 1, 0, 0), (0, 1, -1, 0)))
    ctx.set_schedule(1.0, sched.poly, 0)
    N = 40
    ctx.set_integrator(N, 0.0)
    psi0 = random_state(n, 3)
    ctx.set_initial_state(psi0)
    ctx.propagate(-1)
    ref = O.propagate(H, sched, N, psi0, nthreads=8)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[prec]
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("nonlinear", [False, True])
def test_ec3_n20_first_steps(prec, nonlinear):
    """The n = 20 workload (linear and nonlinear paths, smoothstep s(t), T = 10): the first
    12 steps (3 RK4 + 9 PEC) on the full step grid."""
    inst, ctx, H, sched = _setup_ec3(20, prec, 2, 10.0, nonlinear=nonlinear, s_kind=1)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    st = ctx.propagate(12)
    assert st["steps_done"] == 12
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(20), max_steps=12, nthreads=16)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[prec] * 0.1
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_incremental_propagation_is_bitwise_identical(prec):
    inst, ctx, H, sched = _setup_ec3(10, prec, 1, 5.0)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    ctx.propagate(-1)
    a = ctx.state()
    ctx.set_initial_state("uniform")
    for k in (1, 2, 3, 7):
        ctx.propagate(k)
    ctx.propagate(-1)
    b = ctx.state()
    assert np.array_equal(a, b)
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_short_grids_rk4_only(prec):
    """N <= 3 steps are pure RK4; N = 4 has one PEC step."""
    inst, ctx, H, sched = _setup_ec3(8, prec, 3, 0.5)
    for N in (1, 2, 3, 4, 5):
        ctx.set_integrator(N, 0.0)
        ctx.set_initial_state("uniform")
        st = ctx.propagate(-1)
        ref = O.propagate(H, sched, N, O.uniform_state(8))
        assert st["evaluations"] == ref.evaluations
        assert rel_err(ctx.state(), ref.psi) < TOL_STATE[prec] * 0.1
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_basis_start_and_energy_groups(prec):
    inst, ctx, H, sched = _setup_ec3(9, prec, 4, 3.0, nonlinear=True)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state(5)
    ctx.propagate(-1)
    e0 = np.zeros(1 << 9, complex)
    e0[5] = 1
    ref = O.propagate(H, sched, O.step_count(H, sched), e0)
    psi = ctx.state()
    assert rel_err(psi, ref.psi) < TOL_STATE[prec]
    for g in range(3):
        assert abs(ctx.energy(g) - O.energy(H, ref.psi, g)) < (1e-11 if prec == C128 else 2e-5)
    assert abs(ctx.norm2() - O.norm2(ref.psi)) < (1e-12 if prec == C128 else 1e-6)
    ctx.close()


def test_reruns_are_deterministic():
    inst, ctx, H, sched = _setup_ec3(14, C64, 6, 2.0, nonlinear=True)
    ctx.set_integrator(0, 0.0)
    outs = []
    for _ in range(3):
        ctx.set_initial_state("uniform")
        st = ctx.propagate(-1)
        outs.append((ctx.state(), st["norm2"], st["max_err_est"]))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and o[1] == outs[0][1] and o[2] == outs[0][2]
    ctx.close()


def test_error_codes():
    from paper_1311_3938_gb300 import _native as N

    ctx = _ctx(6, C128)
    with pytest.raises(N.AqcError) as e:
        ctx.load_terms(0, [1 << 6], [0], [1.0])  # mask beyond n
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(N.AqcError) as e:
        ctx.load_clauses(1, [(0, 0, 1)])  # repeated bit
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(N.AqcError) as e:
        ctx.propagate(-1)  # no state, no schedule
    assert e.value.code == N.AQC_E_STATE
    with pytest.raises(N.AqcError) as e:
        ctx.set_schedule(-1.0, ((1, 0, 0, 0), (0, 0, 0, 0), (0, 0, 0, 0)))
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(N.AqcError) as e:
        ctx.fidelity(1 << 6)
    assert e.value.code == N.AQC_E_INVAL
    ctx.close()


@pytest.mark.parametrize("n", [22, 25])
def test_cluster_tiles_match_cta_tiles_and_oracle(n):
    """complex64 states of 22..28 qubits with 8-CTA cluster tiles (tile_bits = 16: two
    layouts), the default per-CTA tiles and the oracle agree."""
    H = O.Hamiltonian(n)
    a = _ctx(n, C64)
    a.set_tile_bits(16)
    terms = random_terms(n, 4000 + n, nterms=28)
    load_both(a, H, terms, random_clauses(n, 4000 + n, m=8))
    b = _ctx(n, C64)
    for g in range(3):
        sel = [t for t in terms if t[0] == g]
        if sel:
            b.load_terms(g, [t[1] for t in sel], [t[2] for t in sel], [t[3] for t in sel])
    for (g, bits, pen, scale) in random_clauses(n, 4000 + n, m=8):
        b.load_clauses(g, [bits], penalty=pen, scale=scale)
    poly = ((0.3, 0.2, -0.1, 0.05), (1.1, -0.4, 0.0, 0.2), (-0.7, 0.0, 0.5, 0.0))
    for c in (a, b):
        c.set_schedule(5.0, poly, 1)
    psi = random_state(n, 7)
    dpsi = torch.from_numpy(psi).cuda()
    ga = a.hpsi(1.3, dpsi).cpu().numpy()
    gb = b.hpsi(1.3, dpsi).cpu().numpy()
    used = dpsi.to(torch.complex64).cpu().numpy().astype(np.complex128)
    ref = O.hpsi(H, O.Schedule(5.0, 1, poly).weights(1.3), used, nthreads=16)
    assert rel_err(ga, ref) < 3e-6 and rel_err(gb, ref) < 3e-6
    assert rel_err(ga, gb) < 3e-6
    a.close()
    b.close()


def test_cluster_tiles_propagation_n22():
    """A propagation with cluster tiles (tile_bits = 16) matches the oracle."""
    inst, ctx, H, sched = _setup_ec3(22, C64, 9, 5.0, nonlinear=True, s_kind=1)
    ctx.set_tile_bits(16)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    ctx.propagate(10)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(22), max_steps=10, nthreads=16)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[C64] * 0.1
    ctx.close()


# ------------------------------------------------------------------ slab-ordered PEC steps
@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("slab_bits", [1, 3, 6])
def test_slab_order_random_terms_full_solve(prec, slab_bits):
    """Slab order (last partial layout and fused step in one launch over slabs of the index
    space) with small tiles: four layouts, so two full partial passes run first; random X/Y/Z
    products (some held by no layout) and clauses; full solve against the oracle."""
    n = 16
    ctx = _ctx(n, prec)
    ctx.set_tile_bits(8 if prec == C64 else 7)
    ctx.set_slab_bits(slab_bits)
    H = O.Hamiltonian(n)
    terms = [(g, x, z, 0.3 * c) for (g, x, z, c) in random_terms(n, 91 + slab_bits, nterms=24)]
    load_both(ctx, H, terms, random_clauses(n, 91 + slab_bits, m=6))
    sched = O.Schedule(1.0, 0, ((1, -1, 0, 0), (0, 1, 0, 0), (0, 1, -1, 0)))
    ctx.set_schedule(1.0, sched.poly, 0)
    N = 40
    ctx.set_integrator(N, 0.0)
    psi0 = random_state(n, 5)
    ctx.set_initial_state(psi0)
    st = ctx.propagate(-1)
    ref = O.propagate(H, sched, N, psi0, nthreads=8)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[prec]
    ref_norm2 = float(np.vdot(ref.psi, ref.psi).real)
    assert abs(st["norm2"] - ref_norm2) < (1e-12 if prec == C128 else 1e-5)
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_slab_order_matches_layer_order(prec):
    """n = 23 EC3, nonlinear path: slab order (automatic for complex64 at this size, forced
    for complex128) and layer order give the same state up to summation-order rounding, and
    both match the oracle over the first 12 steps."""
    n = 23
    states = []
    for slab in (-1 if prec == C64 else 3, 0):
        inst, ctx, H, sched = _setup_ec3(n, prec, 6, 10.0, nonlinear=True, s_kind=1)
        ctx.set_slab_bits(slab)
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state("uniform")
        ctx.propagate(12)
        states.append(ctx.state())
        ctx.close()
    assert rel_err(states[0], states[1]) < (1e-13 if prec == C128 else 1e-6)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(n), max_steps=12, nthreads=16)
    assert rel_err(states[0], ref.psi) < TOL_STATE[prec] * 0.1


def test_slab_bits_argument_checks():
    from paper_1311_3938_gb300 import _native as N

    ctx = _ctx(10, C64)
    for bad in (-2, 12):
        with pytest.raises(N.AqcError) as e:
            ctx.set_slab_bits(bad)
        assert e.value.code == N.AQC_E_INVAL
    ctx.set_slab_bits(0)
    ctx.set_slab_bits(-1)
    ctx.close()


def test_error_codes_of_the_path_extensions():
    """Argument checks of the Dicke start, clause-by-clause sequences, batches, Lanczos."""
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300.engine import Batch

    ctx = _ctx(8, C128)
    with pytest.raises(N.AqcError) as e:
        ctx.set_initial_state(("dicke", 9))  # weight > n
    assert e.value.code == N.AQC_E_INVAL
    ctx.load_clauses(2, [(0, 1, 2), (3, 4, 5)], stepwise=True)
    with pytest.raises(N.AqcError) as e:
        ctx.load_clauses(2, [(1, 2, 3)], stepwise=True)  # one sequence per context
    assert e.value.code == N.AQC_E_INVAL
    ctx.set_schedule(1.0, ((1, -1, 0, 0), (0, 1, 0, 0), (1, 0, 0, 0)))
    ctx.set_initial_state("uniform")
    b = Batch(C128, max_members=2, max_items=64)
    with pytest.raises(N.AqcError) as e:
        b.add(ctx)  # stepwise sequences are not batched
    assert e.value.code == N.AQC_E_UNSUPPORTED
    b.close()
    start = torch.ones(1 << 8, dtype=torch.complex128, device="cuda")
    for bad in ((0, 1), (5, 6)):  # max_iter < 1; n_eig > max_iter
        with pytest.raises(N.AqcError) as e:
            ctx.lanczos(0.5, start, max_iter=bad[0], n_eig=bad[1])
    ctx.close()
