"""Step-size control on the GPU (aqc_set_integrator with adaptive = 1) against the oracle's
or_propagate_adaptive: the same segments of constant step (start, step size, accepted steps, how
each ended), the same rejections and evaluations, and the same final state within the precision's
tolerance.  The accept/reject decisions compare FP64 reductions with tol ||y||; each case first
checks that no decision of the oracle's run lies within rounding of the threshold.  Also: the
energy of H(t) and of group subsets at a given time (aqc_energy with a group mask and t).
"""
import math

import numpy as np
import pytest

from instances import generate_ec3, random_state, xx_pairs
from oracle import oracle as O

from _helpers import C64, C128, TOL_STATE, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def _both(n, seed, T, s_kind, prec, kappa, tol, grow_after, tile_bits=0):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    pairs = xx_pairs(n, seed)
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = O.nonlinear_path(T, s_kind)
    N0 = O.step_count(H, sched, kappa=kappa)
    ref = O.propagate_adaptive(H, sched, T / N0, tol, O.uniform_state(n), grow_after=grow_after, nthreads=8)
    ctx = Context(n, prec, step_control=True)
    if tile_bits:
        ctx.set_tile_bits(tile_bits)
    HB.load_ec3(ctx, inst, pairs=pairs)
    ctx.set_schedule(T, HB.nonlinear_schedule(), s_kind)
    ctx.set_integrator(0, kappa, adaptive=True, tol=tol)
    ctx.set_step_growth(grow_after)
    ctx.set_initial_state("uniform")
    st = ctx.propagate(-1)
    return ctx, st, ref, N0


def _same_segments(got, want):
    assert len(got) == len(want), (got, want)
    for g, w in zip(got, want):
        assert g[2:] == w[2:], (g, w)
        assert g[0] == pytest.approx(w[0], rel=1e-13, abs=1e-15)
        assert g[1] == pytest.approx(w[1], rel=1e-13)


@pytest.mark.parametrize(
    "n,seed,T,kappa,tol,grow,tile_bits",
    [
        (8, 1, 5.0, 0.4, 1e-9, 8, 0),    # unstable first step: rejected down to a stable one
        (10, 3, 3.0, 0.01, 1e-9, 4, 0),  # 10x finer first step than the rule: the step grows
        (14, 6, 2.0, 0.3, 1e-9, 8, 0),   # two tile layouts (partial pass + fused step)
        (12, 4, 2.0, 0.3, 1e-9, 8, 6),   # small tiles: four layouts
    ],
)
def test_complex128_segments_equal_the_oracle(n, seed, T, kappa, tol, grow, tile_bits):
    ctx, st, ref, N0 = _both(n, seed, T, 1, C128, kappa, tol, grow, tile_bits)
    margin = float(np.min(np.abs(ref.ratios - 1.0)))
    assert margin > 1e-8, f"a decision of this case is within {margin:.1e} of the threshold"
    _same_segments(ctx.segments(), ref.segments)
    assert st["rejects"] == ref.rejects and st["steps_done"] == ref.steps_done
    assert st["evaluations"] == ref.evaluations
    assert st["segments"] == len(ref.segments)
    assert st["t"] == pytest.approx(T, rel=1e-12)
    assert rel_err(ctx.state(), ref.psi) < TOL_STATE[C128]
    assert st["max_err_est"] == pytest.approx(ref.max_err_est, rel=1e-8)
    if kappa > 0.1:
        assert ref.rejects >= 1
    if grow < 8:
        assert any(s[3] == O.SEG_GREW for s in ref.segments)
    ctx.close()


def test_complex64_step_control_accuracy():
    """complex64 (FP32 state, FP64 reductions) from a first step ten times the step rule's.
    Its first PEC step is rejected clearly (estimate 7% above the threshold in the oracle, far
    above FP32 rounding), so that segment equals the oracle's.  Later rejections are set off by
    the PEC scheme's parasitic mode, which grows from rounding once steps pass the scheme's
    stability edge on the imaginary axis: it starts from the FP32 floor here and from the FP64
    floor in the oracle, so those decisions may fall on other steps.  What both runs promise is
    accuracy: the state is within the sum of the accepted local tolerances of a converged
    reference (DOP853 on the dense H(t))."""
    from scipy.integrate import solve_ivp

    n, seed, T, tol = 9, 2, 3.0, 3e-6
    ctx, st, ref, N0 = _both(n, seed, T, 1, C64, 1.0, tol, 0)
    assert ref.segments[0][2:] == (0, O.SEG_REJECTED) and ref.ratios[0] > 1.05
    _same_segments(ctx.segments()[:1], ref.segments[:1])
    segs = ctx.segments()
    assert st["rejects"] >= 1 and segs[-1][3] == O.SEG_AT_T
    assert segs[-1][0] + segs[-1][1] * segs[-1][2] == pytest.approx(T, rel=1e-12)
    assert st["max_err_est"] <= tol * math.sqrt(st["norm2"]) * (1 + 1e-6)
    inst = generate_ec3(n, seed)
    H = O.ec3_hamiltonian(inst, pairs=xx_pairs(n, seed))
    sched = O.nonlinear_path(T, 1)
    Mg = [O.dense_matrix(H, [1.0 if g == k else 0.0 for k in range(3)] + [0.0]) for g in range(3)]

    def rhs(t, y):
        w = sched.weights(t)
        return -1j * ((w[0] * Mg[0] + w[1] * Mg[1] + w[2] * Mg[2]) @ y)

    exact = solve_ivp(rhs, (0.0, T), O.uniform_state(n).astype(complex), method="DOP853", rtol=1e-12,
                      atol=1e-13).y[:, -1]
    err = float(np.linalg.norm(ctx.state().astype(np.complex128) - exact))
    assert err < tol * st["steps_done"] + TOL_STATE[C64], (err, st["steps_done"])
    assert float(np.linalg.norm(ref.psi - exact)) < tol * ref.steps_done
    ctx.close()


def test_fixed_grid_is_one_segment_and_unchanged():
    """adaptive = 0: one segment of N steps; the state equals a context without the extra
    workspace vector, bit for bit."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(11, 2)
    states = []
    for sc in (False, True):
        ctx = Context(11, C64, step_control=sc)
        HB.load_ec3(ctx, inst)
        ctx.set_schedule(4.0, HB.linear_schedule())
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state("uniform")
        st = ctx.propagate(-1)
        N, h = ctx.grid()
        assert ctx.segments() == [(0.0, h, N, 1)]
        assert st["rejects"] == 0 and st["segments"] == 1
        states.append(ctx.state())
        ctx.close()
    assert np.array_equal(states[0], states[1])


def test_adaptive_needs_the_step_control_workspace_and_is_not_batched():
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Batch, Context

    ctx = Context(8, C128)
    with pytest.raises(N.AqcError) as e:
        ctx.set_integrator(0, 0.0, adaptive=True, tol=1e-8)
    assert e.value.code == N.AQC_E_NOMEM
    ctx.close()
    ctx = Context(8, C128, step_control=True)
    for bad in (0.0, -1.0, math.inf):
        with pytest.raises(N.AqcError) as e:
            ctx.set_integrator(0, 0.0, adaptive=True, tol=bad)
        assert e.value.code == N.AQC_E_INVAL
    inst = generate_ec3(8, 1)
    HB.load_ec3(ctx, inst)
    ctx.set_schedule(1.0, HB.linear_schedule())
    ctx.set_integrator(0, 0.0, adaptive=True, tol=1e-8)
    ctx.set_initial_state("uniform")
    b = Batch(C128, max_members=2, max_items=64)
    with pytest.raises(N.AqcError) as e:
        b.add(ctx)
    assert e.value.code == N.AQC_E_UNSUPPORTED
    b.close()
    ctx.close()


def test_minimum_step_is_reported():
    """A tolerance below the rounding floor halves h until it falls below 2^-30 T/N."""
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    ctx = Context(6, C128, step_control=True)
    HB.load_ec3(ctx, generate_ec3(6, 1))
    ctx.set_schedule(1.0, HB.linear_schedule())
    ctx.set_integrator(0, 0.0, adaptive=True, tol=1e-30)
    ctx.set_initial_state("uniform")
    with pytest.raises(N.AqcError) as e:
        ctx.propagate(-1)
    assert e.value.code == N.AQC_E_NUMERIC
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_energy_of_group_subsets_at_a_time(prec):
    """<psi| sum_{g in mask} w_g(s(t)) H_g |psi> for every mask and a few t, and unit weights,
    against the oracle's matvec on the same state."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n = 9
    inst = generate_ec3(n, 3)
    pairs = xx_pairs(n, 3)
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = O.nonlinear_path(2.0, 1)
    ctx = Context(n, prec)
    HB.load_ec3(ctx, inst, pairs=pairs)
    ctx.set_schedule(2.0, HB.nonlinear_schedule(), 1)
    psi = random_state(n, 8)
    ctx.set_initial_state(psi)
    used = ctx.state().astype(np.complex128)
    tol = 1e-12 if prec == C128 else 2e-5
    for t in (0.0, 0.7, 2.0):
        w = sched.weights(t)
        for mask in range(1, 8):
            wm = [w[g] if (mask >> g) & 1 else 0.0 for g in range(3)] + [w[3]]
            want = float(np.vdot(used, O.hpsi(H, wm, used)).real)
            groups = [g for g in range(3) if (mask >> g) & 1]
            got = ctx.energy_at(t, groups)
            assert abs(got - want) < tol * max(1.0, abs(want)), (t, mask, got, want)
    for g in range(3):
        assert abs(ctx.energy(g) - O.energy(H, used, g)) < tol * 10
    ctx.close()
