"""Turn of layouts in the PEC step (aqc_set_layout_turns): the fused step alternates between
layouts 0 and 1 and leaves its layout's products of the new predictor for the next step.  The
results equal the plain pass order up to the order in which the layouts' sums are added, and
the oracle within the precision's tolerance; graph replays of turned steps equal single steps
bit for bit; work that overwrites the partial sum between calls (an energy evaluation, a matvec)
makes the next step start a new turn."""
import numpy as np
import pytest

from instances import generate_ec3, xx_pairs
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


def _ctx(n, seed, prec, T, turns, k_steps=0, nonlinear=True, s_kind=1, extra=False):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    ctx = Context(n, prec, extra_vector=extra)
    ctx.set_layout_turns(turns)
    ctx.set_graph_steps(k_steps)
    HB.load_ec3(ctx, inst, pairs=xx_pairs(n, seed) if nonlinear else None)
    ctx.set_schedule(T, HB.nonlinear_schedule() if nonlinear else HB.linear_schedule(), s_kind)
    ctx.set_integrator(0, 0.0)
    return ctx, inst


@pytest.mark.parametrize("prec", [C64, C128])
@pytest.mark.parametrize("n,seed,T,nonlinear", [(14, 5, 4.0, False), (20, 2, 0.4, True), (23, 7, 0.05, True)])
def test_turns_match_the_plain_order_and_the_oracle(prec, n, seed, T, nonlinear):
    """Two layouts (n = 14, linear path: no product spans the layouts), three (n = 20: the
    partial pass on the TMA-fed kernel, XX couplings across layouts in it), and n = 23; the
    full solves up to n = 20 and the first 40 steps at n = 23 against the oracle."""
    out = []
    for turns in (0, 1):
        ctx, inst = _ctx(n, seed, prec, T, turns, nonlinear=nonlinear)
        ctx.set_initial_state("uniform")
        st = ctx.propagate(-1 if n <= 20 else 40)
        out.append((ctx.state(), st))
        ctx.close()
    (a, sa), (b, sb) = out
    assert sa["steps_done"] == sb["steps_done"] and sa["evaluations"] == sb["evaluations"]
    assert rel_err(b, a) < (1e-13 if prec == C128 else 2e-6)
    H = O.ec3_hamiltonian(generate_ec3(n, seed), pairs=xx_pairs(n, seed) if nonlinear else None)
    sched = (O.nonlinear_path if nonlinear else O.linear_path)(T, 1)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(n),
                      max_steps=-1 if n <= 20 else 40, nthreads=16)
    assert rel_err(b, ref.psi) < TOL_STATE[prec]


@pytest.mark.parametrize("prec", [C64, C128])
def test_turned_graph_replays_equal_single_steps(prec):
    states = []
    for k in (0, 8):
        ctx, _ = _ctx(20, 3, prec, 0.3, 1, k_steps=k)
        ctx.set_initial_state("uniform")
        ctx.propagate(-1)
        states.append((ctx.state(), ctx.graph_replays()))
        ctx.close()
    assert states[0][1] == 0 and states[1][1] > 0
    assert np.array_equal(states[0][0], states[1][0])


def test_turns_with_the_compensated_corrector_and_interruptions():
    """y compensation with turns; an energy evaluation and a matvec between propagate calls
    overwrite the partial sum, so the next step starts a new turn: the result stays within
    rounding of an uninterrupted run."""
    from paper_1311_3938_gb300 import _native as N

    ref = None
    for interrupt in (False, True):
        ctx, inst = _ctx(20, 4, C64, 0.5, 1, extra=True)
        ctx.set_y_compensation(True)
        ctx.set_initial_state("uniform")
        for _ in range(6):
            ctx.propagate(37)
            if interrupt:
                ctx.energy(N.AQC_GRP_B)
                ctx.hpsi(0.1, torch.ones(1 << 20, dtype=torch.complex64, device="cuda"))
        ctx.propagate(-1)
        got = ctx.state()
        ctx.close()
        if ref is None:
            ref = got
        else:
            assert rel_err(got, ref) < 2e-6


def test_bad_mode():
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300.engine import Context

    with Context(6, C64) as c:
        for bad in (-2, 2):
            with pytest.raises(N.AqcError) as e:
                c.set_layout_turns(bad)
            assert e.value.code == N.AQC_E_INVAL
