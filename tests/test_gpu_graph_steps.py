"""CUDA-graph replay of PEC steps for lone contexts (aqc_set_graph_steps): the replayed steps
read their schedule weights from the workspace, written by the host before each replay with the
expression the step-by-step path uses, so a solve with replays equals one without, bit for bit.
Also: recapture when the step size or the tables change, runs split into calls that end
inside a replay's span, and the oracle on the small-state workload (n = 10, T = 20)."""
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


def _ec3_ctx(n, seed, prec, T, nonlinear=False, s_kind=0, k_steps=-1):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, seed)
    ctx = Context(n, prec)
    ctx.set_graph_steps(k_steps)
    HB.load_ec3(ctx, inst, pairs=xx_pairs(n, seed) if nonlinear else None)
    ctx.set_schedule(T, HB.nonlinear_schedule() if nonlinear else HB.linear_schedule(), s_kind)
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    return ctx, inst


@pytest.mark.parametrize("prec", [C128, C64])
@pytest.mark.parametrize("n,seed,T,nonlinear,s_kind,k_steps", [
    (10, 1, 20.0, False, 0, -1),   # the small-state workload, automatic K = 16
    (14, 5, 6.0, True, 1, 8),      # nonlinear path, smoothstep, two layouts
    (20, 2, 0.5, True, 0, 4),      # three partial passes per step (TMA-fed) in the graph
])
def test_replay_equals_step_by_step(prec, n, seed, T, nonlinear, s_kind, k_steps):
    states, replays, stats = [], [], []
    for k in (0, k_steps):
        ctx, _ = _ec3_ctx(n, seed, prec, T, nonlinear, s_kind, k)
        st = ctx.propagate(-1)
        states.append(ctx.state())
        replays.append(ctx.graph_replays())
        stats.append(st)
        ctx.close()
    assert replays[0] == 0 and replays[1] > 0
    assert stats[0]["steps_done"] == stats[1]["steps_done"] == stats[0]["n_steps"]
    assert stats[0]["evaluations"] == stats[1]["evaluations"]
    assert np.array_equal(states[0], states[1])
    assert stats[0]["norm2"] == stats[1]["norm2"]
    assert stats[0]["max_err_est"] == stats[1]["max_err_est"]


def test_calls_that_split_a_replay_span_and_recapture():
    """propagate(max_steps) in uneven pieces (steps left over run one by one, the next call
    replays from another ring phase: a new capture), a new step size (recapture) and new terms
    (tables rebuilt: recapture), each against a context without replays."""
    from paper_1311_3938_gb300 import hamiltonians as HB

    def run(k):
        ctx, inst = _ec3_ctx(12, 3, C128, 5.0, k_steps=k)
        out = []
        for m in (7, 37, 5, 61):
            ctx.propagate(m)
            out.append(ctx.state())
        ctx.set_integrator(1234, 0.0)  # new h
        ctx.set_initial_state("uniform")
        ctx.propagate(-1)
        out.append(ctx.state())
        ctx.load_terms(2, *HB.xx_terms(xx_pairs(12, 3)))  # tables change
        ctx.set_schedule(5.0, HB.nonlinear_schedule())
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state("uniform")
        ctx.propagate(-1)
        out.append(ctx.state())
        r = ctx.graph_replays()
        ctx.close()
        return out, r

    a, ra = run(0)
    b, rb = run(12)
    assert ra == 0 and rb > 0
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_xy_driver_in_graph():
    """Y products (general-product loop) inside replayed steps: equal to step by step."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(12, 11)
    out = []
    for k in (0, 16):
        ctx = Context(12, C64)
        ctx.set_graph_steps(k)
        sched, w = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=8.0)
        ctx.set_schedule(3.0, sched)
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state(("dicke", w))
        ctx.propagate(-1)
        out.append((ctx.state(), ctx.graph_replays()))
        ctx.close()
    assert out[0][1] == 0 and out[1][1] > 0
    assert np.array_equal(out[0][0], out[1][0])


def test_small_state_workload_against_the_oracle():
    """n = 10, complex128, linear path, T = 20 (automatic replay): full state against the oracle."""
    ctx, inst = _ec3_ctx(10, 1, C128, 20.0)
    st = ctx.propagate(-1)
    psi = ctx.state()
    assert ctx.graph_replays() > 0
    ctx.close()
    H = O.ec3_hamiltonian(inst)
    sched = O.linear_path(20.0)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(10))
    assert st["steps_done"] == ref.steps_done
    assert rel_err(psi, ref.psi) < TOL_STATE[C128]


def test_not_used_under_step_control_and_bad_arguments():
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    ctx = Context(9, C128, step_control=True)
    for bad in (3, 5, 68, -2):
        with pytest.raises(N.AqcError) as e:
            ctx.set_graph_steps(bad)
        assert e.value.code == N.AQC_E_INVAL
    ctx.set_graph_steps(8)
    HB.load_ec3(ctx, generate_ec3(9, 2))
    ctx.set_schedule(2.0, HB.linear_schedule())
    ctx.set_integrator(0, 0.0, adaptive=True, tol=1e-8)
    ctx.set_initial_state("uniform")
    ctx.propagate(-1)
    assert ctx.graph_replays() == 0
    ctx.close()


@pytest.mark.parametrize("prec", [C64, C128])
def test_grid_limit_keeps_the_state(prec):
    """aqc_set_grid_limit: every layout pass (the TMA-fed partial passes included) on a few CTAs;
    the state is the same bit for bit, with and without graph replays (recaptured)."""
    out = []
    for limit in (0, 7, 1):
        ctx, _ = _ec3_ctx(20, 4, prec, 0.3, nonlinear=True)
        ctx.set_grid_limit(limit)
        ctx.propagate(-1)
        out.append(ctx.state())
        ctx.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_compensated_corrector_replays_and_arguments():
    """y compensation: graph replays give the same bits as single steps; the state differs from
    the plain corrector's by rounding only; complex128, a missing extra vector, step-size
    control and batches are refused."""
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Batch, Context

    inst = generate_ec3(14, 5)
    out = {}
    for comp, k in ((False, 0), (True, 0), (True, 8)):
        ctx = Context(14, C64, extra_vector=True)
        ctx.set_graph_steps(k)
        HB.load_ec3(ctx, inst, pairs=xx_pairs(14, 5))
        ctx.set_schedule(4.0, HB.nonlinear_schedule(), 1)
        ctx.set_integrator(0, 0.0)
        ctx.set_y_compensation(comp)
        ctx.set_initial_state("uniform")
        ctx.propagate(-1)
        out[(comp, k)] = (ctx.state(), ctx.graph_replays())
        ctx.close()
    assert np.array_equal(out[(True, 0)][0], out[(True, 8)][0]) and out[(True, 8)][1] > 0
    assert 0 < rel_err(out[(True, 0)][0], out[(False, 0)][0]) < 1e-5
    with Context(8, C128, extra_vector=True) as c:
        with pytest.raises(N.AqcError) as e:
            c.set_y_compensation(True)
        assert e.value.code == N.AQC_E_UNSUPPORTED
    with Context(8, C64) as c:
        with pytest.raises(N.AqcError) as e:
            c.set_y_compensation(True)
        assert e.value.code == N.AQC_E_NOMEM
    c = Context(8, C64, extra_vector=True)
    c.set_y_compensation(True)
    with pytest.raises(N.AqcError) as e:
        c.set_integrator(0, 0.0, adaptive=True, tol=1e-6)
    assert e.value.code == N.AQC_E_UNSUPPORTED
    HB.load_ec3(c, generate_ec3(8, 1))
    c.set_schedule(1.0, HB.linear_schedule())
    c.set_integrator(0, 0.0)
    c.set_initial_state("uniform")
    b = Batch(C64, max_members=2, max_items=64)
    with pytest.raises(N.AqcError) as e:
        b.add(c)
    assert e.value.code == N.AQC_E_UNSUPPORTED
    b.close()
    c.close()
