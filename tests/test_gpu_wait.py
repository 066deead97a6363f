"""The give-up path of the library's bounded device waits, run on purpose without any fault
(aqc_wait_selftest): a wait on a flag that nothing sets ends after its poll limit, the host
reads AQC_E_TIMEOUT, and the context stays usable for a solve that matches the oracle."""
import pytest

from instances import generate_ec3
from oracle import oracle as O

from _helpers import C64, TOL_STATE, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


def test_wait_gives_up_and_the_context_stays_usable():
    import time

    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(10, 1)
    ctx = Context(10, C64)
    HB.load_ec3(ctx, inst)
    ctx.set_schedule(2.0, HB.linear_schedule())
    ctx.set_integrator(0, 0.0)
    ctx.set_initial_state("uniform")
    for polls in (1, 2000):
        t0 = time.perf_counter()
        with pytest.raises(N.AqcError) as e:
            N.aqc_wait_selftest(ctx.handle, polls)
        assert e.value.code == N.AQC_E_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
    for bad in (0, -5, 10 ** 8):
        with pytest.raises(N.AqcError) as e:
            N.aqc_wait_selftest(ctx.handle, bad)
        assert e.value.code == N.AQC_E_INVAL
    st = ctx.propagate(-1)  # the fault slot was cleared: stats report no timeout
    psi = ctx.state()
    ctx.close()
    H = O.ec3_hamiltonian(inst)
    sched = O.linear_path(2.0)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(10))
    assert st["steps_done"] == ref.steps_done
    assert rel_err(psi, ref.psi) < TOL_STATE[C64]
