"""Staged host transfers (aqc_transfer_attach / aqc_stage_initial_state / aqc_fetch_state):
the copy-engine path gives the same psi(0) and the same final psi as the synchronous host
copies, bit for bit, also when the next input is staged while the current instance
integrates and when the library reorders the index bits; the result matches the oracle."""
import numpy as np
import pytest

from instances import generate_ec3, random_state
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


def _tdt(prec):
    return torch.complex128 if prec == C128 else torch.complex64


def _pinned(v, prec):
    return torch.from_numpy(np.ascontiguousarray(v)).to(_tdt(prec)).pin_memory()


def _ec3_ctx(n, prec, T, N):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    inst = generate_ec3(n, 2)
    ctx = Context(n, prec)
    HB.load_ec3(ctx, inst)
    ctx.set_schedule(T, HB.linear_schedule())
    ctx.set_integrator(N, 0.0)
    return inst, ctx


def _xy_ctx(n, prec, inst):
    """XY driver with a catalyst: pair products span layouts, so the library reorders bits."""
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    ctx = Context(n, prec)
    sched, k = HB.load_xy(ctx, inst, driver="xy", catalyst_alpha=8.0)
    ctx.set_schedule(10.0, sched)
    ctx.set_integrator(0, 0.0)
    return ctx, k


@pytest.mark.parametrize("prec", [C128, C64])
def test_staged_solve_matches_oracle(prec):
    n, T, N = 10, 2.0, 12
    inst, ctx = _ec3_ctx(n, prec, T, N)
    ctx.attach_transfers()
    v = random_state(n, 21)
    host_in = _pinned(v, prec)
    host_out = torch.empty_like(host_in).pin_memory()
    ctx.stage_initial_state(host_in)
    ctx.set_initial_state("staged")
    ctx.propagate(-1)
    ctx.fetch_state(host_out)
    ctx.transfer_wait()
    ref = O.propagate(O.ec3_hamiltonian(inst), O.linear_path(T), N, v.astype(np.complex128))
    assert rel_err(host_out.numpy(), ref.psi) < TOL_STATE[prec]
    assert np.array_equal(host_out.numpy(), ctx.state())
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_pipelined_instances_match_synchronous_copies(prec):
    """Stage instance k+1 while instance k integrates; fetch instance k while k+1 starts."""
    n = 16  # two tile layouts
    inst, ctx = _ec3_ctx(n, prec, 3.0, 40)
    ins = [_pinned(random_state(n, 30 + k), prec) for k in range(3)]
    outs = [torch.empty_like(ins[0]).pin_memory() for _ in range(3)]
    want = []
    for k in range(3):
        ctx.set_initial_state(ins[k])
        ctx.propagate(9)
        want.append(ctx.state())
    ctx.attach_transfers()
    ctx.stage_initial_state(ins[0])
    for k in range(3):
        ctx.set_initial_state("staged")
        if k + 1 < 3:
            ctx.stage_initial_state(ins[k + 1])
        ctx.propagate(9, stats=False)
        ctx.fetch_state(outs[k])
    ctx.transfer_wait()
    for k in range(3):
        assert np.array_equal(outs[k].numpy(), want[k]), k
    ctx.close()


@pytest.mark.parametrize("prec", [C128, C64])
def test_staged_copies_with_reordered_bits(prec):
    n = 21
    inst = generate_ec3(n, 4)
    a, k = _xy_ctx(n, prec, inst)
    v = random_state(n, 8)
    a.set_initial_state(_pinned(v, prec))
    a.propagate(6)
    want = a.state()
    a.attach_transfers()
    host_in = _pinned(v, prec)
    host_out = torch.empty_like(host_in).pin_memory()
    a.stage_initial_state(host_in)
    a.set_initial_state("staged")
    a.fetch_state(host_out)  # psi(0) back through the output staging vector
    a.transfer_wait()
    assert np.array_equal(host_out.numpy(), host_in.numpy())
    a.propagate(6)
    a.fetch_state(host_out)
    a.transfer_wait()
    assert np.array_equal(host_out.numpy(), want)
    a.close()


def test_transfer_argument_and_order_checks():
    from paper_1311_3938_gb300 import _native as N

    n = 12
    _, ctx = _ec3_ctx(n, C64, 1.0, 8)
    h = torch.zeros(1 << n, dtype=torch.complex64).pin_memory()
    with pytest.raises(N.AqcError) as e:
        ctx.stage_initial_state(h)  # nothing attached
    assert e.value.code == N.AQC_E_STATE
    with pytest.raises(N.AqcError) as e:
        ctx.fetch_state(h)
    assert e.value.code == N.AQC_E_STATE
    ctx.attach_transfers()
    with pytest.raises(N.AqcError) as e:
        ctx.set_initial_state("staged")  # nothing staged
    assert e.value.code == N.AQC_E_STATE
    v = torch.empty(3 << n, dtype=torch.complex64, device="cuda")
    with pytest.raises(N.AqcError) as e:  # overlapping staging vectors
        N.aqc_transfer_attach(ctx.handle, v.data_ptr(), v.data_ptr() + 1024)
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(N.AqcError) as e:  # misaligned
        N.aqc_transfer_attach(ctx.handle, v.data_ptr() + 8, v.data_ptr() + (16 << n))
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(N.AqcError) as e:  # inside the workspace
        N.aqc_transfer_attach(ctx.handle, ctx._ws_ptr, v.data_ptr())
    assert e.value.code == N.AQC_E_INVAL
    with pytest.raises(ValueError):
        ctx.stage_initial_state(torch.zeros(1 << n, dtype=torch.complex128))
    ctx.stage_initial_state(h)
    ctx.set_initial_state("staged")
    assert ctx.norm2() == 0.0
    ctx.transfer_wait()
    ctx.close()
