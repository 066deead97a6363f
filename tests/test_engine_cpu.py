"""Host-side bookkeeping of the Python binding's staged transfers (no GPU): the library calls
are replaced by recorders, so only the binding's own logic runs.  A re-attach keeps the previous
staging vectors alive until the library has released them; host tensors of enqueued copies stay
referenced until transfer_wait(); argument checks come before any library call."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def ctx(monkeypatch):
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import engine as E

    calls = []
    real_empty = torch.empty

    class _NoDevice:
        def __init__(self, *_):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *_):
            return False

    monkeypatch.setattr(torch, "empty", lambda n, dtype=None, device=None: real_empty(n, dtype=dtype))
    monkeypatch.setattr(torch.cuda, "device", _NoDevice)
    c = object.__new__(E.Context)  # no CUDA context: only the binding's bookkeeping
    c.precision, c.N, c.dev, c.handle = N.AQC_C64, 16, torch.device("cpu"), None
    c._stage, c._in_flight = None, []
    monkeypatch.setattr(N, "aqc_transfer_attach", lambda h, a, b: calls.append(("attach", a, b, c._stage)))
    monkeypatch.setattr(N, "aqc_stage_initial_state", lambda h, p: calls.append(("stage", p)))
    monkeypatch.setattr(N, "aqc_fetch_state", lambda h, p: calls.append(("fetch", p)))
    monkeypatch.setattr(N, "aqc_transfer_wait", lambda h: calls.append(("wait",)))
    yield c, calls
    c.handle = None  # nothing to destroy


def test_reattach_keeps_previous_vectors_until_released(ctx):
    c, calls = ctx
    c.attach_transfers()
    first = c._stage
    assert calls[0][3] is None and calls[0][1] == first[0].data_ptr() and calls[0][2] == first[1].data_ptr()
    c.attach_transfers()
    assert calls[1][3] is first  # still referenced while the library switched vectors
    assert c._stage is not first


def test_host_tensors_of_enqueued_copies_stay_referenced(ctx):
    c, calls = ctx
    c.attach_transfers()
    h_in = torch.zeros(16, dtype=torch.complex64)
    h_out = torch.zeros(16, dtype=torch.complex64)
    c.stage_initial_state(h_in)
    c.fetch_state(h_out)
    assert [x[0] for x in calls[1:]] == ["stage", "fetch"]
    assert calls[1][1] == h_in.data_ptr() and calls[2][1] == h_out.data_ptr()
    assert c._in_flight == [h_in, h_out]
    c.transfer_wait()
    assert c._in_flight == [] and calls[-1] == ("wait",)


def test_argument_checks_precede_library_calls(ctx):
    c, calls = ctx
    c.attach_transfers()
    n0 = len(calls)
    for bad in (torch.zeros(16, dtype=torch.complex128), torch.zeros(15, dtype=torch.complex64),
                torch.zeros(32, dtype=torch.complex64)[::2]):
        with pytest.raises(ValueError):
            c.stage_initial_state(bad)
        with pytest.raises(ValueError):
            c.fetch_state(bad)
    assert len(calls) == n0 and c._in_flight == []
