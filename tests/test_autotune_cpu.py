"""Host-side logic of the batch autotuner (no GPU): the cache key, the choice of the fastest
shape, and the on-disk cache (hit, bypass, unreadable file).  The timing of a shape is replaced
by a stand-in, since it needs a GPU."""
import json
import os
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def tuner(monkeypatch, tmp_path):
    from paper_1311_3938_gb300 import autotune as A

    monkeypatch.setenv("AQC_CACHE_DIR", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "FakeGPU")
    calls = []
    rates = {(0, 256, 16): 5.0, (0, 256, 64): 9.0, (0, 128, 16): 4.0, (11, 256, 16): 7.0, (12, 256, 16): 8.5}

    def fake_measure(jobs, shape, device=0, rounds=4):
        calls.append(tuple(shape))
        return rates[tuple(shape)]

    monkeypatch.setattr(A, "measure_shape", fake_measure)
    return A, calls, tmp_path


def _jobs(*ns, precision=1):
    return [SimpleNamespace(n=n, precision=precision) for n in ns]


def test_key_is_device_precision_and_size_histogram(tuner):
    A, _, _ = tuner
    assert A._key(_jobs(14, 12, 12), 1) == "FakeGPU|p1|12:2,14:1"
    assert A._key(_jobs(12, 14, 12), 1) == A._key(_jobs(14, 12, 12), 1)  # order-free
    assert A._key(_jobs(12), 0) != A._key(_jobs(12), 1)


def test_fastest_shape_wins_and_is_cached(tuner):
    A, calls, tmp = tuner
    jobs = _jobs(12, 16, 16)
    shape, entry = A.autotune(jobs)
    assert shape == (0, 256, 64)
    assert sorted(calls) == sorted(A.DEFAULT_SHAPES)
    assert [r["amp_steps_per_s"] for r in entry["results"]] == [5.0, 9.0, 4.0, 7.0, 8.5]
    cache = json.load(open(os.path.join(str(tmp), "autotune.json")))
    assert cache[A._key(jobs, 1)]["shape"] == [0, 256, 64]
    calls.clear()
    again, _ = A.autotune(jobs)  # cache hit: nothing is timed
    assert again == shape and calls == []
    A.autotune(jobs, use_cache=False)  # bypass: every shape is timed again
    assert len(calls) == len(A.DEFAULT_SHAPES)


def test_explicit_shapes_and_unreadable_cache(tuner):
    A, calls, tmp = tuner
    with open(os.path.join(str(tmp), "autotune.json"), "w") as f:
        f.write("{not json")
    shape, _ = A.autotune(_jobs(18), shapes=[(11, 256, 16), (0, 128, 16)])
    assert shape == (11, 256, 16) and calls == [(11, 256, 16), (0, 128, 16)]
    cache = json.load(open(os.path.join(str(tmp), "autotune.json")))  # rewritten whole
    assert list(cache) == ["FakeGPU|p1|18:1"]
