"""The entry point that allocates nothing: aqc_norm2_noalloc.

Some callers may not allocate device memory (their framework or host application owns all of
it, or allocation is not allowed where they issue work).  aqc_norm2_noalloc serves them: it
takes their own device vector and keeps its reduction scratch in a static device array of the
library.  This test calls it through the C ABI and checks it against the existing entry point
(aqc_norm2 of a context holding the same state) on two calls in a row, for both precisions.
The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from instances import random_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P
    from paper_1311_3938_gb300 import _native

    P.build()
    L = C.CDLL(_native.LIB_PATH)
    L.aqc_norm2_noalloc.restype = C.c_int
    L.aqc_norm2_noalloc.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_double)]
    L.aqc_last_error.restype = C.c_char_p
    L.aqc_last_error.argtypes = [C.c_void_p]
    return L


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
@pytest.mark.parametrize("n", [6, 17, 22])
def test_norm2_noalloc_matches_context_entry_point(lib, prec, tol, n):
    from paper_1311_3938_gb300.engine import Context

    v = random_state(n, 100 + n) * 1.7  # norm^2 = 2.89
    dt = torch.complex128 if prec == 0 else torch.complex64
    psi = torch.from_numpy(v).to(dt).cuda()
    stream = torch.cuda.current_stream()
    with Context(n, prec) as ctx:
        ctx.set_initial_state(psi)
        ref = ctx.norm2()
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = C.c_double(-1.0)
        rc = lib.aqc_norm2_noalloc(prec, psi.data_ptr(), psi.numel(), stream.cuda_stream, C.byref(out))
        assert rc == 0, lib.aqc_last_error(None)
        assert abs(out.value - ref) <= tol * abs(ref), (out.value, ref)
        assert abs(out.value - 2.89) < (1e-12 if prec == 0 else 1e-5)


def test_norm2_noalloc_rejects_bad_sizes(lib):
    psi = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = C.c_double()
    assert lib.aqc_norm2_noalloc(1, psi.data_ptr(), 0, None, C.byref(out)) == -1
    assert lib.aqc_norm2_noalloc(1, psi.data_ptr(), (1 << 31) + 1, None, C.byref(out)) == -1
    assert b"n_amplitudes" in lib.aqc_last_error(None)
    assert lib.aqc_norm2_noalloc(7, psi.data_ptr(), 4, None, C.byref(out)) == -1


@pytest.mark.parametrize("count,offset", [(1, 0), (3, 0), ((1 << 20) + 1, 0), (5, 1), ((1 << 16) + 3, 1)])
def test_norm2_noalloc_odd_lengths_and_offsets(lib, count, offset):
    """complex64 in FP64 against numpy: an odd length takes its last amplitude apart from the
    16-byte loads; a vector 8 bytes off a 16-byte boundary takes one 8-byte load per amplitude."""
    rng = np.random.default_rng(count)
    v = (rng.standard_normal(count + 1) + 1j * rng.standard_normal(count + 1)).astype(np.complex64)
    buf = torch.from_numpy(v).cuda()  # one spare amplitude: the offset view stays inside
    assert buf.data_ptr() % 256 == 0
    ref = float(np.sum(np.abs(v[offset:offset + count].astype(np.complex128)) ** 2))
    out = C.c_double(-1.0)
    rc = lib.aqc_norm2_noalloc(1, buf.data_ptr() + 8 * offset, count, torch.cuda.current_stream().cuda_stream,
                               C.byref(out))
    assert rc == 0, lib.aqc_last_error(None)
    assert abs(out.value - ref) <= 1e-6 * ref, (out.value, ref)
