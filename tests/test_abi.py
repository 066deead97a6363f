"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol;
host-only logic (workspace sizing, argument checks before any device call) behaves."""
import ctypes as C
import os

import pytest


@pytest.fixture(scope="module")
def native():
    import paper_1311_3938_gb300 as P
    from paper_1311_3938_gb300 import _native as N

    P.build()
    N.lib()
    return N


def test_library_exports_every_header_symbol(native):
    names = native.header_functions()
    assert len(names) >= 17
    raw = C.CDLL(native.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_workspace_bytes(native):
    for prec, amp in ((0, 16), (1, 8)):
        for n in (1, 10, 20, 28):
            b = native.aqc_workspace_bytes(n, prec)
            assert b >= 8 * (1 << n) * amp
            # plus one byte per index (cached clause counts) and small tables
            assert b < 8 * (1 << n) * amp + (1 << n) + 64 * 1024 * 1024
    assert native.aqc_workspace_bytes(0, 0) == 0
    assert native.aqc_workspace_bytes(32, 0) == 0
    assert native.aqc_workspace_bytes(10, 7) == 0


def test_create_rejects_bad_arguments(native):
    h = C.c_void_p()
    L = native.lib()
    assert L.aqc_create(C.byref(h), 0, 0, 0, None, 0, None) == native.AQC_E_INVAL
    assert L.aqc_create(C.byref(h), 0, 5, 10, None, 0, None) == native.AQC_E_INVAL
    assert L.aqc_create(C.byref(h), 0, 0, 10, None, 0, None) == native.AQC_E_NOMEM
    assert b"workspace" in L.aqc_last_error(None)
    assert h.value is None
    assert native.aqc_version().startswith("aqc-gb300")


def test_staged_transfer_entry_points_reject_null_context(native):
    L = native.lib()
    assert L.aqc_transfer_attach(None, None, None) == native.AQC_E_INVAL
    assert L.aqc_stage_initial_state(None, None) == native.AQC_E_INVAL
    assert L.aqc_fetch_state(None, None) == native.AQC_E_INVAL
    assert L.aqc_transfer_wait(None) == native.AQC_E_INVAL
    assert native.AQC_INIT_STAGED == 5


def test_norm2_noalloc_rejects_misaligned_vectors(native):
    """Checked on the host before any device call: the pointer is never dereferenced."""
    L = native.lib()
    L.aqc_norm2_noalloc.restype = C.c_int
    L.aqc_norm2_noalloc.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(C.c_double)]
    out = C.c_double()
    assert L.aqc_norm2_noalloc(native.AQC_C128, 0x10008, 4, None, C.byref(out)) == native.AQC_E_INVAL
    assert b"aligned" in L.aqc_last_error(None)
    assert L.aqc_norm2_noalloc(native.AQC_C64, 0x10004, 4, None, C.byref(out)) == native.AQC_E_INVAL


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle (test infrastructure only)."""
    root = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1311_3938_gb300")
    for dp, _, fs in os.walk(root):
        for f in fs:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower().replace("oracle_", ""), f
