"""ctypes binding of libaqc.so: the C ABI of include/aqc.h under the same names.

Argument marshalling only; every step of the computation runs in the library's CUDA
kernels.  Loading fails loudly if the library has not been built (no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libaqc.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "aqc.h")

AQC_OK = 0
AQC_E_INVAL = -1
AQC_E_NOMEM = -2
AQC_E_CUDA = -3
AQC_E_NUMERIC = -4
AQC_E_STATE = -5
AQC_E_UNSUPPORTED = -6
AQC_E_TIMEOUT = -7
AQC_UNIT_WEIGHTS = -1.0
AQC_SEG_RUNNING, AQC_SEG_AT_T, AQC_SEG_REJECTED, AQC_SEG_GREW = 0, 1, 2, 3
AQC_WS_STEP_CONTROL = 1
AQC_WS_Y_COMPENSATION = AQC_WS_STEP_CONTROL

AQC_C128 = 0
AQC_C64 = 1
AQC_GRP_A, AQC_GRP_B, AQC_GRP_C = 0, 1, 2
AQC_PEN_INDICATOR, AQC_PEN_SQUARED = 0, 1
AQC_CLAUSE_STEPWISE = 0x100
AQC_S_LINEAR, AQC_S_SMOOTHSTEP = 0, 1
AQC_INIT_UNIFORM, AQC_INIT_BASIS, AQC_INIT_USER_HOST, AQC_INIT_USER_DEVICE, AQC_INIT_DICKE = 0, 1, 2, 3, 4
AQC_INIT_STAGED = 5


class AqcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"aqc error {code}: {msg}")
        self.code = code


class aqc_stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64),
        ("n_steps", C.c_int64),
        ("evaluations", C.c_int64),
        ("t", C.c_double),
        ("h", C.c_double),
        ("norm2", C.c_double),
        ("max_err_est", C.c_double),
        ("last_err_est", C.c_double),
        ("elapsed_ms", C.c_double),
        ("launches", C.c_int64),
        ("rejects", C.c_int64),
        ("segments", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class aqc_segment(C.Structure):
    _fields_ = [("t0", C.c_double), ("h", C.c_double), ("steps", C.c_int64), ("end", C.c_int32), ("pad", C.c_int32)]


_lib = None


def lib():
    """The loaded libaqc.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libaqc.so is not built ({LIB_PATH}); run paper_1311_3938_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl, sz = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_size_t
        sig = {
            "aqc_workspace_bytes": (sz, [i32, i32]),
            "aqc_workspace_bytes_ex": (sz, [i32, i32, C.c_uint]),
            "aqc_create": (i32, [C.POINTER(vp), i32, i32, i32, vp, sz, vp]),
            "aqc_destroy": (None, [vp]),
            "aqc_set_stream": (i32, [vp, vp]),
            "aqc_load_terms": (i32, [vp, i32, sz, vp, vp, vp]),
            "aqc_load_clauses": (i32, [vp, i32, sz, vp, i32, dbl]),
            "aqc_clear_hamiltonian": (i32, [vp]),
            "aqc_set_schedule": (i32, [vp, i32, dbl, vp, vp, vp]),
            "aqc_set_integrator": (i32, [vp, i64, dbl, i32, dbl]),
            "aqc_set_step_growth": (i32, [vp, i32]),
            "aqc_get_segments": (i32, [vp, C.POINTER(aqc_segment), i64, C.POINTER(i64)]),
            "aqc_set_tile_bits": (i32, [vp, i32]),
            "aqc_set_slab_bits": (i32, [vp, i32]),
            "aqc_set_relabel": (i32, [vp, i32]),
            "aqc_get_grid": (i32, [vp, C.POINTER(i64), C.POINTER(dbl)]),
            "aqc_set_initial_state": (i32, [vp, i32, u64, vp]),
            "aqc_propagate": (i32, [vp, i64, C.POINTER(aqc_stats)]),
            "aqc_get_state": (i32, [vp, vp, i32]),
            "aqc_transfer_attach": (i32, [vp, vp, vp]),
            "aqc_stage_initial_state": (i32, [vp, vp]),
            "aqc_fetch_state": (i32, [vp, vp]),
            "aqc_transfer_wait": (i32, [vp]),
            "aqc_fidelity": (i32, [vp, u64, C.POINTER(dbl)]),
            "aqc_energy": (i32, [vp, i32, dbl, C.POINTER(dbl)]),
            "aqc_norm2": (i32, [vp, C.POINTER(dbl)]),
            "aqc_hpsi": (i32, [vp, dbl, vp, vp]),
            "aqc_lanczos_workspace_bytes": (sz, [i32, i32, i32]),
            "aqc_lanczos": (i32, [vp, dbl, vp, vp, sz, i32, i32, dbl, C.POINTER(dbl), C.POINTER(dbl),
                                  C.POINTER(i32)]),
            "aqc_lanczos_ground": (i32, [vp, dbl, vp, vp, sz, i32, dbl, C.POINTER(dbl), C.POINTER(dbl), vp,
                                         C.POINTER(i32)]),
            "aqc_tridiag_eigvals": (i32, [i32, C.POINTER(dbl), C.POINTER(dbl), i32, C.POINTER(dbl)]),
            "aqc_tridiag_eigvec": (i32, [i32, C.POINTER(dbl), C.POINTER(dbl), dbl, C.POINTER(dbl)]),
            "aqc_launch_count": (i32, [vp, C.POINTER(i64)]),
            "aqc_set_graph_steps": (i32, [vp, i32]),
            "aqc_set_grid_limit": (i32, [vp, i32]),
            "aqc_set_y_compensation": (i32, [vp, i32]),
            "aqc_set_layout_turns": (i32, [vp, i32]),
            "aqc_wait_selftest": (i32, [vp, i64]),
            "aqc_measure_fp64_fma": (i32, [i32, vp, i32, C.POINTER(dbl), C.POINTER(dbl)]),
            "aqc_get_graph_replays": (i32, [vp, C.POINTER(i64)]),
            "aqc_batch_workspace_bytes": (sz, [i32, i64]),
            "aqc_batch_create": (i32, [C.POINTER(vp), i32, i32, i32, i64, vp, sz, vp]),
            "aqc_batch_destroy": (None, [vp]),
            "aqc_batch_set_shape": (i32, [vp, i32, i32]),
            "aqc_batch_add": (i32, [vp, vp, C.POINTER(i32)]),
            "aqc_batch_remove": (i32, [vp, i32]),
            "aqc_batch_run": (i32, [vp, i64]),
            "aqc_batch_poll": (i32, [vp, vp, C.POINTER(i32), C.POINTER(i64)]),
            "aqc_batch_last_error": (C.c_char_p, [vp]),
            "aqc_norm2_noalloc": (i32, [i32, vp, u64, vp, C.POINTER(dbl)]),
            "aqc_last_error": (C.c_char_p, [vp]),
            "aqc_version": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions(path: str = HEADER_PATH):
    """Names of the functions declared in include/aqc.h."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(aqc_[a-z0-9_]+)\s*\(", txt)))


def _check(ctx, rc):
    if rc != AQC_OK:
        msg = lib().aqc_last_error(ctx)
        raise AqcError(rc, msg.decode() if msg else "")
    return rc


# ---- thin wrappers under the C names ---------------------------------------------------
def aqc_workspace_bytes(n_qubits: int, precision: int) -> int:
    return int(lib().aqc_workspace_bytes(n_qubits, precision))


def aqc_workspace_bytes_ex(n_qubits: int, precision: int, flags: int) -> int:
    return int(lib().aqc_workspace_bytes_ex(n_qubits, precision, int(flags)))


def aqc_create(device: int, precision: int, n_qubits: int, workspace: int, workspace_bytes: int, stream: int):
    h = C.c_void_p()
    rc = lib().aqc_create(C.byref(h), device, precision, n_qubits, C.c_void_p(workspace), workspace_bytes,
                          C.c_void_p(stream))
    _check(None, rc)
    return h


def aqc_destroy(ctx):
    lib().aqc_destroy(ctx)


def aqc_set_stream(ctx, stream: int):
    _check(ctx, lib().aqc_set_stream(ctx, C.c_void_p(stream)))


def aqc_load_terms(ctx, group, n_terms, xmask_ptr, zmask_ptr, coef_ptr):
    _check(ctx, lib().aqc_load_terms(ctx, group, n_terms, xmask_ptr, zmask_ptr, coef_ptr))


def aqc_load_clauses(ctx, group, m, bits_ptr, penalty, scale):
    _check(ctx, lib().aqc_load_clauses(ctx, group, m, bits_ptr, penalty, float(scale)))


def aqc_clear_hamiltonian(ctx):
    _check(ctx, lib().aqc_clear_hamiltonian(ctx))


def aqc_set_schedule(ctx, s_kind, T, coefA, coefB, coefC):
    arr = [(C.c_double * 4)(*[float(v) for v in c]) for c in (coefA, coefB, coefC)]
    _check(ctx, lib().aqc_set_schedule(ctx, s_kind, float(T), arr[0], arr[1], arr[2]))


def aqc_set_integrator(ctx, n_steps, kappa, adaptive=0, tol=0.0):
    _check(ctx, lib().aqc_set_integrator(ctx, int(n_steps), float(kappa), int(adaptive), float(tol)))


def aqc_set_step_growth(ctx, grow_after):
    _check(ctx, lib().aqc_set_step_growth(ctx, int(grow_after)))


def aqc_get_segments(ctx):
    """[(t0, h, steps, end)] of the segments of constant step of the run so far."""
    count = C.c_int64()
    _check(ctx, lib().aqc_get_segments(ctx, None, 0, C.byref(count)))
    arr = (aqc_segment * max(1, count.value))()
    _check(ctx, lib().aqc_get_segments(ctx, arr, count.value, C.byref(count)))
    return [(arr[i].t0, arr[i].h, arr[i].steps, arr[i].end) for i in range(count.value)]


def aqc_get_grid(ctx):
    n = C.c_int64()
    h = C.c_double()
    _check(ctx, lib().aqc_get_grid(ctx, C.byref(n), C.byref(h)))
    return n.value, h.value


def aqc_set_tile_bits(ctx, tile_bits):
    _check(ctx, lib().aqc_set_tile_bits(ctx, int(tile_bits)))


def aqc_set_relabel(ctx, enable):
    _check(ctx, lib().aqc_set_relabel(ctx, 1 if enable else 0))


def aqc_set_slab_bits(ctx, slab_bits):
    _check(ctx, lib().aqc_set_slab_bits(ctx, int(slab_bits)))


def aqc_set_initial_state(ctx, kind, basis, user_ptr):
    _check(ctx, lib().aqc_set_initial_state(ctx, kind, int(basis), C.c_void_p(user_ptr) if user_ptr else None))


def aqc_propagate(ctx, max_steps, want_stats=True):
    st = aqc_stats()
    _check(ctx, lib().aqc_propagate(ctx, int(max_steps), C.byref(st) if want_stats else None))
    return st.as_dict() if want_stats else None


def aqc_get_state(ctx, dst_ptr, dst_on_device):
    _check(ctx, lib().aqc_get_state(ctx, C.c_void_p(dst_ptr), int(dst_on_device)))


def aqc_transfer_attach(ctx, stage_in_ptr, stage_out_ptr):
    _check(ctx, lib().aqc_transfer_attach(ctx, C.c_void_p(stage_in_ptr), C.c_void_p(stage_out_ptr)))


def aqc_stage_initial_state(ctx, host_ptr):
    _check(ctx, lib().aqc_stage_initial_state(ctx, C.c_void_p(host_ptr)))


def aqc_fetch_state(ctx, host_ptr):
    _check(ctx, lib().aqc_fetch_state(ctx, C.c_void_p(host_ptr)))


def aqc_transfer_wait(ctx):
    _check(ctx, lib().aqc_transfer_wait(ctx))


def aqc_fidelity(ctx, w):
    out = C.c_double()
    _check(ctx, lib().aqc_fidelity(ctx, int(w), C.byref(out)))
    return out.value


def aqc_energy(ctx, group_mask, t=AQC_UNIT_WEIGHTS):
    out = C.c_double()
    _check(ctx, lib().aqc_energy(ctx, int(group_mask), float(t), C.byref(out)))
    return out.value


def aqc_norm2(ctx):
    out = C.c_double()
    _check(ctx, lib().aqc_norm2(ctx, C.byref(out)))
    return out.value


def aqc_hpsi(ctx, t, psi_ptr, out_ptr):
    _check(ctx, lib().aqc_hpsi(ctx, float(t), C.c_void_p(psi_ptr), C.c_void_p(out_ptr)))


def aqc_lanczos_workspace_bytes(n, precision, max_iter):
    return int(lib().aqc_lanczos_workspace_bytes(int(n), int(precision), int(max_iter)))


def aqc_lanczos(ctx, t, start_ptr, work_ptr, work_bytes, max_iter, n_eig, tol):
    """(eigenvalues, their last change, iterations) of the lowest n_eig Ritz values."""
    eig = (C.c_double * n_eig)()
    conv = (C.c_double * n_eig)()
    iters = C.c_int()
    _check(ctx, lib().aqc_lanczos(ctx, float(t), C.c_void_p(start_ptr), C.c_void_p(work_ptr), int(work_bytes),
                                  int(max_iter), int(n_eig), float(tol), eig, conv, C.byref(iters)))
    return list(eig), list(conv), iters.value


def aqc_lanczos_ground(ctx, t, start_ptr, work_ptr, work_bytes, max_iter, tol, ground_ptr):
    """(theta, residual, iterations); the unit ground vector is written to ground_ptr."""
    theta = C.c_double()
    resid = C.c_double()
    iters = C.c_int()
    _check(ctx, lib().aqc_lanczos_ground(ctx, float(t), C.c_void_p(start_ptr), C.c_void_p(work_ptr), int(work_bytes),
                                         int(max_iter), float(tol), C.byref(theta), C.byref(resid),
                                         C.c_void_p(ground_ptr), C.byref(iters)))
    return theta.value, resid.value, iters.value


def aqc_tridiag_eigvals(a, b, n_eig):
    k = len(a)
    A = (C.c_double * k)(*a)
    B = (C.c_double * max(1, k - 1))(*b) if k > 1 else (C.c_double * 1)()
    out = (C.c_double * n_eig)()
    rc = lib().aqc_tridiag_eigvals(k, A, B, int(n_eig), out)
    if rc:
        raise AqcError(rc, "aqc_tridiag_eigvals: bad arguments")
    return list(out)


def aqc_tridiag_eigvec(a, b, lam):
    k = len(a)
    A = (C.c_double * k)(*a)
    B = (C.c_double * max(1, k - 1))(*b) if k > 1 else (C.c_double * 1)()
    out = (C.c_double * k)()
    rc = lib().aqc_tridiag_eigvec(k, A, B, float(lam), out)
    if rc:
        raise AqcError(rc, "aqc_tridiag_eigvec: bad arguments")
    return list(out)


def aqc_set_graph_steps(ctx, k_steps):
    _check(ctx, lib().aqc_set_graph_steps(ctx, int(k_steps)))


def aqc_wait_selftest(ctx, polls):
    _check(ctx, lib().aqc_wait_selftest(ctx, int(polls)))


def aqc_set_layout_turns(ctx, mode):
    _check(ctx, lib().aqc_set_layout_turns(ctx, int(mode)))


def aqc_set_y_compensation(ctx, enable):
    _check(ctx, lib().aqc_set_y_compensation(ctx, 1 if enable else 0))


def aqc_set_grid_limit(ctx, max_ctas):
    _check(ctx, lib().aqc_set_grid_limit(ctx, int(max_ctas)))


def aqc_get_graph_replays(ctx):
    out = C.c_int64()
    _check(ctx, lib().aqc_get_graph_replays(ctx, C.byref(out)))
    return out.value


def aqc_measure_fp64_fma(device, stream_ptr, iters):
    """(TFLOP/s, ms of the timed launch)."""
    tf = C.c_double()
    ms = C.c_double()
    _check(None, lib().aqc_measure_fp64_fma(int(device), C.c_void_p(stream_ptr), int(iters), C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def aqc_launch_count(ctx):
    out = C.c_int64()
    _check(ctx, lib().aqc_launch_count(ctx, C.byref(out)))
    return out.value


def _bcheck(b, rc):
    if rc != AQC_OK:
        msg = lib().aqc_batch_last_error(b)
        raise AqcError(rc, msg.decode() if msg else "")
    return rc


def aqc_batch_workspace_bytes(max_members: int, max_items: int) -> int:
    return int(lib().aqc_batch_workspace_bytes(max_members, max_items))


def aqc_batch_create(device, precision, max_members, max_items, workspace, workspace_bytes, stream):
    h = C.c_void_p()
    rc = lib().aqc_batch_create(C.byref(h), device, precision, max_members, max_items, C.c_void_p(workspace),
                                workspace_bytes, C.c_void_p(stream) if stream else None)
    _bcheck(None, rc)
    return h


def aqc_batch_destroy(b):
    lib().aqc_batch_destroy(b)


def aqc_batch_set_shape(b, threads, steps_per_round):
    _bcheck(b, lib().aqc_batch_set_shape(b, int(threads), int(steps_per_round)))


def aqc_batch_add(b, ctx):
    slot = C.c_int()
    _bcheck(b, lib().aqc_batch_add(b, ctx, C.byref(slot)))
    return slot.value


def aqc_batch_remove(b, slot):
    _bcheck(b, lib().aqc_batch_remove(b, int(slot)))


def aqc_batch_run(b, rounds):
    _bcheck(b, lib().aqc_batch_run(b, int(rounds)))


def aqc_batch_poll(b, max_members):
    steps = (C.c_int64 * max_members)()
    active = C.c_int()
    launches = C.c_int64()
    _bcheck(b, lib().aqc_batch_poll(b, steps, C.byref(active), C.byref(launches)))
    return list(steps), active.value, launches.value


def aqc_norm2_noalloc(precision, psi_ptr, n_amplitudes, stream):
    out = C.c_double()
    _check(None, lib().aqc_norm2_noalloc(int(precision), C.c_void_p(psi_ptr), int(n_amplitudes),
                                         C.c_void_p(stream) if stream else None, C.byref(out)))
    return out.value


def aqc_last_error(ctx):
    m = lib().aqc_last_error(ctx)
    return m.decode() if m else ""


def aqc_version():
    return lib().aqc_version().decode()
