"""Python-side context: a torch-allocated device workspace plus the C-ABI handle.

PyTorch provides only device memory (the workspace tensor) and the CUDA stream; all work is
done by libaqc.so kernels.
"""
from __future__ import annotations

import ctypes as C
import warnings

import numpy as np
import torch

from . import _native as N


def _dtype(precision):
    return np.complex128 if precision == N.AQC_C128 else np.complex64


def _torch_dtype(precision):
    return torch.complex128 if precision == N.AQC_C128 else torch.complex64


class Context:
    """One state vector of n qubits on one GPU with its integrator (include/aqc.h)."""

    def __init__(self, n: int, precision: int = N.AQC_C128, device: int = 0, stream=None, step_control=False,
                 extra_vector=None):
        """step_control=True (or extra_vector=True) reserves the workspace's extra vector, which
        step-size control (set_integrator(adaptive=True)) or y compensation
        (set_y_compensation()) uses."""
        if extra_vector is not None:
            step_control = step_control or bool(extra_vector)
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.n = n
        self.precision = precision
        self.device = device
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.ws_bytes = N.aqc_workspace_bytes_ex(n, precision, N.AQC_WS_STEP_CONTROL if step_control else 0)
        if self.ws_bytes == 0:
            raise ValueError("unsupported n / precision")
        # +256 so that the pointer can be aligned
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.dev)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.handle = N.aqc_create(device, precision, n, self._ws_ptr, self.ws_bytes, self.stream.cuda_stream)
        self.N = 1 << n
        self._stage = None  # staging vectors of aqc_transfer_attach
        self._in_flight = []

    # ---- lifetime
    def close(self):
        if getattr(self, "handle", None):
            self.stream.synchronize()  # this context's work only, not the whole device
            N.aqc_destroy(self.handle)  # waits for the staged copies
            self.handle = None
            self.workspace = None
            self._stage = None
            self._in_flight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- Hamiltonian
    def load_terms(self, group, xmask, zmask, coef):
        x = np.ascontiguousarray(xmask, dtype=np.uint64)
        z = np.ascontiguousarray(zmask, dtype=np.uint64)
        c = np.ascontiguousarray(coef, dtype=np.float64)
        if not (len(x) == len(z) == len(c)):
            raise ValueError("term arrays differ in length")
        N.aqc_load_terms(self.handle, group, len(x), x.ctypes.data, z.ctypes.data, c.ctypes.data)

    def load_clauses(self, group, clauses, penalty=N.AQC_PEN_INDICATOR, scale=1.0, stepwise=False):
        """EC3 clauses; stepwise=True makes them (in order) the clause-by-clause sequence."""
        b = np.ascontiguousarray(np.asarray(clauses, dtype=np.int32).reshape(-1))
        kind = penalty | (N.AQC_CLAUSE_STEPWISE if stepwise else 0)
        N.aqc_load_clauses(self.handle, group, len(b) // 3, b.ctypes.data, kind, scale)

    def clear_hamiltonian(self):
        N.aqc_clear_hamiltonian(self.handle)

    # ---- schedule / integrator
    def set_schedule(self, T, weights, s_kind=N.AQC_S_LINEAR):
        N.aqc_set_schedule(self.handle, s_kind, T, *weights)

    def grid(self):
        """(N, h) of the step grid."""
        return N.aqc_get_grid(self.handle)

    def set_tile_bits(self, tile_bits=0):
        N.aqc_set_tile_bits(self.handle, tile_bits)

    def set_relabel(self, enable=True):
        """Qubit relabelling that keeps multi-qubit flips inside tile layouts (transparent)."""
        N.aqc_set_relabel(self.handle, enable)

    def set_slab_bits(self, slab_bits=0):
        """Slab order of the PEC step: 0 off, -1 automatic, k > 0 at most k slab bits."""
        N.aqc_set_slab_bits(self.handle, slab_bits)

    def set_graph_steps(self, k_steps=-1):
        """PEC steps per CUDA-graph replay: 0 off, -1 automatic, or a multiple of 4 up to 64."""
        N.aqc_set_graph_steps(self.handle, k_steps)

    def set_layout_turns(self, mode=1):
        """Turn of layouts of the PEC step (aqc_set_layout_turns): 0 off (default), 1 on."""
        N.aqc_set_layout_turns(self.handle, mode)

    def set_y_compensation(self, enable=True):
        """Compensated complex64 corrector (aqc_set_y_compensation); set the initial state after."""
        N.aqc_set_y_compensation(self.handle, enable)

    def set_grid_limit(self, max_ctas=0):
        """At most max_ctas CTAs per layout-pass launch (0: every SM)."""
        N.aqc_set_grid_limit(self.handle, max_ctas)

    def graph_replays(self):
        return N.aqc_get_graph_replays(self.handle)

    def set_integrator(self, n_steps=0, kappa=0.0, adaptive=False, tol=0.0):
        """Fixed-step grid (n_steps, or the step rule with kappa), or step-size control with a
        relative tolerance tol per PEC step (adaptive=True; aqc.h, aqc_set_integrator)."""
        N.aqc_set_integrator(self.handle, n_steps, kappa, 1 if adaptive else 0, tol)

    def set_step_growth(self, grow_after=16):
        N.aqc_set_step_growth(self.handle, grow_after)

    def segments(self):
        """[(t0, h, accepted steps, end)] of the run's segments of constant step."""
        return N.aqc_get_segments(self.handle)

    def set_initial_state(self, state="uniform"):
        """"uniform" (|S>), a basis index, ("dicke", k) (Eq. initstate), "staged" (the vector of
        the last stage_initial_state), or a host/device vector."""
        if isinstance(state, str) and state == "uniform":
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_UNIFORM, 0, 0)
        elif isinstance(state, str) and state == "staged":
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_STAGED, 0, 0)
        elif isinstance(state, tuple) and len(state) == 2 and state[0] == "dicke":
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_DICKE, int(state[1]), 0)
        elif isinstance(state, (int, np.integer)):
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_BASIS, int(state), 0)
        elif isinstance(state, torch.Tensor) and state.device.type == "cpu":
            t = state.to(_torch_dtype(self.precision)).contiguous()  # host buffer (pinned: async DMA)
            if t.numel() != self.N:
                raise ValueError("state has the wrong length")
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_USER_HOST, 0, t.data_ptr())
            self.stream.synchronize()
        elif isinstance(state, torch.Tensor):
            t = state.to(self.dev, _torch_dtype(self.precision)).contiguous()
            if t.numel() != self.N:
                raise ValueError("state has the wrong length")
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_USER_DEVICE, 0, t.data_ptr())
            self.stream.synchronize()
        else:
            a = np.ascontiguousarray(state, dtype=_dtype(self.precision))
            if a.size != self.N:
                raise ValueError("state has the wrong length")
            N.aqc_set_initial_state(self.handle, N.AQC_INIT_USER_HOST, 0, a.ctypes.data)
            self.stream.synchronize()

    # ---- staged host transfers (copy engines overlap the integrator)
    def attach_transfers(self):
        """Allocate the two device staging vectors and attach them (aqc_transfer_attach).  Called
        again, it keeps the previous vectors alive until the library has finished their copies."""
        dt = _torch_dtype(self.precision)
        with torch.cuda.device(self.dev):
            stage = (torch.empty(self.N, dtype=dt, device=self.dev), torch.empty(self.N, dtype=dt, device=self.dev))
        N.aqc_transfer_attach(self.handle, stage[0].data_ptr(), stage[1].data_ptr())
        self._stage = stage  # the previous pair (if any) is released only now
        self._in_flight = []  # host tensors of enqueued copies (attach waited for the earlier ones)

    @staticmethod
    def _warn_pageable(host_tensor):
        if torch.cuda.is_available() and not host_tensor.is_pinned():
            warnings.warn("pageable host tensor: the staged copy cannot overlap the integration "
                          "(use .pin_memory())", stacklevel=3)

    def stage_initial_state(self, host_tensor):
        """Enqueue the copy of a pinned host vector (qubit order) for the next
        set_initial_state("staged"); returns at once.  The tensor stays referenced (and must not
        change) until transfer_wait()."""
        if host_tensor.device.type != "cpu" or host_tensor.dtype != _torch_dtype(self.precision):
            raise ValueError("a host tensor of the state dtype is required")
        if host_tensor.numel() != self.N or not host_tensor.is_contiguous():
            raise ValueError("state has the wrong length or is not contiguous")
        self._warn_pageable(host_tensor)
        N.aqc_stage_initial_state(self.handle, host_tensor.data_ptr())
        self._in_flight.append(host_tensor)  # alive until its copy is known to be done

    def fetch_state(self, host_tensor):
        """Enqueue the copy of psi into a pinned host tensor; valid after transfer_wait(), which
        also releases the references the context keeps to the tensors of enqueued copies."""
        if host_tensor.device.type != "cpu" or host_tensor.dtype != _torch_dtype(self.precision):
            raise ValueError("a host tensor of the state dtype is required")
        if host_tensor.numel() != self.N or not host_tensor.is_contiguous():
            raise ValueError("state has the wrong length or is not contiguous")
        self._warn_pageable(host_tensor)
        N.aqc_fetch_state(self.handle, host_tensor.data_ptr())
        self._in_flight.append(host_tensor)

    def transfer_wait(self):
        N.aqc_transfer_wait(self.handle)
        self._in_flight.clear()

    def propagate(self, max_steps=-1, stats=True):
        return N.aqc_propagate(self.handle, max_steps, stats)

    # ---- results
    def state(self, device=False):
        if device:
            out = torch.empty(self.N, dtype=_torch_dtype(self.precision), device=self.dev)
            N.aqc_get_state(self.handle, out.data_ptr(), 1)
            return out
        out = np.empty(self.N, dtype=_dtype(self.precision))
        N.aqc_get_state(self.handle, out.ctypes.data, 0)
        return out

    def state_into(self, host_tensor):
        """Copy psi into a (pinned) host torch tensor of the state dtype."""
        N.aqc_get_state(self.handle, host_tensor.data_ptr(), 0)
        return host_tensor

    def fidelity(self, w):
        return N.aqc_fidelity(self.handle, w)

    def energy(self, group=N.AQC_GRP_B):
        """<psi|H_group|psi> with unit weight (the final energy of Sec. II.B for group B)."""
        return N.aqc_energy(self.handle, 1 << group, N.AQC_UNIT_WEIGHTS)

    def energy_at(self, t, groups=(N.AQC_GRP_A, N.AQC_GRP_B, N.AQC_GRP_C)):
        """<psi| sum_{g in groups} w_g(s(t)) H_g |psi> (all groups: <H(t)>)."""
        mask = 0
        for g in groups:
            mask |= 1 << g
        return N.aqc_energy(self.handle, mask, float(t))

    def norm2(self):
        return N.aqc_norm2(self.handle)

    def launch_count(self):
        return N.aqc_launch_count(self.handle)

    def lanczos(self, t, start: torch.Tensor, max_iter=200, n_eig=2, tol=1e-10):
        """Lowest n_eig eigenvalues of H(t) reachable from `start` (aqc_lanczos): returns
        (eigenvalues, last change of each, iterations)."""
        nbytes = N.aqc_lanczos_workspace_bytes(self.n, self.precision, max_iter)
        with torch.cuda.stream(self.stream):
            start = start.to(self.dev, _torch_dtype(self.precision)).contiguous()
            work = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.dev)
            off = (-work.data_ptr()) % 256
            out = N.aqc_lanczos(self.handle, t, start.data_ptr(), work.data_ptr() + off, nbytes, max_iter, n_eig, tol)
            del work, start
        return out

    def lanczos_ground(self, t, start: torch.Tensor, max_iter=300, tol=1e-12):
        """Lowest eigenpair of H(t) reachable from `start` (aqc_lanczos_ground): returns
        (device vector x, theta, residual ||H x - theta x||, iterations)."""
        nbytes = N.aqc_lanczos_workspace_bytes(self.n, self.precision, max_iter)
        with torch.cuda.stream(self.stream):
            start = start.to(self.dev, _torch_dtype(self.precision)).contiguous()
            work = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.dev)
            off = (-work.data_ptr()) % 256
            x = torch.empty(self.N, dtype=_torch_dtype(self.precision), device=self.dev)
            theta, resid, iters = N.aqc_lanczos_ground(self.handle, t, start.data_ptr(), work.data_ptr() + off, nbytes,
                                                       max_iter, tol, x.data_ptr())
            del work, start
        return x, theta, resid, iters

    def hpsi(self, t, psi: torch.Tensor, out: torch.Tensor = None):
        """out = H(t) psi for device tensors of the state dtype."""
        psi = psi.to(self.dev, _torch_dtype(self.precision)).contiguous()
        if out is None:
            out = torch.empty_like(psi)
        N.aqc_hpsi(self.handle, t, psi.data_ptr(), out.data_ptr())
        return out


class Batch:
    """Many contexts stepped together (include/aqc.h, aqc_batch_*): batched PEC launches over
    (member, tile) work items, K steps per CUDA-graph replay."""

    def __init__(self, precision=N.AQC_C64, device=0, max_members=64, max_items=1 << 16, stream=None,
                 threads=256, steps_per_round=16):
        self.precision = precision
        self.device = device
        self.dev = torch.device("cuda", device)
        self.max_members = max_members
        self.stream = stream if stream is not None else torch.cuda.Stream(self.dev)
        self.ws_bytes = N.aqc_batch_workspace_bytes(max_members, max_items)
        if self.ws_bytes == 0:
            raise ValueError("unsupported batch size")
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.dev)
        ptr = (self.workspace.data_ptr() + 255) // 256 * 256
        self.handle = N.aqc_batch_create(device, precision, max_members, max_items, ptr, self.ws_bytes,
                                         self.stream.cuda_stream)
        self.members = {}
        N.aqc_batch_set_shape(self.handle, threads, steps_per_round)
        self.threads = threads
        self.steps_per_round = steps_per_round

    def set_shape(self, threads, steps_per_round):
        N.aqc_batch_set_shape(self.handle, threads, steps_per_round)
        self.threads = threads
        self.steps_per_round = steps_per_round

    def add(self, ctx: Context) -> int:
        slot = N.aqc_batch_add(self.handle, ctx.handle)
        self.members[slot] = ctx
        return slot

    def remove(self, slot) -> Context:
        N.aqc_batch_remove(self.handle, slot)
        return self.members.pop(slot)

    def run(self, rounds=1):
        N.aqc_batch_run(self.handle, rounds)

    def poll(self):
        steps, active, launches = N.aqc_batch_poll(self.handle, self.max_members)
        return steps, active, launches

    def run_to_completion(self, rounds_per_poll=8, max_polls=1 << 30):
        """Replay rounds until every member reached its t = T; returns the number of polls."""
        polls = 0
        while polls < max_polls:
            self.run(rounds_per_poll)
            _, active, _ = self.poll()
            polls += 1
            if active == 0:
                break
        return polls

    def close(self):
        if getattr(self, "handle", None):
            self.stream.synchronize()
            N.aqc_batch_destroy(self.handle)
            self.handle = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
