"""Python side of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package's smoke check and by the bench's
CPU-baseline leg, never by the product path.  It shares no code with the CUDA path.

Contents
  * Hamiltonian construction from Exact-Cover-3 data, written from the paper's equations:
      H_i = sum_i c_i (1 - sigma^x_i)                       (Eq. Hix; c_i = 1/2 or n_i/2)
      H_f = sum_clauses Omega * pen(#ones)                  (Eq. hci; or the Z/ZZ form Eq. final_ham)
      H_c = sum_(i,j) J_ij sigma^x_i sigma^x_j              (third path term, cf. Eq. nlpath)
      H^xyz = Omega sum_{i<j} n_ij/2 (1 - sigma_i . sigma_j)  (Eq. Hixyz)
      H^xy  = 3 m Omega 1 - Omega sum_{i<j} n_ij/2 (X_i X_j + Y_i Y_j)   (Eq. Hixy)
  * `dicke_state`: the balanced superposition over one Hamming weight (Eq. initstate).
  * `xy_sector_ground_state`: the ground state of H^xy in one Hamming-weight sector (the XY
    algorithm's start, Sec. III.A.3), by dense diagonalisation of the sector block.
  * `hpsi` / `propagate`: thin ctypes calls into aqc_oracle.c (scatter-form SQH matvec, RK4
    start-up + Adams-Bashforth-Moulton-4 PEC integrator).
  * `dense_matrix`: explicit 2x2 Pauli matrices combined with Kronecker products, qubit 1 as
    the least significant bit (Eq. ztensor and the index formula after it).
  * observables: P_1 = |<w|psi>|^2 and E = <psi|H_f|psi> (Sec. II.B).
  * `step_count`: the fixed-step rule h = T/N, N = ceil(T * Lambda / kappa).

Every function here is pinned by tests/test_oracle_pins.py, tests/test_oracle_xy_pins.py and
tests/test_oracle_cbc_pins.py against closed forms, dense linear algebra, brute force or a
library ODE solver; none is "parity unpinned".  tests/test_oracle_mutations.py plants mistakes
in the builders of the XY/XYZ algorithms and checks that a pin catches each.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aqc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

PEN_INDICATOR = 0
PEN_SQUARED = 1
KAPPA = 0.1  # h * Lambda per step; the PEC scheme is stable on the imaginary axis up to ~0.22


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Ham(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("nterms", C.c_int),
        ("xmask", C.POINTER(C.c_uint64)),
        ("zmask", C.POINTER(C.c_uint64)),
        ("coef", C.POINTER(C.c_double)),
        ("term_group", C.POINTER(C.c_int)),
        ("nclauses", C.c_int),
        ("clause_bits", C.POINTER(C.c_int)),
        ("clause_group", C.POINTER(C.c_int)),
        ("clause_penalty", C.POINTER(C.c_int)),
        ("clause_scale", C.POINTER(C.c_double)),
        ("clause_step", C.POINTER(C.c_int)),
        ("step_m", C.c_int),
    ]


class _Sched(C.Structure):
    _fields_ = [("s_kind", C.c_int), ("T", C.c_double), ("poly", (C.c_double * 4) * 3)]


class _Stats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64),
        ("evaluations", C.c_int64),
        ("max_err_est", C.c_double),
        ("last_err_est", C.c_double),
        ("t_end", C.c_double),
    ]


class _AStats(C.Structure):
    _fields_ = [
        ("steps_done", C.c_int64),
        ("evaluations", C.c_int64),
        ("rejects", C.c_int64),
        ("segments", C.c_int64),
        ("pec_attempts", C.c_int64),
        ("max_err_est", C.c_double),
        ("t_end", C.c_double),
    ]


class _Segment(C.Structure):
    _fields_ = [("t0", C.c_double), ("h", C.c_double), ("steps", C.c_int64), ("end", C.c_int32), ("pad", C.c_int32)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.or_hpsi.argtypes = [C.POINTER(_Ham), C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_int]
        lib.or_hpsi.restype = C.c_int
        lib.or_propagate.argtypes = [C.POINTER(_Ham), C.POINTER(_Sched), C.c_int64, C.c_int64, C.c_void_p,
                                     C.POINTER(_Stats), C.c_int]
        lib.or_propagate.restype = C.c_int
        lib.or_hpsi_at.argtypes = [C.POINTER(_Ham), C.POINTER(C.c_double), C.c_void_p, C.c_int64, C.c_void_p,
                                   C.c_void_p]
        lib.or_hpsi_at.restype = C.c_int
        lib.or_propagate_adaptive.argtypes = [C.POINTER(_Ham), C.POINTER(_Sched), C.c_double, C.c_double, C.c_int,
                                              C.c_double, C.c_int64, C.c_void_p, C.POINTER(_AStats),
                                              C.POINTER(_Segment), C.c_int64, C.c_void_p, C.c_int64, C.c_int]
        lib.or_propagate_adaptive.restype = C.c_int
        lib.or_weights.argtypes = [C.POINTER(_Sched), C.c_double, C.POINTER(C.c_double)]
        lib.or_weights.restype = None
        _lib = lib
    return _lib


# ----------------------------------------------------------------------------------------
# Hamiltonian data (SQH form: list of Pauli products with real prefactors + EC3 clauses)
# ----------------------------------------------------------------------------------------
@dataclass
class Hamiltonian:
    n: int
    terms: list = field(default_factory=list)    # (group, xmask, zmask, coef)
    clauses: list = field(default_factory=list)  # (group, (a, b, c), penalty, scale, step)

    def add_term(self, group, xmask, zmask, coef):
        self.terms.append((int(group), int(xmask), int(zmask), float(coef)))

    def add_clause(self, group, bits, penalty=PEN_INDICATOR, scale=1.0, step=0):
        """step = j >= 1 marks clause h_j of the clause-by-clause sequence (Eq. kpath)."""
        self.clauses.append((int(group), tuple(int(b) for b in bits), int(penalty), float(scale), int(step)))

    def _ctypes(self):
        nt, nc = len(self.terms), len(self.clauses)
        keep = {}
        keep["x"] = np.array([t[1] for t in self.terms] or [0], dtype=np.uint64)
        keep["z"] = np.array([t[2] for t in self.terms] or [0], dtype=np.uint64)
        keep["c"] = np.array([t[3] for t in self.terms] or [0.0], dtype=np.float64)
        keep["g"] = np.array([t[0] for t in self.terms] or [0], dtype=np.int32)
        keep["cb"] = np.array([b for c in self.clauses for b in c[1]] or [0, 0, 0], dtype=np.int32)
        keep["cg"] = np.array([c[0] for c in self.clauses] or [0], dtype=np.int32)
        keep["cp"] = np.array([c[2] for c in self.clauses] or [0], dtype=np.int32)
        keep["cs"] = np.array([c[3] for c in self.clauses] or [0.0], dtype=np.float64)
        keep["st"] = np.array([c[4] for c in self.clauses] or [0], dtype=np.int32)
        step_m = sum(1 for c in self.clauses if c[4] > 0)
        h = _Ham(
            self.n, nt,
            keep["x"].ctypes.data_as(C.POINTER(C.c_uint64)),
            keep["z"].ctypes.data_as(C.POINTER(C.c_uint64)),
            keep["c"].ctypes.data_as(C.POINTER(C.c_double)),
            keep["g"].ctypes.data_as(C.POINTER(C.c_int)),
            nc,
            keep["cb"].ctypes.data_as(C.POINTER(C.c_int)),
            keep["cg"].ctypes.data_as(C.POINTER(C.c_int)),
            keep["cp"].ctypes.data_as(C.POINTER(C.c_int)),
            keep["cs"].ctypes.data_as(C.POINTER(C.c_double)),
            keep["st"].ctypes.data_as(C.POINTER(C.c_int)),
            step_m,
        )
        return h, keep

    def norm_bound(self, group):
        """sum |coef| over the group's terms + max penalty * |scale| over its clauses."""
        b = sum(abs(t[3]) for t in self.terms if t[0] == group)
        b += sum(abs(c[3]) * (4.0 if c[2] == PEN_SQUARED else 1.0) for c in self.clauses if c[0] == group)
        return b


def x_driver(n, group=0, weights=None):
    """Eq. Hix: H^x = sum_i c_i (1 - sigma^x_i), c_i = weights[i] (default 1/2 each)."""
    H = Hamiltonian(n)
    add_x_driver(H, group, weights)
    return H


def add_x_driver(H, group=0, weights=None):
    n = H.n
    if weights is None:
        weights = [0.5] * n
    H.add_term(group, 0, 0, float(sum(weights)))  # identity part
    for i in range(n):
        H.add_term(group, 1 << i, 0, -float(weights[i]))


def add_ec3_clauses(H, clauses, group=1, penalty=PEN_INDICATOR, scale=1.0):
    """Eq. hci summed over clauses (Eq. final_ham, left side)."""
    for c in clauses:
        H.add_clause(group, c, penalty, scale)


def add_ec3_zz_form(H, n, clauses, group=1, scale=1.0):
    """Eq. final_ham, right side: Omega m 1 - Omega sum n_i/2 Z_i + Omega sum n_ij/2 Z_i Z_j.
    Equal to the squared clause penalty summed over clauses."""
    ni = [0] * n
    nij = {}
    for c in clauses:
        for a in c:
            ni[a] += 1
        for x in range(3):
            for y in range(x + 1, 3):
                k = (min(c[x], c[y]), max(c[x], c[y]))
                nij[k] = nij.get(k, 0) + 1
    H.add_term(group, 0, 0, scale * len(clauses))
    for i in range(n):
        if ni[i]:
            H.add_term(group, 0, 1 << i, -scale * ni[i] / 2.0)
    for (i, j), v in sorted(nij.items()):
        H.add_term(group, 0, (1 << i) | (1 << j), scale * v / 2.0)


def add_xx_terms(H, pairs, group=2):
    """H_c = sum J_ij sigma^x_i sigma^x_j over the given (i, j, J) pairs."""
    for (i, j, J) in pairs:
        H.add_term(group, (1 << i) | (1 << j), 0, J)


def clause_pair_counts(clauses):
    """n_ij of Eq. final_ham: the number of clauses holding both bits i < j."""
    nij = {}
    for c in clauses:
        b = sorted(c)
        for x in range(3):
            for y in range(x + 1, 3):
                nij[(b[x], b[y])] = nij.get((b[x], b[y]), 0) + 1
    return nij


def add_xyz_driver(H, clauses, group=0, omega=1.0):
    """Eq. Hixyz: Omega sum_{i<j} n_ij/2 (1 - X_i X_j - Y_i Y_j - Z_i Z_j) (Heisenberg ferromagnet
    on the clause graph).  A Y on qubit q is written with both mask bits of q set."""
    for (i, j), v in sorted(clause_pair_counts(clauses).items()):
        m = (1 << i) | (1 << j)
        a = omega * v / 2.0
        H.add_term(group, 0, 0, a)
        H.add_term(group, m, 0, -a)  # X_i X_j
        H.add_term(group, m, m, -a)  # Y_i Y_j
        H.add_term(group, 0, m, -a)  # Z_i Z_j


def add_xy_driver(H, clauses, group=0, omega=1.0):
    """Eq. Hixy: 3 m Omega 1 - Omega sum_{i<j} n_ij/2 (X_i X_j + Y_i Y_j)."""
    H.add_term(group, 0, 0, 3.0 * len(clauses) * omega)
    for (i, j), v in sorted(clause_pair_counts(clauses).items()):
        m = (1 << i) | (1 << j)
        H.add_term(group, m, 0, -omega * v / 2.0)
        H.add_term(group, m, m, -omega * v / 2.0)


def dicke_state(n, k):
    """Eq. initstate: C(n, k)^{-1/2} times the sum of all basis states with k one-bits."""
    N = 1 << n
    w = np.array([bin(z).count("1") for z in range(N)])
    psi = np.zeros(N, dtype=np.complex128)
    psi[w == k] = 1.0 / math.sqrt(math.comb(n, k))
    return psi


def xy_sector_ground_state(n, clauses, k, omega=1.0):
    """Sec. III.A.3: the ground state of H^xy (Eq. Hixy) inside the sector of Hamming weight k
    (Eq. Sigmaz), the start of the XY algorithm.  The sector block <u|H^xy|v> (|u| = |v| = k) is
    built column by column from the oracle's matvec, diagonalised densely (numpy eigh), and the
    lowest eigenvector embedded in the 2^n space with the sign fixed so that its amplitudes sum
    to a non-negative number.  Returns (energy, state).  Sizes up to C(n, k) of a few thousand."""
    H = Hamiltonian(n)
    add_xy_driver(H, clauses, 0, omega)
    w = [1.0, 0.0, 0.0, 0.0]
    idx = np.array([z for z in range(1 << n) if bin(z).count("1") == k], dtype=np.int64)
    if idx.size == 0:
        raise ValueError("empty sector")
    block = np.empty((idx.size, idx.size), dtype=np.complex128)
    e = np.zeros(1 << n, dtype=np.complex128)
    for c, z in enumerate(idx):
        e[z] = 1.0
        block[:, c] = hpsi(H, w, e)[idx]
        e[z] = 0.0
    lam, V = np.linalg.eigh(block)
    v = V[:, 0]
    if v.sum().real < 0:
        v = -v
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[idx] = v
    return float(lam[0]), psi


def xy_hamiltonian(inst, driver="xy", penalty=PEN_INDICATOR, catalyst=None):
    """The XY or XYZ algorithm (Sec. III.A.2-3): driver (group 0), H_f (group 1) and, with
    `catalyst` = the list of kept clauses, H_{m-1} of Eq. nlpath as clauses in group 2."""
    H = Hamiltonian(inst.n)
    (add_xy_driver if driver == "xy" else add_xyz_driver)(H, inst.clauses, 0)
    add_ec3_clauses(H, inst.clauses, 1, penalty)
    if catalyst is not None:
        add_ec3_clauses(H, catalyst, 2, penalty)
    return H


def add_clause_by_clause(H, clauses, group=2, penalty=PEN_INDICATOR, scale=1.0):
    """H_d(s) of Eq. kpath over `clauses` in the given order (clause j of the list is h_j);
    use with a group weight of 1 (Eq. cbc: H = (1-s) H_i + s H_f + H_d(s))."""
    for j, c in enumerate(clauses):
        H.add_clause(group, c, penalty, scale, step=j + 1)


def ec3_hamiltonian(inst, penalty=PEN_INDICATOR, pairs=None, x_weights=None):
    """The workload Hamiltonian: H_i (group 0), H_f (group 1) and optional H_c (group 2)."""
    H = Hamiltonian(inst.n)
    add_x_driver(H, 0, x_weights)
    add_ec3_clauses(H, inst.clauses, 1, penalty)
    if pairs:
        add_xx_terms(H, pairs, 2)
    return H


# ----------------------------------------------------------------------------------------
# schedules
# ----------------------------------------------------------------------------------------
S_LINEAR = 0
S_SMOOTHSTEP = 1


@dataclass
class Schedule:
    T: float
    s_kind: int = S_LINEAR
    poly: tuple = ((1.0, -1.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0))

    def _ctypes(self):
        sc = _Sched()
        sc.s_kind = self.s_kind
        sc.T = self.T
        for g in range(3):
            for k in range(4):
                sc.poly[g][k] = float(self.poly[g][k])
        return sc

    def s_of(self, t):
        tau = t / self.T
        return tau if self.s_kind == S_LINEAR else 3 * tau * tau - 2 * tau ** 3

    def weights(self, t):
        """[w_A, w_B, w_C, s] at time t (s is used by clause-by-clause sequences)."""
        s = self.s_of(t)
        return [sum(self.poly[g][k] * s ** k for k in range(4)) for g in range(3)] + [s]


def linear_path(T, s_kind=S_LINEAR):
    """Eq. aqc: H(s) = (1 - s) H_i + s H_f."""
    return Schedule(T, s_kind, ((1.0, -1.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0)))


def nonlinear_path(T, s_kind=S_LINEAR, alpha=1.0):
    """Eq. nlpath form: H(s) = (1 - s) H_i + s H_f + alpha s (1 - s) H_c."""
    return Schedule(T, s_kind, ((1.0, -1.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0), (0.0, alpha, -alpha, 0.0)))


def clause_by_clause_path(T, s_kind=S_LINEAR):
    """Eq. cbc: A = 1 - s, B = s, C = 1 (the clause-by-clause term carries its own s-dependence)."""
    return Schedule(T, s_kind, ((1.0, -1.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0), (1.0, 0.0, 0.0, 0.0)))


# ----------------------------------------------------------------------------------------
# calls into the C oracle
# ----------------------------------------------------------------------------------------
def hpsi(H: Hamiltonian, weights, psi, nthreads=1):
    """out = sum_g w_g H_g psi (complex128)."""
    lib = _load()
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if psi.shape != (1 << H.n,):
        raise ValueError("psi must have 2**n entries")
    out = np.zeros_like(psi)
    h, keep = H._ctypes()
    w = (C.c_double * 4)(*[float(x) for x in list(weights)[:4]] + [0.0] * (4 - min(4, len(weights))))
    rc = lib.or_hpsi(C.byref(h), w, psi.ctypes.data, out.ctypes.data, int(nthreads))
    if rc != 0:
        raise RuntimeError("or_hpsi failed")
    return out


def hpsi_at(H: Hamiltonian, weights, psi, zs):
    """(H psi)(z) for the given indices only (complex128 array)."""
    lib = _load()
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if psi.shape != (1 << H.n,):
        raise ValueError("psi must have 2**n entries")
    zs = np.ascontiguousarray(zs, dtype=np.uint64)
    out = np.zeros(len(zs), dtype=np.complex128)
    h, keep = H._ctypes()
    w = (C.c_double * 4)(*[float(x) for x in list(weights)[:4]] + [0.0] * (4 - min(4, len(weights))))
    rc = lib.or_hpsi_at(C.byref(h), w, psi.ctypes.data, len(zs), zs.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError("or_hpsi_at failed")
    return out


@dataclass
class PropagateResult:
    psi: np.ndarray
    steps_done: int
    evaluations: int
    max_err_est: float
    last_err_est: float
    t_end: float


def propagate(H: Hamiltonian, sched: Schedule, nsteps: int, psi0, max_steps: int = -1, nthreads=1):
    """Integrate i psi' = H(t) psi on h = T/nsteps for max_steps steps (-1: to T)."""
    lib = _load()
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    if psi.shape != (1 << H.n,):
        raise ValueError("psi0 must have 2**n entries")
    h, keep = H._ctypes()
    sc = sched._ctypes()
    st = _Stats()
    rc = lib.or_propagate(C.byref(h), C.byref(sc), int(nsteps), int(max_steps), psi.ctypes.data, C.byref(st),
                          int(nthreads))
    if rc != 0:
        raise RuntimeError(f"or_propagate failed ({rc})")
    return PropagateResult(psi, st.steps_done, st.evaluations, st.max_err_est, st.last_err_est, st.t_end)


SEG_RUNNING, SEG_AT_T, SEG_REJECTED, SEG_GREW = 0, 1, 2, 3


@dataclass
class AdaptiveResult:
    psi: np.ndarray
    steps_done: int
    evaluations: int
    rejects: int
    max_err_est: float
    t_end: float
    segments: list  # (t0, h, accepted steps, end) per segment of constant step
    ratios: np.ndarray  # Milne estimate / (tol ||y||) of every PEC attempt (accepted iff <= 1)


def propagate_adaptive(H: Hamiltonian, sched: Schedule, h0, tol, psi0, grow_after=16, hmin=None, max_steps=-1,
                       nthreads=1, log_cap=100000):
    """Integrate with step-size control (or_propagate_adaptive): segments of constant h that
    land on T, a PEC step accepted if its Milne estimate <= tol ||y||, otherwise a new segment
    with h/2; 2h after `grow_after` accepted steps with estimates <= tol ||y|| / 32."""
    lib = _load()
    psi = np.array(psi0, dtype=np.complex128, copy=True)
    if psi.shape != (1 << H.n,):
        raise ValueError("psi0 must have 2**n entries")
    h, keep = H._ctypes()
    sc = sched._ctypes()
    st = _AStats()
    log = (_Segment * log_cap)()
    hmin = float(h0) * 2.0 ** -30 if hmin is None else float(hmin)
    ratios = np.zeros(log_cap)
    rc = lib.or_propagate_adaptive(C.byref(h), C.byref(sc), float(h0), float(tol), int(grow_after), hmin,
                                   int(max_steps), psi.ctypes.data, C.byref(st), log, int(log_cap),
                                   ratios.ctypes.data, int(log_cap), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"or_propagate_adaptive failed ({rc})")
    segs = [(log[i].t0, log[i].h, log[i].steps, log[i].end) for i in range(min(st.segments, log_cap))]
    ratios = ratios[: min(log_cap, st.pec_attempts)]
    return AdaptiveResult(psi, st.steps_done, st.evaluations, st.rejects, st.max_err_est, st.t_end, segs, ratios)


def uniform_state(n):
    """|S> = 2^{-n/2} sum_z |z> (Sec. II.A.1)."""
    N = 1 << n
    return np.full(N, 1.0 / math.sqrt(N), dtype=np.complex128)


# ----------------------------------------------------------------------------------------
# step rule
# ----------------------------------------------------------------------------------------
def step_count(H: Hamiltonian, sched: Schedule, kappa=KAPPA, min_steps=4):
    """N = max(min_steps, ceil(T * Lambda / kappa)); Lambda = max over s in [0,1] (1025-point
    grid) of sum_g |w_g(s)| * norm_bound(g)."""
    b = [H.norm_bound(g) for g in range(3)]
    lam = 0.0
    for i in range(1025):
        s = i / 1024.0
        w = [sum(sched.poly[g][k] * s ** k for k in range(4)) for g in range(3)]
        lam = max(lam, sum(abs(w[g]) * b[g] for g in range(3)))
    return max(min_steps, int(math.ceil(sched.T * lam / kappa)))


# ----------------------------------------------------------------------------------------
# dense reference (small n) and observables
# ----------------------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def pauli_string_matrix(n, xmask, zmask):
    """Kronecker product of single-qubit Paulis.  Qubit q (bit q-1 of z) is the
    least-significant tensor factor, so the leftmost factor is qubit n (the index formula
    after Eq. ztensor)."""
    M = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        xq, zq = (xmask >> q) & 1, (zmask >> q) & 1
        P = _Y if (xq and zq) else _X if xq else _Z if zq else _I2
        M = np.kron(M, P)
    return M


def clause_diagonal(n, bits, penalty):
    z = np.arange(1 << n)
    k = sum((z >> b) & 1 for b in bits)
    if penalty == PEN_SQUARED:
        return ((1 - k) ** 2).astype(np.float64)
    return (k != 1).astype(np.float64)


def dense_matrix(H: Hamiltonian, weights):
    """sum_g w_g H_g as a dense 2^n x 2^n matrix (n <= 10)."""
    n = H.n
    if n > 10:
        raise ValueError("dense matrices only for n <= 10")
    N = 1 << n
    M = np.zeros((N, N), dtype=np.complex128)
    for (g, x, z, c) in H.terms:
        M += weights[g] * c * pauli_string_matrix(n, x, z)
    plain = [c for c in H.clauses if c[4] == 0]
    steps = sorted((c for c in H.clauses if c[4] > 0), key=lambda c: c[4])
    for (g, bits, pen, scale, _) in plain:
        M += np.diag(weights[g] * scale * clause_diagonal(n, bits, pen))
    if steps:
        # Eq. kpath, segment by segment: on s_k in [0, 1), H_d = (1 - s_k) H_{k-1} + s_k H_k with
        # H_j the first j clauses of the sequence (1 <= j <= m-1) and H_0 = H_m = 0
        m, s = len(steps), float(weights[3])

        def H_j(j):
            d = np.zeros(N)
            if 1 <= j <= m - 1:
                for (g, bits, pen, scale, _) in steps[:j]:
                    d += weights[g] * scale * clause_diagonal(n, bits, pen)
            return d

        k = min(int(math.floor(m * s)) + 1, m)
        sk = m * s - k + 1
        if 0.0 <= sk < 1.0:
            M += np.diag((1.0 - sk) * H_j(k - 1) + sk * H_j(k))
    return M


def fidelity(psi, w):
    """P_1 = |<w|psi>|^2 (Sec. II.B)."""
    return float(abs(psi[w]) ** 2)


def energy(H: Hamiltonian, psi, group=1):
    """<psi|H_group|psi> (Sec. II.B: E = sum_n E_n P_n)."""
    w = [0.0, 0.0, 0.0]
    w[group] = 1.0
    return float(np.vdot(psi, hpsi(H, w, psi)).real)


def norm2(psi):
    return float(np.vdot(psi, psi).real)
