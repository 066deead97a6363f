"""SQH term lists of the paper's Hamiltonians, as arrays for aqc_load_terms / aqc_load_clauses.

Qubit q of the paper is bit q-1 of the basis index (Eq. ztensor).  All builders return plain
numpy arrays (xmask uint64, zmask uint64, coef float64) or clause bit triples (int32).
"""
from __future__ import annotations

import numpy as np

from . import _native as N

# path weights as cubics in s (w(s) = c0 + c1 s + c2 s^2 + c3 s^3)
W_ONE_MINUS_S = (1.0, -1.0, 0.0, 0.0)
W_S = (0.0, 1.0, 0.0, 0.0)
W_ZERO = (0.0, 0.0, 0.0, 0.0)


def w_s_one_minus_s(alpha: float = 1.0):
    """alpha * s (1 - s), the weight of the third path term (Eq. nlpath)."""
    return (0.0, float(alpha), -float(alpha), 0.0)


def x_driver_terms(n: int, weights=None):
    """Eq. Hix: H^x = sum_i c_i (1 - sigma^x_i); c_i = 1/2 by default (n_i/2 in the paper).
    Returns the identity prefactor sum c_i and one -c_i sigma^x_i product per qubit."""
    c = np.full(n, 0.5) if weights is None else np.asarray(weights, dtype=np.float64)
    x = np.concatenate([[0], 1 << np.arange(n, dtype=np.uint64)]).astype(np.uint64)
    z = np.zeros(n + 1, dtype=np.uint64)
    coef = np.concatenate([[c.sum()], -c]).astype(np.float64)
    return x, z, coef


def xx_terms(pairs):
    """sum_(i,j) J_ij sigma^x_i sigma^x_j over (i, j, J) triples."""
    x = np.array([(1 << i) | (1 << j) for (i, j, _) in pairs], dtype=np.uint64)
    z = np.zeros(len(pairs), dtype=np.uint64)
    coef = np.array([J for (_, _, J) in pairs], dtype=np.float64)
    return x, z, coef


def ec3_zz_terms(n: int, clauses, omega: float = 1.0):
    """Eq. final_ham: Omega m 1 - Omega sum_i n_i/2 sigma^z_i + Omega sum_{i<j} n_ij/2 sigma^z_i sigma^z_j."""
    ni = np.zeros(n)
    nij = {}
    for c in clauses:
        for a in c:
            ni[a] += 1
        for u in range(3):
            for v in range(u + 1, 3):
                key = (min(c[u], c[v]), max(c[u], c[v]))
                nij[key] = nij.get(key, 0) + 1
    xs, zs, cs = [0], [0], [omega * len(clauses)]
    for i in range(n):
        if ni[i]:
            xs.append(0)
            zs.append(1 << i)
            cs.append(-omega * ni[i] / 2)
    for (i, j), v in sorted(nij.items()):
        xs.append(0)
        zs.append((1 << i) | (1 << j))
        cs.append(omega * v / 2)
    return np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cs, np.float64)


def _pair_weights(clauses):
    """n_ij (Eq. final_ham): clauses holding both bits i < j, as {(i, j): count}."""
    out = {}
    for c in clauses:
        a, b, d = sorted(int(v) for v in c)
        for key in ((a, b), (a, d), (b, d)):
            out[key] = out.get(key, 0) + 1
    return out


def xyz_driver_terms(clauses, omega: float = 1.0):
    """Eq. Hixyz: Omega sum_{i<j} n_ij/2 (1 - X_i X_j - Y_i Y_j - Z_i Z_j), the Heisenberg
    ferromagnet on the clause graph.  A Y on qubit q sets bit q in both masks."""
    xs, zs, cs = [], [], []
    ident = 0.0
    for (i, j), v in sorted(_pair_weights(clauses).items()):
        m = (1 << i) | (1 << j)
        a = omega * v / 2.0
        ident += a
        xs += [m, m, 0]
        zs += [0, m, m]
        cs += [-a, -a, -a]
    return (np.array([0] + xs, np.uint64), np.array([0] + zs, np.uint64), np.array([ident] + cs, np.float64))


def xy_driver_terms(clauses, omega: float = 1.0):
    """Eq. Hixy: 3 m Omega 1 - Omega sum_{i<j} n_ij/2 (X_i X_j + Y_i Y_j), the x,y ferromagnet."""
    xs, zs, cs = [0], [0], [3.0 * len(clauses) * omega]
    for (i, j), v in sorted(_pair_weights(clauses).items()):
        m = (1 << i) | (1 << j)
        xs += [m, m]
        zs += [0, m]
        cs += [-omega * v / 2.0, -omega * v / 2.0]
    return np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cs, np.float64)


def removable_clauses(n: int, clauses):
    """Indices of clauses whose removal keeps the clause graph connected (bits joined by shared
    clauses), the clauses the paper allows to drop for H_{m-1} (Sec. IV.A.1)."""
    used = sorted({int(b) for c in clauses for b in c})  # the bits of the full clause graph

    def connected(cl):
        parent = list(range(n))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        for c in cl:
            r = find(int(c[0]))
            for b in c[1:]:
                parent[find(int(b))] = r
        return len({find(b) for b in used}) <= 1

    base = connected(clauses)
    return [k for k in range(len(clauses)) if connected(clauses[:k] + clauses[k + 1:]) or not base]


def clause_by_clause_schedule():
    """Eq. cbc: A = 1 - s, B = s, C = 1 (the sequence in group C carries the s-dependence of
    Eq. kpath itself)."""
    return (W_ONE_MINUS_S, W_S, (1.0, 0.0, 0.0, 0.0))


def load_xy(ctx, inst, driver: str = "xy", catalyst_alpha: float = 0.0, removed: int = None,
            penalty=N.AQC_PEN_INDICATOR, clause_by_clause: bool = False):
    """The XY or XYZ algorithm (Sec. III.A.2-3) with optional catalyst (Eq. nlpath): driver in
    group A, H_f clauses in group B and, if catalyst_alpha != 0, H_{m-1} (every clause but
    `removed`; default: the last removable clause) in group C; or, with clause_by_clause, the
    clauses in stored order as the sequence of Eq. kpath in group C (Eq. cbc).  Returns the
    schedule (use with ctx.set_schedule) and the Hamming weight of the solution (the start
    sector: set_xy_ground_start for the XY driver, the Dicke state for XYZ)."""
    terms = xy_driver_terms(inst.clauses) if driver == "xy" else xyz_driver_terms(inst.clauses)
    ctx.load_terms(N.AQC_GRP_A, *terms)
    ctx.load_clauses(N.AQC_GRP_B, inst.clauses, penalty=penalty)
    sched = linear_schedule()
    if clause_by_clause:
        ctx.load_clauses(N.AQC_GRP_C, list(inst.clauses), penalty=penalty, stepwise=True)
        return clause_by_clause_schedule(), bin(int(inst.solution)).count("1")
    if catalyst_alpha:
        cl = list(inst.clauses)
        if removed is None:
            rem = removable_clauses(inst.n, cl)
            removed = rem[-1] if rem else len(cl) - 1
        keep = cl[:removed] + cl[removed + 1:]
        ctx.load_clauses(N.AQC_GRP_C, keep, penalty=penalty)
        sched = nonlinear_schedule(catalyst_alpha)
    return sched, bin(int(inst.solution)).count("1")


def set_xy_ground_start(ctx, k: int, max_iter: int = 200, tol: float = None):
    """psi(0) of the XY algorithm (Sec. III.A.3): the ground state of H(0) in the sector of
    Hamming weight k.  On the XY paths here H(0) is the driver H^xy alone (weight 1 for group A,
    0 for B and for the catalyst; the clause-by-clause term H_d(0) vanishes).  The eigenpair is
    computed by aqc_lanczos_ground from the Dicke state of weight k (Eq. initstate), which lies
    in the sector and overlaps the ground state: the sector block of H^xy has non-positive
    off-diagonal entries, so its ground state has positive amplitudes.  tol is the relative Ritz
    residual (default 1e-12 for complex128, 2e-6 for complex64); the Krylov space is capped at
    the sector dimension C(n, k).  Returns (energy, residual ||H x - E x||, iterations)."""
    import math

    if not 0 <= k <= ctx.n:
        raise ValueError("Hamming weight out of range")
    if tol is None:
        tol = 1e-12 if ctx.precision == N.AQC_C128 else 2e-6
    ctx.set_initial_state(("dicke", k))
    start = ctx.state(device=True)
    iters = max(1, min(int(max_iter), math.comb(ctx.n, k)))
    x, theta, resid, used = ctx.lanczos_ground(0.0, start, max_iter=iters, tol=tol)
    del start
    ctx.set_initial_state(x)
    return theta, resid, used


def clause_bits(clauses):
    """EC3 clauses (Eq. 1clause) as a flat int32 array of 0-based bits."""
    return np.ascontiguousarray(np.array(clauses, dtype=np.int32).reshape(-1))


def load_ec3(ctx, inst, pairs=None, penalty=N.AQC_PEN_INDICATOR, x_weights=None):
    """Load H_i (group A), the clause penalties of H_f (group B) and optional H_c (group C)."""
    ctx.load_terms(N.AQC_GRP_A, *x_driver_terms(inst.n, x_weights))
    ctx.load_clauses(N.AQC_GRP_B, inst.clauses, penalty=penalty)
    if pairs:
        ctx.load_terms(N.AQC_GRP_C, *xx_terms(pairs))


def linear_schedule():
    """Eq. aqc: A = 1 - s, B = s."""
    return (W_ONE_MINUS_S, W_S, W_ZERO)


def nonlinear_schedule(alpha: float = 1.0):
    """Eq. nlpath form: A = 1 - s, B = s, C = alpha s (1 - s)."""
    return (W_ONE_MINUS_S, W_S, w_s_one_minus_s(alpha))
