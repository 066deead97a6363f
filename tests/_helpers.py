"""Test helpers: load the same seeded problem data into the CUDA path and into the oracle."""
import numpy as np

from oracle import oracle as O

C128, C64 = 0, 1
TOL_STATE = {C128: 1e-10, C64: 1e-5}  # relative state error bounds of the two precisions


def tol_fidelity(prec, psi_ref):
    """Bar for |P_1 - P_1(oracle)| implied by the state bar: for one amplitude,
    ||a|^2 - |b|^2| <= (|a| + |b|) |a - b| <= (2 ||b|| + ||a - b||) ||a - b||."""
    nb = float(np.linalg.norm(psi_ref))
    d = TOL_STATE[prec] * nb
    return (2 * nb + d) * d


def rel_err(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def random_terms(n, seed, nterms=16, with_y=True):
    """Seeded raw Pauli products (group, xmask, zmask, coef): single/two-bit flips spread over
    all bits, random multi-qubit strings, Z strings and identities."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nterms):
        g = int(rng.integers(0, 3))
        kind = k % 4
        if kind == 0:  # single-bit X or Y
            b = int(rng.integers(0, n))
            x = 1 << b
            z = x if (with_y and rng.random() < 0.3) else 0
        elif kind == 1 and n >= 2:  # two-bit flip
            i, j = rng.choice(n, size=2, replace=False)
            x = (1 << int(i)) | (1 << int(j))
            z = int(rng.integers(0, 1 << n)) if with_y else 0
        elif kind == 2:  # general string
            x = int(rng.integers(0, 1 << n))
            z = int(rng.integers(0, 1 << n)) if with_y else 0
        else:  # diagonal
            x = 0
            z = int(rng.integers(0, 1 << n))
        out.append((g, x, z, float(rng.normal())))
    out.append((1, 0, 0, 0.75))  # identity shift
    return out


def random_clauses(n, seed, m=6):
    rng = np.random.default_rng(seed + 7)
    out = []
    if n < 3:
        return out
    for k in range(m):
        bits = tuple(int(b) for b in rng.choice(n, size=3, replace=False))
        out.append((int(rng.integers(0, 3)), bits, k % 2, float(rng.uniform(0.5, 1.5))))
    return out


def load_both(ctx, H_oracle, terms, clauses):
    """Feed raw terms/clauses to a Context and to an oracle Hamiltonian."""
    for g in range(3):
        sel = [t for t in terms if t[0] == g]
        if sel:
            ctx.load_terms(g, [t[1] for t in sel], [t[2] for t in sel], [t[3] for t in sel])
        for t in sel:
            H_oracle.add_term(*t)
    for (g, bits, pen, scale) in clauses:
        ctx.load_clauses(g, [bits], penalty=pen, scale=scale)
        H_oracle.add_clause(g, bits, pen, scale)
