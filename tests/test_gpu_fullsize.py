"""Full-size checks (n = 28, the benchmark's launch configuration) and a three-layout parity run.

* H(t) psi at n = 28 for a seeded random state, both precisions: sampled outputs against the
  oracle's single-output evaluation (edges, tile boundaries, the solution, random indices).
* A product-state property at n = 28: for a Hamiltonian without couplings the exact evolution
  factorises; sampled amplitudes of the GPU state equal products of single-qubit oracle states.
* n = 24 (three layouts plus products no layout holds): the first 12 grid steps against the
  FP64 oracle, both precisions.
"""
import math

import numpy as np
import pytest

from instances import generate_ec3, random_state, xx_pairs
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


def _sample_indices(n, w, seed=0, count=3000):
    N = 1 << n
    rng = np.random.default_rng(seed)
    edges = [0, 1, N - 1, N - 2, w, w ^ 1, (1 << 13) - 1, 1 << 13, (1 << 20) - 1, 1 << 21, N >> 1]
    return np.unique(np.concatenate([np.array(edges, dtype=np.uint64),
                                     rng.integers(0, N, count, dtype=np.uint64)]))


@pytest.mark.parametrize("prec", [C64, C128])
def test_hpsi_n28_sampled_against_oracle(prec):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, T, t = 28, 100.0, 37.5
    inst = generate_ec3(n, 3)
    psi = random_state(n, 28)
    with Context(n, prec) as ctx:
        HB.load_ec3(ctx, inst)
        ctx.set_schedule(T, HB.linear_schedule())
        dt = torch.complex128 if prec == C128 else torch.complex64
        dpsi = torch.from_numpy(psi).to(dt).cuda()
        out = ctx.hpsi(t, dpsi).cpu().numpy()
        used = dpsi.cpu().numpy().astype(np.complex128)  # the input as the GPU saw it
        del dpsi
    H = O.ec3_hamiltonian(inst)
    zs = _sample_indices(n, inst.solution)
    ref = O.hpsi_at(H, O.linear_path(T).weights(t), used, zs)
    got = out[zs.astype(np.int64)]
    scale = np.abs(ref).max()
    tol = 1e-13 if prec == C128 else 2e-6
    assert np.max(np.abs(got - ref)) < tol * scale


def _one_qubit_state(c, b, T, nsteps):
    """Qubit evolution under (1-s) c (1 - X) + s b Z from |+>, by the oracle at n = 1."""
    H1 = O.Hamiltonian(1)
    O.add_x_driver(H1, 0, [c])
    H1.add_term(1, 0, 1, b)
    return O.propagate(H1, O.linear_path(T), nsteps, O.uniform_state(1)).psi


def test_product_state_n28():
    from paper_1311_3938_gb300.engine import Context

    n, T = 28, 1.0
    rng = np.random.default_rng(28)
    c = rng.uniform(0.3, 1.0, n)
    b = rng.uniform(-1.0, 1.0, n)
    with Context(n, C64) as ctx:
        ctx.load_terms(0, [0] + [1 << q for q in range(n)], [0] * (n + 1), [float(c.sum())] + list(-c))
        ctx.load_terms(1, [0] * n, [1 << q for q in range(n)], list(b))
        ctx.set_schedule(T, ((1, -1, 0, 0), (0, 1, 0, 0), (0, 0, 0, 0)))
        ctx.set_integrator(0, 0.02)
        ctx.set_initial_state("uniform")
        st = ctx.propagate(-1)
        assert abs(st["t"] - T) < 1e-12
        psi = ctx.state()
    qubits = [_one_qubit_state(c[q], b[q], T, 20000) for q in range(n)]
    zs = _sample_indices(n, 12345, seed=1, count=2000)
    ref = np.array([np.prod([qubits[q][(int(z) >> q) & 1] for q in range(n)]) for z in zs])
    got = psi[zs.astype(np.int64)].astype(np.complex128)
    # amplitudes are ~2^-14; compare relative to the amplitude scale
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) < 2e-5 * scale
    assert abs(st["norm2"] - 1.0) < 1e-4


@pytest.mark.parametrize("prec", [C64, C128])
def test_n24_three_layouts_first_steps(prec):
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.engine import Context

    n, T = 24, 10.0
    inst = generate_ec3(n, 4)
    pairs = xx_pairs(n, 4)
    with Context(n, prec) as ctx:
        HB.load_ec3(ctx, inst, pairs=pairs)
        ctx.set_schedule(T, HB.nonlinear_schedule(), 1)
        ctx.set_integrator(0, 0.0)
        ctx.set_initial_state("uniform")
        ctx.propagate(12)
        got = ctx.state()
    H = O.ec3_hamiltonian(inst, pairs=pairs)
    sched = O.nonlinear_path(T, 1)
    ref = O.propagate(H, sched, O.step_count(H, sched), O.uniform_state(n), max_steps=12, nthreads=16)
    assert rel_err(got, ref.psi) < TOL_STATE[prec] * 0.1


@pytest.mark.parametrize("n", [22, 27])
def test_x_string_partial_passes_sampled(n):
    """Strided layouts holding only X strings run the TMA-fed partial kernel: single X on every
    qubit, XX pairs inside one strided layout (some on its register-held tile bits, some not),
    XX pairs spanning layouts (products no layout holds) and a diagonal; sampled outputs of
    H(t) psi against the oracle's single-output evaluation."""
    from paper_1311_3938_gb300.engine import Context

    rng = np.random.default_rng(n)
    terms = [(0, 1 << q, 0, float(rng.uniform(0.2, 1.0))) for q in range(n)]
    for (a, b) in [(13, 14), (14, 16), (15, 20), (19, 20), (21, 22), (n - 1, n - 3), (n - 2, 21), (3, 25 % n),
                   (0, 13), (6, n - 1), (17, n - 1)]:
        if a != b and a < n and b < n:
            terms.append((2, (1 << a) | (1 << b), 0, float(rng.uniform(-1.0, 1.0))))
    terms.append((1, 0, (1 << 2) | (1 << (n - 1)), 0.7))
    H = O.Hamiltonian(n)
    ctx = Context(n, C64)
    for g in range(3):
        sel = [t for t in terms if t[0] == g]
        if sel:
            ctx.load_terms(g, [t[1] for t in sel], [t[2] for t in sel], [t[3] for t in sel])
            for t in sel:
                H.add_term(g, t[1], t[2], t[3])
    poly = ((1, -1, 0, 0), (0, 1, 0, 0), (0, 1, -1, 0))
    ctx.set_schedule(10.0, poly, 0)
    psi = random_state(n, 99)
    dpsi = torch.from_numpy(psi).to(torch.complex64).cuda()
    out = ctx.hpsi(3.3, dpsi).cpu().numpy()
    used = dpsi.cpu().numpy().astype(np.complex128)
    del dpsi
    ctx.close()
    zs = _sample_indices(n, 1234, seed=n, count=3000)
    ref = O.hpsi_at(H, O.Schedule(10.0, 0, poly).weights(3.3), used, zs)
    got = out[zs.astype(np.int64)]
    assert np.max(np.abs(got - ref)) < 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("n,relabel", [(22, False), (27, False), (27, True)])
def test_hop_partial_passes_sampled(n, relabel):
    """Hops X_iX_j + Y_iY_j (Eq. Hixy) on pairs inside strided layouts (with and without the
    pair bit and the register-held tile bits), across layouts, plus an X driver: H(t) psi at
    sampled outputs against the oracle's single-output evaluation; the TMA-fed partial kernel
    runs the strided layouts that hold only X strings and hops."""
    from paper_1311_3938_gb300.engine import Context

    rng = np.random.default_rng(100 + n)
    H = O.Hamiltonian(n)
    ctx = Context(n, C64)
    ctx.set_relabel(relabel)
    xs, zs, cs = [0], [0], [0.25 * n]
    for q in range(n):
        xs.append(1 << q); zs.append(0); cs.append(-0.5)
    for (a, b) in [(0, 13), (1, 14), (13, 19), (14, 15), (16, 20), (0, 21), (2, n - 1), (21, 22), (n - 2, n - 1),
                   (5, 17), (3, 9), (0, 5)]:
        if not (a < n and b < n):
            continue
        c = float(rng.uniform(-1.0, -0.2))
        m = (1 << a) | (1 << b)
        xs += [m, m]; zs += [0, m]; cs += [c, c]
    for x, z, c in zip(xs, zs, cs):
        H.add_term(0, x, z, c)
    ctx.load_terms(0, xs, zs, cs)
    ctx.load_terms(1, [0], [(1 << 3) | (1 << (n - 1))], [0.3])
    H.add_term(1, 0, (1 << 3) | (1 << (n - 1)), 0.3)
    poly = ((1, -1, 0, 0), (0, 1, 0, 0), (0, 0, 0, 0))
    ctx.set_schedule(10.0, poly, 0)
    psi = random_state(n, 7 + n)
    dpsi = torch.from_numpy(psi).to(torch.complex64).cuda()
    out = ctx.hpsi(2.7, dpsi).cpu().numpy()
    used = dpsi.cpu().numpy().astype(np.complex128)
    del dpsi
    ctx.close()
    zs_ = _sample_indices(n, 4321, seed=n, count=3000)
    ref = O.hpsi_at(H, O.Schedule(10.0, 0, poly).weights(2.7), used, zs_)
    got = out[zs_.astype(np.int64)]
    assert np.max(np.abs(got - ref)) < 2e-6 * np.abs(ref).max()
