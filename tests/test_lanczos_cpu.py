"""Host part of the Lanczos spectrum (no GPU): the Sturm-bisection tridiagonal eigensolver of
libaqc.so against numpy's dense symmetric eigensolver, and the workspace sizing."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def native():
    import paper_1311_3938_gb300 as P

    P.build()
    from paper_1311_3938_gb300 import _native as N

    return N


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (7, 2), (40, 3), (200, 4)])
def test_tridiagonal_eigenvalues(native, k, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=k) * 3.0
    b = rng.normal(size=max(0, k - 1))
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ref = np.linalg.eigvalsh(T)
    m = min(k, 5)
    got = native.aqc_tridiag_eigvals(list(a), list(b), m)
    assert np.max(np.abs(np.array(got) - ref[:m])) < 1e-12 * max(1.0, np.abs(ref).max())


def test_tridiagonal_with_clustered_and_zero_couplings(native):
    # a zero coupling splits the matrix; equal diagonals give degenerate eigenvalues
    a = [1.0, 1.0, 1.0, 5.0, -2.0, -2.0]
    b = [0.0, 0.5, 0.0, 1e-9, 0.0]
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ref = np.linalg.eigvalsh(T)
    got = native.aqc_tridiag_eigvals(a, b, 6)
    assert np.max(np.abs(np.array(got) - ref)) < 1e-12


def test_lanczos_workspace_sizing(native):
    for prec, amp in ((0, 16), (1, 8)):
        b = native.aqc_lanczos_workspace_bytes(12, prec, 50)
        assert b >= 51 * (1 << 12) * amp
        assert b < 51 * (1 << 12) * amp + 2 * 1024 * 1024
    assert native.aqc_lanczos_workspace_bytes(12, 0, 0) == 0
    assert native.aqc_lanczos_workspace_bytes(40, 0, 10) == 0
    with pytest.raises(native.AqcError):
        native.aqc_tridiag_eigvals([1.0, 2.0], [0.1], 3)


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (9, 2), (60, 3), (250, 4)])
def test_tridiagonal_ground_eigenvector(native, k, seed):
    """aqc_tridiag_eigvec at the lowest eigenvalue: numpy's eigenvector up to its sign, which the
    library fixes by a non-negative first entry (the Ritz coefficients of aqc_lanczos_ground)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(size=k) * 3.0
    b = rng.uniform(0.2, 1.0, size=max(0, k - 1))  # non-zero couplings: unreduced, simple spectrum
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    lam, V = np.linalg.eigh(T)
    theta = native.aqc_tridiag_eigvals(list(a), list(b), 1)[0]
    got = np.array(native.aqc_tridiag_eigvec(list(a), list(b), theta))
    # sign: the library's rule (first entry >= 0) where the first entry is not at rounding level
    # (a localised eigenvector can have a first entry of 1e-24), else numpy's sign aligned
    want = V[:, 0] * (1.0 if (V[0, 0] >= 0 if abs(V[0, 0]) > 1e-8 else np.dot(V[:, 0], got) >= 0) else -1.0)
    assert got[0] >= 0
    assert abs(np.linalg.norm(got) - 1.0) < 1e-13
    assert np.max(np.abs(got - want)) < 1e-9
    assert np.linalg.norm(T @ got - theta * got) < 1e-11 * max(1.0, np.abs(lam).max())
