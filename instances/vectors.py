"""Seeded synthetic state vectors (numpy PCG64 + standard normals: identical on every host)."""
from __future__ import annotations

import numpy as np


def random_state(n: int, seed: int, normalize: bool = True) -> np.ndarray:
    """Complex128 vector of 2**n amplitudes with i.i.d. standard-normal parts."""
    g = np.random.Generator(np.random.PCG64(seed))
    N = 1 << n
    v = g.standard_normal(N) + 1j * g.standard_normal(N)
    if normalize:
        v /= np.sqrt(np.vdot(v, v).real)
    return v.astype(np.complex128)


def uniform_state_value(n: int) -> float:
    """Amplitude of the uniform superposition |S> on n qubits (Sec. II.A.1)."""
    return 1.0 / np.sqrt(float(1 << n))
