"""GB300-native adiabatic-evolution hot path (arXiv:1311.3938): SQH matvec fused with the
fourth-order predictor-corrector integrator, as hand-written sm_103a CUDA behind a C ABI
(include/aqc.h), with a thin Python binding."""
from . import _native
from ._native import (  # noqa: F401
    AQC_C64,
    AQC_C128,
    AQC_GRP_A,
    AQC_GRP_B,
    AQC_GRP_C,
    AQC_CLAUSE_STEPWISE,
    AQC_INIT_BASIS,
    AQC_INIT_DICKE,
    AQC_INIT_STAGED,
    AQC_INIT_UNIFORM,
    AQC_PEN_INDICATOR,
    AQC_PEN_SQUARED,
    AQC_S_LINEAR,
    AQC_S_SMOOTHSTEP,
    AqcError,
)

__version__ = "0.1.0"


def build(force=False, verbose=False):
    from .buildlib import build as _b

    return _b(force=force, verbose=verbose)


def Context(*a, **k):
    from .engine import Context as _C

    return _C(*a, **k)
