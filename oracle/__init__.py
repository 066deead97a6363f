"""FP64 CPU oracle for the adiabatic-evolution hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package's smoke check and by the bench's
CPU-baseline leg, never by the product path.  It shares no code with the CUDA path; its only
common dependency is the seeded input generator package `instances`.
"""
from . import oracle  # noqa: F401
