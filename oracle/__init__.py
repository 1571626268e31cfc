"""FP64 CPU oracle for synchronized tracing of blobtree implicit surfaces.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  The arithmetic lives
in ``oracle.c`` (plain C, FP64, compiled without FMA contraction); this module
builds it with gcc and marshals numpy arrays.  It shares no code with the CUDA
path; both only read scenes made by ``paper_2304_09673_b300.scenegen``.
"""
from .oracle import *  # noqa: F401,F403
