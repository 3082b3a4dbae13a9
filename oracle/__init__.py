"""Plain FP64 CPU oracle for the mixed-precision H-matrix vector product and
BiCG-STAB of arXiv:1911.00093 (see hmat_oracle.c for what is computed and the
passages it follows).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are its only users.  It shares no code with the
GPU path and never calls it.
"""
from .oracle import *  # noqa: F401,F403
