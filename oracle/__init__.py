"""FP64 CPU oracle for TVOLAP (arxiv 2310.00319, Section 2, Eqs. 1-12).

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the CPU-baseline leg of
bench.py may import this package; the product library never does. It shares
no code with the CUDA path. See ``oracle.reference`` for the functions.
"""
from .reference import *  # noqa: F401,F403
