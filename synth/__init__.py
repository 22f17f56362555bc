"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This package only draws inputs: signals, impulse responses and filter
schedules. It holds none of the method's arithmetic (no windows, transforms
or convolutions) and imports neither the CUDA library nor the oracle.
"""
from .workloads import *  # noqa: F401,F403
