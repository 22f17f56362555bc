"""GB300-native (sm_103a) time-variant overlap-add in partitions (TVOLAP).

Time-variant partitioned convolution of many audio channels after arxiv
2310.00319, Section 2: hand-written CUDA kernels behind the C ABI in
include/tvolap.h, with this package as the thin Python binding.

    from paper_2310_00319_gb300 import Plan
    plan = Plan(L=256, M=94, n_in=64, n_slots=512)
    plan.load_bank(0, irs)                       # [512, 48000] float32 on cuda
    y = plan.process_signal(x, sched_a, sched_b, sched_alpha)
"""
from .tvolap import Plan, n_blocks_for  # noqa: F401
from ._lib import TvolapError  # noqa: F401
from . import costmodel  # noqa: F401
