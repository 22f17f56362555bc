"""The paper's operation-count model (arxiv 2310.00319, Section 3, Tables 1-2)
and the byte / flop counts this library reports against its rooflines.

Paper model: a real FFT of length 2N costs 5 log2(N) + 14 operations per
sample (N/2 log2 N butterflies of 10 operations, plus 4N multiplications and
10N additions); TVOLAP transforms every sample forth and back twice (50%
overlap), does 2M complex multiply-adds of 8 operations per sample and
2 * 2 * 1 multiplications for the window and the overlap-add.
"""
from __future__ import annotations

import math


def fft_ops_per_sample(n: int) -> float:
    """5 log2(n) + 14 operations per sample for a real FFT of a block of n
    samples zero-padded to 2n (Section 3)."""
    return 5.0 * math.log2(n) + 14.0


def direct_ops_per_sample(n_ir: int) -> float:
    """Direct convolution: one multiply and one add per tap (Eq. 13)."""
    return 2.0 * n_ir


def ola_ops_per_sample(n_ir: int) -> float:
    """OLA with block N_IR: forward and inverse transform, a complex
    multiplication (6) and an addition (1) per sample."""
    return 2.0 * fft_ops_per_sample(n_ir) + 6.0 + 1.0


def wola_ops_per_sample(n_ir: int) -> float:
    """WOLA: OLA twice (50% overlap) plus analysis and synthesis windows and the
    overlapping summation (3 operations)."""
    return 2.0 * (ola_ops_per_sample(n_ir) + 3.0)


def tvolap_ops_per_sample(L: int, M: int) -> float:
    """TVOLAP with block 2L and M partitions:
    2 * 2 * (5 log2(2L) + 14) + 2M * 8 + 2 * 2 * 1."""
    return 4.0 * fft_ops_per_sample(2 * L) + 16.0 * M + 4.0


def mflops(ops_per_sample: float, fs: float = 48000.0) -> float:
    return ops_per_sample * fs / 1e6


# --------------------------------------------------------------------------- library counts
def mac_flops_per_block_bin_partition(interp: bool) -> int:
    """FP32 operations of Eq. 7 per (output block, bin, partition): a complex
    multiply-add (8) and, for a mix of two filters, the mix h_a + alpha (h_b -
    h_a) (2 multiply-adds = 4)."""
    return 12 if interp else 8


def mac_flops(n_out: int, n_blocks: int, P: int, M: int, interp: bool) -> float:
    """Algorithmic flops of the offline multiply-accumulate over all blocks."""
    return float(n_out) * n_blocks * P * M * mac_flops_per_block_bin_partition(interp)


def stream_mac_bytes_per_tick(n_out: int, P: int, M: int, n_filters: int,
                              shared_inputs: int | None = None) -> float:
    """HBM bytes one streaming tick of Eq. 7 must move at least: every output
    reads M delay-line spectra of its input (shared between outputs of the
    same input when ``shared_inputs`` counts the distinct inputs) and M
    spectra of each of its n_filters (1 or 2) filters, 8 bytes per bin, and
    writes one spectrum."""
    n_fdl = n_out if shared_inputs is None else shared_inputs
    return 8.0 * P * (M * (n_fdl + n_out * n_filters) + n_out)
