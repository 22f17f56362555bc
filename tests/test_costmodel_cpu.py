"""The counts behind the bench's roofline numbers, against brute force: the
(block, partition) products of Eq. 7 that exist (t - 2m >= 0, m < M), the
flops per product, and the least bytes a streaming tick of Eq. 7 moves."""
import itertools

import pytest

import bench
from paper_2310_00319_gb300 import costmodel


@pytest.mark.parametrize("nb,M", [(1, 1), (2, 3), (7, 2), (40, 5), (41, 94), (1876, 94)])
def test_mac_terms_counts_the_products_that_exist(nb, M):
    brute = sum(1 for t, m in itertools.product(range(nb), range(M)) if t - 2 * m >= 0)
    assert bench.mac_terms(nb, M) == brute


def test_flops_per_product_and_benchmark_total():
    # a complex multiply-add is 4 real multiply-adds (8 flops); a two-filter mix
    # h_a + alpha (h_b - h_a) adds one real multiply-add per component (4 flops)
    assert costmodel.mac_flops_per_block_bin_partition(False) == 8
    assert costmodel.mac_flops_per_block_bin_partition(True) == 12
    assert costmodel.mac_flops(3, 10, 64, 4, True) == 3 * 10 * 64 * 4 * 12
    # benchmark: 64 channels, 1876 blocks, P = 512, M = 94, a mix in every block
    flops = bench.mac_terms(1876, 94) * 512 * 64 * 12
    per_sample = flops / (64 * 480000)
    # 2 M 12 = 2256 at full depth (two blocks of 2L per hop); the first 2M - 1
    # blocks sum fewer partitions, which leaves 2145.3 over 1876 blocks
    assert per_sample == pytest.approx(2145.3056, abs=1e-3)
    assert per_sample < 2 * 94 * 12


def test_stream_bytes_per_tick_by_enumeration():
    P, M = 64, 5
    for n_out, n_f, shared in [(1, 1, None), (2, 2, None), (2, 1, 1), (4, 2, 2)]:
        n_in = n_out if shared is None else shared
        reads = n_in * M * P * 8                     # each input's delay line, once
        reads += n_out * n_f * M * P * 8             # each output's filters
        writes = n_out * P * 8                       # one spectrum per output
        assert costmodel.stream_mac_bytes_per_tick(n_out, P, M, n_f, shared) == reads + writes
